"""ctypes wrapper of the CPU reference interpreter (oracle/rtl_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`.  The simulator package never
imports it and shares no code with it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "rtl_oracle.c")
_lock = threading.Lock()
_lib = None

# operator kinds, in the order of the C enum
KINDS = ("input", "reg", "const", "memrd", "add", "sub", "mul", "and", "or", "xor",
         "shl", "shr", "eq", "lt", "mux", "slice", "concat")
KIND = {k: i for i, k in enumerate(KINDS)}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (plain gcc, -O2)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(_SRC):
        tmp = f"{LIB_PATH}.tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            u64, i64, vp, cp = C.c_uint64, C.c_int64, C.c_void_p, C.c_char_p
            sigs = {
                "orc_net_load_file": (vp, [cp, cp, C.c_size_t]),
                "orc_net_load_text": (vp, [cp, C.c_size_t, cp, C.c_size_t]),
                "orc_net_free": (None, [vp]),
                "orc_net_counts": (None, [vp, C.POINTER(C.c_int)]),
                "orc_net_mem_lg": (C.c_int, [vp, C.c_int]),
                "orc_sim_new": (vp, [vp, u64, u64]),
                "orc_sim_free": (None, [vp]),
                "orc_sim_reset": (None, [vp, u64, u64]),
                "orc_sim_run": (None, [vp, u64, vp]),
                "orc_sim_digest": (u64, [vp]),
                "orc_sim_cycle": (u64, [vp]),
                "orc_sim_set_cycle": (None, [vp, u64]),
                "orc_sim_get_reg": (u64, [vp, C.c_int]),
                "orc_sim_set_reg": (None, [vp, C.c_int, u64]),
                "orc_sim_get_regs": (None, [vp, vp]),
                "orc_sim_get_mem": (u64, [vp, C.c_int, u64]),
                "orc_sim_set_mem": (None, [vp, C.c_int, u64, u64]),
                "orc_sim_hold_input": (None, [vp, C.c_int, u64]),
                "orc_sim_release_input": (None, [vp, C.c_int]),
                "orc_sim_node_value": (u64, [vp, i64]),
                "orc_op": (u64, [C.c_int, C.c_int, u64, u64, u64, C.c_int, C.c_int]),
                "orc_mix64": (u64, [u64]),
                "orc_instance_key": (u64, [u64, u64]),
                "orc_stimulus": (u64, [u64, u64, u64, C.c_uint32, C.c_uint32, C.c_int]),
            }
            for name, (res, args) in sigs.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


class Net:
    """A parsed, checked and ordered netlist."""

    def __init__(self, path: str | None = None, text: str | None = None):
        err = C.create_string_buffer(512)
        L = lib()
        if text is not None:
            b = text.encode()
            h = L.orc_net_load_text(b, len(b), err, 512)
        else:
            h = L.orc_net_load_file(path.encode(), err, 512)
        if not h:
            raise OracleError(err.value.decode())
        self._h = h
        c = (C.c_int * 5)()
        L.orc_net_counts(h, c)
        self.n_in, self.n_reg, self.n_mem, self.n_node, self.n_wport = list(c)

    def mem_depth(self, m):
        return 1 << lib().orc_net_mem_lg(self._h, m)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_net_free(self._h)
            self._h = None


class Sim:
    """One simulated instance: registers, memories and the cycle counter."""

    def __init__(self, net: Net, seed: int = 42, inst: int = 0):
        self.net = net
        self._h = lib().orc_sim_new(net._h, seed, inst)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_sim_free(self._h)
            self._h = None

    def reset(self, seed, inst):
        lib().orc_sim_reset(self._h, seed, inst)

    def run(self, n: int, digests: bool = False):
        """Advance n cycles; with digests=True return the digest after each cycle."""
        if digests:
            out = np.zeros(max(n, 1), dtype=np.uint64)
            lib().orc_sim_run(self._h, n, out.ctypes.data)
            return out[:n]
        lib().orc_sim_run(self._h, n, None)
        return None

    @property
    def cycle(self):
        return lib().orc_sim_cycle(self._h)

    def set_cycle(self, c):
        """Set the cycle counter (resuming from a state taken at cycle c: the
        stimulus of cycle t depends on t)."""
        lib().orc_sim_set_cycle(self._h, c)

    def digest(self):
        return lib().orc_sim_digest(self._h)

    def reg(self, r):
        return lib().orc_sim_get_reg(self._h, r)

    def regs(self):
        out = np.zeros(max(self.net.n_reg, 1), dtype=np.uint64)
        lib().orc_sim_get_regs(self._h, out.ctypes.data)
        return out[: self.net.n_reg]

    def set_reg(self, r, v):
        lib().orc_sim_set_reg(self._h, r, v)

    def mem(self, m, a):
        return lib().orc_sim_get_mem(self._h, m, a)

    def mem_all(self, m):
        return np.array([self.mem(m, a) for a in range(self.net.mem_depth(m))], dtype=np.uint64)

    def set_mem(self, m, a, v):
        lib().orc_sim_set_mem(self._h, m, a, v)

    def hold_input(self, k, v):
        lib().orc_sim_hold_input(self._h, k, v)

    def release_input(self, k):
        lib().orc_sim_release_input(self._h, k)

    def node_value(self, i):
        return lib().orc_sim_node_value(self._h, i)


def op(kind: str, w: int, a: int, b: int = 0, c: int = 0, wb: int = 0, lo: int = 0) -> int:
    return lib().orc_op(KIND[kind], w, a, b, c, wb, lo)


def mix64(z: int) -> int:
    return lib().orc_mix64(z)


def stimulus(seed, inst, t, k, n_in, w) -> int:
    return lib().orc_stimulus(seed, inst, t, k, n_in, w)


def run_digests(path: str, seed: int, inst: int, n: int) -> np.ndarray:
    """Digests of states 0..n of one instance (index t = state after t cycles)."""
    net = Net(path)
    s = Sim(net, seed, inst)
    out = np.zeros(n + 1, dtype=np.uint64)
    out[0] = s.digest()
    out[1:] = s.run(n, digests=True)
    return out
