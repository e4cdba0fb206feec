"""Python binding of the simulator's C ABI (include/sim.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library libgb300sim.so.  If the library is missing this module raises; there
is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgb300sim.so")

SIM_OK = 0
ERRORS = {
    -1: "SIM_ERR_PARSE", -2: "SIM_ERR_COMB_LOOP", -3: "SIM_ERR_WIDTH", -4: "SIM_ERR_CAPACITY",
    -5: "SIM_ERR_OOM", -6: "SIM_ERR_TIMEOUT", -7: "SIM_ERR_CUDA", -8: "SIM_ERR_BADARG",
    -9: "SIM_ERR_ADMISSION", -10: "SIM_ERR_STATE",
}
SIM_SIG_INPUT, SIM_SIG_REG = 0, 1
SIM_MODE_AUTO, SIM_MODE_LANE_OP, SIM_MODE_LANE_INST = 0, 1, 2
SIM_KERNEL_PERSISTENT, SIM_KERNEL_PER_CYCLE, SIM_KERNEL_PER_CYCLE_GRAPH = 0, 1, 2
MODES = {"auto": 0, "lane_op": 1, "lane_inst": 2}
LOWERINGS = {"bytecode": 0, "generated": 1}
ORDERS = {"auto": 0, "group_major": 1, "process_major": 2, "cta_major": 3}
PARTITIONERS = {"slb": 0, "hypergraph": 1}
# generated-CUDA modules are cached here across processes
os.environ.setdefault("RTLSIM_GENCACHE", os.path.join(os.path.dirname(PKG), "_build", "gencache"))
KERNELS = {"persistent": 0, "per_cycle": 1, "graph": 2, "persistent_graph": 3}


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class sim_config(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("mode", C.c_int32), ("kernel", C.c_int32),
        ("target_processes", C.c_uint32), ("warps_per_cta", C.c_uint32), ("max_slots", C.c_uint32),
        ("digest_capacity", C.c_uint32), ("timeout_ms", C.c_uint32), ("big_array_bytes", C.c_uint64),
        ("disable_stage3", C.c_uint32), ("seed_partition", C.c_uint32), ("lowering", C.c_uint32),
        ("task_order", C.c_uint32), ("phase_samples", C.c_uint32), ("wave_groups", C.c_uint32),
        ("cluster_size", C.c_uint32), ("partitioner", C.c_uint32), ("chain", C.c_uint32),
        ("reserved", C.c_uint32 * 1),
    ]


class sim_netlist_info(C.Structure):
    _fields_ = [
        ("n_inputs", C.c_uint32), ("n_regs", C.c_uint32), ("n_mems", C.c_uint32), ("n_wports", C.c_uint32),
        ("n_nodes", C.c_uint64), ("n_ops", C.c_uint64), ("n_fibers", C.c_uint32), ("n_processes", C.c_uint32),
        ("fiber_cost_sum", C.c_uint64), ("process_cost_sum", C.c_uint64), ("process_cost_max", C.c_uint64),
        ("fiber_cost_max", C.c_uint64), ("max_bundles", C.c_uint32), ("max_slots", C.c_uint32),
        ("instr_count", C.c_uint64), ("cut_words", C.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()

EXPORTS = {
    "sim_config_default": (None, [C.c_void_p]),
    "sim_load_netlist": (C.c_int, [C.c_char_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "sim_netlist_get_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sim_netlist_destroy": (None, [C.c_void_p]),
    "sim_create_instances": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64, C.c_void_p, C.c_void_p]),
    "sim_batch_destroy": (None, [C.c_void_p]),
    "sim_poke": (C.c_int, [C.c_void_p, C.c_uint32, C.c_int32, C.c_uint32, C.c_uint64]),
    "sim_unpoke": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32]),
    "sim_poke_mem": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64]),
    "sim_step": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sim_sync": (C.c_int, [C.c_void_p]),
    "sim_peek": (C.c_int, [C.c_void_p, C.c_uint32, C.c_int32, C.c_uint32, C.c_void_p]),
    "sim_peek_mem": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_void_p]),
    "sim_peek_regs": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p]),
    "sim_peek_mems": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p]),
    "sim_cycle": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sim_state_digests": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sim_track_digests": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32]),
    "sim_digests": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_void_p]),
    "sim_step_host": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "sim_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sim_free_blob": (None, [C.c_void_p]),
    "sim_launch_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_debug_skip_arrival": (C.c_int, [C.c_void_p, C.c_uint32]),
    "sim_last_error": (C.c_char_p, []),
    "sim_netlist_table": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "sim_state_digests_noalloc": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sim_measure_int_peak": (C.c_int, [C.c_uint32, C.c_void_p]),
    "sim_netlist_compile_generated": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "sim_phase_times": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p]),
    "sim_server_config_default": (None, [C.c_void_p]),
    "sim_server_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sim_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p]),
    "sim_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint32]),
    "sim_job_digests": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p]),
    "sim_server_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_server_destroy": (None, [C.c_void_p]),
    "sim_server_footprint": (C.c_size_t, [C.c_void_p, C.c_uint32]),
}

JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class sim_server_config(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("pool_slots", C.c_uint32), ("hbm_cap_bytes", C.c_uint64),
                ("chunk_cycles", C.c_uint32), ("persistent", C.c_uint32), ("reserved", C.c_uint32 * 6)]


class sim_job(C.Structure):
    _fields_ = [("netlist", C.c_void_p), ("n_inst", C.c_uint32), ("seed", C.c_uint64), ("n_cycles", C.c_uint64)]


class sim_job_status(C.Structure):
    _fields_ = [("state", C.c_int32), ("n_inst", C.c_uint32), ("cycles_done", C.c_uint64),
                ("t_arrive", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]

TABLES = {"s_ins": (0, None), "s_off": (1, np.uint32), "s_len": (2, np.uint32), "b_ins": (3, None),
          "b_off": (4, np.uint32), "b_len": (5, np.uint32), "fiber_proc": (6, np.int32),
          "fiber_sink": (7, np.int32), "fiber_cost": (8, np.uint64), "proc_cost": (9, np.uint64),
          "reg_cls": (10, np.uint8), "reg_idx": (11, np.uint32), "s_slots": (12, np.uint32),
          "b_slots": (13, np.uint32), "c_words": (14, np.uint32), "c_off": (15, np.uint32),
          "c_size": (16, np.uint32), "warp_proc": (17, np.uint32), "mir_off": (18, np.uint32),
          "mir_reg": (19, np.uint32), "cluster_plan": (20, np.uint64), "mem_lg": (21, np.uint8)}
# one 16-byte instruction of the device bytecode
DINS = np.dtype([("op", np.uint8), ("w", np.uint8), ("dst", np.uint16), ("a", np.uint16), ("b", np.uint16),
                 ("c", np.uint16), ("x", np.uint16), ("imm", np.uint32)])


def lib(build_if_missing: bool = False):
    """Load libgb300sim.so (raises if it is missing and not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                if not build_if_missing:
                    raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                       "`python -m paper_2403_04714_gb300.build`")
                from .build import build
                build()
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in EXPORTS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc):
    if rc != SIM_OK:
        raise SimError(rc, lib().sim_last_error().decode(errors="replace"))


def default_config(**kw) -> sim_config:
    cfg = sim_config()
    lib().sim_config_default(C.byref(cfg))
    for k, v in kw.items():
        if k == "mode" and isinstance(v, str):
            v = MODES[v]
        if k == "kernel" and isinstance(v, str):
            v = KERNELS[v]
        if k == "lowering" and isinstance(v, str):
            v = LOWERINGS[v]
        if k == "task_order" and isinstance(v, str):
            v = ORDERS[v]
        if k == "partitioner" and isinstance(v, str):
            v = PARTITIONERS[v]
        setattr(cfg, k, v)
    return cfg


def measure_int_peak(iters: int = 4096) -> float:
    """sim_measure_int_peak: integer lane-operations per second of the current GPU."""
    v = C.c_double()
    _check(lib().sim_measure_int_peak(iters, C.byref(v)))
    return v.value


class Netlist:
    """sim_load_netlist: parse, check, partition (fibers -> SLB processes) and lower."""

    def __init__(self, text: str | bytes, **cfg):
        if isinstance(text, str):
            text = text.encode()
        self.config = default_config(**cfg)
        h = C.c_void_p()
        _check(lib().sim_load_netlist(text, len(text), C.byref(self.config), C.byref(h)))
        self._h = h

    @classmethod
    def from_file(cls, path, **cfg):
        with open(path, "rb") as f:
            return cls(f.read(), **cfg)

    def compile_generated(self, mode) -> dict:
        """sim_netlist_compile_generated: build the generated-CUDA lowering (no GPU needed)."""
        sec, cached = C.c_double(), C.c_int32()
        m = MODES[mode] if isinstance(mode, str) else mode
        _check(lib().sim_netlist_compile_generated(self._h, m, C.byref(sec), C.byref(cached)))
        return {"seconds": sec.value, "cached": bool(cached.value)}

    def table(self, name: str) -> np.ndarray:
        which, dt = TABLES[name]
        n = C.c_size_t(0)
        _check(lib().sim_netlist_table(self._h, which, None, C.byref(n)))
        raw = np.zeros(n.value, dtype=np.uint8)
        _check(lib().sim_netlist_table(self._h, which, raw.ctypes.data, C.byref(n)))
        return raw.view(DINS if dt is None else dt)

    def info(self) -> dict:
        out = sim_netlist_info()
        _check(lib().sim_netlist_get_info(self._h, C.byref(out)))
        return out.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().sim_netlist_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Batch:
    """sim_create_instances: n_inst independently seeded instances on the device."""

    def __init__(self, netlist: Netlist, n_inst: int, seed: int = 42, stream=None, track=None):
        self.netlist = netlist
        self.n_inst = n_inst
        self.info = netlist.info()
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", 0))
        _check(lib().sim_create_instances(netlist._h, n_inst, seed, C.c_void_p(s) if s else None, C.byref(h)))
        self._h = h
        if track is not None:
            self.track_digests(track)

    def close(self):
        if getattr(self, "_h", None):
            lib().sim_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # -- stepping -------------------------------------------------------------
    def step(self, n_cycles: int):
        _check(lib().sim_step(self._h, n_cycles))

    def sync(self):
        _check(lib().sim_sync(self._h))

    @property
    def cycle(self) -> int:
        v = C.c_uint64()
        _check(lib().sim_cycle(self._h, C.byref(v)))
        return v.value

    def step_host(self, n_cycles: int, held_inputs: np.ndarray | None, out: np.ndarray):
        """sim_step_host: held inputs (n_inst x n_inputs) in, per-instance digests out."""
        hp = None
        if held_inputs is not None:
            assert held_inputs.dtype == np.uint64 and held_inputs.flags.c_contiguous
            hp = held_inputs.ctypes.data
        assert out.dtype == np.uint64 and out.size >= self.n_inst
        _check(lib().sim_step_host(self._h, n_cycles, hp, out.ctypes.data))
        return out

    # -- signals -------------------------------------------------------------
    def poke(self, inst: int, kind: int, index: int, value: int):
        _check(lib().sim_poke(self._h, inst, kind, index, value & (2 ** 64 - 1)))

    def poke_reg(self, inst, r, value):
        self.poke(inst, SIM_SIG_REG, r, value)

    def hold_input(self, inst, k, value):
        self.poke(inst, SIM_SIG_INPUT, k, value)

    def unpoke(self, inst, k):
        _check(lib().sim_unpoke(self._h, inst, k))

    def poke_mem(self, inst, m, addr, value):
        _check(lib().sim_poke_mem(self._h, inst, m, addr, value & (2 ** 64 - 1)))

    def peek(self, inst: int, kind: int, index: int) -> int:
        v = C.c_uint64()
        _check(lib().sim_peek(self._h, inst, kind, index, C.byref(v)))
        return v.value

    def peek_reg(self, inst, r):
        return self.peek(inst, SIM_SIG_REG, r)

    def peek_mem(self, inst, m, addr) -> int:
        v = C.c_uint64()
        _check(lib().sim_peek_mem(self._h, inst, m, addr, C.byref(v)))
        return v.value

    def mem_all(self, inst: int, m: int) -> np.ndarray:
        """sim_peek_mems: every word of memory m of one instance, in address order."""
        depth = 1 << int(self.netlist.table("mem_lg")[m])
        out = np.zeros(depth, dtype=np.uint64)
        _check(lib().sim_peek_mems(self._h, inst, m, out.ctypes.data))
        return out

    def regs(self, inst: int) -> np.ndarray:
        out = np.zeros(max(1, self.info["n_regs"]), dtype=np.uint64)
        _check(lib().sim_peek_regs(self._h, inst, out.ctypes.data))
        return out[: self.info["n_regs"]]

    # -- digests -------------------------------------------------------------
    def state_digests(self) -> np.ndarray:
        out = np.zeros(self.n_inst, dtype=np.uint64)
        _check(lib().sim_state_digests(self._h, out.ctypes.data))
        return out

    def state_digests_noalloc(self, out_ptr: int):
        """sim_state_digests_noalloc: digests into caller memory (device or host
        pointer, n_inst 64-bit words) with no allocation inside the library."""
        _check(lib().sim_state_digests_noalloc(self._h, C.c_void_p(out_ptr)))

    def track_digests(self, insts):
        arr = (C.c_uint32 * len(insts))(*insts)
        _check(lib().sim_track_digests(self._h, arr, len(insts)))

    def digests(self, inst: int, first: int, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1), dtype=np.uint64)
        _check(lib().sim_digests(self._h, inst, first, n, out.ctypes.data))
        return out[:n]

    # -- checkpoints ---------------------------------------------------------
    def save(self) -> bytes:
        p = C.c_void_p()
        n = C.c_size_t()
        _check(lib().sim_save(self._h, C.byref(p), C.byref(n)))
        try:
            return C.string_at(p, n.value)
        finally:
            lib().sim_free_blob(p)

    def restore(self, blob: bytes):
        _check(lib().sim_restore(self._h, blob, len(blob)))

    def phase_times(self, n: int) -> np.ndarray:
        """sim_phase_times: per cycle (compute ns, sync ns, cycle ns) of the last persistent launch."""
        out = np.zeros((max(n, 1), 3), dtype=np.float64)
        _check(lib().sim_phase_times(self._h, n, out.ctypes.data))
        return out[:n]

    def launch_info(self) -> dict:
        a, b, c, d = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint64()
        _check(lib().sim_launch_info(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return {"ctas": a.value, "warps_per_cta": b.value, "tasks_per_cycle": c.value, "kernels_launched": d.value}

    def debug_skip_arrival(self, timeout_ms: int):
        _check(lib().sim_debug_skip_arrival(self._h, timeout_ms))


class Server:
    """sim_server_create: continuous-batching job server (one pool per netlist)."""

    def __init__(self, **cfg):
        c = sim_server_config()
        lib().sim_server_config_default(C.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        h = C.c_void_p()
        _check(lib().sim_server_create(C.byref(c), C.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, netlist: Netlist, n_inst: int, seed: int, n_cycles: int) -> int:
        j = sim_job(netlist._h.value, n_inst, seed, n_cycles)
        jid = C.c_uint64()
        _check(lib().sim_submit(self._h, C.byref(j), C.byref(jid)))
        self._keep[jid.value] = netlist          # the netlist must outlive its job
        return jid.value

    def poll(self, job_id: int) -> dict:
        st = sim_job_status()
        _check(lib().sim_poll(self._h, job_id, C.byref(st)))
        return {"state": JOB_STATES[st.state], "n_inst": st.n_inst, "cycles_done": st.cycles_done,
                "t_arrive": st.t_arrive, "t_start": st.t_start, "t_done": st.t_done}

    def wait(self, job_id: int, timeout_ms: int = 600_000):
        _check(lib().sim_server_wait(self._h, job_id, timeout_ms))

    def digests(self, job_id: int, n_inst: int) -> np.ndarray:
        out = np.zeros(n_inst, dtype=np.uint64)
        _check(lib().sim_job_digests(self._h, job_id, out.ctypes.data))
        return out

    @staticmethod
    def footprint(netlist: Netlist, slots: int) -> int:
        return lib().sim_server_footprint(netlist._h, slots)

    def stats(self) -> dict:
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().sim_server_stats(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return {"instance_cycles": a.value, "kernels": b.value, "bytes_in_use": c.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().sim_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
