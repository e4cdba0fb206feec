"""Parity at depth: the GPU runs a workload to its full length; at sampled
cycles K its complete state (registers and memories) is loaded into a fresh
oracle set to cycle K, and the oracle's next W cycles are compared with the
GPU's, digest by digest.  The oracle alone could not reach these cycles in a
test's time (the 2M-op mesh at 1M cycles is ~2 x 10^12 operator
evaluations)."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim
from test_gpu_dumps import assert_same_state
from test_gpu_parity import first_mismatch

pytestmark = pytest.mark.gpu


def oracle_at(net, b, inst, seed, k):
    """A fresh oracle holding the GPU's state of instance `inst` after k cycles."""
    ref = oracle.Sim(net, seed, inst)
    for r, v in enumerate(b.regs(inst)):
        ref.set_reg(r, int(v))
    for m in range(net.n_mem):
        for a, v in enumerate(b.mem_all(inst, m)):
            ref.set_mem(m, a, int(v))
    ref.set_cycle(k)
    return ref


def windows(path, cfg, n_inst, insts, seed, ks, w):
    net = oracle.Net(path=path)
    nl = sim.Netlist(open(path, "rb").read(), digest_capacity=w + 1, **cfg)
    b = sim.Batch(nl, n_inst, seed=seed, track=insts)
    done = 0
    for k in ks:
        b.step(k - done)
        b.sync()
        refs = [oracle_at(net, b, i, seed, k) for i in insts]
        gpu_state = b.state_digests()
        for i, ref in zip(insts, refs):
            assert ref.digest() == gpu_state[i], (k, i)
        b.step(w)
        b.sync()
        done = k + w
        with cf.ThreadPoolExecutor(len(insts)) as ex:
            wants = list(ex.map(lambda ref: ref.run(w, digests=True), refs))
        for i, want in zip(insts, wants):
            got = b.digests(i, k + 1, w)
            assert first_mismatch(got, want) is None, (k, i, first_mismatch(got, want))
        # and the full state at the end of the window, word by word
        for i, ref in zip(insts, refs):
            assert_same_state(b, i, ref, (k + w, i))
    return b


def test_mid_full_run_windows():
    # the headline workload: 100k cycles, windows after 50k and at the end
    path = netgen.cached_netlist("mid")
    windows(path, dict(mode="lane_op"), 1, [0], 42, [50_000, 99_000], 1000)


def test_mid_cluster_full_run_windows():
    path = netgen.cached_netlist("mid")
    windows(path, dict(mode="lane_op", cluster_size=2, warps_per_cta=4), 1, [0], 42, [99_000], 1000)


def test_mesh_deep_windows_and_closed_forms():
    # the 2M-op mesh to 1M cycles: windows at 250k and 999k, then the
    # embedded closed-form registers at the last cycle
    from test_oracle_closed_forms import fib_pair, mac_closed
    path = netgen.cached_netlist("mesh")
    b = windows(path, dict(mode="lane_op"), 1, [0], 42, [250_000, 999_000], 400)
    names = netgen.parse_names(open(path).read())
    b.step(1_000_000 - b.cycle)
    b.sync()
    t = 1_000_000
    assert b.peek_reg(0, names["chk_counter16"]) == t % 65536
    assert b.peek_reg(0, names["chk_fib_b"]) == fib_pair(t)[1]
    assert b.peek_reg(0, names["chk_mac"]) == mac_closed(t)


def test_batched_full_run_sampled_windows():
    # 4,096 instances for the full 100k cycles; 16 sampled instances checked
    path = netgen.cached_netlist("mid")
    insts = [0, 1, 4095, 31, 32, 1000, 2047, 2048, 3071, 777, 1234, 2500, 3333, 4000, 64, 96]
    windows(path, dict(mode="lane_inst", lowering="generated", kernel="persistent_graph"), 4096, insts, 42,
            [99_700], 300)
