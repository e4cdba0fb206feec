"""GPU parity of the cluster-exchange kernel against the oracle, bit-exact.

Register values pass between processes of one thread-block cluster through
distributed shared memory (D_STX into the consumer CTA's mirror, D_LDM from
it) and across clusters through global memory.  A grid that is one cluster
synchronises with the bounded cluster barrier; a grid of several clusters
with the grid barrier.
"""
import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim
from test_gpu_parity import first_mismatch, oracle_digests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_text():
    return open(netgen.cached_netlist("tiny")).read()


def run_cluster(text, C, W, target, n, seed=42, chunks=(None,)):
    nl = sim.Netlist(text, mode="lane_op", cluster_size=C, warps_per_cta=W, target_processes=target,
                     digest_capacity=n + 1)
    plan = nl.table("cluster_plan")
    b = sim.Batch(nl, 1, seed=seed)
    done = 0
    for k in chunks:
        step = n - done if k is None else k
        b.step(step)
        done += step
    assert done == n
    b.sync()
    return b, plan


@pytest.mark.parametrize("C,W,target", [(8, 1, 8), (4, 2, 8), (2, 2, 8), (16, 4, 64), (6, 2, 24), (3, 1, 7)])
def test_tiny_cluster(tiny_text, C, W, target):
    n = 3000
    b, plan = run_cluster(tiny_text, C, W, target, n, chunks=(1000, 1, 999, None))
    assert plan[4] > 0          # some reads really go through a mirror
    want, ref = oracle_digests(tiny_text, 42, 0, n)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())


def test_one_cluster_with_memories():
    # memories: write records cross CTAs under the cluster barrier alone
    text = netgen.gen_flat(11, n_ops=20_000, n_regs=2_000, depth=30, n_inputs=16,
                           rams=((9, 64), (6, 32))).to_text()
    n = 2000
    b, plan = run_cluster(text, 16, 8, 128, n)
    assert plan[2] == 16        # the whole grid is one cluster
    want, ref = oracle_digests(text, 42, 0, n)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())


def test_mid_clusters():
    path = netgen.cached_netlist("mid")
    text = open(path).read()
    n = 1500
    b, plan = run_cluster(text, 8, 8, 0, n, chunks=(700, None))
    assert plan[2] > 8          # several clusters: grid barrier plus mirrors
    want, ref = oracle_digests(path, 42, 0, n, is_path=True)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())


def test_mid_clusters_of_six():
    # a cluster size that is not a power of two (6 CTAs x 4 warps)
    path = netgen.cached_netlist("mid")
    text = open(path).read()
    n = 1500
    b, plan = run_cluster(text, 6, 4, 0, n, chunks=(700, None))
    assert plan[0] == 6 and plan[2] % 6 == 0 and plan[4] > 0
    want, ref = oracle_digests(path, 42, 0, n, is_path=True)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())


def test_mesh_clusters():
    from test_oracle_closed_forms import fib_pair, mac_closed
    path = netgen.cached_netlist("mesh")
    text = open(path).read()
    n = 150
    b = None
    for C, W in ((2, 8), (4, 4), (2, 4), (2, 2)):
        try:            # the first geometry whose clusters fit the GPU at once
            b, plan = run_cluster(text, C, W, 0, n)
            break
        except sim.SimError as e:
            assert e.name == "SIM_ERR_CAPACITY"
    assert b is not None
    want, ref = oracle_digests(path, 42, 0, n, is_path=True)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())
    names = netgen.parse_names(text)
    b.step(2000 - n)
    b.sync()
    assert b.peek_reg(0, names["chk_counter16"]) == 2000
    assert b.peek_reg(0, names["chk_fib_b"]) == fib_pair(2000)[1]
    assert b.peek_reg(0, names["chk_mac"]) == mac_closed(2000)


def test_cluster_poke_between_steps(tiny_text):
    # a poked register reaches the mirrors: each launch refills them from
    # the global state
    nl = sim.Netlist(tiny_text, mode="lane_op", cluster_size=4, warps_per_cta=2, target_processes=8)
    b = sim.Batch(nl, 1, seed=3)
    ref = oracle.Sim(oracle.Net(text=tiny_text), seed=3, inst=0)
    b.step(50)
    ref.run(50)
    for r in (0, 5, 17):
        b.poke_reg(0, r, 0x5A5A5A5A5A5A5A5A)
        ref.set_reg(r, 0x5A5A5A5A5A5A5A5A)
    b.step(50)
    ref.run(50)
    b.sync()
    assert np.array_equal(b.regs(0), ref.regs())


def test_cluster_barrier_timeout_is_reported(tiny_text):
    # one CTA of a single-cluster grid skips its first arrivals: every CTA's
    # bounded wait expires, the step reports SIM_ERR_TIMEOUT and the context
    # stays usable
    nl = sim.Netlist(tiny_text, mode="lane_op", cluster_size=8, warps_per_cta=1, target_processes=8)
    b = sim.Batch(nl, 1, seed=1)
    b.debug_skip_arrival(20)
    b.step(10)
    with pytest.raises(sim.SimError) as e:
        b.sync()
    assert e.value.name == "SIM_ERR_TIMEOUT"
    b2 = sim.Batch(nl, 1, seed=1)
    b2.step(100)
    b2.sync()
    want, ref = oracle_digests(tiny_text, 1, 0, 100)
    assert np.array_equal(b2.regs(0), ref.regs())


def test_cluster_save_restore(tiny_text):
    # checkpoint taken from a cluster run resumes to the same trace
    nl = sim.Netlist(tiny_text, mode="lane_op", cluster_size=4, warps_per_cta=2, target_processes=8,
                     digest_capacity=301)
    b = sim.Batch(nl, 1, seed=5)
    b.step(100)
    blob = b.save()
    b.step(200)
    b.sync()
    first = b.digests(0, 101, 200)
    b.restore(blob)
    b.step(200)
    b.sync()
    assert np.array_equal(b.digests(0, 101, 200), first)
    want, _ = oracle_digests(tiny_text, 5, 0, 300)
    assert first_mismatch(first, want[101:301]) is None


def test_cluster_grid_barrier_timeout_is_reported(tiny_text):
    # a grid of two clusters: the cluster holding the skipping CTA withholds
    # its arrival at the grid counter; every cluster's bounded wait expires
    nl = sim.Netlist(tiny_text, mode="lane_op", cluster_size=2, warps_per_cta=2, target_processes=8)
    assert nl.table("cluster_plan")[2] == 4
    b = sim.Batch(nl, 1, seed=1)
    b.debug_skip_arrival(20)
    b.step(10)
    with pytest.raises(sim.SimError) as e:
        b.sync()
    assert e.value.name == "SIM_ERR_TIMEOUT"
    b2 = sim.Batch(nl, 1, seed=1)
    b2.step(100)
    b2.sync()
    want, ref = oracle_digests(tiny_text, 1, 0, 100)
    assert np.array_equal(b2.regs(0), ref.regs())
