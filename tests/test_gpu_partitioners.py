"""GPU parity of the hypergraph partition (the alternative to the bottom-up
merge, Sec. 7): the same netlists partitioned by either strategy give the
oracle's digests on every cycle, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim

pytestmark = pytest.mark.gpu


def oracle_digests(text, seed, inst, n):
    s = oracle.Sim(oracle.Net(text=text), seed, inst)
    return np.concatenate([np.array([s.digest()], dtype=np.uint64), s.run(n, digests=True)]), s


@pytest.mark.parametrize("name,n", [("tiny", 5000), ("mid", 2000), ("mesh_small", 2000)])
def test_single_instance_every_cycle(name, n):
    text = open(netgen.cached_netlist(name)).read()
    want, ref = oracle_digests(text, 42, 0, n)
    nl = sim.Netlist(text, mode="lane_op", partitioner="hypergraph", digest_capacity=n + 1)
    b = sim.Batch(nl, 1, seed=42)
    b.step(n)
    b.sync()
    assert np.array_equal(b.digests(0, 0, n + 1), want)
    assert np.array_equal(b.regs(0), ref.regs())


def test_cluster_exchange_and_lane_inst():
    text = open(netgen.cached_netlist("mid")).read()
    n = 1000
    want, _ = oracle_digests(text, 3, 0, n)
    nl = sim.Netlist(text, mode="lane_op", partitioner="hypergraph", cluster_size=2, warps_per_cta=4,
                     digest_capacity=n + 1)
    b = sim.Batch(nl, 1, seed=3)
    b.step(n)
    b.sync()
    assert np.array_equal(b.digests(0, 0, n + 1), want)
    nl = sim.Netlist(text, mode="lane_inst", partitioner="hypergraph", digest_capacity=n + 1)
    b = sim.Batch(nl, 40, seed=3, track=[0, 39])
    b.step(n)
    b.sync()
    assert np.array_equal(b.digests(0, 0, n + 1), want)
    assert np.array_equal(b.digests(39, 0, n + 1), oracle_digests(text, 3, 39, n)[0])
