"""GPU parity of the experiment circuits (the paper's scaling experiments).

The sweeps of the bench time these netlists; here each runs every cycle of a
prefix against the oracle, bit-exact, in the configurations the sweeps use:
  - the synchronisation experiment's independent xorshift fibers (Sec. 4.1),
    on the grid barrier with one fiber per process and in one 16-CTA cluster;
  - the communication experiment's circuit under a random partition, where
    nearly every read crosses processes (Sec. 4.2);
  - the weak-scaling mesh at its largest size, 6 x 6 blocks (Sec. 6), with
    the grid barrier, the cluster exchange and the hypergraph partitioning
    strategy (Sec. 7).
"""
import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim
from test_gpu_dumps import assert_same_state
from test_gpu_parity import first_mismatch

pytestmark = pytest.mark.gpu


def every_cycle(text, cfg, n, seed=1):
    nl = sim.Netlist(text, mode="lane_op", digest_capacity=n + 1, **cfg)
    b = sim.Batch(nl, 1, seed=seed)
    b.step(n)
    b.sync()
    ref = oracle.Sim(oracle.Net(text=text), seed, 0)
    want = np.concatenate([np.array([ref.digest()], dtype=np.uint64), ref.run(n, digests=True)])
    got = b.digests(0, 0, n + 1)
    assert first_mismatch(got, want) is None, (cfg, first_mismatch(got, want))
    assert_same_state(b, 0, ref, cfg)
    return nl, b


@pytest.mark.parametrize("cfg", [dict(target_processes=1216),
                                 dict(cluster_size=16, warps_per_cta=8, target_processes=128)],
                         ids=["grid_barrier_1216", "one_cluster_16"])
def test_prng_fibers(cfg):
    every_cycle(netgen.gen_prng(1216).to_text(), cfg, 2000)


def test_prng_many_fibers_per_process():
    # 32 fibers per process on 608 processes (a point of the sweep)
    every_cycle(netgen.gen_prng(608 * 32).to_text(), dict(target_processes=608), 300)


@pytest.mark.parametrize("reads,procs", [(1, 152), (4, 608), (16, 152)])
def test_exchange_random_partition(reads, procs):
    text = netgen.gen_exchange(procs * 32, reads).to_text()
    nl, _ = every_cycle(text, dict(target_processes=procs, seed_partition=1), 500)
    assert nl.info()["cut_words"] > 0


@pytest.fixture(scope="module")
def mesh6_text():
    return netgen.gen_mesh(1106, mesh=6, ops_per_block=30_000, regs_per_block=2_000, depth=40,
                           inputs_per_block=8).to_text()


@pytest.mark.parametrize("cfg", [dict(), dict(cluster_size=2, warps_per_cta=8), dict(partitioner="hypergraph")],
                         ids=["grid_barrier", "cluster2x8", "hypergraph"])
def test_weak_scaling_mesh_6x6(mesh6_text, cfg):
    every_cycle(mesh6_text, cfg, 60, seed=42)
