"""Full state dumps against the oracle, element by element.

The per-cycle parity tests compare a 64-bit digest of the whole state; here
every register and every memory word of the GPU state is compared with the
oracle's at cycles 0, 1, 2, 10, 100 and the last cycle of the run (the
current values of Sec. 3.2 after that many cycles), for each kernel and lane
mapping, so that a mistake that a digest collision could hide still fails.
"""
import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim
from test_oracle_digest import ROM_RAM

pytestmark = pytest.mark.gpu

DUMPS = (0, 1, 2, 10, 100)


def assert_same_state(b, inst, ref, tag):
    got = b.regs(inst)
    want = ref.regs()
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, (tag, "register", int(bad[0]), int(got[bad[0]]), int(want[bad[0]]))
    for m in range(ref.net.n_mem):
        g, w = b.mem_all(inst, m), ref.mem_all(m)
        bad = np.nonzero(g != w)[0]
        assert len(bad) == 0, (tag, "memory", m, int(bad[0]))


def run_dumps(text, cfg, n_inst, insts, seed, last):
    net = oracle.Net(text=text)
    nl = sim.Netlist(text, **cfg)
    b = sim.Batch(nl, n_inst, seed=seed)
    refs = {i: oracle.Sim(net, seed, i) for i in insts}
    done = 0
    for c in DUMPS + (last,):
        if c > done:
            b.step(c - done)
            for r in refs.values():
                r.run(c - done)
            done = c
        b.sync()
        for i, r in refs.items():
            assert_same_state(b, i, r, (cfg, i, c))


@pytest.fixture(scope="module")
def tiny_text():
    return open(netgen.cached_netlist("tiny")).read()


@pytest.fixture(scope="module")
def mid_text():
    return open(netgen.cached_netlist("mid")).read()


TINY_CASES = [
    (dict(mode="lane_op"), 1, [0]),
    (dict(mode="lane_op", chain=2), 1, [0]),
    (dict(mode="lane_op", chain=2, cluster_size=4, warps_per_cta=2, target_processes=16), 1, [0]),
    (dict(mode="lane_op", lowering="generated"), 1, [0]),
    (dict(mode="lane_op", kernel="per_cycle"), 1, [0]),
    (dict(mode="lane_op", cluster_size=8, warps_per_cta=2, target_processes=16), 1, [0]),
    (dict(mode="lane_op", cluster_size=2, warps_per_cta=2, target_processes=8), 1, [0]),
    (dict(mode="lane_inst"), 70, [0, 45, 69]),
    (dict(mode="lane_inst", lowering="generated", kernel="persistent_graph"), 70, [0, 33, 69]),
]


@pytest.mark.parametrize("cfg,n_inst,insts", TINY_CASES, ids=[str(i) for i in range(len(TINY_CASES))])
def test_tiny_dumps(tiny_text, cfg, n_inst, insts):
    run_dumps(tiny_text, cfg, n_inst, insts, 42, 1000)


@pytest.mark.parametrize("cfg,n_inst,insts", [
    (dict(mode="lane_op"), 1, [0]),
    (dict(mode="lane_op", lowering="generated"), 1, [0]),
    (dict(mode="lane_op", cluster_size=2, warps_per_cta=1, target_processes=2), 1, [0]),
    (dict(mode="lane_inst"), 33, [0, 32]),
    (dict(mode="lane_inst", lowering="generated"), 33, [0, 32]),
    (dict(mode="lane_op", chain=2), 1, [0]),
], ids=["lane_op", "lane_op_gen", "cluster", "lane_inst", "lane_inst_gen", "lane_op_pairs"])
def test_rom_ram_dumps(cfg, n_inst, insts):
    run_dumps(ROM_RAM, cfg, n_inst, insts, 7, 300)


@pytest.mark.parametrize("cfg,n_inst,insts", [
    (dict(mode="lane_op"), 1, [0]),
    (dict(mode="lane_op", chain=2), 1, [0]),
    (dict(mode="lane_op", cluster_size=4, warps_per_cta=4), 1, [0]),
    (dict(mode="lane_op", cluster_size=6, warps_per_cta=4, chain=2), 1, [0]),
    (dict(mode="lane_inst", lowering="generated", kernel="persistent_graph"), 64, [0, 63]),
], ids=["grid_barrier", "grid_barrier_pairs", "cluster4x4", "cluster6x4_pairs", "batched_generated"])
def test_mid_dumps(mid_text, cfg, n_inst, insts):
    run_dumps(mid_text, cfg, n_inst, insts, 42, 1000)
