"""GPU parity of gated and divided clocks: the design with a divide-by-2 and
a divide-by-4 clock and gated registers, lowered to a single clock by the
compiler, against the oracle (which simulates the clock domains phase by
phase), every cycle, bit-exact; in both lane mappings, both lowerings and
the cluster exchange; plus the closed forms of its check registers."""
import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim

pytestmark = pytest.mark.gpu

N = 3000


@pytest.fixture(scope="module")
def clocked():
    text = netgen.gen_clocked().to_text()
    net = oracle.Net(text=text)
    return text, net


def oracle_digests(net, seed, inst, n):
    s = oracle.Sim(net, seed, inst)
    return np.concatenate([np.array([s.digest()], dtype=np.uint64), s.run(n, digests=True)]), s


@pytest.mark.parametrize("cfg", [dict(mode="lane_op"),
                                 dict(mode="lane_op", lowering="generated"),
                                 dict(mode="lane_op", cluster_size=4, warps_per_cta=2, target_processes=16),
                                 dict(mode="lane_op", kernel="per_cycle")],
                         ids=["lane_op", "lane_op_generated", "cluster", "per_cycle"])
def test_single_instance_every_cycle(clocked, cfg):
    text, net = clocked
    nl = sim.Netlist(text, digest_capacity=N + 1, **cfg)
    b = sim.Batch(nl, 1, seed=42)
    b.step(N)
    b.sync()
    want, ref = oracle_digests(net, 42, 0, N)
    assert np.array_equal(b.digests(0, 0, N + 1), want)
    assert np.array_equal(b.regs(0), ref.regs())


@pytest.mark.parametrize("lowering", ["bytecode", "generated"])
def test_lane_inst_instances(clocked, lowering):
    text, net = clocked
    n, n_inst = 1000, 70          # ragged: three warps, the last one partial
    nl = sim.Netlist(text, mode="lane_inst", lowering=lowering, kernel="persistent_graph", digest_capacity=n + 1)
    insts = (0, 1, 33, 69)
    b = sim.Batch(nl, n_inst, seed=7, track=list(insts))
    b.step(n)
    b.sync()
    for i in insts:
        want, ref = oracle_digests(net, 7, i, n)
        assert np.array_equal(b.digests(i, 0, n + 1), want), i
        assert np.array_equal(b.regs(i), ref.regs()), i


def test_check_registers_closed_forms(clocked):
    text, _ = clocked
    names = netgen.parse_names(text)
    nl = sim.Netlist(text, mode="lane_op")
    b = sim.Batch(nl, 1, seed=1)
    T = 100_001
    b.step(T)
    b.sync()
    e = (T + 1) // 2
    assert b.peek_reg(0, names["cnt_div2"]) == e % 65536
    assert b.peek_reg(0, names["clk_div4"]) == e % 2
    assert b.peek_reg(0, names["cnt_div4"]) == ((e + 1) // 2) % 65536
    assert b.peek_reg(0, names["sample_div2"]) == T % 65536          # T odd: the counter after the edge


def test_divided_clock_beside_memories():
    from test_clocks_lowering import clocked_with_memories
    text = clocked_with_memories().to_text()
    n = 2000
    want, ref = oracle_digests(oracle.Net(text=text), 5, 0, n)
    for cfg in (dict(mode="lane_op"), dict(mode="lane_op", cluster_size=2, warps_per_cta=2, target_processes=12)):
        nl = sim.Netlist(text, digest_capacity=n + 1, **cfg)
        b = sim.Batch(nl, 1, seed=5)
        b.step(n)
        b.sync()
        assert np.array_equal(b.digests(0, 0, n + 1), want), cfg
        assert np.array_equal(b.regs(0), ref.regs()), cfg


def test_ripple_counter_sixteen_domains_deep():
    from test_oracle_clocks import ripple_counter
    n_bits, n = 16, 5000
    text = ripple_counter(n_bits).to_text()
    want, _ = oracle_digests(oracle.Net(text=text), 1, 0, n)
    nl = sim.Netlist(text, mode="lane_op", digest_capacity=n + 1)
    b = sim.Batch(nl, 1, seed=1)
    b.step(n)
    b.sync()
    assert np.array_equal(b.digests(0, 0, n + 1), want)
    assert sum(int(b.peek_reg(0, i)) << i for i in range(n_bits)) == (-n) % (1 << n_bits)
