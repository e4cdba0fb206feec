"""The lowered bytecode, run by a Python emulator of the instruction set,
reproduces the oracle cycle by cycle (CPU only): checks the schedule steps,
value-slot reuse, register addressing and memory write records before any
GPU run."""
import random

import pytest

import oracle
from bytecode_emu import Emu
from paper_2403_04714_gb300 import netgen, sim
from test_oracle_bruteforce import random_tiny_circuit


def run_compare(text, mode, cycles, target=0, seed_partition=0, shuffle=False, cluster=None, partitioner="slb",
                chain=0):
    extra = {"partitioner": partitioner, "chain": chain}
    if cluster:
        extra = dict(cluster_size=cluster[0], warps_per_cta=cluster[1], chain=chain)
    base_mode = mode.replace("_compact", "").replace("_cluster", "")
    nl = sim.Netlist(text, mode=base_mode, target_processes=target, seed_partition=seed_partition, **extra)
    emu = Emu(text, nl, mode, seed=42, inst=0)
    ref = oracle.Sim(oracle.Net(text=text), seed=42, inst=0)
    rng = random.Random(1)
    n_proc = len(emu.off)
    for t in range(cycles):
        order = list(range(n_proc))
        if shuffle:
            rng.shuffle(order)
        emu.step(order)
        ref.run(1)
        assert emu.regs == [int(v) for v in ref.regs()], (mode, t)
    emu.finish()
    for m in range(len(emu.mems)):
        assert emu.mems[m] == [ref.mem(m, a) for a in range(len(emu.mems[m]))]


@pytest.mark.parametrize("mode", ["lane_op", "lane_op_compact", "lane_inst"])
def test_tiny_workload(mode):
    text = open(netgen.cached_netlist("tiny")).read()
    run_compare(text, mode, 40, shuffle=True)


@pytest.mark.parametrize("mode", ["lane_op", "lane_op_compact", "lane_inst"])
@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_with_memory(mode, seed):
    text = random_tiny_circuit(seed).to_text()
    for target in (1, 2, 4):
        run_compare(text, mode, 25, target=target, shuffle=True)


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_flat_netlist_with_rams(mode):
    text = netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text()
    for target, sp in ((16, 0), (40, 3)):
        run_compare(text, mode, 30, target=target, seed_partition=sp, shuffle=True)


# Cluster exchange: reads from producers in the same cluster come from the
# CTA's mirror (D_LDM), which the producers write with D_STX; the emulator
# checks every mirror read against the register and every mirror entry for
# exactly one write per cycle.
@pytest.mark.parametrize("C,W,target", [(2, 2, 8), (2, 1, 5), (4, 2, 16), (6, 2, 24), (3, 1, 7)])
def test_cluster_tiny(C, W, target):
    text = open(netgen.cached_netlist("tiny")).read()
    run_compare(text, "lane_op_cluster", 30, target=target, shuffle=True, cluster=(C, W))


@pytest.mark.parametrize("seed", range(4))
def test_cluster_random_circuits_with_memory(seed):
    text = random_tiny_circuit(seed).to_text()
    for C, W, target in ((2, 1, 2), (2, 1, 4), (4, 1, 4), (2, 2, 3)):
        run_compare(text, "lane_op_cluster", 20, target=target, shuffle=True, cluster=(C, W))


def test_cluster_flat_netlist_with_rams():
    text = netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text()
    for C, W, target in ((4, 2, 16), (4, 2, 8), (8, 4, 40)):
        run_compare(text, "lane_op_cluster", 20, target=target, shuffle=True, cluster=(C, W))


# Operator chains (sim_config.chain = 2): a lane runs a dependent pair of
# operators in one step; the emulator reads a chain step as two rows.
@pytest.mark.parametrize("seed", range(6))
def test_chained_random_circuits_with_memory(seed):
    text = random_tiny_circuit(seed).to_text()
    for target in (1, 2, 4):
        run_compare(text, "lane_op_compact", 25, target=target, shuffle=True, chain=2)
    run_compare(text, "lane_op_cluster", 20, target=2, shuffle=True, cluster=(2, 1), chain=2)


def test_chained_tiny_and_flat():
    run_compare(open(netgen.cached_netlist("tiny")).read(), "lane_op_compact", 40, shuffle=True, chain=2)
    run_compare(open(netgen.cached_netlist("tiny")).read(), "lane_op_cluster", 30, target=16, shuffle=True,
                cluster=(4, 2), chain=2)
    text = netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text()
    run_compare(text, "lane_op_compact", 30, target=16, shuffle=True, chain=2)
    run_compare(text, "lane_op_compact", 30, target=8, shuffle=True, chain=2)
