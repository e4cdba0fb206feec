"""Gated and divided clocks on the CUDA path's side (CPU only): the compiler
lowers them to a single clock, and the lowered bytecode, run by the Python
emulator of the instruction set, reproduces the oracle (which simulates the
clock domains phase by phase) cycle by cycle.  The loader rejects what the
oracle rejects."""
import pytest

from paper_2403_04714_gb300 import netgen, sim
from test_lowering_emulated import run_compare
from test_oracle_clocks import random_clocked_circuit


@pytest.mark.parametrize("mode", ["lane_op", "lane_op_compact", "lane_inst"])
def test_clocked_design(mode):
    text = netgen.gen_clocked().to_text()
    run_compare(text, mode, 40, shuffle=True)


def test_clocked_design_with_cluster_exchange():
    text = netgen.gen_clocked().to_text()
    run_compare(text, "lane_op_cluster", 30, target=16, cluster=(4, 2))


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
@pytest.mark.parametrize("seed", range(8))
def test_random_clocked_circuits(mode, seed):
    text = random_clocked_circuit(seed).to_text()
    for target in (1, 2, 4):
        run_compare(text, mode, 25, target=target, shuffle=True)


def test_registers_and_signals_unchanged_by_the_lowering():
    nl = netgen.gen_clocked()
    info = sim.Netlist(nl.to_text(), mode="lane_op").info()
    assert info["n_regs"] == len(nl.regs) and info["n_inputs"] == len(nl.inputs)


def test_loader_rejections():
    base = ["rtlnet 1", "reg 1 0", "reg 1 0", "reg 8 0", "n reg 1 0", "n reg 1 1", "n reg 8 2",
            "next 0 0", "next 1 1", "next 2 2"]
    bad = [base + ["clock 0 1", "clock 1 0", "end"],
           base + ["clock 0 2", "end"],
           base + ["clock 2 0", "clock 2 1", "end"],
           base + ["gate 2 9", "end"],
           ["rtlnet 1", "reg 1 0", "reg 8 0", "mem 2 8", "n reg 1 0", "n reg 8 1", "n memrd 8 0 1",
            "next 0 0", "next 1 2", "clock 1 0", "end"]]
    for lines in bad:
        with pytest.raises(sim.SimError):
            sim.Netlist("\n".join(lines), mode="lane_op")


def clocked_with_memories(seed=21):
    """A flat design with two RAMs (write ports on the top clock), plus a
    divide-by-2 clock for the registers whose cones read no memory."""
    nl = netgen.gen_flat(seed, n_ops=2500, n_regs=120, depth=14, n_inputs=6, rams=((4, 64), (3, 16)))
    div = nl.add_reg(1, 0, "clk_div2")
    nl.set_next(div, nl.node("xor", 1, nl.node("reg", 1, div), nl.node("const", 1, 1)))

    def reads_memory(root):
        seen, st = set(), [root]
        while st:
            i = st.pop()
            if i in seen:
                continue
            seen.add(i)
            op, _, a = nl.nodes[i]
            if op == "memrd":
                return True
            if op in ("input", "reg", "const"):
                continue
            st.extend([a[0]] if op == "slice" else a)
        return False

    ones = [i for i, (op, w, _) in enumerate(nl.nodes) if w == 1 and not reads_memory(i)]
    for r in range(0, 120, 3):
        if not reads_memory(nl.regs[r][2]):
            nl.clocks[r] = div
            if r % 2:
                nl.gates[r] = ones[r % len(ones)]
    return nl


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_divided_clock_beside_memories(mode):
    nl = clocked_with_memories()
    assert len(nl.clocks) > 10
    run_compare(nl.to_text(), mode, 30, target=12, shuffle=True)


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_deep_chain_of_divided_clocks(mode):
    from test_oracle_clocks import ripple_counter
    run_compare(ripple_counter(16).to_text(), mode, 70, target=4, shuffle=True)


@pytest.mark.parametrize("seed", range(30, 36))
def test_random_designs_every_lowering_and_partitioner(seed):
    # clocks, gates and memories together, both partitioning strategies,
    # both lane mappings and the cluster exchange
    text = clocked_with_memories(seed).to_text()
    part = "hypergraph" if seed % 2 else "slb"
    run_compare(text, "lane_op", 12, target=7, shuffle=True, partitioner=part)
    run_compare(text, "lane_inst", 12, target=5, partitioner=part)
    run_compare(text, "lane_op_cluster", 12, target=12, cluster=(3, 2), partitioner=part)


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_gated_clock_register(mode):
    from test_oracle_clocks import gated_divider
    run_compare(gated_divider()[0].to_text(), mode, 60, target=2, shuffle=True)
