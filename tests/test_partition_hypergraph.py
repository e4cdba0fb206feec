"""The alternative partitioning strategy the paper compares with its
bottom-up merge (Sec. 7, "Partitioning Strategies", after RepCut): a k-way
hypergraph partition of the fibers whose hyperedges are the shared nodes, so
that the cut is the duplicated work.  Checked on the CPU: every process's
cost is the deduplicated union of its fibers (brute force), independent
modules are separated without duplicating anything, the quality stays near
the bottom-up merge's on the mid workload, and the lowered program of a
hypergraph partition reproduces the oracle."""
import pytest

from paper_2403_04714_gb300 import netgen, sim
from test_lowering_emulated import run_compare
from test_partition import cone, netgen_nodes, node_cost


@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("target", [1, 7, 30])
def test_process_cost_is_deduplicated_union(seed, target):
    text = netgen.gen_flat(seed, n_ops=600, n_regs=40, depth=12, n_inputs=4).to_text()
    nodes = netgen_nodes(text)
    nexts = {int(t[1]): int(t[2]) for t in (l.split() for l in text.splitlines()) if t and t[0] == "next"}
    nl = sim.Netlist(text, target_processes=target, partitioner="hypergraph")
    proc, sink, pcost = nl.table("fiber_proc"), nl.table("fiber_sink"), nl.table("proc_cost")
    assert sorted(set(proc.tolist())) == list(range(len(pcost)))
    assert len(pcost) == min(target, len(sink))
    for p in range(len(pcost)):
        members = [sink[f] for f in range(len(sink)) if proc[f] == p]
        u = set()
        for r in members:
            u |= cone(nodes, nexts[r])
        assert pcost[p] == sum(node_cost(nodes[i]) for i in u) + len(members)


def modules_netlist(k, m, chain):
    """k disjoint modules; in each, m registers whose next values all use one
    shared chain of `chain` ops (the shared cone of the module)."""
    nl = netgen.Netlist()
    for j in range(k):
        regs = [nl.add_reg(32, j * m + i) for i in range(m)]
        x = nl.node("add", 32, nl.node("reg", 32, regs[0]), nl.node("reg", 32, regs[1]))
        for c in range(chain):
            x = nl.node("xor" if c % 2 else "mul", 32, x, nl.node("const", 32, 2 * c + 3))
        for r in regs:
            nl.set_next(r, nl.node("add", 32, x, nl.node("reg", 32, r)))
    return nl


@pytest.mark.parametrize("k", [2, 4, 6])
def test_independent_modules_split_without_duplication(k):
    m = 6
    nl = modules_netlist(k, m, 12)
    c = sim.Netlist(nl.to_text(), target_processes=k, partitioner="hypergraph")
    proc = c.table("fiber_proc")
    sink = c.table("fiber_sink")
    groups = {}
    for f in range(len(sink)):
        groups.setdefault(int(proc[f]), set()).add(int(sink[f]) // m)
    assert all(len(g) == 1 for g in groups.values()) and len(groups) == k
    # zero cut: the processes' costs add up to the unduplicated cost
    one = sim.Netlist(nl.to_text(), target_processes=1, partitioner="hypergraph")
    assert c.info()["process_cost_sum"] == one.info()["process_cost_sum"]


def test_mid_workload_quality_near_bottom_up():
    text = open(netgen.cached_netlist("mid")).read()
    b = sim.Netlist(text, target_processes=608).info()
    h = sim.Netlist(text, target_processes=608, partitioner="hypergraph").info()
    assert h["n_processes"] == 608
    assert h["process_cost_max"] <= 1.2 * b["process_cost_max"]
    assert h["process_cost_sum"] <= 1.3 * b["process_cost_sum"]
    assert h["process_cost_sum"] < 0.25 * h["fiber_cost_sum"]


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_lowered_hypergraph_partition_matches_oracle(mode):
    text = netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text()
    for target in (5, 16, 40):
        run_compare(text, mode, 25, target=target, shuffle=True, partitioner="hypergraph")


def test_stage1_array_groups_kept():
    # the fibers reading one big array (stage 1, Sec. 5.1 footnote) stay in one
    # process under the hypergraph partition too
    nl = netgen.Netlist()
    big = nl.add_mem(15, 64)                       # 256 KiB
    small = [nl.add_mem(10, 64) for _ in range(3)]
    owner = {}
    for m in [big] + small:
        for k in range(4):
            r = nl.add_reg(64, 0)
            nl.set_next(r, nl.node("xor", 64, nl.node("memrd", 64, m, nl.node("const", 15, k)),
                                   nl.node("reg", 64, r)))
            owner[r] = m
    c = sim.Netlist(nl.to_text(), target_processes=4, partitioner="hypergraph")
    proc, sink = c.table("fiber_proc"), c.table("fiber_sink")
    assert len({int(proc[f]) for f in range(len(sink)) if owner[int(sink[f])] == big}) == 1
