"""Pins of the fiber extraction and submodular-load-balancing partitioner
(paper Sec. 3.2, Sec. 4.3 and Sec. 5.1), checked on the compiled tables."""
import random

import numpy as np
import pytest

from paper_2403_04714_gb300 import netgen, sim


def cone(nl_text_nodes, root):
    """Brute-force backward crawl (nodes as (op, w, args))."""
    seen, st = set(), [root]
    while st:
        i = st.pop()
        if i in seen:
            continue
        seen.add(i)
        op, _, a = nl_text_nodes[i]
        if op in ("input", "reg", "const"):
            continue
        st.extend([a[0]] if op == "slice" else [a[1]] if op == "memrd" else a)
    return seen


def node_cost(node):
    op, w, _ = node
    if op in ("input", "memrd"):
        return 3
    if op == "mul":
        return 3 if w > 32 else 2
    return 1


def staircase_netlist(n):
    """n independent, equal fibers: r_i' = r_i + 1 with private constants."""
    nl = netgen.Netlist()
    for i in range(n):
        r = nl.add_reg(8, i)
        nl.set_next(r, nl.node("add", 8, nl.node("reg", 8, r), nl.node("const", 8, 1)))
    return nl


@pytest.mark.parametrize("P,worst_fibers", [(4, 3), (5, 3), (6, 2), (12, 1), (1, 12)])
def test_staircase_footnote(P, worst_fibers):
    # Sec. 6 footnote: 12 equal fibers on 4/5/6 processes give a worst
    # process of 3/3/2 fibers (5 processes do not help over 4).
    nl = sim.Netlist(staircase_netlist(12).to_text(), target_processes=P)
    fiber_cost = nl.table("fiber_cost")
    assert len(set(fiber_cost.tolist())) == 1
    i = nl.info()
    assert i["n_processes"] == P
    assert i["process_cost_max"] == worst_fibers * int(fiber_cost[0])


def test_bsp_figure_fibers_and_shared_node():
    # Fig. bsp_sim: three registers, three fibers; a1 and a2 in one fiber,
    # a3 feeding two fibers (duplicated when they sit in different processes).
    text = """rtlnet 1
reg 8 1
reg 8 2
reg 8 3
n reg 8 0
n reg 8 1
n reg 8 2
n add 8 0 1
n xor 8 3 2
n sub 8 1 2
n or 8 5 4
n and 8 5 0
next 0 6
next 1 7
next 2 2
end
"""
    # nodes: 3=a1 (add), 4=a2 (xor a1 r2), 5=a3 (sub r1 r2)
    #        write1 = or(a3, a2), write2 = and(a3, r0), write3 = r2
    nodes = netgen_nodes(text)
    nl3 = sim.Netlist(text, target_processes=3)
    assert nl3.info()["n_fibers"] == 3
    fc = nl3.table("fiber_cost").astype(int)
    f1, f2 = cone(nodes, 6), cone(nodes, 7)
    assert 5 in f1 and 5 in f2                  # a3 shared
    assert {3, 4} <= f1 and 3 not in f2         # a1, a2 in the same fiber
    for f, c in zip((f1, f2, cone(nodes, 2)), fc):
        assert c == sum(node_cost(nodes[i]) for i in f) + 1
    # one process: shared nodes counted once, tau(f1 u f2) = t1 + t2 - tau(f1 n f2)
    nl1 = sim.Netlist(text, target_processes=1)
    union = f1 | f2 | cone(nodes, 2)
    assert nl1.info()["process_cost_max"] == sum(node_cost(nodes[i]) for i in union) + 3
    # two processes: whichever pair merges, its cost counts the shared nodes once
    nl2 = sim.Netlist(text, target_processes=2)
    proc, sink = nl2.table("fiber_proc"), nl2.table("fiber_sink")
    cones = {0: f1, 1: f2, 2: cone(nodes, 2)}
    for p, c in enumerate(nl2.table("proc_cost")):
        u = set().union(*[cones[sink[f]] for f in range(3) if proc[f] == p])
        assert c == sum(node_cost(nodes[i]) for i in u) + sum(1 for f in range(3) if proc[f] == p)


def netgen_nodes(text):
    out = []
    for line in text.splitlines():
        t = line.split()
        if t and t[0] == "n":
            out.append((t[1], int(t[2]), [int(x) for x in t[3:]]))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("target", [1, 7, 30])
def test_process_cost_is_deduplicated_union(seed, target):
    # any partition: tau(process) = sum of costs over the union of its fibers'
    # nodes (brute force) plus one unit per register store
    text = netgen.gen_flat(seed, n_ops=600, n_regs=40, depth=12, n_inputs=4).to_text()
    nodes = netgen_nodes(text)
    nexts = {}
    for line in text.splitlines():
        t = line.split()
        if t and t[0] == "next":
            nexts[int(t[1])] = int(t[2])
    for seed_part in (0, seed):
        nl = sim.Netlist(text, target_processes=target, seed_partition=seed_part)
        proc = nl.table("fiber_proc")
        sink = nl.table("fiber_sink")
        pcost = nl.table("proc_cost")
        assert len(pcost) == min(target, len(sink))
        for p in range(len(pcost)):
            members = [sink[f] for f in range(len(sink)) if proc[f] == p]
            u = set()
            for r in members:
                u |= cone(nodes, nexts[r])
            assert pcost[p] == sum(node_cost(nodes[i]) for i in u) + len(members)


def test_memory_footnote_stage1():
    # Sec. 5.1 footnote: one 256 KiB array and four 64 KiB arrays, each read
    # by three equal fibers, three processes.  Stage 1 (threshold 128 KiB)
    # pre-merges the big array's fibers; no process then needs more than
    # 384 KiB of arrays.
    nl = netgen.Netlist()
    arrays = [nl.add_mem(15, 64)] + [nl.add_mem(13, 64) for _ in range(4)]   # 256 KiB, 4 x 64 KiB
    reg_array = {}
    for m in arrays:
        for k in range(3):
            r = nl.add_reg(64, 0)
            a = nl.node("const", 13, k)
            nl.set_next(r, nl.node("memrd", 64, m, a))
            reg_array[r] = m
    text = nl.to_text()
    kib = {arrays[0]: 256}
    kib.update({m: 64 for m in arrays[1:]})
    for big, expect_premerged in ((128 * 1024, True), (1 << 40, False)):
        cfg = sim.Netlist(text, target_processes=3, big_array_bytes=big)
        proc = cfg.table("fiber_proc")
        sink = cfg.table("fiber_sink")
        a_procs = {proc[f] for f in range(len(sink)) if reg_array[sink[f]] == arrays[0]}
        if expect_premerged:
            assert len(a_procs) == 1
            for p in set(proc.tolist()):
                used = {reg_array[sink[f]] for f in range(len(sink)) if proc[f] == p}
                assert sum(kib[m] for m in used) <= 384


def test_prng_circuit_has_no_exchange():
    # Sec. 4.1: independent xorshift PRNG fibers (3 XORs, 3 shifts each):
    # every fiber reads only its own register, so no value crosses processes.
    nl = netgen.Netlist()
    for i in range(64):
        r = nl.add_reg(64, i + 1)
        x = nl.node("reg", 64, r)
        for sh, kind in ((13, "shl"), (7, "shr"), (17, "shl")):
            x = nl.node("xor", 64, x, nl.node(kind, 64, x, nl.node("const", 7, sh)))
        nl.set_next(r, x)
    for target in (1, 8, 64):
        c = sim.Netlist(nl.to_text(), target_processes=target)
        assert c.info()["cut_words"] == 0
        assert c.info()["n_processes"] == target


def test_mid_workload_partition_quality():
    c = sim.Netlist.from_file(netgen.cached_netlist("mid"), target_processes=1216)
    i = c.info()
    assert i["n_processes"] == 1216
    # conservative merge keeps the worst process at the slowest fiber
    assert i["process_cost_max"] == i["fiber_cost_max"]
    # merging removes most duplicated work
    assert i["process_cost_sum"] < 0.35 * i["fiber_cost_sum"]
