"""Cluster placement and exchange lowering, checked statically on the CPU:
the placement is a permutation of the processes over the grid's warps, every
CTA's mirror holds exactly the registers its processes read from producers
of its own cluster, every mirror read and write addresses the right entry,
and a 2x2 mesh keeps its blocks inside clusters."""
import numpy as np
import pytest

from paper_2403_04714_gb300 import netgen, sim

NOPROC = 0xFFFFFFFF
D_LDR, D_LDM, D_STX = 1, 21, 22


def plan_of(text, C, W, tp):
    nl = sim.Netlist(text, mode="lane_op", cluster_size=C, warps_per_cta=W, target_processes=tp)
    C_, W_, grid, mirror_words, local, remote = (int(v) for v in nl.table("cluster_plan"))
    assert (C_, W_) == (C, W)
    warp_proc = nl.table("warp_proc")
    n_proc = nl.info()["n_processes"]
    cta = {}
    for w, p in enumerate(warp_proc):
        if p != NOPROC:
            cta[int(p)] = w // W
    # producer process of every register
    producer = {}
    for f, (p, sink) in enumerate(zip(nl.table("fiber_proc"), nl.table("fiber_sink"))):
        if sink >= 0:
            producer[int(sink)] = int(p)
    ins, off, ln = nl.table("s_ins"), nl.table("s_off"), nl.table("s_len")
    progs = {p: ins[int(off[p]) * 32:(int(off[p]) + int(ln[p])) * 32] for p in range(n_proc)}
    return nl, dict(grid=grid, mirror_words=mirror_words, local=local, remote=remote, warp_proc=warp_proc,
                    cta=cta, producer=producer, progs=progs, mir_off=nl.table("mir_off"),
                    mir_reg=nl.table("mir_reg"), n_proc=n_proc)


@pytest.fixture(scope="module")
def tiny_text():
    return open(netgen.cached_netlist("tiny")).read()


@pytest.mark.parametrize("C,W,tp", [(2, 2, 8), (4, 2, 16), (2, 1, 5), (8, 1, 8)])
def test_placement_and_mirrors_are_consistent(tiny_text, C, W, tp):
    _, P = plan_of(tiny_text, C, W, tp)
    wp = P["warp_proc"]
    assert len(wp) == P["grid"] * W and P["grid"] % C == 0
    placed = sorted(int(p) for p in wp if p != NOPROC)
    assert placed == list(range(P["n_proc"]))            # every process exactly once
    mir_off, mir_reg = P["mir_off"], P["mir_reg"]
    assert len(mir_off) == P["grid"] + 1 and mir_off[-1] == len(mir_reg)
    reads = {c: set() for c in range(P["grid"])}
    for p, rows in P["progs"].items():
        c = P["cta"][p]
        for d in rows[rows["op"] != 0]:
            op, imm = int(d["op"]), int(d["imm"])
            idx = int(d["b"]) | (int(d["x"]) << 16)
            same = P["cta"][P["producer"][imm]] // C == c // C if op in (D_LDR, D_LDM, D_STX) else None
            if op == D_LDM:
                assert same, "mirror read of a register produced in another cluster"
                assert mir_reg[mir_off[c] + idx] == imm
                reads[c].add(imm)
            elif op == D_LDR:
                assert not same, "in-cluster read left in global memory"
            elif op == D_STX:
                assert P["producer"][imm] == p
                target = c // C * C + int(d["c"])
                assert mir_reg[mir_off[target] + idx] == imm
    for c in range(P["grid"]):
        entries = [int(r) for r in mir_reg[mir_off[c]:mir_off[c + 1]]]
        assert entries == sorted(set(entries))
        assert set(entries) == reads[c]                     # no unused and no missing entry
        assert len(entries) <= P["mirror_words"]


def test_every_mirror_entry_has_exactly_one_writer(tiny_text):
    _, P = plan_of(tiny_text, 4, 2, 16)
    writes = {}
    for p, rows in P["progs"].items():
        c = P["cta"][p]
        for d in rows[rows["op"] == D_STX]:
            key = (c // 4 * 4 + int(d["c"]), int(d["b"]) | (int(d["x"]) << 16))
            writes[key] = writes.get(key, 0) + 1
    total = int(P["mir_off"][-1])
    assert len(writes) == total and set(writes.values()) == {1}


def test_mesh_blocks_stay_inside_clusters():
    # 2x2 mesh, 4 clusters of 32 processes: the placement keeps each block's
    # logic in one cluster, so only the mesh links cross clusters
    text = open(netgen.cached_netlist("mesh_small")).read()
    _, P = plan_of(text, 4, 8, 128)
    frac = P["local"] / (P["local"] + P["remote"])
    assert frac >= 0.8, frac
