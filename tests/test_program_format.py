"""Static checks of the shared-memory programs the per-operation interpreter
runs (CPU only): the step words describe the instructions exactly, a step's
flags match its contents (operator steps hold operators only, leaf steps
leaves only, up to 128 of them), no step writes a slot twice, every operand
slot was written by an earlier step, and no step reads a slot that it also
writes."""
import pytest

from paper_2403_04714_gb300 import netgen, sim

D_LDR, D_LDI, D_CONST, D_MEMRD = 1, 2, 3, 4
ALU = set(range(5, 18))
D_MUX, D_SLICE = 15, 16
D_STR, D_WREC, D_COMMIT, D_LDM, D_STX = 18, 19, 20, 21, 22
LEAVES = {D_LDR, D_LDI, D_CONST, D_LDM}
GENERIC, LEAF = 1 << 31, 1 << 30


def reads(d):
    op = int(d["op"])
    if op in ALU:
        if op == D_MUX:
            return [int(d["a"]), int(d["b"]), int(d["c"])]
        if op == D_SLICE:
            return [int(d["a"])]
        return [int(d["a"]), int(d["b"])]
    if op in (D_MEMRD, D_STR, D_STX):
        return [int(d["a"])]
    if op == D_WREC:
        return [int(d["a"]), int(d["b"]), int(d["c"])]
    return []


def writes(d):
    return int(d["dst"]) if int(d["op"]) in ALU or int(d["op"]) in LEAVES | {D_MEMRD} else None


def check_programs(nl):
    words, off, size = nl.table("c_words"), nl.table("c_off"), nl.table("c_size")
    slots = nl.table("s_slots")
    for p in range(len(off)):
        prog = words[int(off[p]):int(off[p]) + int(size[p])]
        nb = int(prog[0])
        table = prog[1:1 + nb]
        ins = prog[(nb + 4) // 4 * 4:].copy().view(sim.DINS)
        first_expected = 0
        valid = {}                     # slot -> step that wrote it
        for b, e in enumerate(int(x) for x in table):
            first, cnt = e & 0xFFFF, (e >> 16) & 0xFF
            assert first == first_expected and cnt >= 1
            first_expected += cnt
            step = ins[first:first + cnt]
            ops = [int(d["op"]) for d in step]
            if not e & GENERIC:
                assert all(o in ALU for o in ops), (p, b, "operator step holds another kind")
            if e & LEAF:
                assert all(o in LEAVES for o in ops) and cnt <= 128, (p, b)
            else:
                assert cnt <= 32 or all(o == D_STX for o in ops), (p, b)
            dsts = [writes(d) for d in step if writes(d) is not None]
            assert len(dsts) == len(set(dsts)), (p, b, "slot written twice in one step")
            step_reads = set()
            for d in step:
                for s in reads(d):
                    assert s in valid, (p, b, "operand slot read before any write")
                    step_reads.add(s)
            assert not step_reads & set(dsts), (p, b, "slot read and written in one step")
            for s in dsts:
                assert s < int(slots[p])
                valid[s] = b
        assert first_expected == len(ins), (p, "instructions not covered by the steps")


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_programs_of_the_workloads(name):
    check_programs(sim.Netlist(open(netgen.cached_netlist(name)).read(), mode="lane_op"))


def test_programs_with_memories_and_clusters():
    text = netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text()
    check_programs(sim.Netlist(text, mode="lane_op", target_processes=16))
    check_programs(sim.Netlist(text, mode="lane_op", cluster_size=4, warps_per_cta=2, target_processes=16))
