"""Static checks of the shared-memory programs the per-operation interpreter
runs (CPU only): the step words describe the instructions exactly, a step's
flags match its contents (operator steps hold operators only, leaf steps
leaves only and store steps register and mirror stores only, up to 128 of
them, the latter only in programs without operator pairs), no step writes a slot twice, every operand
slot was written by an earlier step, and no step reads a slot that it also
writes."""
import pytest

from paper_2403_04714_gb300 import netgen, sim

D_LDR, D_LDI, D_CONST, D_MEMRD = 1, 2, 3, 4
ALU = set(range(5, 18))
D_MUX, D_SLICE = 15, 16
D_STR, D_WREC, D_COMMIT, D_LDM, D_STX = 18, 19, 20, 21, 22
LEAVES = {D_LDR, D_LDI, D_CONST, D_LDM}
GENERIC, LEAF, CHAIN, STORE = 1 << 31, 1 << 30, 1 << 29, 1 << 28


def _reads(d):
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


def check_chain_step(p, b, e, step, valid, slots):
    """A chain step: R rows (bits 24-27) of n operators; lane i runs the
    operators i, n + i, ... in order (D_NOP after the end of its chain).  An
    operand flagged in imm bits 0/1/2 names the slot of the lane's previous
    operator; every other operand was written by an earlier step or earlier
    in the lane's own chain; no slot is written twice, and no slot written in
    the step is read there by another lane."""
    rows = (e >> 24) & 0xF
    assert e & GENERIC and rows >= 2 and len(step) % rows == 0 and len(step) // rows <= 32, (p, b)
    n = len(step) // rows
    grid = [step[r * n:(r + 1) * n] for r in range(rows)]
    assert all(int(d["op"]) in ALU for d in grid[0]), (p, b)
    dsts = [int(d["dst"]) for row in grid for d in row if int(d["op"]) != 0]
    assert len(dsts) == len(set(dsts)), (p, b, "slot written twice in one step")
    chained = 0
    for lane in range(n):
        own = set()                     # slots this lane wrote earlier in the step
        ended = False
        for r in range(rows):
            d = grid[r][lane]
            if int(d["op"]) == 0:
                ended = True
                continue
            assert int(d["op"]) in ALU and not ended, (p, b, "chains are contiguous operator runs")
            flags = int(d["imm"]) if r else 0
            names = ["a", "b", "c"][:len(_reads(d))]
            assert not flags >> len(names), (p, b)
            for k, name in enumerate(names):
                sl = int(d[name])
                if flags >> k & 1:
                    assert sl == int(grid[r - 1][lane]["dst"]), (p, b, "chained operand names the previous result")
                    chained += 1
                else:
                    assert sl in valid or sl in own, (p, b, "operand slot read before any write")
                    assert sl in own or sl not in dsts, (p, b, "slot written in this step read by another lane")
            own.add(int(d["dst"]))
    assert chained > 0
    for s in dsts:
        assert s < int(slots[p])
        valid[s] = b


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
            if e & CHAIN:
                check_chain_step(p, b, e, step, valid, slots)
                continue
            if not e & GENERIC:
                assert all(o in ALU for o in ops), (p, b, "operator step holds another kind")
            if e & LEAF:
                assert all(o in LEAVES for o in ops) and cnt <= 128, (p, b)
            elif e & STORE:
                assert e & GENERIC and all(o in (D_STR, D_STX) for o in ops) and cnt <= 128, (p, b)
                assert nl.config.chain < 2, (p, b, "store steps only without operator pairs")
            else:
                assert cnt <= 32, (p, b)
            dsts = [writes(d) for d in step if writes(d) is not None]
            assert len(dsts) == len(set(dsts)), (p, b, "slot written twice in one step")
            step_reads = set()
            for d in step:
                for s in _reads(d):
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


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_chained_programs_of_the_workloads(name):
    text = open(netgen.cached_netlist(name)).read()
    check_programs(sim.Netlist(text, mode="lane_op", chain=2))
    check_programs(sim.Netlist(text, mode="lane_op", chain=2, cluster_size=4, warps_per_cta=4))


def test_chained_programs_with_memories():
    text = netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text()
    check_programs(sim.Netlist(text, mode="lane_op", target_processes=16, chain=2))
    with pytest.raises(sim.SimError):
        sim.Netlist(text, mode="lane_op", chain=3)
