"""Test helper: a Python emulator of the simulator's device bytecode.

Written from the instruction-set definition (the DIns layout and opcode
list of the compiler header), not from the CUDA kernels, so that the lowered
program (schedule steps, slot allocation, register addressing, write records)
can be checked against the oracle on the CPU.  Registers are addressed by
their netlist index (instruction field imm).
"""
import oracle

D_NOP, D_LDR, D_LDI, D_CONST, D_MEMRD = 0, 1, 2, 3, 4
D_ADD, D_SUB, D_MUL, D_AND, D_OR, D_XOR, D_SHL, D_SHR, D_EQ, D_LT = range(5, 15)
D_MUX, D_SLICE, D_CONCAT, D_STR, D_WREC, D_COMMIT, D_LDM, D_STX = range(15, 23)
M64 = (1 << 64) - 1


def mask(w):
    return (1 << w) - 1


class Emu:
    def __init__(self, net_text, netlist, mode, seed=42, inst=0):
        from pyeval import PyNet
        self.py = PyNet(net_text)
        self.mode = mode
        self.seed, self.inst = seed, inst
        self.cluster = None
        if mode == "lane_op_cluster":
            # cluster exchange: per-CTA mirrors written by D_STX, read by D_LDM
            C, W, grid = (int(v) for v in netlist.table("cluster_plan")[:3])
            warp_proc = netlist.table("warp_proc")
            mir_off, mir_reg = netlist.table("mir_off"), netlist.table("mir_reg")
            cta = {int(pr): w // W for w, pr in enumerate(warp_proc) if pr != 0xFFFFFFFF}
            self.cluster = dict(C=C, cta=cta, mir_off=[int(v) for v in mir_off], mir_reg=[int(v) for v in mir_reg])
            mode = "lane_op_compact"
        if mode == "lane_op_compact":
            # rebuild 32-wide rows from the shared-memory program format
            words = netlist.table("c_words")
            c_off, c_size = netlist.table("c_off"), netlist.table("c_size")
            rows = []
            self.off = []
            import numpy as np
            from paper_2403_04714_gb300.sim import DINS
            lens = []
            for p in range(len(c_off)):
                # word 0: step count; then the step words; instructions from
                # the next multiple of 4 words.  A wide leaf or store step (up
                # to 128 independent instructions) becomes several 32-lane rows.
                prog = words[int(c_off[p]):int(c_off[p]) + int(c_size[p])]
                nb = int(prog[0])
                table = prog[1:1 + nb]
                ins = prog[(nb + 4) // 4 * 4:].copy().view(DINS)
                self.off.append(len(rows) // 32)
                n_rows = 0
                for e in table:
                    first, cnt = int(e) & 0xffff, (int(e) >> 16) & 0xff
                    chain = (int(e) >> 29) & 1
                    n_rows_step = (int(e) >> 24) & 0xF if chain else 1
                    assert cnt <= 32 or (int(e) >> 30) & 1 or (int(e) >> 28) & 1 or \
                        (chain and cnt <= 32 * n_rows_step), "only leaf, store and chain steps may exceed 32 lanes"
                    # a chain step holds rows of the lanes' operators, each
                    # lane's next operator in the next row (reading the
                    # previous result's slot): as many sequential rows
                    width = cnt // n_rows_step if chain else 32
                    for k in range(0, max(cnt, 1), width):
                        row = np.zeros(32, dtype=DINS)
                        n = min(width, cnt - k)
                        row[:n] = ins[first + k:first + k + n]
                        rows.extend(row)
                        n_rows += 1
                lens.append(n_rows)
            self.ins = np.array(rows, dtype=DINS)
            self.len = lens
            self.nslots = netlist.table("s_slots")
            mode = "lane_op"
        elif mode == "lane_op":
            self.ins = netlist.table("s_ins")
            self.off = netlist.table("s_off")
            self.len = netlist.table("s_len")
            self.nslots = netlist.table("s_slots")
        else:
            self.ins = netlist.table("b_ins")
            self.off = netlist.table("b_off")
            self.len = netlist.table("b_len")
            self.nslots = netlist.table("b_slots")
        self.mode = mode
        self.regs, self.mems = self.py.initial_state()
        if self.cluster:
            cl = self.cluster
            cl["cur"] = [[self.regs[r] for r in cl["mir_reg"][cl["mir_off"][c]:cl["mir_off"][c + 1]]]
                         for c in range(len(cl["mir_off"]) - 1)]
        self.cycle = 0
        self.pending = {}           # port -> (en, addr, data) of the previous cycle
        self.n_in = len(self.py.inputs)

    def _read_mem(self, m, addr):
        v = self.mems[m][addr]
        for port in sorted(self.pending):
            pm = self.py.wports[port][0]
            en, a, d = self.pending[port]
            if pm == m and en and a == addr:
                v = d
        return v

    def _commit(self, m):
        for port in sorted(self.pending):
            en, a, d = self.pending[port]
            if self.py.wports[port][0] == m and en:
                self.mems[m][a] = d

    def _exec(self, d, slots, nxt, recs):
        op, w = int(d["op"]), int(d["w"])
        S = lambda k: slots[int(d[k])]
        if op == D_NOP:
            return None
        if op == D_LDR:
            return self.regs[int(d["imm"])]
        if op == D_LDI:
            k = int(d["imm"])
            return oracle.stimulus(self.seed, self.inst, self.cycle, k, self.n_in, w)
        if op == D_CONST:
            return int(d["imm"]) | (int(d["a"]) << 32) | (int(d["b"]) << 48)
        if op == D_MEMRD:
            m = int(d["imm"])
            depth = 2 ** self.py.mems[m][0]
            return self._read_mem(m, S("a") % depth)
        if op == D_STR:
            r = int(d["imm"])
            assert nxt[r] is None, f"register {r} stored twice"
            nxt[r] = S("a") & mask(w)
            return None
        if op == D_WREC:
            port = int(d["imm"])
            recs[port] = (S("a") != 0, S("b") & mask(int(d["x"])), S("c") & mask(w))
            return None
        if op == D_COMMIT:
            if self.pending:
                self._commit(int(d["imm"]))
            return None
        if op == D_LDM:
            cl = self.cluster
            c = cl["cta"][self.proc]
            i = int(d["b"]) | (int(d["x"]) << 16)
            assert cl["mir_reg"][cl["mir_off"][c] + i] == int(d["imm"]), "mirror entry holds another register"
            v = cl["cur"][c][i]
            assert v == self.regs[int(d["imm"])], "stale mirror value"
            return v
        if op == D_STX:
            cl = self.cluster
            c = cl["cta"][self.proc] // cl["C"] * cl["C"] + int(d["c"])
            i = int(d["b"]) | (int(d["x"]) << 16)
            assert cl["mir_reg"][cl["mir_off"][c] + i] == int(d["imm"]), "mirror write to the wrong entry"
            assert cl["nxt"][c][i] is None, "mirror entry written twice"
            cl["nxt"][c][i] = S("a") & mask(w)
            return None
        a, b = S("a"), S("b")
        if op == D_MUX:
            v = b if a != 0 else S("c")
        elif op == D_SLICE:
            v = a >> int(d["x"])
        elif op == D_CONCAT:
            v = (a << int(d["x"])) | b
        elif op == D_SHL:
            v = 0 if b >= 64 else (a << b) & M64
        elif op == D_SHR:
            v = 0 if b >= 64 else a >> b
        else:
            v = {D_ADD: a + b, D_SUB: a - b, D_MUL: a * b, D_AND: a & b, D_OR: a | b, D_XOR: a ^ b,
                 D_EQ: int(a == b), D_LT: int(a < b)}[op]
        return v & mask(w)

    def step(self, order=None):
        nxt = [None] * len(self.regs)
        recs = {}
        procs = order if order is not None else range(len(self.off))
        if self.cluster:
            self.cluster["nxt"] = [[None] * len(v) for v in self.cluster["cur"]]
        for p in procs:
            self.proc = p
            slots = [None] * int(self.nslots[p])
            if self.mode == "lane_op":
                for b in range(int(self.len[p])):
                    row = self.ins[(int(self.off[p]) + b) * 32:(int(self.off[p]) + b + 1) * 32]
                    outs = [(int(d["dst"]), self._exec(d, slots, nxt, recs)) for d in row]
                    for dst, v in outs:        # all 32 lanes read before any writes
                        if v is not None:
                            slots[dst] = v
            else:
                base = int(self.off[p])
                for i in range(int(self.len[p])):
                    d = self.ins[base + i]
                    v = self._exec(d, slots, nxt, recs)
                    if v is not None:
                        slots[int(d["dst"])] = v
        assert all(v is not None for v in nxt), "a register got no next value"
        if self.cluster:
            for c, v in enumerate(self.cluster["nxt"]):
                assert all(x is not None for x in v), f"mirror of CTA {c} not fully written"
            self.cluster["cur"] = self.cluster["nxt"]
        self.regs = nxt
        self.pending = recs
        self.cycle += 1

    def finish(self):
        for m in range(len(self.mems)):
            self._commit(m)
        self.pending = {}
