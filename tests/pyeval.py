"""Second, independent evaluator of `rtlnet 1` netlists (test helper).

Written separately from the C oracle: its own parser, recursive evaluation
with Python integers, and every result reduced modulo 2**width at each node.
Used to cross-check one oracle step by brute force on tiny circuits.

Clocks (`gate`, `clock` items): `cycle` follows the event order of a Verilog
simulator with nonblocking assignments, written out directly: the top clock's
registers and the memories update first; then, for each divided clock whose
register rose (0 before the cycle, 1 after its own update), the registers on
it are evaluated again on the updated state and update together.
"""


class PyNet:
    def __init__(self, text):
        self.inputs, self.regs, self.mems, self.nodes = [], [], [], []
        self.next, self.wports, self.minit = {}, [], []
        self.gates, self.clocks = {}, {}
        for line in text.splitlines():
            t = line.split("#")[0].split()
            if not t or t[0] in ("rtlnet", "end"):
                continue
            if t[0] == "in":
                self.inputs.append(int(t[1]))
            elif t[0] == "reg":
                self.regs.append((int(t[1]), int(t[2], 0)))
            elif t[0] == "mem":
                self.mems.append((int(t[1]), int(t[2])))
            elif t[0] == "n":
                self.nodes.append((t[1], int(t[2]), [int(x, 0) for x in t[3:]]))
            elif t[0] == "next":
                self.next[int(t[1])] = int(t[2])
            elif t[0] == "wport":
                self.wports.append(tuple(int(x) for x in t[1:5]))
            elif t[0] == "gate":
                self.gates[int(t[1])] = int(t[2])
            elif t[0] == "clock":
                self.clocks[int(t[1])] = int(t[2])
            elif t[0] == "minit":
                self.minit.append(tuple(int(x, 0) for x in t[1:4]))

    def initial_state(self):
        regs = [init % (2 ** w) for (w, init) in self.regs]
        mems = [[0] * (2 ** lg) for (lg, w) in self.mems]
        for m, a, v in self.minit:
            mems[m][a] = v % (2 ** self.mems[m][1])
        return regs, mems

    def step(self, regs, mems, inputs):
        """One clock cycle: returns (next regs, next mems, node values)."""
        ev = self._evaluator(regs, mems, inputs)
        new_regs = [ev(self.next[r]) % (2 ** w) for r, (w, _) in enumerate(self.regs)]
        new_mems = [list(m) for m in mems]
        for (m, en, addr, data) in self.wports:       # ascending port order
            if ev(en) != 0:
                lg, w = self.mems[m]
                new_mems[m][ev(addr) % (2 ** lg)] = ev(data) % (2 ** w)
        vals = {i: ev(i) for i in range(len(self.nodes))}
        return new_regs, new_mems, vals

    def clock_depth(self, r):
        d = 0
        while r in self.clocks:
            r = self.clocks[r]
            d += 1
            assert d <= len(self.regs), "loop of clock registers"
        return d

    def cycle(self, regs, mems, inputs):
        """One top-clock cycle with gated and divided clocks: (regs, mems)."""
        depth = [self.clock_depth(r) for r in range(len(self.regs))]

        def takes(r, ev, cur):
            g = self.gates.get(r)
            if g is not None and ev(g) == 0:
                return cur[r]
            return ev(self.next[r]) % (2 ** self.regs[r][0])

        start = list(regs)
        ev = self._evaluator(regs, mems, inputs)
        cur = [takes(r, ev, regs) if depth[r] == 0 else regs[r] for r in range(len(regs))]
        new_mems = [list(m) for m in mems]
        for (m, en, addr, data) in self.wports:
            if ev(en) != 0:
                lg, w = self.mems[m]
                new_mems[m][ev(addr) % (2 ** lg)] = ev(data) % (2 ** w)
        for k in range(1, max(depth, default=0) + 1):
            ev = self._evaluator(cur, new_mems, inputs)
            upd = {}
            for r in range(len(regs)):
                if depth[r] == k:
                    d = self.clocks[r]
                    upd[r] = takes(r, ev, cur) if start[d] == 0 and cur[d] != 0 else cur[r]
            for r, v in upd.items():
                cur[r] = v
        return cur, new_mems

    def _evaluator(self, regs, mems, inputs):
        memo = {}

        def ev(i):
            if i in memo:
                return memo[i]
            op, w, a = self.nodes[i]
            mod = 2 ** w
            if op == "input":
                v = inputs[a[0]]
            elif op == "reg":
                v = regs[a[0]]
            elif op == "const":
                v = a[0]
            elif op == "memrd":
                depth = 2 ** self.mems[a[0]][0]
                v = mems[a[0]][ev(a[1]) % depth]
            elif op == "add":
                v = ev(a[0]) + ev(a[1])
            elif op == "sub":
                v = ev(a[0]) - ev(a[1])
            elif op == "mul":
                v = ev(a[0]) * ev(a[1])
            elif op == "and":
                v = ev(a[0]) & ev(a[1])
            elif op == "or":
                v = ev(a[0]) | ev(a[1])
            elif op == "xor":
                v = ev(a[0]) ^ ev(a[1])
            elif op == "shl":
                s = ev(a[1])
                v = 0 if s >= 64 else ev(a[0]) * 2 ** s
            elif op == "shr":
                s = ev(a[1])
                v = 0 if s >= 64 else ev(a[0]) // 2 ** s
            elif op == "eq":
                v = 1 if ev(a[0]) == ev(a[1]) else 0
            elif op == "lt":
                v = 1 if ev(a[0]) < ev(a[1]) else 0
            elif op == "mux":
                v = ev(a[1]) if ev(a[0]) != 0 else ev(a[2])
            elif op == "slice":
                v = ev(a[0]) // 2 ** a[1]
            elif op == "concat":
                wb = self.nodes[a[1]][1]
                v = ev(a[0]) * 2 ** wb + ev(a[1])
            else:
                raise ValueError(op)
            v %= mod
            memo[i] = v
            return v

        return ev
