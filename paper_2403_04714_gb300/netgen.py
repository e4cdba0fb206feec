"""Seeded synthetic word-level netlist generator and the `rtlnet` text format.

This module is the shared input generator: it writes netlist *descriptions* and
holds none of the simulation arithmetic (no operator is ever evaluated here).
Both the CPU oracle and the CUDA path read the files it writes, each with its
own parser.

The paper's benchmark designs (Chipyard SoCs, vta, mc; Sec. 6) are not
available, so seeded synthetic netlists stand in for them.  Their shape follows
what the paper reports about real designs: many small fibers (about 4.4 DDG
nodes per fiber, Table perf_smackdown), shared combinational logic between
neighbouring register cones (Sec. 3.2, Fig. bsp_sim node a3), a few very
popular signals (power-law fan-out), and arrays read and written through ports
(Sec. 5.2, differential exchange).

File format (`rtlnet 1`), one item per line, `#` starts a comment:

    rtlnet 1
    in   <width> [name]                 input k (k counts `in` lines from 0)
    reg  <width> <init> [name]          register r (counts `reg` lines from 0)
    mem  <log2 depth> <width> [name]    memory m (counts `mem` lines from 0)
    n    <op> <width> <args...>         node i (counts `n` lines from 0)
    next <r> <node>                     next-state node of register r
    wport <m> <en> <addr> <data>        write port p of memory m (p counts `wport` lines)
    gate <r> <node>                     register r's clock is gated by node (optional)
    clock <r> <d>                       register r is clocked by the rising edge of the
                                        1-bit register d, a divided clock (optional;
                                        default: the top-level clock)
    minit <m> <addr> <value>            initial memory word (default 0)
    end

Node ops and their arguments (node ids may refer forward; the file must be
acyclic through nodes, registers break cycles):

    input k | reg r | const v | memrd m a
    add a b | sub a b | mul a b | and a b | or a b | xor a b
    shl a b | shr a b | eq a b | lt a b | mux s a b
    slice a lo | concat a b
"""

from __future__ import annotations

import io
import os
import random
from dataclasses import dataclass, field

BIN_OPS = ("add", "sub", "mul", "and", "or", "xor", "shl", "shr", "eq", "lt")
ALL_OPS = BIN_OPS + ("mux", "slice", "concat")          # the 13 comb op kinds
LFSR32_MASK = 0x80200003   # Galois mask for taps 32,22,2,1
LFSR16_MASK = 0xD008       # Galois mask for taps 16,15,13,4
MAC_K = 0x9E3779B97F4A7C15


@dataclass
class Netlist:
    """In-memory netlist under construction (plain lists; no evaluation)."""
    inputs: list = field(default_factory=list)   # (width, name)
    regs: list = field(default_factory=list)     # [width, init, next_node, name]
    mems: list = field(default_factory=list)     # (log2depth, width, name)
    nodes: list = field(default_factory=list)    # (op, width, args tuple)
    wports: list = field(default_factory=list)   # (mem, en, addr, data)
    minit: list = field(default_factory=list)    # (mem, addr, value)
    gates: dict = field(default_factory=dict)    # register -> gate node
    clocks: dict = field(default_factory=dict)   # register -> clock register

    # -- construction helpers -------------------------------------------------
    def add_input(self, width, name=""):
        self.inputs.append((width, name))
        return len(self.inputs) - 1

    def add_reg(self, width, init=0, name=""):
        self.regs.append([width, init, -1, name])
        return len(self.regs) - 1

    def add_mem(self, log2depth, width, name=""):
        self.mems.append((log2depth, width, name))
        return len(self.mems) - 1

    def node(self, op, width, *args):
        self.nodes.append((op, width, tuple(int(a) for a in args)))
        return len(self.nodes) - 1

    def set_next(self, r, node):
        self.regs[r][2] = node

    def width(self, node):
        return self.nodes[node][1]

    # -- serialisation --------------------------------------------------------
    def write(self, f):
        w = f.write
        w("rtlnet 1\n")
        for width, name in self.inputs:
            w(f"in {width} {name}\n" if name else f"in {width}\n")
        for width, init, _, name in self.regs:
            w(f"reg {width} {init} {name}\n" if name else f"reg {width} {init}\n")
        for lg, width, name in self.mems:
            w(f"mem {lg} {width} {name}\n" if name else f"mem {lg} {width}\n")
        buf = []
        for op, width, args in self.nodes:
            buf.append("n %s %d %s\n" % (op, width, " ".join(map(str, args))))
            if len(buf) >= 65536:
                w("".join(buf))
                buf.clear()
        w("".join(buf))
        for r, (_, _, nxt, _) in enumerate(self.regs):
            if nxt < 0:
                raise ValueError(f"register {r} has no next node")
            w(f"next {r} {nxt}\n")
        for m, en, addr, data in self.wports:
            w(f"wport {m} {en} {addr} {data}\n")
        for r, g in sorted(self.gates.items()):
            w(f"gate {r} {g}\n")
        for r, d in sorted(self.clocks.items()):
            w(f"clock {r} {d}\n")
        for m, a, v in self.minit:
            w(f"minit {m} {a} {v}\n")
        w("end\n")

    def to_text(self) -> str:
        s = io.StringIO()
        self.write(s)
        return s.getvalue()

    def save(self, path):
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            self.write(f)
        os.replace(tmp, path)

    def reg_index(self, name):
        for i, r in enumerate(self.regs):
            if r[3] == name:
                return i
        raise KeyError(name)


def node_depths(nl: Netlist, prev=None):
    """Combinational depth of each node (leaves 0); nodes are built in topological order.

    `prev` holds already-known depths of a prefix of the node list."""
    d = list(prev or []) + [0] * (len(nl.nodes) - len(prev or []))
    for i in range(len(prev or []), len(nl.nodes)):
        op, _, args = nl.nodes[i]
        if op in ("reg", "input", "const"):
            continue
        srcs = (args[0],) if op == "slice" else (args[1],) if op == "memrd" else args
        d[i] = 1 + max(d[j] for j in srcs)
    return d


def parse_names(text: str):
    """Map register names to indices from rtlnet text (used by tests)."""
    names, r = {}, 0
    for line in text.splitlines():
        t = line.split()
        if t and t[0] == "reg":
            if len(t) > 3:
                names[t[3]] = r
            r += 1
    return names


# ---------------------------------------------------------------------------
# Closed-form blocks embedded in every generated netlist.  Their traces have
# known closed forms (counter, maximal LFSR, Fibonacci, multiply-accumulate),
# which pin the oracle and give a size-independent check on long GPU runs.
# ---------------------------------------------------------------------------
def add_check_blocks(nl: Netlist, prefix="chk_"):
    c = nl.add_reg(16, 0, prefix + "counter16")
    rc = nl.node("reg", 16, c)
    nl.set_next(c, nl.node("add", 16, rc, nl.node("const", 16, 1)))

    s = nl.add_reg(32, 1, prefix + "lfsr32")
    rs = nl.node("reg", 32, s)
    sh = nl.node("shr", 32, rs, nl.node("const", 6, 1))
    lsb = nl.node("slice", 1, rs, 0)
    tap = nl.node("mux", 32, lsb, nl.node("const", 32, LFSR32_MASK), nl.node("const", 32, 0))
    nl.set_next(s, nl.node("xor", 32, sh, tap))

    s16 = nl.add_reg(16, 1, prefix + "lfsr16")
    r16 = nl.node("reg", 16, s16)
    sh16 = nl.node("shr", 16, r16, nl.node("const", 4, 1))
    # -(s & 1) & mask, written with sub/and instead of mux
    neg = nl.node("sub", 16, nl.node("const", 16, 0), nl.node("and", 16, r16, nl.node("const", 16, 1)))
    nl.set_next(s16, nl.node("xor", 16, sh16, nl.node("and", 16, neg, nl.node("const", 16, LFSR16_MASK))))

    fa = nl.add_reg(64, 0, prefix + "fib_a")
    fb = nl.add_reg(64, 1, prefix + "fib_b")
    ra, rb = nl.node("reg", 64, fa), nl.node("reg", 64, fb)
    nl.set_next(fa, rb)
    nl.set_next(fb, nl.node("add", 64, ra, rb))

    acc = nl.add_reg(64, 0, prefix + "mac")
    racc = nl.node("reg", 64, acc)
    prod = nl.node("mul", 64, rc, nl.node("const", 64, MAC_K))
    nl.set_next(acc, nl.node("add", 64, racc, prod))
    return {"counter16": c, "lfsr32": s, "lfsr16": s16, "fib_a": fa, "fib_b": fb, "mac": acc}


# ---------------------------------------------------------------------------
# Random module-structured logic.
# ---------------------------------------------------------------------------
def _powerlaw_table(alpha_num=2, cap=512):
    """Integer cumulative weights for a discrete power law P(k) ~ k^-alpha, k in [1, cap]."""
    cum, tot = [], 0
    for k in range(1, cap + 1):
        tot += (1 << 40) // (k ** alpha_num)
        cum.append(tot)
    return cum


def _draw(rng, cum):
    import bisect
    return bisect.bisect_right(cum, rng.randrange(cum[-1])) + 1


class _Weighted:
    """Pick items with probability proportional to integer weights (append-only)."""

    def __init__(self):
        self.items, self.cum = [], []

    def add(self, item, weight):
        self.items.append(item)
        self.cum.append((self.cum[-1] if self.cum else 0) + weight)

    def __len__(self):
        return len(self.items)

    def pick(self, rng):
        import bisect
        return self.items[bisect.bisect_right(self.cum, rng.randrange(self.cum[-1]))]


@dataclass
class GenParams:
    n_ops: int                   # combinational ops (leaf/const nodes are extra)
    n_regs: int
    depth: int
    n_inputs: int
    reg_width_mix: tuple = ((1, 30), (32, 40), (64, 30))   # (width, percent)
    regs_per_module: int = 10
    p_leaf: float = 0.55          # extra operand is a leaf (reg/input/const)
    p_global: float = 0.30        # a register leaf is drawn from the whole design
    p_share: float = 0.10         # extra operand taken from the neighbouring module
    rams: tuple = ()              # ((log2depth, width, sync_read_ports, comb_read_ports, write_ports), ...)
    fanout_cap: int = 512
    check_blocks: bool = True


def _pick_width(rng, mix):
    x = rng.randrange(100)
    acc = 0
    for w, pct in mix:
        acc += pct
        if x < acc:
            return w
    return mix[-1][0]


def generate_logic(nl: Netlist, rng: random.Random, p: GenParams, in_ids, reg_ids,
                   ext_regs=None):
    """Generate `p.n_ops` ops driving the registers in `reg_ids` (already declared).

    Structure: registers are grouped into modules of ~regs_per_module; each
    module owns ~n_ops/n_modules ops arranged in levels 1..d (d <= depth, one
    module reaches depth exactly).  An op at level L takes its first operand
    from level L-1 of its module, so the longest path is exact.  Extra operands
    come from leaves, lower levels of the module, or the previous module's
    logic (shared logic, which SLB must deduplicate).  Register reads across
    the design follow a power-law popularity, capped at fanout_cap.
    """
    n_mod = max(1, len(reg_ids) // p.regs_per_module)
    cum_pop = _powerlaw_table(2, p.fanout_cap)

    # design-wide register pool with power-law popularity
    global_regs = _Weighted()
    for r in (ext_regs if ext_regs is not None else reg_ids):
        global_regs.add(r, _draw(rng, cum_pop))
    reg_leaf = {}

    def leaf_reg(r):
        nid = reg_leaf.get(r)
        if nid is None:
            nid = nl.node("reg", nl.regs[r][0], r)
            reg_leaf[r] = nid
        return nid

    in_leaf = {}

    def leaf_in(k):
        nid = in_leaf.get(k)
        if nid is None:
            nid = nl.node("input", nl.inputs[k][0], k)
            in_leaf[k] = nid
        return nid

    def const_node(width):
        v = rng.getrandbits(width)
        if rng.randrange(4) == 0:
            v = rng.randrange(min(1 << width, 8))
        return nl.node("const", width, v)

    ops_per_mod = [p.n_ops // n_mod + (1 if i < p.n_ops % n_mod else 0) for i in range(n_mod)]
    regs_of_mod = [reg_ids[i::n_mod] for i in range(n_mod)]
    prev_levels = None
    made = 0
    for mi in range(n_mod):
        n_here = ops_per_mod[mi]
        d = p.depth if mi == 0 else rng.randrange(max(2, p.depth // 4), p.depth + 1)
        d = max(1, min(d, n_here))
        lvl_count = [1] * d
        for _ in range(n_here - d):
            # skew toward low levels: min of two uniform draws
            lvl_count[min(rng.randrange(d), rng.randrange(d))] += 1
        own_regs = regs_of_mod[mi]
        local_regs = _Weighted()
        for r in own_regs:
            local_regs.add(r, 4)
        levels = []          # per level: _Weighted of node ids
        all_nodes = _Weighted()
        narrow = []          # nodes of width <= 6, usable as shift amounts

        def pick_leaf(width_hint):
            x = rng.randrange(100)
            if x < 8 and in_ids:
                return leaf_in(in_ids[rng.randrange(len(in_ids))])
            if x < 22:
                return const_node(width_hint)
            if x < 22 + int(p.p_global * 78) and len(global_regs):
                return leaf_reg(global_regs.pick(rng))
            return leaf_reg(local_regs.pick(rng))

        def pick_lower(L):
            # an op from a lower level of this module, or the previous module
            if prev_levels and rng.random() < p.p_share:
                lv = prev_levels[min(L - 1, len(prev_levels)) - 1] if L > 1 else prev_levels[0]
                return lv.pick(rng)
            if L <= 1 or not len(all_nodes):
                return pick_leaf(rng.choice((1, 8, 16, 32, 64)))
            return levels[rng.randrange(L - 1)].pick(rng)

        def pick_extra(L, width_hint):
            if rng.random() < p.p_leaf or L <= 1:
                return pick_leaf(width_hint)
            return pick_lower(L)

        for L in range(1, d + 1):
            lv = _Weighted()
            n_narrow = len(narrow)      # shift amounts come from lower levels only
            for _ in range(lvl_count[L - 1]):
                first = levels[L - 2].pick(rng) if L >= 2 else pick_leaf(rng.choice((8, 16, 32, 64)))
                wa = nl.width(first)
                kind = ALL_OPS[rng.randrange(len(ALL_OPS))]
                if kind in ("shl", "shr"):
                    if n_narrow and rng.randrange(2):
                        amt = narrow[rng.randrange(n_narrow)]
                    else:
                        amt = nl.node("const", 7, rng.randrange(0, min(wa + 3, 127)))
                    nid = nl.node(kind, wa, first, amt)
                elif kind in ("eq", "lt"):
                    b = pick_extra(L, wa)
                    nid = nl.node(kind, 1, first, b)
                elif kind == "mux":
                    s = pick_extra(L - 1, 1)     # may get a slice wrapper: one level lower
                    if nl.width(s) != 1 and L >= 2 and rng.randrange(2):
                        s = nl.node("slice", 1, s, rng.randrange(nl.width(s)))
                    b = pick_extra(L, wa)
                    if rng.randrange(2):
                        nid = nl.node("mux", max(wa, nl.width(b)), s, first, b)
                    else:
                        nid = nl.node("mux", max(wa, nl.width(b)), s, b, first)
                elif kind == "slice":
                    wo = rng.randrange(1, wa + 1)
                    nid = nl.node("slice", wo, first, rng.randrange(0, wa - wo + 1))
                elif kind == "concat":
                    b = pick_extra(L - 1, max(1, 64 - wa))
                    wb = nl.width(b)
                    if wa + wb > 64:
                        if wa >= 64:
                            nid = nl.node("slice", 32, first, rng.randrange(33))
                            lv.add(nid, _draw(rng, cum_pop))
                            all_nodes.add(nid, 1)
                            made += 1
                            continue
                        if L >= 2:
                            b = nl.node("slice", 64 - wa, b, rng.randrange(wb - (64 - wa) + 1))
                        else:
                            b = const_node(64 - wa)
                        wb = 64 - wa
                    if rng.randrange(2):
                        nid = nl.node("concat", wa + wb, first, b)
                    else:
                        nid = nl.node("concat", wa + wb, b, first)
                else:
                    b = pick_extra(L, wa)
                    nid = nl.node(kind, max(wa, nl.width(b)), first, b)
                if nl.width(nid) <= 6:
                    narrow.append(nid)
                lv.add(nid, _draw(rng, cum_pop))
                all_nodes.add(nid, 1)
                made += 1
            levels.append(lv)

        # register next-state nodes: the deepest op feeds a register so the
        # module depth is realised; the others come from any level
        deepest = levels[-1].items
        for j, r in enumerate(own_regs):
            if j == 0:
                src = deepest[rng.randrange(len(deepest))]
            else:
                lv = levels[rng.randrange(len(levels))]
                src = lv.items[rng.randrange(len(lv.items))]
            nl.set_next(r, src)
        prev_levels = levels
    return made


def add_ram(nl, rng, log2depth, width, addr_src, data_src, en_src, n_sync=1, n_comb=0,
            n_wports=1, name="ram", ext_regs=None):
    """A RAM with synchronous read ports (memrd feeding a register), combinational
    read ports (memrd nodes returned for use by logic) and write ports."""
    m = nl.add_mem(log2depth, width, name)
    comb = []
    for i in range(n_sync):
        a = nl.node("slice", log2depth, addr_src(), 0)
        rd = nl.node("memrd", width, m, a)
        r = nl.add_reg(width, 0, f"{name}_rd{i}")
        nl.set_next(r, rd)
        if ext_regs is not None:
            ext_regs.append(r)
    for i in range(n_comb):
        a = nl.node("slice", log2depth, addr_src(), 0)
        comb.append(nl.node("memrd", width, m, a))
    for i in range(n_wports):
        en = nl.node("slice", 1, en_src(), 0)
        a = nl.node("slice", log2depth, addr_src(), 0)
        nl.wports.append((m, en, a, data_src()))
    return m, comb


# ---------------------------------------------------------------------------
# The five workload shapes.
# ---------------------------------------------------------------------------
def gen_flat(seed, n_ops, n_regs, depth, n_inputs, rams=(), reg_width_mix=None,
             regs_per_module=10) -> Netlist:
    """A flat netlist (configs 'tiny' and 'mid')."""
    rng = random.Random(seed)
    nl = Netlist()
    in_ids = [nl.add_input(rng.choice((1, 8, 16, 32, 64))) for _ in range(n_inputs)]
    mix = reg_width_mix or ((1, 30), (32, 40), (64, 30))
    reg_ids = [nl.add_reg(_pick_width(rng, mix), 0) for _ in range(n_regs)]
    for r in reg_ids:
        if rng.randrange(8) == 0:
            w = nl.regs[r][0]
            nl.regs[r][1] = rng.getrandbits(w)
    p = GenParams(n_ops=n_ops, n_regs=n_regs, depth=depth, n_inputs=n_inputs,
                  regs_per_module=regs_per_module)
    generate_logic(nl, rng, p, in_ids, reg_ids)
    # RAMs: addresses/data/enables taken from existing wide nodes shallow enough
    # that the added slice/memrd/xor levels keep the design depth exact
    dep = node_depths(nl)
    wide = [i for i, nd in enumerate(nl.nodes) if nd[1] >= 16 and nd[0] != "const"
            and dep[i] <= depth - 2]
    shallow_regs = [r for r in reg_ids if dep[nl.regs[r][2]] <= depth - 1]
    for k, (lg, width) in enumerate(rams):
        src = lambda: wide[rng.randrange(len(wide))]
        m, _ = add_ram(nl, rng, lg, width, src, src, src, name=f"ram{k}")
        # make the read register visible to logic: route it into an existing register's cone
        rd_reg = len(nl.regs) - 1
        tgt = shallow_regs[rng.randrange(len(shallow_regs))]
        old = nl.regs[tgt][2]
        x = nl.node("xor", max(nl.width(old), width), old, nl.node("reg", width, rd_reg))
        nl.set_next(tgt, x)
    add_check_blocks(nl)
    return nl


def gen_tiny(seed=1000) -> Netlist:
    """64 registers (widths uniform in {1,8,16,32,64}), 2,000 ops, depth 20, 8 inputs."""
    mix = ((1, 20), (8, 20), (16, 20), (32, 20), (64, 20))
    return gen_flat(seed, n_ops=2000, n_regs=64, depth=20, n_inputs=8, reg_width_mix=mix,
                    regs_per_module=8)


def gen_mid(seed=1001) -> Netlist:
    """200k ops, 20k registers (30% 1b / 40% 32b / 30% 64b), depth 60, two 512x64 RAMs."""
    return gen_flat(seed, n_ops=200_000, n_regs=20_000, depth=60, n_inputs=64,
                    rams=((9, 64), (9, 64)))


def gen_mesh(seed=1002, mesh=4, ops_per_block=120_000, regs_per_block=8_000, depth=60,
             inputs_per_block=16) -> Netlist:
    """mesh x mesh replicated core-like blocks on a 2-D mesh with 64-bit valid/ready links.

    Each block: `ops_per_block` ops, `regs_per_block` registers, a 32x64-bit
    register file (two combinational reads, one write) and a 16 KB RAM
    (2048x64-bit, one synchronous read, one write).  Each block drives one
    outgoing link per mesh neighbour (64-bit data register, 1-bit valid,
    1-bit ready); a block reads only its neighbours' link registers.
    """
    rng = random.Random(seed)
    nl = Netlist()
    nb = mesh * mesh
    # declare per block: inputs, registers, link registers
    blk = []
    for b in range(nb):
        in_ids = [nl.add_input(rng.choice((1, 8, 16, 32, 64)), f"b{b}_in{k}") for k in range(inputs_per_block)]
        reg_ids = [nl.add_reg(_pick_width(rng, ((1, 30), (32, 40), (64, 30))), 0)
                   for _ in range(regs_per_block)]
        blk.append({"in": in_ids, "regs": reg_ids, "links": {}})
    dirs = ((0, 1, "e"), (0, -1, "w"), (1, 0, "s"), (-1, 0, "n"))
    for b in range(nb):
        y, x = divmod(b, mesh)
        for dy, dx, nm in dirs:
            yy, xx = y + dy, x + dx
            if 0 <= yy < mesh and 0 <= xx < mesh:
                data = nl.add_reg(64, 0, f"b{b}_{nm}_data")
                valid = nl.add_reg(1, 0, f"b{b}_{nm}_valid")
                ready = nl.add_reg(1, 0, f"b{b}_{nm}_ready")
                blk[b]["links"][nm] = (yy * mesh + xx, data, valid, ready)
    dep_known = []
    for b in range(nb):
        brng = random.Random(rng.getrandbits(64))
        y, x = divmod(b, mesh)
        # registers visible to this block's logic: its own + neighbours' links towards it
        incoming = []
        for ob in range(nb):
            for nm, (dst, data, valid, ready) in blk[ob]["links"].items():
                if dst == b:
                    incoming += [data, valid]
        own_out = []
        for nm, (dst, data, valid, ready) in blk[b]["links"].items():
            own_out += [data, valid, ready]
        ext = blk[b]["regs"] + incoming
        p = GenParams(n_ops=ops_per_block, n_regs=regs_per_block, depth=depth,
                      n_inputs=inputs_per_block)
        first_node = len(nl.nodes)
        generate_logic(nl, brng, p, blk[b]["in"], blk[b]["regs"], ext_regs=ext)
        dep = node_depths(nl, dep_known)
        dep_known = dep
        wide = [i for i in range(first_node, len(nl.nodes)) if nl.nodes[i][1] >= 16
                and nl.nodes[i][0] != "const" and dep[i] <= depth - 3]
        shallow = [r for r in blk[b]["regs"] if dep[nl.regs[r][2]] <= depth - 1]
        src = lambda: wide[brng.randrange(len(wide))]
        # register file: 32 x 64, 2 comb reads, 1 write
        _, comb = add_ram(nl, brng, 5, 64, src, src, src, n_sync=0, n_comb=2, n_wports=1,
                          name=f"b{b}_rf")
        # 16 KB RAM: 2048 x 64, 1 sync read, 1 write
        add_ram(nl, brng, 11, 64, src, src, src, n_sync=1, n_comb=0, n_wports=1,
                name=f"b{b}_ram")
        ram_rd = len(nl.regs) - 1
        # fold memory reads into some register cones
        for c in comb + [nl.node("reg", 64, ram_rd)]:
            tgt = shallow[brng.randrange(len(shallow))]
            old = nl.regs[tgt][2]
            nl.set_next(tgt, nl.node("add", 64, old, c))
        # outgoing links: data/valid from block logic; ready from the incoming valid
        for nm, (dst, data, valid, ready) in blk[b]["links"].items():
            nl.set_next(data, nl.node("mux", 64, nl.node("slice", 1, src(), 0), src(),
                                      nl.node("reg", 64, data)))
            nl.set_next(valid, nl.node("slice", 1, src(), 0))
            back = blk[dst]["links"]
            opp = {"e": "w", "w": "e", "s": "n", "n": "s"}[nm]
            vin = back[opp][2] if opp in back else None
            nl.set_next(ready, nl.node("eq", 1, nl.node("reg", 1, vin), nl.node("const", 1, 0))
                        if vin is not None else nl.node("const", 1, 1))
    add_check_blocks(nl)
    return nl


def gen_prng(n_fibers: int, seed: int = 5) -> Netlist:
    """Independent 64-bit xorshift generators (three XORs, three shifts each):
    one fiber per register, no value crosses fibers (the synchronisation
    experiment's circuit, Sec. 4.1)."""
    rng = random.Random(seed)
    nl = Netlist()
    for i in range(n_fibers):
        r = nl.add_reg(64, rng.getrandbits(64) | 1)
        x = nl.node("reg", 64, r)
        for sh, kind in ((13, "shl"), (7, "shr"), (17, "shl")):
            x = nl.node("xor", 64, x, nl.node(kind, 64, x, nl.node("const", 7, sh)))
        nl.set_next(r, x)
    return nl


def gen_clocked(seed=1004, n_ops=2_000, n_regs=64, depth=20, n_inputs=8, gated_frac=0.25,
                divided_frac=0.25) -> Netlist:
    """A design with one top-level clock, a divide-by-2 and a divide-by-4
    clock (toggle registers, the second clocked by the first) and gated
    clocks: random logic like `gen_flat`, then a share of its registers moved
    to the divided clocks and a share gated by a 1-bit signal of the logic.
    Check registers with closed forms: a counter on each divided clock, a
    register on the divide-by-2 clock sampling a top-clock counter, and a
    counter gated by bit 0 of the 32-bit LFSR."""
    nl = gen_flat(seed, n_ops, n_regs, depth, n_inputs)      # includes the check blocks
    rng = random.Random(seed + 1)
    reg_ids = list(range(n_regs))
    chk = {name[len("chk_"):]: nl.reg_index(name) for name in ("chk_counter16", "chk_lfsr32")}
    div2 = nl.add_reg(1, 0, "clk_div2")
    nl.set_next(div2, nl.node("xor", 1, nl.node("reg", 1, div2), nl.node("const", 1, 1)))
    div4 = nl.add_reg(1, 0, "clk_div4")
    nl.set_next(div4, nl.node("xor", 1, nl.node("reg", 1, div4), nl.node("const", 1, 1)))
    nl.clocks[div4] = div2
    for name, clk in (("cnt_div2", div2), ("cnt_div4", div4)):
        c = nl.add_reg(16, 0, name)
        nl.set_next(c, nl.node("add", 16, nl.node("reg", 16, c), nl.node("const", 16, 1)))
        nl.clocks[c] = clk
    smp = nl.add_reg(16, 0, "sample_div2")          # samples the top-clock counter
    nl.set_next(smp, nl.node("reg", 16, chk["counter16"]))
    nl.clocks[smp] = div2
    gc = nl.add_reg(16, 0, "cnt_gated")             # counts cycles with LFSR bit 0 set
    nl.set_next(gc, nl.node("add", 16, nl.node("reg", 16, gc), nl.node("const", 16, 1)))
    nl.gates[gc] = nl.node("slice", 1, nl.node("reg", 32, chk["lfsr32"]), 0)
    # random logic registers onto the divided and gated clocks
    bits = [i for i, (op, w, _) in enumerate(nl.nodes) if w == 1 and op != "memrd"]
    for r in reg_ids:
        u = rng.random()
        if u < divided_frac:
            nl.clocks[r] = rng.choice((div2, div4))
        if rng.random() < gated_frac:
            nl.gates[r] = rng.choice(bits)
    return nl


def gen_exchange(n_fibers: int, reads: int, seed: int = 9) -> Netlist:
    """The communication experiment's circuit (Sec. 4.2) as a netlist: 64-bit
    registers, each of whose next value combines its own value with `reads`
    registers drawn at random from the whole design (an xor tree, then one
    xorshift step).  Under a random partition nearly every read crosses
    processes, so the values exchanged per process grow with `reads`."""
    rng = random.Random(seed)
    nl = Netlist()
    regs = [nl.add_reg(64, rng.getrandbits(64) | 1) for _ in range(n_fibers)]
    for r in regs:
        terms = [nl.node("reg", 64, r)]
        for _ in range(reads):
            q = rng.randrange(n_fibers - 1)
            terms.append(nl.node("reg", 64, q if q < r else q + 1))
        while len(terms) > 1:
            terms = [nl.node("xor", 64, terms[i], terms[i + 1]) if i + 1 < len(terms) else terms[i]
                     for i in range(0, len(terms), 2)]
        x = terms[0]
        nl.set_next(r, nl.node("xor", 64, x, nl.node("shl", 64, x, nl.node("const", 7, 13))))
    return nl


def gen_mesh_small(seed=1003) -> Netlist:
    """A 2x2 mesh of 30k-op blocks: the mesh shape at served-job scale."""
    return gen_mesh(seed, mesh=2, ops_per_block=30_000, regs_per_block=2_000, depth=40, inputs_per_block=8)


CONFIGS = {
    "tiny": dict(gen=gen_tiny, seed=1000, n_inst=1, cycles=10_000, stim_seed=42),
    "mid": dict(gen=gen_mid, seed=1001, n_inst=1, cycles=100_000, stim_seed=42),
    "mesh": dict(gen=gen_mesh, seed=1002, n_inst=1, cycles=1_000_000, stim_seed=42),
    "batched": dict(gen=gen_mid, seed=1001, n_inst=4096, cycles=100_000, stim_seed=42),
    "mesh_small": dict(gen=gen_mesh_small, seed=1003, n_inst=1, cycles=10_000, stim_seed=42),
}


def cached_netlist(name: str, cache_dir: str | None = None, **overrides) -> str:
    """Generate (once) the named workload netlist and return its file path."""
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    cache_dir = cache_dir or os.environ.get("RTLSIM_NETCACHE",
                                            os.path.join(os.path.dirname(os.path.dirname(
                                                os.path.abspath(__file__))), "_build", "nets"))
    os.makedirs(cache_dir, exist_ok=True)
    path = os.path.join(cache_dir, f"{cfg['gen'].__name__}_{cfg['seed']}.rtlnet")
    if not os.path.exists(path):
        cfg["gen"](cfg["seed"]).save(path)
    return path


def served_trace(n_jobs=40, rate=200.0, seed=7, inst_max=1024, cycles_lo=1e2, cycles_hi=3e3,
                 shapes=(("tiny", 0.6), ("mid", 0.3), ("mesh_small", 0.1))):
    """Seeded job trace: Poisson arrivals, shape by weight, instances and
    cycle budgets log-uniform.  Returns (arrival_s, shape, pool_index, n_inst, n_cycles, seed)."""
    import math
    rng = random.Random(seed)
    t, out = 0.0, []
    for j in range(n_jobs):
        t += rng.expovariate(rate)
        x, acc, shape = rng.random(), 0.0, shapes[-1][0]
        for name, wgt in shapes:
            acc += wgt
            if x < acc:
                shape = name
                break
        n_inst = max(1, min(inst_max, int(round(math.exp(rng.uniform(0, math.log(inst_max)))))))
        cyc = int(round(math.exp(rng.uniform(math.log(cycles_lo), math.log(cycles_hi)))))
        out.append((t, shape, rng.randrange(1 << 30), n_inst, cyc, 1000 + j))
    return out
