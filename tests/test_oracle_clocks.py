"""Pins of the oracle's gated and divided clocks (paper Sec. 5, limitations:
one top-level clock plus gated or divided ones).

* Closed forms on the seeded multi-clock design: a divide-by-2 and a
  divide-by-4 toggle register, a counter on each divided clock, a register on
  the divide-by-2 clock that samples a top-clock counter (its value tells the
  post-edge reading from the clock-enable one), and a counter gated by bit 0
  of the 32-bit LFSR, counted here from the LFSR's own recurrence.
* Brute force: on tiny random circuits with a divided and a gated clock, one
  oracle cycle equals the independent Python evaluator for every register
  state and input.
* Special cases: a gate that is always 1 changes nothing; a clock register
  that never rises freezes its registers.
* Loader rejections: a loop of clock registers, a clock register wider than
  one bit, two clock items for one register, a memory read under a divided
  clock.
"""
import itertools
import random

import pytest

import oracle
from paper_2403_04714_gb300 import netgen
from pyeval import PyNet

LFSR32_MASK = 0x80200003


@pytest.fixture(scope="module")
def clocked():
    nl = netgen.gen_clocked()
    text = nl.to_text()
    return nl, text, netgen.parse_names(text)


def run_regs(text, cycles, names, seed=42):
    net = oracle.Net(text=text)
    sim = oracle.Sim(net, seed=seed, inst=0)
    out = {k: [] for k in names}
    for _ in range(cycles):
        for k, r in names.items():
            out[k].append(sim.reg(r))
        sim.run(1)
    return out


def test_divided_clock_closed_forms(clocked):
    _, text, names = clocked
    want = ("clk_div2", "clk_div4", "cnt_div2", "cnt_div4", "sample_div2", "chk_counter16")
    got = run_regs(text, 600, {k: names[k] for k in want})
    for t in range(600):
        edges2 = (t + 1) // 2                 # rising edges of div2 in cycles 0..t-1
        assert got["chk_counter16"][t] == t
        assert got["clk_div2"][t] == t % 2
        assert got["cnt_div2"][t] == edges2
        assert got["clk_div4"][t] == edges2 % 2
        assert got["cnt_div4"][t] == (edges2 + 1) // 2
        # the divided clock's edge follows the top clock's: the sampled counter
        # is the value after that edge (t + 1 at the edge of cycle t, t even)
        assert got["sample_div2"][t] == (t if t % 2 else max(t - 1, 0))


def test_gated_counter_counts_lfsr_bits(clocked):
    _, text, names = clocked
    got = run_regs(text, 800, {k: names[k] for k in ("cnt_gated", "chk_lfsr32")})
    s, count = 1, 0
    for t in range(800):
        assert got["chk_lfsr32"][t] == s
        assert got["cnt_gated"][t] == count
        count += s & 1
        s = (s >> 1) ^ (LFSR32_MASK if s & 1 else 0)


def random_clocked_circuit(seed):
    """2 inputs, registers of 3, 2 and 1 bits plus two 1-bit clock registers
    (divide-by-2 on the top clock, a second one clocked by the first)."""
    rng = random.Random(seed)
    nl = netgen.Netlist()
    i0, i1 = nl.add_input(2), nl.add_input(2)
    regs = [nl.add_reg(w, rng.randrange(2 ** w)) for w in (3, 2, 1)]
    c1, c2 = nl.add_reg(1, 0), nl.add_reg(1, 0)
    pool = [nl.node("input", 2, i0), nl.node("input", 2, i1)]
    pool += [nl.node("reg", nl.regs[r][0], r) for r in regs + [c1, c2]]
    pool.append(nl.node("const", 3, rng.randrange(8)))
    for _ in range(rng.randrange(10, 20)):
        kind = rng.choice(netgen.ALL_OPS)
        a, b, c = (pool[rng.randrange(len(pool))] for _ in range(3))
        wa, wb = nl.width(a), nl.width(b)
        if kind in ("eq", "lt"):
            n = nl.node(kind, 1, a, b)
        elif kind == "mux":
            n = nl.node("mux", rng.randrange(1, 6), a, b, c)
        elif kind == "slice":
            w = rng.randrange(1, wa + 1)
            n = nl.node("slice", w, a, rng.randrange(wa - w + 1))
        elif kind == "concat":
            n = nl.node("concat", wa + wb, a, b)
        else:
            n = nl.node(kind, rng.randrange(1, 7), a, b)
        pool.append(n)
    for r in regs + [c1, c2]:
        nl.set_next(r, pool[rng.randrange(len(pool))])
    nl.clocks[c2] = c1
    ones = [n for n in pool if nl.width(n) == 1]
    for r in regs:
        choice = rng.randrange(3)
        if choice:
            nl.clocks[r] = (c1, c2)[choice - 1]
        if ones and rng.randrange(2):
            nl.gates[r] = ones[rng.randrange(len(ones))]
    return nl


@pytest.mark.parametrize("seed", range(10))
def test_one_cycle_matches_python_evaluator_for_every_state(seed):
    nl = random_clocked_circuit(seed)
    text = nl.to_text()
    py = PyNet(text)
    sim = oracle.Sim(oracle.Net(text=text), seed=1, inst=0)
    n_regs = len(nl.regs)
    widths = [w for w, *_ in nl.regs]
    for state in itertools.product(*(range(2 ** w) for w in widths)):
        for x0, x1 in itertools.product(range(4), range(4)):
            for r, v in enumerate(state):
                sim.set_reg(r, v)
            sim.hold_input(0, x0)
            sim.hold_input(1, x1)
            sim.run(1)
            want, _ = py.cycle(list(state), [], [x0, x1])
            got = [sim.reg(r) for r in range(n_regs)]
            assert got == want, (seed, state, x0, x1)


def test_gate_that_is_always_one_changes_nothing():
    base = netgen.gen_flat(11, n_ops=600, n_regs=40, depth=10, n_inputs=4)
    gated = netgen.gen_flat(11, n_ops=600, n_regs=40, depth=10, n_inputs=4)
    one = gated.node("const", 1, 1)
    for r in range(len(gated.regs)):
        gated.gates[r] = one
    a = oracle.Sim(oracle.Net(text=base.to_text()), seed=3, inst=0)
    b = oracle.Sim(oracle.Net(text=gated.to_text()), seed=3, inst=0)
    assert a.run(200, digests=True).tolist() == b.run(200, digests=True).tolist()


def test_clock_register_that_never_rises_freezes_its_registers():
    nl = netgen.gen_flat(12, n_ops=400, n_regs=30, depth=8, n_inputs=4)
    stuck = nl.add_reg(1, 0, "stuck")
    nl.set_next(stuck, nl.node("const", 1, 0))
    frozen = list(range(0, 30, 3))
    for r in frozen:
        nl.clocks[r] = stuck
    sim = oracle.Sim(oracle.Net(text=nl.to_text()), seed=5, inst=0)
    init = [sim.reg(r) for r in frozen]
    sim.run(100)
    assert [sim.reg(r) for r in frozen] == init


def _reject(text, what):
    with pytest.raises(Exception, match=what):
        oracle.Net(text=text)


def test_loader_rejections():
    base = ["rtlnet 1", "reg 1 0", "reg 1 0", "reg 8 0", "n reg 1 0", "n reg 1 1", "n reg 8 2",
            "next 0 0", "next 1 1", "next 2 2"]
    _reject("\n".join(base + ["clock 0 1", "clock 1 0", "end"]), "loop of clock registers")
    _reject("\n".join(base + ["clock 0 2", "end"]), "clock register must be 1 bit")
    _reject("\n".join(base + ["clock 2 0", "clock 2 1", "end"]), "two clock items")
    mem = ["rtlnet 1", "reg 1 0", "reg 8 0", "mem 2 8", "n reg 1 0", "n reg 8 1", "n memrd 8 0 1",
           "next 0 0", "next 1 2", "clock 1 0", "end"]
    _reject("\n".join(mem), "memory read under a divided clock")


def ripple_counter(n):
    """n toggle registers, stage i clocked by the rising edge of stage i - 1
    (stage 0 on the top clock): a ripple counter n clock domains deep."""
    nl = netgen.Netlist()
    q = [nl.add_reg(1, 0, f"q{i}") for i in range(n)]
    for i, r in enumerate(q):
        nl.set_next(r, nl.node("xor", 1, nl.node("reg", 1, r), nl.node("const", 1, 1)))
        if i:
            nl.clocks[r] = q[i - 1]
    return nl


def test_ripple_counter_counts_down():
    # stage i toggles when stage i - 1 goes 0 -> 1, within the same top cycle
    # for the whole cascade: the bits read as (-t) mod 2^n
    n = 12
    sim = oracle.Sim(oracle.Net(text=ripple_counter(n).to_text()), seed=1, inst=0)
    for t in range(5000):
        v = sum(sim.reg(i) << i for i in range(n))
        assert v == (-t) % (1 << n), t
        sim.run(1)


def gated_divider():
    """A divide-by-2 toggle whose own clock is gated by bit 0 of the 32-bit
    LFSR, and a counter on its rising edge."""
    nl = netgen.Netlist()
    chk = netgen.add_check_blocks(nl)
    d = nl.add_reg(1, 0, "div")
    nl.set_next(d, nl.node("xor", 1, nl.node("reg", 1, d), nl.node("const", 1, 1)))
    nl.gates[d] = nl.node("slice", 1, nl.node("reg", 32, chk["lfsr32"]), 0)
    c = nl.add_reg(16, 0, "cnt")
    nl.set_next(c, nl.node("add", 16, nl.node("reg", 16, c), nl.node("const", 16, 1)))
    nl.clocks[c] = d
    return nl, d, c


def test_gated_divider_counts_every_second_enabled_cycle():
    nl, d, c = gated_divider()
    sim = oracle.Sim(oracle.Net(text=nl.to_text()), seed=1, inst=0)
    s, enabled = 1, 0
    for t in range(2000):
        assert sim.reg(d) == enabled % 2
        assert sim.reg(c) == (enabled + 1) // 2          # rising edges: enabled cycles 1, 3, 5, ...
        enabled += s & 1
        s = (s >> 1) ^ (LFSR32_MASK if s & 1 else 0)
        sim.run(1)


@pytest.mark.parametrize("seed", range(6))
def test_many_cycles_match_python_evaluator_with_memories(seed):
    # larger designs (RAMs on the top clock, a divided and gated clock) over
    # many cycles with random held inputs: oracle against the Python evaluator
    from test_clocks_lowering import clocked_with_memories
    nl = clocked_with_memories(500 + seed) if seed % 2 else random_clocked_circuit(10_000 + seed)
    text = nl.to_text()
    py = PyNet(text)
    sim = oracle.Sim(oracle.Net(text=text), seed=3, inst=0)
    regs, mems = py.initial_state()
    rng = random.Random(seed)
    for t in range(25):
        ins = [rng.getrandbits(w) for w in py.inputs]
        for k, v in enumerate(ins):
            sim.hold_input(k, v)
        sim.run(1)
        regs, mems = py.cycle(regs, mems, ins)
        assert [int(x) for x in sim.regs()] == regs, (seed, t)
        assert [[sim.mem(m, a) for a in range(len(mems[m]))] for m in range(len(mems))] == mems, (seed, t)
