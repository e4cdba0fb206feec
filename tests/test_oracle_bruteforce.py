"""Brute-force and semantic pins of the oracle.

* Tiny random circuits (at most 14 bits of register, memory and input state):
  for every state and input, one oracle step (next registers, next memory,
  every node value) equals the independent Python evaluator in pyeval.py.
* The seeded tiny workload: its first cycles equal the Python evaluator driven
  with the same inputs.
* Memory semantics with closed forms: read-before-write at the clock edge,
  highest write port wins, address wrap, initial images.
* Loader rejections: combinational loop (paper Sec. 5.3), width and slice
  errors.
"""
import itertools
import random

import pytest

import oracle
from paper_2403_04714_gb300 import netgen
from pyeval import PyNet


def random_tiny_circuit(seed):
    """A random circuit over 2 inputs, 3 registers and one 4x2-bit memory."""
    rng = random.Random(seed)
    nl = netgen.Netlist()
    i0, i1 = nl.add_input(2), nl.add_input(2)
    regs = [nl.add_reg(w, rng.randrange(2 ** w)) for w in (3, 2, 1)]
    m = nl.add_mem(2, 2)
    pool = [nl.node("input", 2, i0), nl.node("input", 2, i1)]
    pool += [nl.node("reg", nl.regs[r][0], r) for r in regs]
    pool.append(nl.node("const", 3, rng.randrange(8)))
    pool.append(nl.node("memrd", 2, m, pool[rng.randrange(len(pool))]))
    for _ in range(rng.randrange(10, 24)):
        kind = rng.choice(netgen.ALL_OPS)
        a = pool[rng.randrange(len(pool))]
        b = pool[rng.randrange(len(pool))]
        wa, wb = nl.width(a), nl.width(b)
        if kind in ("eq", "lt"):
            n = nl.node(kind, 1, a, b)
        elif kind == "mux":
            n = nl.node("mux", rng.randrange(1, 6), a, b, pool[rng.randrange(len(pool))])
        elif kind == "slice":
            w = rng.randrange(1, wa + 1)
            n = nl.node("slice", w, a, rng.randrange(wa - w + 1))
        elif kind == "concat":
            if wa + wb > 64:
                continue
            n = nl.node("concat", wa + wb, a, b)
        elif kind in ("shl", "shr"):
            n = nl.node(kind, rng.randrange(1, 7), a, b)
        else:
            n = nl.node(kind, rng.randrange(1, 7), a, b)
        pool.append(n)
    for r in regs:
        nl.set_next(r, pool[rng.randrange(len(pool))])
    for _ in range(2):   # two write ports: exercises port priority
        nl.wports.append((m, pool[rng.randrange(len(pool))], pool[rng.randrange(len(pool))],
                          pool[rng.randrange(len(pool))]))
    return nl


@pytest.mark.parametrize("seed", range(12))
def test_one_step_matches_python_evaluator_for_every_state(seed):
    nl = random_tiny_circuit(seed)
    text = nl.to_text()
    py = PyNet(text)
    net = oracle.Net(text=text)
    sim = oracle.Sim(net, seed=1, inst=0)
    # state bits: regs 3+2+1, memory 4x2 = 8 -> 14 bits; inputs 2+2 (every
    # memory image is sampled, the rest is exhaustive)
    rng = random.Random(seed)
    mem_images = [[rng.randrange(4) for _ in range(4)] for _ in range(6)] + [[0, 1, 2, 3]]
    for mem in mem_images:
        for r0, r1, r2, x0, x1 in itertools.product(range(8), range(4), range(2), range(4), range(4)):
            regs = [r0, r1, r2]
            for r, v in enumerate(regs):
                sim.set_reg(r, v)
            for a, v in enumerate(mem):
                sim.set_mem(0, a, v)
            sim.hold_input(0, x0)
            sim.hold_input(1, x1)
            sim.run(1)
            exp_regs, exp_mems, vals = py.step(regs, [mem], [x0, x1])
            assert [sim.reg(r) for r in range(3)] == exp_regs, (seed, regs, mem, x0, x1)
            assert [sim.mem(0, a) for a in range(4)] == exp_mems[0]
            for i, v in vals.items():
                assert sim.node_value(i) == v, (seed, i, nl.nodes[i])


def test_tiny_workload_first_cycles_match_python_evaluator(netcache):
    path = netgen.cached_netlist("tiny", cache_dir=netcache)
    text = open(path).read()
    py = PyNet(text)
    sim = oracle.Sim(oracle.Net(path), seed=42, inst=0)
    regs, mems = py.initial_state()
    n_in = len(py.inputs)
    for t in range(60):
        ins = [oracle.stimulus(42, 0, t, k, n_in, w) for k, w in enumerate(py.inputs)]
        regs, mems, _ = py.step(regs, mems, ins)
        sim.run(1)
        assert list(sim.regs()) == regs, t


def _counter_mem_net(wport_lines, read_addr="c", extra=""):
    return f"""rtlnet 1
reg 8 0 c
reg 8 0 q
mem 4 8
n reg 8 0
n const 8 1
n add 8 0 1
n memrd 8 0 0
n const 1 1
n const 8 100
n add 8 0 5
n slice 1 0 0
{extra}next 0 2
next 1 3
{wport_lines}end
"""


def test_memory_read_before_write():
    # write c at address c mod 16 every cycle; q <= mem[c mod 16] (sync read).
    # Writes land at the clock edge, so the read sees the value written 16
    # cycles earlier: q_{t+1} = (t-16) mod 256 for t >= 16, else 0.
    text = _counter_mem_net("wport 0 4 0 0\n")
    sim = oracle.Sim(oracle.Net(text=text))
    for t in range(600):
        sim.run(1)
        expect = (t - 16) % 256 if t >= 16 else 0
        assert sim.reg(1) == expect, t


def test_memory_highest_port_wins():
    # port 0 always writes c at address c; port 1 writes c+100 at the same
    # address on odd c; q <= mem[c]: q_{t+1} = mem_t[c_t], written 16 cycles before
    text = _counter_mem_net("wport 0 4 0 0\nwport 0 7 0 6\n")
    sim = oracle.Sim(oracle.Net(text=text))
    for t in range(600):
        sim.run(1)
        if t < 16:
            expect = 0
        else:
            tw = t - 16
            expect = (tw + 100) % 256 if tw % 2 else tw % 256
        assert sim.reg(1) == expect, t


def test_memory_address_wraps_and_initial_image():
    text = """rtlnet 1
reg 8 0 q
mem 2 8
n const 8 6
n memrd 8 0 0
next 0 1
minit 0 2 77
end
"""
    sim = oracle.Sim(oracle.Net(text=text))
    sim.run(1)
    assert sim.reg(0) == 77          # address 6 wraps to 2 in a 4-word memory


@pytest.mark.parametrize("text,msg", [
    ("rtlnet 1\nreg 4 0\nn add 4 1 2\nn reg 4 0\nn add 4 0 1\nnext 0 0\nend\n", "loop"),
    ("rtlnet 1\nreg 4 0\nn reg 4 0\nn slice 4 0 1\nnext 0 1\nend\n", "slice"),
    ("rtlnet 1\nreg 4 0\nn reg 4 0\nn concat 7 0 0\nnext 0 1\nend\n", "concat"),
    ("rtlnet 1\nreg 4 0\nn reg 4 0\nn eq 2 0 0\nnext 0 1\nend\n", "compare"),
    ("rtlnet 1\nreg 4 0\nn reg 4 0\nend\n", "next"),
    ("rtlnet 1\nreg 65 0\nn reg 65 0\nnext 0 0\nend\n", "width"),
    ("rtlnet 2\nend\n", "rtlnet"),
    ("rtlnet 1\nreg 4 0\nn reg 4 0\nn frob 4 0 0\nnext 0 0\nend\n", "unknown op"),
])
def test_loader_rejects(text, msg):
    with pytest.raises(oracle.OracleError, match=msg):
        oracle.Net(text=text)
