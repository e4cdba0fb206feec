"""Pins of the oracle's state digest (orc_sim_digest).

Every per-cycle parity claim compares the GPU's digest with the oracle's, so
the oracle's digest must be pinned to something other than itself.  The
digest is a definition of this project (the paper has none; it supports the
current/next state split of Sec. 3.2 being checked cycle by cycle):

    D(S) = sum over registers r of mix(H(r) ^ reg[r])
         + sum over memories m and words a of mix(H(2^40 + m 2^24 + a) ^ mem[m][a])   (mod 2^64)
    H(x) = x * 0x9E3779B97F4A7C15 + 1 (mod 2^64),  mix = the SplitMix64 output function.

Here it is recomputed in Python big integers from the oracle's dumped
registers and memory words, with mix written from its published definition
(Steele, Lea, Flood 2014) and pinned by the published SplitMix64 vector.
A second property checks that the digest moves by exactly one term when one
register or one memory word changes, which fails for a digest that skips a
word, hashes a word under the wrong index, or counts a word twice.
"""
import os
import random

import pytest

import oracle
from paper_2403_04714_gb300 import netgen

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def py_mix(z):
    # SplitMix64 output function, from its published definition
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def py_hash(x):
    return (x * GAMMA + 1) & M64


def reg_term(r, v):
    return py_mix(py_hash(r) ^ v)


def mem_term(m, a, v):
    return py_mix(py_hash((1 << 40) + (m << 24) + a) ^ v)


def py_digest(regs, mems):
    d = 0
    for r, v in enumerate(regs):
        d += reg_term(r, int(v))
    for m, words in enumerate(mems):
        for a, v in enumerate(words):
            d += mem_term(m, a, int(v))
    return d & M64


def dump(s):
    return s.regs(), [s.mem_all(m) for m in range(s.net.n_mem)]


def test_python_mix_is_splitmix64():
    # the published SplitMix64 vector (tests/golden), stream seeded 1234567
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
    vals = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    seed = int(vals[0][1])
    want = [int(v[0]) for v in vals[1:]]
    assert [py_mix((seed + (n + 1) * GAMMA) & M64) for n in range(len(want))] == want


# a design with a ROM (a memory without write ports and with an initial
# image), a RAM with two write ports, and registers of several widths
ROM_RAM = """rtlnet 1
in 8
in 3
reg 8 0 c
reg 16 0 q
reg 16 0 rom_q
reg 1 1 b
reg 64 18446744073709551615 w
mem 4 16 ram
mem 3 16 rom
mem 2 64 ram2
n reg 8 0
n const 8 1
n add 8 0 1
n memrd 16 0 0
n const 1 1
n concat 16 0 0
n input 3 1
n memrd 16 1 6
n reg 1 3
n xor 1 8 4
n reg 64 4
n input 8 0
n mul 64 10 11
n memrd 64 2 6
n add 64 12 13
n slice 2 0 0
next 0 2
next 1 3
next 2 7
next 3 9
next 4 14
wport 0 4 0 5
wport 0 8 6 3
wport 2 8 15 12
minit 1 5 4242
minit 1 0 17
minit 1 7 65535
minit 0 3 7
minit 2 1 123456789123
end
"""


def _designs():
    return {"tiny": open(netgen.cached_netlist("tiny")).read(),
            "mid": open(netgen.cached_netlist("mid")).read(),
            "rom_ram": ROM_RAM}


@pytest.mark.parametrize("name,cycles", [("tiny", (0, 1, 2, 10, 100, 537)), ("mid", (0, 1, 7)),
                                         ("rom_ram", (0, 1, 2, 10, 100, 300))])
def test_digest_is_the_definition(name, cycles):
    text = _designs()[name]
    net = oracle.Net(text=text)
    s = oracle.Sim(net, seed=42, inst=3)
    done = 0
    for c in cycles:
        s.run(c - done)
        done = c
        regs, mems = dump(s)
        assert len(regs) == net.n_reg and len(mems) == net.n_mem
        assert s.digest() == py_digest(regs, mems), (name, c)


@pytest.mark.parametrize("name", ["tiny", "rom_ram"])
def test_digest_moves_by_one_term(name):
    text = _designs()[name]
    net = oracle.Net(text=text)
    s = oracle.Sim(net, seed=9, inst=0)
    s.run(25)
    rng = random.Random(5)
    regs = list(range(net.n_reg))
    picks = sorted(set([0, net.n_reg - 1] + rng.sample(regs, min(24, net.n_reg))))
    for r in picks:
        old = s.reg(r)
        d0 = s.digest()
        new = rng.getrandbits(64)
        s.set_reg(r, new)
        new = s.reg(r)                  # reduced to the register's width
        assert (s.digest() - d0) & M64 == (reg_term(r, new) - reg_term(r, old)) & M64, r
        s.set_reg(r, old)
        assert s.digest() == d0
    for m in range(net.n_mem):
        depth = net.mem_depth(m)
        for a in sorted(set([0, depth - 1] + [rng.randrange(depth) for _ in range(6)])):
            old = s.mem(m, a)
            d0 = s.digest()
            s.set_mem(m, a, rng.getrandbits(64))
            new = s.mem(m, a)
            assert (s.digest() - d0) & M64 == (mem_term(m, a, new) - mem_term(m, a, old)) & M64, (m, a)
            s.set_mem(m, a, old)
            assert s.digest() == d0


def test_digest_tells_registers_apart():
    # swapping the values of two registers changes the digest (each term is
    # keyed by its register's index), unless the values are equal
    net = oracle.Net(text=ROM_RAM)
    s = oracle.Sim(net, seed=1, inst=0)
    s.set_reg(1, 5)
    s.set_reg(2, 6)
    d = s.digest()
    s.set_reg(1, 6)
    s.set_reg(2, 5)
    assert s.digest() != d
    s.set_reg(2, 6)
    assert s.digest() == py_digest(*dump(s))
