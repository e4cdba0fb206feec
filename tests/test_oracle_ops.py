"""Pins of the oracle's operator semantics and stimulus generator.

Each operator of the oracle is compared with a restatement in Python big
integers (results taken modulo 2**w, shifts as multiplication/floor division
by powers of two), exhaustively for small widths and on edge/random values for
wide ones.  The stimulus generator is pinned to the published SplitMix64 test
vector and to the generator's sequential definition.
"""
import os
import random

import pytest

import oracle

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def ref_op(kind, w, a, b=0, c=0, wb=0, lo=0):
    mod = 2 ** w
    if kind == "add":
        v = a + b
    elif kind == "sub":
        v = a - b                      # Python % below gives the 2-adic wrap
    elif kind == "mul":
        v = a * b
    elif kind == "and":
        v = a & b
    elif kind == "or":
        v = a | b
    elif kind == "xor":
        v = a ^ b
    elif kind == "shl":
        v = 0 if b >= 64 else a * 2 ** b
    elif kind == "shr":
        v = 0 if b >= 64 else a // 2 ** b
    elif kind == "eq":
        v = int(a == b)
    elif kind == "lt":
        v = int(a < b)
    elif kind == "mux":
        v = b if a != 0 else c
    elif kind == "slice":
        v = a // 2 ** lo
    elif kind == "concat":
        v = a * 2 ** wb + b
    else:
        raise ValueError(kind)
    return v % mod


BINARY = ("add", "sub", "mul", "and", "or", "xor", "eq", "lt")


@pytest.mark.parametrize("kind", BINARY)
def test_binary_ops_exhaustive_small(kind):
    # result widths 1..6, operands up to two bits wider than the result
    for w in range(1, 7):
        if kind in ("eq", "lt") and w != 1:
            continue
        top = 2 ** (w + 2)
        for a in range(top):
            for b in range(top):
                assert oracle.op(kind, w, a, b) == ref_op(kind, w, a, b), (kind, w, a, b)


@pytest.mark.parametrize("kind", ("shl", "shr"))
def test_shifts_exhaustive(kind):
    for w in range(1, 9):
        for a in range(256):
            for s in range(0, 71):
                assert oracle.op(kind, w, a, s) == ref_op(kind, w, a, s), (kind, w, a, s)
    # amounts far beyond the width
    for s in (64, 65, 127, 2 ** 32, 2 ** 63, M64):
        assert oracle.op(kind, 64, M64, s) == 0


def test_mux_slice_concat_exhaustive():
    for w in range(1, 7):
        for s in range(4):
            for a in range(2 ** w):
                for b in range(0, 2 ** w, max(1, 2 ** w // 8)):
                    assert oracle.op("mux", w, s, a, b) == ref_op("mux", w, s, a, b)
    for wa in range(1, 9):
        for w in range(1, wa + 1):
            for lo in range(0, wa - w + 1):
                for a in range(2 ** wa):
                    assert oracle.op("slice", w, a, lo=lo) == ref_op("slice", w, a, lo=lo)
    for wa in range(1, 6):
        for wb in range(1, 6):
            for a in range(2 ** wa):
                for b in range(2 ** wb):
                    got = oracle.op("concat", wa + wb, a, b, wb=wb)
                    assert got == ref_op("concat", wa + wb, a, b, wb=wb)


def test_wide_ops_random_and_edges():
    rng = random.Random(5)
    edges = [0, 1, 2, 3, 2 ** 31, 2 ** 32 - 1, 2 ** 32, 2 ** 63, 2 ** 63 - 1, M64, M64 - 1]
    for _ in range(20000):
        w = rng.randrange(9, 65)
        a = rng.choice(edges) if rng.randrange(3) == 0 else rng.getrandbits(64)
        b = rng.choice(edges) if rng.randrange(3) == 0 else rng.getrandbits(64)
        a &= (1 << rng.randrange(1, 65)) - 1
        for kind in ("add", "sub", "mul", "and", "or", "xor"):
            assert oracle.op(kind, w, a, b) == ref_op(kind, w, a, b), (kind, w, a, b)
        s = rng.randrange(0, 80)
        for kind in ("shl", "shr"):
            assert oracle.op(kind, w, a, s) == ref_op(kind, w, a, s)
        assert oracle.op("eq", 1, a, b) == ref_op("eq", 1, a, b)
        assert oracle.op("eq", 1, a, a) == 1
        assert oracle.op("lt", 1, a, b) == ref_op("lt", 1, a, b)
        wb = rng.randrange(1, 64)
        wa = rng.randrange(1, 65 - wb)
        x, y = a % 2 ** wa, b % 2 ** wb
        assert oracle.op("concat", wa + wb, x, y, wb=wb) == ref_op("concat", wa + wb, x, y, wb=wb)
        lo = rng.randrange(0, 64)
        ws = rng.randrange(1, 65 - lo)
        assert oracle.op("slice", ws, a, lo=lo) == ref_op("slice", ws, a, lo=lo)


def _golden_splitmix():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
    vals = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    seed = int(vals[0][1])
    return seed, [int(v[0]) for v in vals[1:]]


def test_splitmix64_published_vector():
    seed, expect = _golden_splitmix()
    got = [oracle.mix64((seed + (n + 1) * GAMMA) & M64) for n in range(len(expect))]
    assert got == expect


def test_stimulus_is_the_sequential_generator():
    # output n of the counter form equals the n-th step of the sequential
    # SplitMix64 (state += gamma; output mix(state)), restated here
    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    seed, inst, n_in = 42, 3, 5
    st = seed
    key = None
    for _ in range(inst + 1):
        st = (st + GAMMA) & M64
        key = mix(st)
    assert oracle.lib().orc_instance_key(seed, inst) == key
    st = key
    for t in range(20):
        for k in range(n_in):
            st = (st + GAMMA) & M64
            w = 1 + (7 * k + t) % 64
            assert oracle.stimulus(seed, inst, t, k, n_in, w) == mix(st) % 2 ** w
