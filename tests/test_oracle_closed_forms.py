"""Closed-form pins of the oracle's cycle semantics.

The check blocks embedded in every generated netlist (16-bit counter, 16- and
32-bit Galois LFSRs, Fibonacci pair, multiply-accumulate) have traces with
closed forms that do not depend on the oracle: these tests run the oracle on
the seeded tiny netlist and compare its register values with them, which pins
the register commit (current/next split, paper Sec. 3.2) and the arithmetic.
"""
import pytest

import oracle
from paper_2403_04714_gb300 import netgen

M64 = (1 << 64) - 1


def fib_pair(n):
    """(F(n), F(n+1)) mod 2^64 by fast doubling."""
    if n == 0:
        return 0, 1
    a, b = fib_pair(n >> 1)
    c = (a * ((2 * b - a) % 2 ** 64)) % 2 ** 64
    d = (a * a + b * b) % 2 ** 64
    return (d, (c + d) % 2 ** 64) if n & 1 else (c, d)


def gf2_matmul(A, B):
    """32x32 GF(2) matrices as lists of row bitmasks."""
    out = []
    for row in A:
        acc = 0
        j = 0
        while row:
            if row & 1:
                acc ^= B[j]
            row >>= 1
            j += 1
        out.append(acc)
    return out


def gf2_pow(M, e, n=32):
    R = [1 << i for i in range(n)]
    while e:
        if e & 1:
            R = gf2_matmul(R, M)
        M = gf2_matmul(M, M)
        e >>= 1
    return R


def gf2_apply(M, v):
    out = 0
    for i, row in enumerate(M):
        out |= (bin(row & v).count("1") & 1) << i
    return out


def galois_matrix(mask, n=32):
    """Companion matrix of s' = (s >> 1) ^ (s_0 ? mask : 0): row i = bits feeding bit i."""
    rows = []
    for i in range(n):
        r = 0
        if i + 1 < n:
            r |= 1 << (i + 1)         # bit i <- bit i+1 (shift right)
        if mask >> i & 1:
            r |= 1                    # bit i <- bit 0 when the tap is set
        rows.append(r)
    return rows


def test_lfsr32_polynomial_is_maximal():
    # the state matrix has multiplicative order exactly 2^32-1
    M = galois_matrix(netgen.LFSR32_MASK)
    I = [1 << i for i in range(32)]
    order = 2 ** 32 - 1
    assert gf2_pow(M, order) == I
    for p in (3, 5, 17, 257, 65537):
        assert gf2_pow(M, order // p) != I


def mac_closed(t):
    q, r = divmod(t, 1 << 16)
    s = q * ((1 << 16) * ((1 << 16) - 1) // 2) + r * (r - 1) // 2
    return (netgen.MAC_K * s) % 2 ** 64


@pytest.fixture(scope="module")
def tiny(netcache):
    path = netgen.cached_netlist("tiny", cache_dir=netcache)
    names = netgen.parse_names(open(path).read())
    return path, names


def test_check_blocks_every_cycle(tiny):
    path, names = tiny
    net = oracle.Net(path)
    sim = oracle.Sim(net, seed=42, inst=0)
    M = galois_matrix(netgen.LFSR32_MASK)
    c, l32, fa, fb, mac = (names["chk_counter16"], names["chk_lfsr32"], names["chk_fib_a"],
                           names["chk_fib_b"], names["chk_mac"])
    for t in range(0, 10_001):
        if t:
            sim.run(1)
        assert sim.reg(c) == t % 65536
        a, b = fib_pair(t)
        assert sim.reg(fa) == a and sim.reg(fb) == b
        assert sim.reg(mac) == mac_closed(t)
        if t % 250 == 0 or t == 10_000:
            assert sim.reg(l32) == gf2_apply(gf2_pow(M, t), 1), t


def test_lfsr16_period_by_brute_force(tiny):
    path, names = tiny
    net = oracle.Net(path)
    sim = oracle.Sim(net, seed=1, inst=0)
    r = names["chk_lfsr16"]
    s0 = sim.reg(r)
    seen = {s0}
    for t in range(1, 65535):
        sim.run(1)
        v = sim.reg(r)
        assert v != s0, t
        seen.add(v)
    sim.run(1)
    assert sim.reg(r) == s0
    assert len(seen) == 65535 and 0 not in seen


def test_long_run_closed_forms(tiny):
    # counter/LFSR/Fibonacci/MAC after 100k cycles in one call
    path, names = tiny
    sim = oracle.Sim(oracle.Net(path), seed=7, inst=3)
    sim.run(100_000)
    t = 100_000
    assert sim.reg(names["chk_counter16"]) == t % 65536
    assert sim.reg(names["chk_fib_a"]) == fib_pair(t)[0]
    assert sim.reg(names["chk_mac"]) == mac_closed(t)
    M = galois_matrix(netgen.LFSR32_MASK)
    assert sim.reg(names["chk_lfsr32"]) == gf2_apply(gf2_pow(M, t), 1)
