"""GPU parity: the CUDA simulator against the oracle, bit-exact.

Every comparison is on the digest of the full state after every cycle (and
on full register dumps), for both lane mappings, all three launch schemes,
SLB and random partitions, memories, pokes and checkpoints.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim

pytestmark = pytest.mark.gpu


def oracle_digests(text_or_path, seed, inst, n, is_path=False):
    net = oracle.Net(path=text_or_path) if is_path else oracle.Net(text=text_or_path)
    s = oracle.Sim(net, seed, inst)
    return np.concatenate([np.array([s.digest()], dtype=np.uint64), s.run(n, digests=True)]), s


def oracle_many(text, seed, insts, n):
    with cf.ThreadPoolExecutor(max(1, len(insts))) as ex:
        return list(ex.map(lambda i: oracle_digests(text, seed, i, n)[0], insts))


def first_mismatch(a, b):
    bad = np.nonzero(np.asarray(a) != np.asarray(b))[0]
    return None if len(bad) == 0 else int(bad[0])


@pytest.fixture(scope="module")
def tiny_text():
    return open(netgen.cached_netlist("tiny")).read()


@pytest.fixture(scope="module")
def mid_text():
    return open(netgen.cached_netlist("mid")).read()


LOWERINGS = ["bytecode", "generated"]


@pytest.mark.parametrize("lowering", LOWERINGS)
def test_tiny_every_cycle_persistent(tiny_text, lowering):
    n = 10_000
    nl = sim.Netlist(tiny_text, mode="lane_op", digest_capacity=n + 1, lowering=lowering)
    b = sim.Batch(nl, 1, seed=42)
    b.step(n)
    b.sync()
    want, ref = oracle_digests(tiny_text, 42, 0, n)
    got = b.digests(0, 0, n + 1)
    assert first_mismatch(got, want) is None
    assert np.array_equal(b.regs(0), ref.regs())


@pytest.mark.parametrize("lowering", LOWERINGS)
@pytest.mark.parametrize("kernel", ["per_cycle", "graph", "persistent", "persistent_graph"])
def test_tiny_launch_schemes(tiny_text, kernel, lowering):
    n = 700      # not a multiple of the graph chunk
    nl = sim.Netlist(tiny_text, mode="lane_op", kernel=kernel, digest_capacity=n + 1, lowering=lowering)
    b = sim.Batch(nl, 1, seed=9)
    b.step(300)
    b.step(n - 300)
    b.sync()
    want, _ = oracle_digests(tiny_text, 9, 0, n)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None


@pytest.mark.parametrize("lowering", LOWERINGS)
def test_tiny_lane_inst_ragged_instances(tiny_text, lowering):
    # 70 instances: two full 32-lane groups and a ragged tail
    n, insts = 2000, [0, 1, 31, 32, 45, 69]
    nl = sim.Netlist(tiny_text, mode="lane_inst", digest_capacity=n + 1, lowering=lowering)
    b = sim.Batch(nl, 70, seed=5, track=insts)
    b.step(n)
    b.sync()
    wants = oracle_many(tiny_text, 5, insts, n)
    for i, want in zip(insts, wants):
        assert first_mismatch(b.digests(i, 0, n + 1), want) is None, i
    # final state digest of every instance
    ref_final = [oracle_digests(tiny_text, 5, i, n)[0][-1] for i in range(0, 70, 7)]
    assert np.array_equal(b.state_digests()[0:70:7], ref_final)


@pytest.mark.parametrize("lowering", LOWERINGS)
@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_partition_invariance(tiny_text, mode, lowering):
    n = 500
    want, _ = oracle_digests(tiny_text, 3, 0, n)
    for target, seed_part, chain in ((1, 0, 0), (5, 0, 2), (33, 7, 0), (70, 0, 2), (16, 11, 0), (16, 11, 2)):
        nl = sim.Netlist(tiny_text, mode=mode, target_processes=target, seed_partition=seed_part,
                         digest_capacity=n + 1, lowering=lowering, chain=chain)
        b = sim.Batch(nl, 32 if mode == "lane_inst" else 1, seed=3)
        b.step(n)
        b.sync()
        assert first_mismatch(b.digests(0, 0, n + 1), want) is None, (target, seed_part)


@pytest.mark.parametrize("lowering,chain", [("bytecode", 0), ("bytecode", 2), ("generated", 0)])
def test_mid_single_instance(mid_text, lowering, chain):
    n = 3000
    nl = sim.Netlist(mid_text, mode="lane_op", digest_capacity=n + 1, lowering=lowering, chain=chain)
    b = sim.Batch(nl, 1, seed=42)
    b.step(n)
    b.sync()
    want, ref = oracle_digests(mid_text, 42, 0, n)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())
    for m in range(nl.info()["n_mems"]):
        for a in (0, 1, 100, 511):
            assert b.peek_mem(0, m, a) == ref.mem(m, a)


@pytest.mark.parametrize("lowering", LOWERINGS)
def test_mid_batched_sampled(mid_text, lowering):
    n, n_inst = 300, 4096
    insts = [0, 1, 4095, 31, 32, 1000, 2047, 2048, 3071, 777, 1234, 2500, 3333, 4000, 64, 96]
    nl = sim.Netlist(mid_text, mode="lane_inst", digest_capacity=n + 1, lowering=lowering,
                     kernel="persistent_graph")
    b = sim.Batch(nl, n_inst, seed=42, track=insts)
    b.step(100)
    b.step(100)
    b.step(n - 200)
    b.sync()
    wants = oracle_many(mid_text, 42, insts, n)
    for i, want in zip(insts, wants):
        assert first_mismatch(b.digests(i, 0, n + 1), want) is None, i


def test_mid_closed_forms_at_depth(mid_text):
    # long run: embedded counter / LFSR / Fibonacci registers follow their
    # closed forms at any length (the oracle-independent check for long runs)
    from test_oracle_closed_forms import fib_pair, galois_matrix, gf2_apply, gf2_pow, mac_closed
    names = netgen.parse_names(mid_text)
    n = 20_000
    nl = sim.Netlist(mid_text, mode="lane_op")
    b = sim.Batch(nl, 1, seed=42)
    b.step(n)
    b.sync()
    assert b.peek_reg(0, names["chk_counter16"]) == n % 65536
    assert b.peek_reg(0, names["chk_fib_a"]) == fib_pair(n)[0]
    assert b.peek_reg(0, names["chk_mac"]) == mac_closed(n)
    assert b.peek_reg(0, names["chk_lfsr32"]) == gf2_apply(gf2_pow(galois_matrix(netgen.LFSR32_MASK), n), 1)


@pytest.mark.parametrize("cfg", [{}, dict(cluster_size=8, warps_per_cta=1, target_processes=8),
                                 dict(cluster_size=2, warps_per_cta=2, target_processes=8)],
                         ids=["grid_barrier", "one_cluster", "two_clusters"])
def test_poke_peek_and_checkpoint(tiny_text, cfg):
    n = 200
    nl = sim.Netlist(tiny_text, mode="lane_op", digest_capacity=1000, **cfg)
    b = sim.Batch(nl, 1, seed=4)
    ref = oracle.Sim(oracle.Net(text=tiny_text), seed=4, inst=0)
    b.step(n)
    ref.run(n)
    # register poke, input hold
    b.poke_reg(0, 3, 0xDEADBEEF)
    ref.set_reg(3, 0xDEADBEEF)
    b.hold_input(0, 2, 0x1234)
    ref.hold_input(2, 0x1234)
    from pyeval import PyNet
    w_in = PyNet(tiny_text).inputs[2]
    assert b.peek(0, sim.SIM_SIG_INPUT, 2) == 0x1234 % 2 ** w_in
    blob = b.save()
    b.step(150)
    ref.run(150)
    assert np.array_equal(b.regs(0), ref.regs())
    d_after = b.state_digests()[0]
    assert d_after == ref.digest()
    # restore and replay: same result
    b.restore(blob)
    b.step(150)
    assert b.state_digests()[0] == d_after
    b.unpoke(0, 2)
    ref.release_input(2)
    b.step(50)
    ref.run(50)
    assert np.array_equal(b.regs(0), ref.regs())


@pytest.mark.parametrize("kernel", ["per_cycle", "graph", "persistent", "persistent_graph"])
def test_held_inputs_generated(tiny_text, kernel):
    # generated code reads its inputs from a buffer filled one cycle ahead:
    # holds set and released between steps, steps that end inside a graph
    # chunk, and instances with and without holds all match the oracle
    nl = sim.Netlist(tiny_text, mode="lane_inst", lowering="generated", kernel=kernel)
    b = sim.Batch(nl, 64, seed=9)
    net = oracle.Net(text=tiny_text)
    refs = {i: oracle.Sim(net, seed=9, inst=i) for i in (0, 5, 40, 63)}

    def step(n):
        b.step(n)
        for r in refs.values():
            r.run(n)
        got = b.state_digests()
        for i, r in refs.items():
            assert got[i] == r.digest(), (kernel, i)

    step(70)
    b.hold_input(5, 2, 0x1234)
    refs[5].hold_input(2, 0x1234)
    b.hold_input(40, 0, 0xFFFFFFFFFFFFFFFF)
    refs[40].hold_input(0, 0xFFFFFFFFFFFFFFFF)
    step(131)
    b.unpoke(5, 2)
    refs[5].release_input(2)
    step(1)
    step(64)
    for i, r in refs.items():
        assert np.array_equal(b.regs(i), r.regs()), (kernel, i)


@pytest.mark.parametrize("lowering", LOWERINGS)
def test_memory_poke_and_rom(lowering):
    text = """rtlnet 1
reg 8 0 c
reg 16 0 q
reg 16 0 rom
mem 4 16
mem 3 16
n reg 8 0
n const 8 1
n add 8 0 1
n memrd 16 0 0
n const 1 1
n concat 16 0 0
n memrd 16 1 0
next 0 2
next 1 3
next 2 6
wport 0 4 0 5
minit 1 5 4242
minit 0 3 7
end
"""
    cases = [("lane_op", 1, {}), ("lane_inst", 33, {})]
    if lowering == "bytecode":      # cluster exchange runs the bytecode
        cases.append(("lane_op", 1, dict(cluster_size=2, warps_per_cta=1, target_processes=2)))
    for mode, n_inst, extra in cases:
        nl = sim.Netlist(text, mode=mode, digest_capacity=400, lowering=lowering, **extra)
        b = sim.Batch(nl, n_inst, seed=1, track=[0, n_inst - 1])
        ref = oracle.Sim(oracle.Net(text=text), seed=1, inst=0)
        want = [ref.digest()]
        for t in range(60):
            if t == 20:
                b.poke_mem(0, 0, 9, 999)
                ref.set_mem(0, 9, 999)
            b.step(1)
            ref.run(1)
            want.append(ref.digest())
            assert np.array_equal(b.regs(0), ref.regs()), (mode, t)
        got = b.digests(0, 0, 61)
        assert first_mismatch(got, np.array(want, dtype=np.uint64)) is None


@pytest.mark.parametrize("lowering", LOWERINGS)
def test_degenerate_netlists(lowering):
    cases = [
        # one register, no inputs, next = itself
        "rtlnet 1\nreg 64 12345\nn reg 64 0\nnext 0 0\nend\n",
        # constant next value, 1-bit register
        "rtlnet 1\nreg 1 1\nn const 1 0\nnext 0 0\nend\n",
        # 64-bit concat/slice edges, shifts by >= 64
        "rtlnet 1\nin 64\nreg 64 1\nreg 32 0\nn reg 64 0\nn input 64 0\nn slice 32 1 32\nn slice 32 0 0\n"
        "n concat 64 2 3\nn shl 64 0 1\nn xor 64 4 5\nn const 7 64\nn shr 64 1 7\nn add 64 6 8\nn slice 32 9 16\n"
        "next 0 9\nnext 1 10\nend\n",
    ]
    for text in cases:
        for mode, n_inst in (("lane_op", 1), ("lane_inst", 32)):
            n = 100
            nl = sim.Netlist(text, mode=mode, digest_capacity=n + 1, lowering=lowering)
            b = sim.Batch(nl, n_inst, seed=8)
            b.step(n)
            b.sync()
            want, ref = oracle_digests(text, 8, 0, n)
            assert first_mismatch(b.digests(0, 0, n + 1), want) is None, (text, mode)


@pytest.mark.parametrize("lowering", LOWERINGS)
def test_barrier_timeout_is_reported(tiny_text, lowering):
    # one CTA skips its arrival: the others' bounded waits expire and the
    # step reports SIM_ERR_TIMEOUT (no fault, no unbounded wait)
    nl = sim.Netlist(tiny_text, mode="lane_op", warps_per_cta=1, lowering=lowering)
    b = sim.Batch(nl, 1, seed=1)
    b.step(5)
    blob = b.save()
    b.debug_skip_arrival(20)
    b.step(10)
    with pytest.raises(sim.SimError) as e:
        b.sync()
    assert e.value.name == "SIM_ERR_TIMEOUT"
    # the failed launch left the state part-way through a cycle: the batch
    # refuses to go on until a checkpoint is restored
    for call in (lambda: b.step(1), b.sync, b.state_digests, lambda: b.regs(0)):
        with pytest.raises(sim.SimError) as e:
            call()
        assert e.value.name == "SIM_ERR_STATE"
    b.restore(blob)
    b.step(95)          # the configured (long) barrier wait applies again
    b.sync()
    want, ref = oracle_digests(tiny_text, 1, 0, 100)
    assert b.state_digests()[0] == want[-1]
    assert np.array_equal(b.regs(0), ref.regs())


def test_mesh_single_instance():
    # the 2M-op 4x4 mesh: every cycle of a prefix against the oracle, then the
    # closed-form registers after a longer run
    from test_oracle_closed_forms import fib_pair, mac_closed
    path = netgen.cached_netlist("mesh")
    text = open(path).read()
    n = 200
    nl = sim.Netlist(text, mode="lane_op", digest_capacity=n + 1)
    b = sim.Batch(nl, 1, seed=42)
    b.step(n)
    b.sync()
    want, ref = oracle_digests(path, 42, 0, n, is_path=True)
    assert first_mismatch(b.digests(0, 0, n + 1), want) is None
    assert np.array_equal(b.regs(0), ref.regs())
    names = netgen.parse_names(text)
    b.step(4800)
    b.sync()
    assert b.peek_reg(0, names["chk_counter16"]) == 5000
    assert b.peek_reg(0, names["chk_fib_b"]) == fib_pair(5000)[1]
    assert b.peek_reg(0, names["chk_mac"]) == mac_closed(5000)


def test_mesh_batched_sampled():
    path = netgen.cached_netlist("mesh")
    text = open(path).read()
    n, insts = 40, [0, 63, 17]
    nl = sim.Netlist(text, mode="lane_inst", target_processes=2432, digest_capacity=n + 1)
    b = sim.Batch(nl, 64, seed=3, track=insts)
    b.step(n)
    b.sync()
    wants = [oracle_digests(path, 3, i, n, is_path=True)[0] for i in insts]
    for i, want in zip(insts, wants):
        assert first_mismatch(b.digests(i, 0, n + 1), want) is None, i


def test_batches_with_different_shared_memory_coexist(tiny_text, mid_text):
    # the kernel's shared-memory limit is process-wide: creating a batch that
    # needs less must not break a batch that needs more
    big = sim.Batch(sim.Netlist(mid_text, mode="lane_inst", target_processes=256), 64, seed=1)
    small = sim.Batch(sim.Netlist(tiny_text, mode="lane_inst"), 32, seed=1)
    big.step(3)
    small.step(3)
    big.sync()
    small.sync()
    ref = oracle.Sim(oracle.Net(text=mid_text), 1, 0)
    ref.run(3)
    assert big.state_digests()[0] == ref.digest()


def test_measured_int_peak_is_plausible():
    # the integer issue rate: at most one warp instruction per SM sub-partition
    # and clock (152 SMs x 4 x 32 lanes x ~2.07 GHz = 40.3 T lane-ops/s)
    v = sim.measure_int_peak(1 << 12)
    assert 5e12 < v < 45e12, v
