"""Serving with continuous batching: each job's results are the same alone and
in the mix (bit-exact), and equal the oracle for small jobs; admission by
device-memory footprint."""
import concurrent.futures as cf
import time

import numpy as np
import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim

pytestmark = pytest.mark.gpu


def solo(netlist_text, n_inst, seed, cycles):
    nl = sim.Netlist(netlist_text, mode="lane_inst" if n_inst >= 32 else "lane_op")
    b = sim.Batch(nl, n_inst, seed=seed)
    b.step(cycles)
    return b.state_digests()


def oracle_final(text, seed, inst, cycles):
    s = oracle.Sim(oracle.Net(text=text), seed, inst)
    s.run(cycles)
    return s.digest()


@pytest.fixture(scope="module")
def nets():
    tiny = open(netgen.cached_netlist("tiny")).read()
    flat = netgen.gen_flat(77, n_ops=5000, n_regs=400, depth=18, n_inputs=6, rams=((6, 64),)).to_text()
    return {"tiny": tiny, "flat": flat}


@pytest.mark.parametrize("persistent", [1, 0], ids=["persistent_pools", "per_cycle_pools"])
def test_jobs_alone_and_in_the_mix(nets, persistent):
    handles = {k: sim.Netlist(v) for k, v in nets.items()}
    srv = sim.Server(pool_slots=256, chunk_cycles=97, persistent=persistent)
    # (netlist, instances, seed, cycles, submit delay): arrivals overlap running jobs
    jobs = [("tiny", 1, 5, 1000, 0.0), ("flat", 40, 6, 700, 0.0), ("tiny", 33, 7, 2500, 0.01),
            ("tiny", 3, 8, 300, 0.02), ("flat", 1, 9, 1234, 0.03), ("tiny", 100, 10, 600, 0.05),
            ("flat", 7, 11, 50, 0.06), ("tiny", 1, 12, 1, 0.07)]
    ids = []
    t0 = time.time()
    for name, n, seed, cyc, delay in jobs:
        while time.time() - t0 < delay:
            time.sleep(0.001)
        ids.append(srv.submit(handles[name], n, seed, cyc))
    for jid in ids:
        srv.wait(jid)
    for (name, n, seed, cyc, _), jid in zip(jobs, ids):
        st = srv.poll(jid)
        assert st["state"] == "done" and st["cycles_done"] == cyc
        got = srv.digests(jid, n)
        assert np.array_equal(got, solo(nets[name], n, seed, cyc)), (name, n, seed)
    # oracle parity of the small jobs' sampled instances
    checks = [(name, seed, i, cyc, jid) for (name, n, seed, cyc, _), jid in zip(jobs, ids)
              for i in sorted({0, n - 1}) if n * cyc <= 60_000]
    with cf.ThreadPoolExecutor(8) as ex:
        want = list(ex.map(lambda c: oracle_final(nets[c[0]], c[1], c[2], c[3]), checks))
    for (name, seed, i, cyc, jid), w in zip(checks, want):
        n = srv.poll(jid)["n_inst"]
        assert srv.digests(jid, n)[i] == w, (name, seed, i)
    assert srv.stats()["instance_cycles"] >= sum(n * c for _, n, _, c, _ in jobs)
    srv.close()


def test_admission_under_a_tight_cap(nets):
    a, b = sim.Netlist(nets["tiny"]), sim.Netlist(nets["flat"])
    # a cap that holds one pool at a time: the two netlists' jobs take turns
    fa, fb = sim.Server.footprint(a, 64), sim.Server.footprint(b, 64)
    assert max(fa, fb) < fa + fb
    srv = sim.Server(pool_slots=64, chunk_cycles=50, hbm_cap_bytes=max(fa, fb) + 1024)
    ids = [srv.submit(a, 5, 1, 200), srv.submit(b, 5, 2, 200), srv.submit(a, 2, 3, 100)]
    for jid in ids:
        srv.wait(jid)
        assert srv.poll(jid)["state"] == "done"
    assert np.array_equal(srv.digests(ids[1], 5), solo(nets["flat"], 5, 2, 200))
    with pytest.raises(sim.SimError) as e:
        srv.submit(b, 100_000, 1, 10)
    assert e.value.name == "SIM_ERR_ADMISSION"
    srv.close()


def test_pool_of_a_cluster_lowered_netlist(nets):
    # a netlist loaded for cluster exchange (one instance) still serves
    # multi-instance jobs: pools run its lane = instance program
    nl = sim.Netlist(nets["tiny"], mode="lane_op", cluster_size=2, warps_per_cta=2, target_processes=8)
    srv = sim.Server(pool_slots=64, chunk_cycles=64)
    jid = srv.submit(nl, 40, 21, 300)
    srv.wait(jid)
    assert srv.poll(jid)["state"] == "done"
    assert np.array_equal(srv.digests(jid, 40), solo(nets["tiny"], 40, 21, 300))
    srv.close()


def test_job_admitted_while_a_persistent_step_runs(nets):
    # a long job keeps its pool stepping (one persistent launch per 2,000
    # cycles); jobs of the same netlist that arrive meanwhile join the pool at
    # the next step boundary and overlap the long one, and every result equals
    # the same job run alone
    nl = sim.Netlist(nets["tiny"])
    srv = sim.Server(pool_slots=256, chunk_cycles=2000, persistent=1)
    long_id = srv.submit(nl, 64, 31, 60_000)
    t0 = time.time()
    while srv.poll(long_id)["cycles_done"] < 2000 and time.time() - t0 < 60:
        time.sleep(0.001)
    late = [srv.submit(nl, 5, 32, 3000), srv.submit(nl, 40, 33, 1500)]
    for jid in late:
        srv.wait(jid)
    assert srv.poll(long_id)["state"] == "running"          # the late jobs finished inside the long one
    srv.wait(long_id)
    st_long = srv.poll(long_id)
    for jid, (n, seed, cyc) in zip(late, ((5, 32, 3000), (40, 33, 1500))):
        st = srv.poll(jid)
        assert st["state"] == "done" and st_long["t_start"] < st["t_start"] < st["t_done"] < st_long["t_done"]
        assert np.array_equal(srv.digests(jid, n), solo(nets["tiny"], n, seed, cyc))
    assert np.array_equal(srv.digests(long_id, 64), solo(nets["tiny"], 64, 31, 60_000))
    srv.close()
