"""Benchmark: simulated cycles per second of the BSP RTL simulator on GB300.

Headline workload: the mid netlist (200k ops, 20k registers: 30% 1-bit,
40% 32-bit, 30% 64-bit, depth 60, two 512x64-bit synchronous RAMs), one
instance, 100,000 simulated cycles, persistent kernel; partition size, warps
per CTA and thread-block-cluster exchange picked by the autotuner.
A step is one sim_step of `--cycles` simulated cycles (default 10,000), so
the default 10 timed steps simulate the full 100k-cycle workload.

Also reported in the same JSON line (`rows`): the launch-per-cycle baseline
and its CUDA-graph replay on the same workload, and the batched workload
(the same netlist x 4,096 independently seeded instances, lane = instance).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--cycles C] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "simulated cycles/s (1 instance) and instance-cycles/s (batched), p50/p99 job latency"
UNIT = "simulated cycles/s"
# bytes of one instance's register state (1-bit packed, 32-bit and 64-bit planes)
STATE_BYTES_MID = 6126 / 8 + 7955 * 4 + 5927 * 8
# dram__bytes_read.sum + dram__bytes_write.sum of one 10,000-cycle launch of
# the headline kernel (ncu, 1 pass): the one-time program and table load; the
# per-cycle exchange stays in L2 (capture: ncu --metrics dram__bytes_read.sum,
# dram__bytes_write.sum -k regex:k_cycles -s 1 -c 1 on `bench.py --no-rows
# --steps 2 --warmup 1`, operator pairs in 2-CTA clusters, hypergraph partition)
HEADLINE_TRAFFIC = 5.218e6 + 0.104e6
HBM_PEAK_GBS = 6790.0       # overwritten from MEASURED_PEAKS.json when present
WORKLOAD = ("mid netlist: 200k ops, 20k registers (30% 1b / 40% 32b / 30% 64b), depth 60, "
            "fan-out power law (alpha 2, max 512), two 512x64b synchronous RAMs; 1 instance, "
            "100k cycles; persistent kernel, autotuned geometry (grid barrier, optional cluster exchange)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# Integer ALU peak (no measured integer peak in the driver's file): 152 SMs x
# 4 sub-partitions x 16 lanes per clock of the integer ALU pipe (IADD3, LOP3,
# SHF, ISETP, SEL: half a warp instruction per clock per sub-partition, as the
# pipe utilisation ncu reports for the interpreter confirms) at the maximum SM
# clock.  bench also reports sim_measure_int_peak beside it.
def alu_peak_ops(p):
    return 152 * 4 * 16 * float(p.get("sm_max_mhz", 2070.0)) * 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return dist.get_rank(), dist.get_world_size(), local, dist


def barrier(dist):
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if dist:
        dist.barrier()


def max_over_ranks(dist, x):
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(dist, world, units_per_rank, seconds):
    """Whole-job rate of N independent replicas (weak scaling, no data-path
    collective): the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(dist, seconds)


def time_steps(batch, stream, steps, warmup, cycles, flush):
    """Device-timed steps (CUDA events on the batch's stream), L2 flushed between steps."""
    import torch
    for _ in range(warmup):
        batch.step(cycles)
    batch.sync()
    ms = []
    k0 = batch.launch_info()["kernels_launched"]
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.step(cycles)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    batch.sync()
    launches = batch.launch_info()["kernels_launched"] - k0
    return ms, launches


def mesh_row(stream, flush):
    """The 4x4 mesh netlist (2M ops), one instance, persistent kernel: the grid
    barrier kernel and the cluster exchange (2-CTA clusters, 8 warps per CTA)."""
    from paper_2403_04714_gb300 import netgen, sim
    text = open(netgen.cached_netlist("mesh"), "rb").read()
    out = {}
    for name, cfg in (("grid_barrier", dict(target_processes=1216, warps_per_cta=8)),
                      ("cluster", dict(cluster_size=2, warps_per_cta=8))):
        try:
            nl = sim.Netlist(text, mode="lane_op", **cfg)
            b = sim.Batch(nl, 1, seed=42, stream=stream)
        except sim.SimError as e:
            out[name] = {"unavailable": str(e)}
            continue
        ms, lk = time_steps(b, stream, 3, 1, 1000, flush)
        i = nl.info()
        out[name] = {"value": 3000 / (sum(ms) / 1000.0), "unit": UNIT, "cycles_timed": 3000, "kernels": lk,
                     "processes": i["n_processes"], "max_bundles": i["max_bundles"], "config": cfg}
        del b, nl
    best = max((v for v in out.values() if "value" in v), key=lambda v: v["value"])
    return dict(best, workload="4x4 mesh of 120k-op blocks (2.0M ops, 128k registers), 1 instance", variants=out)


def phase_row(text, stream, cycles=500, cfg=None):
    """Decomposition of a simulated cycle of the headline workload (Eq. sim_rate)."""
    from paper_2403_04714_gb300 import sim
    import numpy as np
    cfg = dict(cfg or {"mode": "lane_op"})
    nl = sim.Netlist(text, kernel="persistent", phase_samples=cycles, **cfg)
    b = sim.Batch(nl, 1, seed=42, stream=stream)
    b.step(cycles)
    b.step(cycles)
    ph = b.phase_times(cycles)[50:]          # skip the first cycles of the launch
    med = np.median(ph, axis=0)
    steps = nl.info()["max_bundles"]
    return {"compute_ns": float(med[0]), "sync_ns": float(med[1]), "cycle_ns": float(med[2]),
            "steps_slowest_process": steps, "ns_per_step": float(med[0]) / max(1, steps), "config": cfg,
            "note": "medians over cycles 50..500 of one persistent launch; compute = earliest CTA start "
                    "to last CTA arrival (straggler t_comp + t_comm), sync = last arrival to last release"}


def prng_row(stream, per_proc=(1, 8, 64), procs=1216, cycles=2000):
    """Sec. 4.1 synchronisation experiment on GB300: independent xorshift fibers
    (t_comm = 0), `procs` processes with 1/8/64 fibers each, one instance."""
    from paper_2403_04714_gb300 import netgen, sim
    import numpy as np
    out = {}
    for k in per_proc:
        text = netgen.gen_prng(procs * k).to_text()
        nl = sim.Netlist(text, mode="lane_op", target_processes=procs, phase_samples=cycles)
        b = sim.Batch(nl, 1, seed=1, stream=stream)
        b.step(cycles)
        b.sync()
        t = time.perf_counter()
        b.step(cycles)
        b.sync()
        sec = time.perf_counter() - t
        ph = np.median(b.phase_times(cycles)[100:], axis=0)
        out[f"fibers_per_process_{k}"] = {"cycles_per_s": cycles / sec, "compute_ns": float(ph[0]),
                                          "sync_ns": float(ph[1]), "cycle_ns": float(ph[2]),
                                          "ctas": b.launch_info()["ctas"]}
    return out


def sync_sweep_row(stream, per_proc=(1, 32, 256), procs=(38, 152, 608, 1216, 2432), cycles=2000):
    """Sec. 4.1 synchronisation experiment as a sweep (the paper's PRNG rate
    figure): the number of processes (warps, the GPU's counterpart of tiles)
    grows with the number of independent xorshift fibers, fibers per process
    held fixed; t_comm = 0, so the rate falls only through the barrier and
    through warps sharing an SM.  Rates are normalised to the smallest grid."""
    from paper_2403_04714_gb300 import netgen, sim
    import numpy as np
    out = {}
    for k in per_proc:
        line, base = {}, None
        for P in procs:
            if P * k > 400_000:        # generation alone would take tens of seconds
                continue
            try:
                nl = sim.Netlist(netgen.gen_prng(P * k).to_text(), mode="lane_op", target_processes=P,
                                 phase_samples=cycles)
                b = sim.Batch(nl, 1, seed=1, stream=stream)
            except sim.SimError as e:
                line[str(P)] = {"unavailable": str(e)}
                continue
            b.step(cycles)
            b.sync()
            t = time.perf_counter()
            b.step(cycles)
            b.sync()
            rate = cycles / (time.perf_counter() - t)
            base = base or rate
            ph = np.median(b.phase_times(cycles)[100:], axis=0)
            line[str(P)] = {"cycles_per_s": rate, "normalised": rate / base, "compute_ns": float(ph[0]),
                            "sync_ns": float(ph[1]), "steps": nl.info()["max_bundles"],
                            "launch": b.launch_info()}
            del b, nl
        out[f"fibers_per_process_{k}"] = line
    return out


def mesh_weak_row(stream, flush, sides=(2, 3, 4, 5, 6)):
    """Weak scaling of the mesh design (the paper's srN / lrN series, Sec. 6):
    N x N blocks of 30k ops and 2k registers each, N = 2..6, one instance, the
    plain grid-barrier kernel and the cluster exchange (2-CTA clusters, 8 warps
    per CTA)."""
    from paper_2403_04714_gb300 import netgen, sim
    out = {}
    for n in sides:
        text = netgen.gen_mesh(1100 + n, mesh=n, ops_per_block=30_000, regs_per_block=2_000, depth=40,
                               inputs_per_block=8).to_text()
        r = {}
        for kind, cfg in (("grid_barrier", dict()), ("cluster", dict(cluster_size=2, warps_per_cta=8))):
            try:
                nl = sim.Netlist(text, mode="lane_op", **cfg)
                b = sim.Batch(nl, 1, seed=42, stream=stream)
            except sim.SimError as e:
                r[kind] = {"unavailable": str(e)}
                continue
            ms, lk = time_steps(b, stream, 3, 1, 1000, flush)
            i = nl.info()
            r[kind] = {"cycles_per_s": 3000 / (sum(ms) / 1000.0), "processes": i["n_processes"],
                       "steps": i["max_bundles"], "launch": b.launch_info()}
            r["ops"], r["registers"] = i["n_ops"], i["n_regs"]
            del b, nl
        out[f"{n}x{n}"] = r
    return out


def partitioner_row(stream, flush, names=("tiny", "mid", "mesh_small")):
    """The paper's comparison of partitioning strategies (Sec. 7): the
    bottom-up merge (SLB) against a k-way hypergraph partition of the fibers,
    one instance, the grid-barrier kernel with the default partition size."""
    from paper_2403_04714_gb300 import netgen, sim
    import numpy as np
    out = {}
    for name in names:
        text = open(netgen.cached_netlist(name), "rb").read()
        r = {}
        for part in ("slb", "hypergraph"):
            t = time.perf_counter()
            nl = sim.Netlist(text, mode="lane_op", partitioner=part, phase_samples=500)
            compile_s = time.perf_counter() - t
            b = sim.Batch(nl, 1, seed=42, stream=stream)
            ms, _ = time_steps(b, stream, 3, 1, 2000, flush)
            b.step(500)
            ph = np.median(b.phase_times(500)[50:], axis=0)
            i = nl.info()
            r[part] = {"cycles_per_s": 6000 / (sum(ms) / 1000.0), "compute_ns": float(ph[0]), "sync_ns": float(ph[1]),
                       "processes": i["n_processes"], "process_cost_sum": i["process_cost_sum"],
                       "process_cost_max": i["process_cost_max"], "cut_words": i["cut_words"],
                       "steps": i["max_bundles"], "compile_s": compile_s}
            del b, nl
        out[name] = r
    return out


def exchange_sweep_row(stream, procs=(152, 608, 2432), reads=(1, 4, 16, 64), per_proc=32, cycles=2000):
    """Sec. 4.2 communication experiment on GB300: every process holds 32
    registers and each register reads `reads` registers of random other
    processes (a random balanced partition), so a process imports about
    8 x 32 x reads bytes per cycle; the grid size m varies at fixed bytes
    per process b.  On the paper's IPU the on-chip exchange time depended on
    b but not on m."""
    from paper_2403_04714_gb300 import netgen, sim
    import numpy as np
    out = {}
    for d in reads:
        line = {}
        for P in procs:
            if P * d > 40_000:         # the random partition of the largest cases takes tens of seconds
                continue
            try:
                nl = sim.Netlist(netgen.gen_exchange(P * per_proc, d).to_text(), mode="lane_op",
                                 target_processes=P, seed_partition=1, phase_samples=cycles)
                b = sim.Batch(nl, 1, seed=1, stream=stream)
            except sim.SimError as e:
                line[str(P)] = {"unavailable": str(e)}
                continue
            b.step(cycles)
            b.sync()
            t = time.perf_counter()
            b.step(cycles)
            b.sync()
            rate = cycles / (time.perf_counter() - t)
            ph = np.median(b.phase_times(cycles)[100:], axis=0)
            i = nl.info()
            line[str(P)] = {"cycles_per_s": rate, "compute_ns": float(ph[0]), "sync_ns": float(ph[1]),
                            "bytes_in_per_process": 8.0 * i["cut_words"] / P, "steps": i["max_bundles"],
                            "launch": b.launch_info()}
            del b, nl
        out[f"reads_{d}"] = line
    return out


def cluster_row(stream, flush):
    """Cluster exchange against the plain grid-barrier kernel, one instance: a
    design that fits one 16-CTA cluster synchronises with the cluster barrier
    and exchanges every value through distributed shared memory."""
    from paper_2403_04714_gb300 import netgen, sim
    import numpy as np
    cases = {
        "tiny": (open(netgen.cached_netlist("tiny"), "rb").read(), dict(), dict(cluster_size=8, warps_per_cta=2,
                                                                              target_processes=16)),
        "prng_1216_fibers": (netgen.gen_prng(1216).to_text(), dict(target_processes=1216),
                             dict(cluster_size=16, warps_per_cta=8, target_processes=128)),
        "mid": (open(netgen.cached_netlist("mid"), "rb").read(), dict(warps_per_cta=4, target_processes=576),
                dict(cluster_size=4, warps_per_cta=4)),
    }
    out = {}
    for name, (text, plain, clus) in cases.items():
        r = {}
        for kind, cfg in (("grid_barrier", plain), ("cluster", clus)):
            nl = sim.Netlist(text, mode="lane_op", phase_samples=500, **cfg)
            b = sim.Batch(nl, 1, seed=42, stream=stream)
            cyc = 5000 if name != "mid" else 2000
            ms, _ = time_steps(b, stream, 3, 1, cyc, flush)
            b.step(500)
            ph = np.median(b.phase_times(500)[50:], axis=0)
            r[kind] = {"cycles_per_s": 3 * cyc / (sum(ms) / 1000.0), "compute_ns": float(ph[0]),
                       "sync_ns": float(ph[1]), "processes": nl.info()["n_processes"],
                       "ctas": b.launch_info()["ctas"], "config": cfg}
            if kind == "cluster":
                plan = nl.table("cluster_plan")
                r[kind]["reads_in_cluster"] = int(plan[4])
                r[kind]["reads_across_clusters"] = int(plan[5])
            del b, nl
        out[name] = r
    return out


def served_row(n_jobs=40, rate=200.0):
    """Continuous batching over a seeded Poisson trace of jobs (p50/p99 latency):
    the configured arrival rate with persistent pool steps (the server's
    default) and with per-cycle graph replays, then the same trace at ~70 % of
    the job rate the first run sustained (queueing separated from service
    time)."""
    out = served_run(n_jobs, rate, persistent=1)
    out["per_cycle_pools"] = served_run(n_jobs, rate, persistent=0)
    light = 0.7 * n_jobs / out["makespan_s"]
    out["rate_scaled"] = dict(served_run(n_jobs, light, persistent=1), arrival_rate_per_s=light)
    return out


def served_full_row():
    """The served mix as specified: the first 256 arrivals of the Poisson trace
    (200 jobs/s), shapes tiny / mid / the 4x4 mesh of 120k-op blocks with
    weights 0.6/0.3/0.1 drawn from pools of 8/4/2 netlists, instances
    log-uniform 1-1,024, cycle budgets log-uniform 1e3-1e6, admission under a
    150 GiB cap; then the same trace at ~70 % of the sustained job rate.
    Minutes of GPU time: opt-in (--rows served_full)."""
    from paper_2403_04714_gb300 import netgen
    pools = {"tiny": [netgen.gen_tiny(2000 + k).to_text() for k in range(8)],
             "mid": [open(netgen.cached_netlist("mid")).read()] + [netgen.gen_mid(2100 + k).to_text() for k in range(3)],
             "mesh": [open(netgen.cached_netlist("mesh")).read(), netgen.gen_mesh(2200).to_text()]}
    shapes = (("tiny", 0.6), ("mid", 0.3), ("mesh", 0.1))
    kw = dict(pools=pools, shapes=shapes, cycles_hi=1e6, chunk=2000, pools_desc="8/4/2",
              large="4x4 mesh of 120k-op blocks (2M ops)")
    out = served_run(256, 200.0, persistent=1, **kw)
    print(json.dumps({"served_full": out}), file=sys.stderr, flush=True)    # kept if the second run is cut short
    light = 0.7 * 256 / out["makespan_s"]
    out["rate_scaled"] = dict(served_run(256, light, persistent=1, **kw), arrival_rate_per_s=light)
    return out


def served_run(n_jobs, rate, persistent=1, pools=None, shapes=(("tiny", 0.6), ("mid", 0.3), ("mesh_small", 0.1)),
               cycles_hi=3e4, chunk=250, pools_desc="4/2/1", large="2x2-mesh"):
    from paper_2403_04714_gb300 import netgen, sim
    if pools is None:
        pools = {"tiny": [netgen.gen_tiny(2000 + k).to_text() for k in range(4)],
                 "mid": [open(netgen.cached_netlist("mid")).read(), netgen.gen_mid(2101).to_text()],
                 "mesh_small": [open(netgen.cached_netlist("mesh_small")).read()]}
    handles = {k: [sim.Netlist(t, mode="lane_inst", lowering="generated") for t in v] for k, v in pools.items()}
    t_compile = time.perf_counter()
    for hs in handles.values():          # compile (or load from the cache) before the trace starts
        for h in hs:
            h.compile_generated("lane_inst")
    t_compile = time.perf_counter() - t_compile
    trace = netgen.served_trace(n_jobs=n_jobs, rate=rate, cycles_lo=1e3, cycles_hi=cycles_hi, shapes=shapes)
    srv = sim.Server(pool_slots=1024, chunk_cycles=chunk, persistent=persistent)
    t0 = time.perf_counter()
    ids = []
    for arrive, shape, pick, n_inst, cyc, seed in trace:
        while time.perf_counter() - t0 < arrive:
            time.sleep(0.0005)
        nl = handles[shape][pick % len(handles[shape])]
        ids.append((srv.submit(nl, n_inst, seed, cyc), n_inst, cyc))
    lat, wait, work = [], [], 0
    for jid, n_inst, cyc in ids:
        srv.wait(jid, 3_600_000)
        st = srv.poll(jid)
        lat.append(st["t_done"] - st["t_arrive"])
        wait.append(st["t_start"] - st["t_arrive"])
        work += n_inst * cyc
    makespan = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat.sort()
    wait.sort()
    pct = lambda v, q: v[min(len(v) - 1, int(q * len(v)))]
    hi = "1e6" if cycles_hi >= 1e6 else f"{cycles_hi:.0e} (upper end scaled down from 1e6 to fit the bench)"
    return {"value": work / makespan, "unit": "instance-cycles/s", "p50_s": pct(lat, 0.5), "p99_s": pct(lat, 0.99),
            "queue_p50_s": pct(wait, 0.5), "queue_p99_s": pct(wait, 0.99),
            "makespan_s": makespan, "jobs": n_jobs, "instance_cycles": work, "kernels": stats["kernels"],
            "pool_steps": "persistent launch per step" if persistent else "per-cycle graph replays",
            "compile_s": t_compile,
            "trace": f"Poisson {rate:.0f} jobs/s, shapes tiny/mid/{large} weights 0.6/0.3/0.1 (pools of {pools_desc} "
                     f"netlists), instances log-uniform 1-1024, cycles log-uniform 1e3-{hi}, cap 150 GiB, 1024 slots "
                     f"per pool, {chunk}-cycle steps"}


def rows_summary(rows):
    """The other configurations' headline numbers in a few short fields."""
    out = {}
    for key in ("batched_4096_generated", "batched_4096_bytecode"):
        r = rows.get(key)
        if r:
            out[key] = {"instance_cycles_per_s": round(r["value"]), "cycles_timed": r["cycles_timed"],
                        "hbm_frac_algorithmic": round(r["hbm_gbs_algorithmic"] / HBM_PEAK_GBS, 4)}
    if "mesh_single" in rows:
        out["mesh_2M_ops_cycles_per_s"] = round(rows["mesh_single"]["value"])
    for key in ("served", "served_full"):
        if key in rows:
            r = rows[key]
            out[key] = {"instance_cycles_per_s": round(r["value"]), "p50_s": round(r["p50_s"], 4),
                        "p99_s": round(r["p99_s"], 4), "jobs": r["jobs"], "makespan_s": round(r["makespan_s"], 2)}
    return out


def run_cpu_baseline(path, cycles, seed=42):
    import oracle
    net = oracle.Net(path)
    s = oracle.Sim(net, seed, 0)
    t = time.perf_counter()
    s.run(cycles)
    dt = time.perf_counter() - t
    return cycles / dt, dt


def run_cpu_baseline_batched(path, cycles, threads, seed=42):
    """The oracle as it stands on `threads` host threads, each simulating its
    own instance (the oracle's C calls release the interpreter lock), for the
    batched rows: instance-cycles per second over the bounded sample."""
    import concurrent.futures as cf
    import oracle
    net = oracle.Net(path)
    sims = [oracle.Sim(net, seed, i) for i in range(threads)]
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda s: s.run(cycles), sims))
    dt = time.perf_counter() - t
    return threads * cycles / dt, dt


def host_cpu():
    """The host the oracle ran on: logical cores and CPU model."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu": model}


def reference_arm(args, rank):
    """The oracle, as it stands, on the host cores (the reference arm)."""
    if rank != 0:
        return
    from paper_2403_04714_gb300 import netgen
    import oracle
    oracle.build()
    path = netgen.cached_netlist("mid")
    per_step = args.ref_cycles
    net = oracle.Net(path)
    s = oracle.Sim(net, 42, 0)
    s.run(per_step * args.warmup)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        s.run(per_step)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = args.steps * per_step / total
    sample = f"{per_step} cycles of the mid netlist (1 instance) per step on one host core"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--cycles", type=int, default=10_000, help="simulated cycles per step")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-cycles", type=int, default=300)
    ap.add_argument("--cpu-cycles", type=int, default=10_000, help="oracle sample for cpu_baseline (~10 s)")
    ap.add_argument("--batched-cycles", type=int, default=1000)
    ap.add_argument("--no-rows", action="store_true", help="headline only (profiling runs)")
    ap.add_argument("--rows", default="single,batched,mesh,cluster,served",
                    help="comma list of extra rows: single, batched, mesh, cluster, served; "
                         "opt-in: sync_sweep, exchange_sweep, mesh_weak, partitioners, served_full")
    args = ap.parse_args()
    rank, world, local, dist = (0, 1, 0, None)
    if args.impl == "reference":
        if "RANK" in os.environ and int(os.environ["RANK"]) != 0:
            return
        reference_arm(args, 0)
        return
    rank, world, local, dist = dist_setup(args.gpus)

    import numpy as np
    import torch
    from paper_2403_04714_gb300 import netgen, sim
    from paper_2403_04714_gb300.build import build
    if rank == 0:
        build()
    barrier(dist)
    path = netgen.cached_netlist("mid")
    text = open(path, "rb").read()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    p = peaks()
    global HBM_PEAK_GBS
    HBM_PEAK_GBS = float(p.get("hbm_gbs", HBM_PEAK_GBS))

    # ---- headline: single instance, persistent kernel, autotuned geometry ------
    from paper_2403_04714_gb300 import autotune
    tuned = autotune.autotune(text, 1)
    nl = sim.Netlist(text, kernel="persistent", **tuned["config"])
    info = nl.info()
    b = sim.Batch(nl, 1, seed=42 + rank, stream=stream)
    barrier(dist)
    with ClockSampler(local) as clk:
        ms, launches = time_steps(b, stream, args.steps, args.warmup, args.cycles, flush)
    value = replica_rate(dist, world, args.steps * args.cycles, sum(ms) / 1000.0)
    per_launch_s = sum(ms) / 1000.0 / max(1, launches)
    cycles_per_launch = args.steps * args.cycles / max(1, launches)
    ops = info["n_ops"]
    achieved = ops * cycles_per_launch / per_launch_s
    peak = alu_peak_ops(p)
    geo = b.launch_info()

    # ---- e2e through the public call: sim_step_host, per-instance digest out ----
    # the timed workload itself (free-running on-device stimulus, the paper's
    # on-device test driver), host-timed around each call, which copies the
    # step's state digest back to pinned host memory
    out_pinned = torch.zeros(1, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    b2 = sim.Batch(nl, 1, seed=42 + rank, stream=stream)
    for _ in range(args.warmup):
        b2.step_host(args.cycles, None, out_pinned)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b2.step_host(args.cycles, None, out_pinned)
    e2e = {"value": replica_rate(dist, world, args.steps * args.cycles, time.perf_counter() - t0), "unit": UNIT,
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8,
           "call": "sim_step_host(held_inputs=NULL): the timed workload (stimulus generated on the device), "
                   "host-timed, state digest read back each step"}
    del b2
    # the same call with every input held from pinned host memory (h2d each step)
    b3 = sim.Batch(nl, 1, seed=42 + rank, stream=stream)
    n_in = info["n_inputs"]
    held = np.arange(n_in, dtype=np.uint64).reshape(1, n_in) * np.uint64(0x9E3779B1)
    held_pinned = torch.from_numpy(held).pin_memory().numpy()
    for _ in range(args.warmup):
        b3.step_host(args.cycles, held_pinned, out_pinned)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b3.step_host(args.cycles, held_pinned, out_pinned)
    e2e_held = {"value": replica_rate(dist, world, args.steps * args.cycles, time.perf_counter() - t0), "unit": UNIT,
                "h2d_bytes_per_step": int(held.nbytes), "d2h_bytes_per_step": 8,
                "call": "sim_step_host (all inputs held from pinned host memory, state digest read back)"}
    del b3

    rows = {}
    want = set() if args.no_rows else set(args.rows.split(","))
    if want:
        # launch-per-cycle baseline and its graph replay, same workload
        for kname in (("per_cycle", "graph") if "single" in want else ()):
            nlk = sim.Netlist(text, mode="lane_op", kernel=kname)
            bk = sim.Batch(nlk, 1, seed=42, stream=stream)
            cyc = min(args.cycles, 2000)
            msk, lk = time_steps(bk, stream, 3, 1, cyc, flush)
            rows[f"single_{kname}"] = {"value": 3 * cyc / (sum(msk) / 1000.0), "unit": UNIT,
                                       "cycles_timed": 3 * cyc, "kernels": lk}
            del bk, nlk
        # batched: same netlist x 4096 instances, lane = instance, both lowerings
        for low in (("generated", "bytecode") if "batched" in want else ()):
            cfg_b = {"mode": "lane_inst", "lowering": low}
            tuned_b = None
            if low == "generated":
                # instances per CTA (32 x warps), the task order and the number
                # of processes, by measurement (the autotuner's candidates)
                cands = autotune.default_candidates(4096, torch.cuda.get_device_properties(0).multi_processor_count)
                tuned_b = autotune.autotune(text, 4096, candidates=cands, cycles=40)
                cfg_b = tuned_b["config"]
            nlb = sim.Netlist(text, kernel="persistent_graph", **cfg_b)
            comp = nlb.compile_generated("lane_inst") if low == "generated" else None
            bb = sim.Batch(nlb, 4096, seed=42, stream=stream)
            cyc = args.batched_cycles if low == "generated" else max(10, args.batched_cycles // 5)
            msb, lb = time_steps(bb, stream, 3, 1, cyc, flush)
            sec = sum(msb) / 1000.0
            ib = nlb.info()
            ic = 3 * cyc * 4096 / sec
            rows[f"batched_4096_{low}"] = {
                "value": ic, "unit": "instance-cycles/s", "cycles_timed": 3 * cyc, "kernels": lb,
                "launch": bb.launch_info(), "processes": ib["n_processes"], "ops_per_cycle": ib["n_ops"],
                "alu_frac": ib["n_ops"] * ic / peak,
                "hbm_gbs_algorithmic": ic * 2 * STATE_BYTES_MID / 1e9,
                "compile": comp,
                "autotuned": None if tuned_b is None else {"config": tuned_b["config"], "cached": tuned_b["cached"],
                                                           "candidates": tuned_b["results"]},
            }
            del bb, nlb
        if "single" in want:
            rows["phases"] = phase_row(text, stream, cfg=tuned["config"])
            rows["prng_sync"] = prng_row(stream)
        if "mesh" in want:
            rows["mesh_single"] = mesh_row(stream, flush)
        if "cluster" in want:
            rows["cluster_exchange"] = cluster_row(stream, flush)
        if "served" in want:
            rows["served"] = served_row()
        if "served_full" in want:
            rows["served_full"] = served_full_row()
        if "sync_sweep" in want:
            rows["sync_sweep"] = sync_sweep_row(stream)
        if "mesh_weak" in want:
            rows["mesh_weak"] = mesh_weak_row(stream, flush)
        if "exchange_sweep" in want:
            rows["exchange_sweep"] = exchange_sweep_row(stream)
        if "partitioners" in want:
            rows["partitioners"] = partitioner_row(stream, flush)

    # ---- measured integer issue rate (the ALU roof, next to the derived one) ---
    int_peak = sim.measure_int_peak(1 << 14)

    # ---- CPU baseline: the oracle on one host core, bounded sample -------------
    cpu = None
    if rank == 0:
        import oracle
        oracle.build()
        v, dt = run_cpu_baseline(path, args.cpu_cycles)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {args.cpu_cycles} cycles of the mid netlist, 1 instance ({dt:.1f} s)",
               "host": host_cpu()}
        for key in ("batched_4096_generated", "batched_4096_bytecode"):
            if key in rows:
                threads = os.cpu_count() or 1
                cyc = max(10, args.cpu_cycles // 10)
                vb, dtb = run_cpu_baseline_batched(path, cyc, threads)
                rows[key]["cpu_baseline"] = {
                    "value": vb, "unit": "instance-cycles/s", "cores": threads, "kind": "oracle",
                    "sample": f"{threads} instances of the mid netlist, first {cyc} cycles each, one thread "
                              f"per instance ({dtb:.1f} s)"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cycles_per_step": args.cycles, "instances": 1,
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1 else "1 GPU",
                       "processes": info["n_processes"], "launch": geo,
                       "autotuned": {"config": tuned["config"], "cached": tuned["cached"],
                                     "candidates": tuned["results"]},
                       "rows_summary": rows_summary(rows)},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": int_peak / 1e12, "unit": "Tops/s",
                         "frac": achieved / int_peak, "traffic": HEADLINE_TRAFFIC,
                         "kernel": "k_cycles_cl (cluster exchange)" if tuned["config"].get("cluster_size")
                                   else "k_cycles<LANE_OP> (persistent)",
                         "peak_source": "measured: sim_measure_int_peak (independent IADD3/LOP3 chains on every SM, "
                                        "this run)",
                         "derived_peak": peak / 1e12, "frac_of_derived": achieved / peak,
                         "note": "word ops (algorithmic, unduplicated) per second of the dominant kernel; "
                                 "derived_peak = 152 SMs x 64 integer-ALU lanes x max SM clock; single-instance BSP is "
                                 "latency-bound, see rows.phases for the cycle decomposition"},
            "cpu_baseline": cpu, "e2e": e2e, "e2e_held_inputs": e2e_held, "gpu_launches": launches,
            "clocks": clk.summary(),
            "rows": rows,
            "netlist": {k: info[k] for k in ("n_ops", "n_regs", "n_fibers", "n_processes", "fiber_cost_sum",
                                             "process_cost_sum", "process_cost_max", "fiber_cost_max",
                                             "max_bundles", "cut_words")},
        }
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
