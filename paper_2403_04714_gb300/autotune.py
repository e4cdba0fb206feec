"""Autotuner for the launch configuration of a netlist on this GPU.

Candidates vary what the compiler cannot decide alone: the partition size
(SLB target process count), the partitioning strategy, warps per CTA (with
lane = instance: instances per CTA = 32 x warps), the task order, the
lowering, operator pairs and, for one instance, the thread-block cluster size
of the distributed-shared-memory exchange.  Each candidate is
timed on a short run of the real workload with CUDA events; the best one is
persisted in a JSON cache keyed by a hash of the netlist text, the instance
count, the GPU name and the built library, so later runs with the same
library reuse it without measuring.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import sim

CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "autotune.json")


_LIB_HASH = None


def _lib_hash() -> str:
    """Hash of the built simulator library: a rebuilt kernel is measured anew."""
    global _LIB_HASH
    if _LIB_HASH is None:
        try:
            with open(sim.LIB_PATH, "rb") as f:
                _LIB_HASH = hashlib.sha256(f.read()).hexdigest()[:16]
        except OSError:
            _LIB_HASH = "nolib"
    return _LIB_HASH


def _key(text: bytes, n_inst: int, device: str) -> str:
    return hashlib.sha256(text + f"|{n_inst}|{device}|{_lib_hash()}".encode()).hexdigest()[:24]


def default_candidates(n_inst: int, sms: int = 152):
    if n_inst >= 32:
        # each warp's staging area of shared memory bounds the warps per SM:
        # smaller CTAs let more of them share an SM.  The default partition
        # has two processes per SM (fewer fibers duplicated across processes
        # than with four: mid 210k instead of 220k generated instructions per
        # instance-cycle, measured 4-7 % faster); four stay candidates
        return ([dict(mode="lane_inst", lowering="generated", warps_per_cta=w, task_order="process_major")
                 for w in (12, 8, 6, 4)] +
                [dict(mode="lane_inst", lowering="generated", warps_per_cta=8, task_order="group_major")] +
                [dict(mode="lane_inst", lowering="generated", warps_per_cta=w, task_order="process_major",
                      target_processes=4 * sms) for w in (12, 8)])
    # operator pairs chained in one step (chain=2) measured faster on every
    # geometry; the unchained adaptive geometry stays as the reference
    cands = [dict(mode="lane_op", lowering="bytecode", chain=0),              # adaptive: 4 or 8 per SM
             dict(mode="lane_op", lowering="bytecode", chain=2),
             dict(mode="lane_op", lowering="bytecode", chain=2, warps_per_cta=8, target_processes=8 * sms),
             dict(mode="lane_op", lowering="bytecode", chain=2, warps_per_cta=3, target_processes=3 * sms)]
    if n_inst == 1:     # cluster exchange (one instance): several clusters, and one 16-CTA cluster
        cands += [dict(mode="lane_op", lowering="bytecode", chain=2, cluster_size=c, warps_per_cta=w)
                  for c, w in ((4, 4), (6, 4), (2, 4), (16, 8))]
        # the hypergraph partitioning strategy (Sec. 7) on the two cluster shapes
        # that measured best with the bottom-up merge
        cands += [dict(mode="lane_op", lowering="bytecode", chain=2, cluster_size=c, warps_per_cta=4,
                       partitioner="hypergraph") for c in (2, 4)]
    return cands


def measure(text: bytes, n_inst: int, cfg: dict, cycles: int, seed: int = 1) -> float:
    """Simulated instance-cycles per second of one candidate (after a warm-up step)."""
    import torch
    nl = sim.Netlist(text, **cfg)
    if cfg.get("lowering") == "generated":
        nl.compile_generated(cfg.get("mode", "lane_inst"))
    stream = torch.cuda.Stream()
    b = sim.Batch(nl, n_inst, seed=seed, stream=stream)
    b.step(cycles)
    b.sync()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    b.step(cycles)
    e.record(stream)
    e.synchronize()
    sec = a.elapsed_time(e) / 1000.0
    b.close()
    return n_inst * cycles / sec


def choose(results):
    """Best candidate: highest throughput, ties to the earlier candidate."""
    best = None
    for cfg, v in results:
        if best is None or v > best[1]:
            best = (cfg, v)
    return best


def autotune(text: bytes | str, n_inst: int, candidates=None, cycles: int | None = None,
             cache_path: str = CACHE, measure_fn=measure, device: str | None = None, force: bool = False) -> dict:
    """Pick the fastest candidate configuration; returns {"config", "value", "results", "cached"}."""
    if isinstance(text, str):
        text = text.encode()
    if device is None:
        import torch
        device = torch.cuda.get_device_name(0)
    key = _key(text, n_inst, device)
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        out = dict(cache[key])
        out["cached"] = True
        return out
    if candidates is None:
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count if torch.cuda.is_available() else 152
        candidates = default_candidates(n_inst, sms)
    cycles = cycles or (50 if n_inst >= 32 else 2000)
    results = []
    t0 = time.time()
    for cfg in candidates:
        try:
            results.append((cfg, measure_fn(text, n_inst, cfg, cycles)))
        except sim.SimError:               # a candidate that does not fit scores 0
            results.append((cfg, 0.0))
    cfg, value = choose(results)
    out = {"config": cfg, "value": value, "results": [[c, v] for c, v in results],
           "seconds": time.time() - t0, "device": device}
    cache[key] = out
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = f"{cache_path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    out = dict(out)
    out["cached"] = False
    return out
