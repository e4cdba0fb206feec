"""Autotuner host logic (CPU, with a stand-in measurement) and, on the GPU,
that the configuration it picks simulates bit-exactly."""
import numpy as np
import pytest

from paper_2403_04714_gb300 import autotune, netgen


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def fake(text, n_inst, cfg, cycles):
        calls.append(cfg)
        return {12: 90.0, 8: 100.0, 6: 120.0, 4: 250.0}[cfg["warps_per_cta"]] + \
            (1 if cfg["task_order"] == "process_major" else 0)

    cache = str(tmp_path / "at.json")
    n = len(autotune.default_candidates(64))
    r = autotune.autotune("rtlnet 1\nend\n", 64, cache_path=cache, measure_fn=fake, device="fake")
    assert r["config"]["warps_per_cta"] == 4 and r["config"]["task_order"] == "process_major"
    assert not r["cached"] and len(calls) == n
    r2 = autotune.autotune("rtlnet 1\nend\n", 64, cache_path=cache, measure_fn=fake, device="fake")
    assert r2["cached"] and r2["config"] == r["config"] and len(calls) == n
    # another instance count or device is another key
    autotune.autotune("rtlnet 1\nend\n", 1, cache_path=cache, measure_fn=lambda *a: 1.0, device="fake")
    autotune.autotune("rtlnet 1\nend\n", 64, cache_path=cache, measure_fn=lambda *a: 1.0, device="other")
    assert len(calls) == n


def test_candidate_that_fails_scores_zero(tmp_path):
    from paper_2403_04714_gb300 import sim

    def fake(text, n_inst, cfg, cycles):
        if cfg["warps_per_cta"] != 4:
            raise sim.SimError(-4, "does not fit")
        return 5.0

    r = autotune.autotune("x", 64, cache_path=str(tmp_path / "a.json"), measure_fn=fake, device="fake")
    assert r["config"]["warps_per_cta"] == 4


@pytest.mark.gpu
def test_tuned_config_is_exact(tmp_path):
    import oracle
    from paper_2403_04714_gb300 import sim
    text = open(netgen.cached_netlist("tiny")).read()
    r = autotune.autotune(text, 64, cycles=200, cache_path=str(tmp_path / "at.json"))
    nl = sim.Netlist(text, **r["config"])
    b = sim.Batch(nl, 64, seed=5)
    b.step(300)
    ref = oracle.Sim(oracle.Net(text=text), 5, 63)
    ref.run(300)
    assert b.state_digests()[63] == ref.digest()
