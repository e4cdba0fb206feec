"""sim_state_digests_noalloc: the allocation-free digest entry point.

Callers whose device memory is owned by someone else (a host runtime with
its own memory pool, or a loop that must not trigger the synchronisation of
cudaMalloc) use this entry point instead of sim_state_digests.  It must give
exactly the same digests, call after call, although every call reuses one
fixed device array inside the library.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2403_04714_gb300 import netgen, sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_text():
    return open(netgen.cached_netlist("tiny")).read()


@pytest.mark.parametrize("mode,n_inst", [("lane_op", 3), ("lane_inst", 70)])
def test_noalloc_digests_equal_the_allocating_entry_point(tiny_text, mode, n_inst):
    import torch
    nl = sim.Netlist(tiny_text, mode=mode)
    b = sim.Batch(nl, n_inst, seed=11)
    b.step(257)
    dev_out = torch.zeros(n_inst, dtype=torch.int64, device="cuda")   # caller-owned device memory
    host_out = np.zeros(n_inst, dtype=np.uint64)                       # caller-owned host memory
    for call in range(2):                                              # two calls in a row
        want = b.state_digests()
        b.state_digests_noalloc(dev_out.data_ptr())
        got = dev_out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), (mode, call)
        b.state_digests_noalloc(host_out.ctypes.data)
        assert np.array_equal(host_out, want), (mode, call)
        b.step(13)


def test_noalloc_rejects_batches_beyond_its_array(tiny_text):
    nl = sim.Netlist(tiny_text, mode="lane_inst")
    b = sim.Batch(nl, (1 << 16) + 1, seed=1)
    out = np.zeros((1 << 16) + 1, dtype=np.uint64)
    with pytest.raises(sim.SimError) as e:
        b.state_digests_noalloc(out.ctypes.data)
    assert e.value.name == "SIM_ERR_CAPACITY"
