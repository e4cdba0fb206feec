"""Randomised differential test of the CUDA path's host side (CPU): random
netlists (random circuits with clocks and memories, flat designs with RAMs)
are lowered in a random configuration (lane mapping, compact or full
programs, cluster exchange, partitioning strategy, partition size), and the
lowered program, run by the Python emulator of the instruction set, must
reproduce the oracle register by register and word by word.  A
configuration the loader rejects (capacity) is skipped."""
import random

import pytest

from paper_2403_04714_gb300 import netgen, sim
from test_clocks_lowering import clocked_with_memories
from test_lowering_emulated import run_compare
from test_oracle_bruteforce import random_tiny_circuit
from test_oracle_clocks import random_clocked_circuit


def random_case(rng):
    kind = rng.randrange(4)
    seed = rng.randrange(10 ** 6)
    if kind == 0:
        return random_clocked_circuit(seed)
    if kind == 1:
        return random_tiny_circuit(seed)
    if kind == 2:
        return clocked_with_memories(seed % 1000)
    return netgen.gen_flat(seed % 5000, n_ops=rng.randrange(50, 1500), n_regs=rng.randrange(5, 80),
                           depth=rng.randrange(4, 12), n_inputs=rng.randrange(1, 5),
                           rams=tuple((rng.randrange(1, 6), rng.choice((8, 16, 64))) for _ in range(rng.randrange(0, 3))))


@pytest.mark.parametrize("seed", range(4))
def test_random_configurations_match_the_oracle(seed):
    rng = random.Random(1000 + seed)
    done = 0
    for _ in range(80):
        try:
            nl = random_case(rng)
        except ValueError:          # a generator draw without room for its RAMs
            continue
        mode = rng.choice(["lane_op", "lane_op_compact", "lane_inst", "lane_op_cluster"])
        kw = {"cluster": (rng.choice((2, 3, 4)), rng.choice((1, 2)))} if mode == "lane_op_cluster" else {}
        try:
            run_compare(nl.to_text(), mode, rng.randrange(3, 10), target=rng.randrange(1, 12),
                        shuffle=rng.random() < 0.5, partitioner=rng.choice(["slb", "hypergraph"]),
                        chain=rng.choice((0, 2)), **kw)
        except sim.SimError as e:
            # only a capacity rejection (a process that does not fit the
            # on-chip budget) is an expected outcome of a random draw
            if e.name != "SIM_ERR_CAPACITY":
                raise
            continue
        done += 1
    assert done > 60
