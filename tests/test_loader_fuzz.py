"""Both loaders (the CUDA path's compiler and the oracle) survive malformed
netlists: random token edits of small valid netlists, including the clock
items, either load or fail with an error, never crash, and the two agree on
whether a netlist is valid; a valid mutant's lowered program, run by the
Python emulator, reproduces the oracle for a few cycles."""
import random

import pytest

import oracle
from paper_2403_04714_gb300 import netgen, sim
from test_lowering_emulated import run_compare
from test_oracle_clocks import random_clocked_circuit

TOKENS = ["0", "1", "2", "7", "63", "64", "65", "-1", "999999", "n", "reg", "in", "mem", "next", "gate",
          "clock", "wport", "minit", "add", "mux", "slice", "concat", "memrd", "const", "end", "x"]


def mutate(text, rng):
    lines = text.splitlines()
    for _ in range(rng.randrange(1, 4)):
        k = rng.randrange(len(lines))
        toks = lines[k].split()
        action = rng.randrange(4)
        if action == 0 and toks:
            toks[rng.randrange(len(toks))] = rng.choice(TOKENS)
        elif action == 1:
            toks.insert(rng.randrange(len(toks) + 1), rng.choice(TOKENS))
        elif action == 2 and toks:
            toks.pop(rng.randrange(len(toks)))
        else:
            lines.insert(rng.randrange(len(lines) + 1), lines[rng.randrange(len(lines))])
        lines[k] = " ".join(toks) if k < len(lines) and action != 3 else lines[k]
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("seed", range(4))
def test_mutated_netlists_load_or_fail_cleanly(seed):
    rng = random.Random(seed)
    base = random_clocked_circuit(seed).to_text()
    disagree, valid = [], 0
    for _ in range(300):
        text = mutate(base, rng)
        try:
            sim.Netlist(text, mode="lane_op", target_processes=3)
            ok_gpu_path = True
        except sim.SimError:
            ok_gpu_path = False
        try:
            oracle.Net(text=text)
            ok_oracle = True
        except Exception:
            ok_oracle = False
        if ok_gpu_path != ok_oracle:
            disagree.append(text)
        elif ok_gpu_path:
            run_compare(text, "lane_op", 6, target=3)
            valid += 1
    assert not disagree, disagree[0]
    assert valid > 0
