"""The generated-CUDA lowering compiles and links for sm_103a on the CPU
(NVRTC + nvJitLink need no GPU): every operator kind, memories with write
ports and read-only memories, degenerate netlists, a design with gated and
divided clocks, both lane mappings."""
import pytest

from paper_2403_04714_gb300 import netgen, sim
from test_oracle_bruteforce import random_tiny_circuit

DEGENERATE = [
    "rtlnet 1\nreg 64 12345\nn reg 64 0\nnext 0 0\nend\n",
    "rtlnet 1\nreg 1 1\nn const 1 0\nnext 0 0\nend\n",
    "rtlnet 1\nin 64\nreg 64 1\nreg 32 0\nn reg 64 0\nn input 64 0\nn slice 32 1 32\nn slice 32 0 0\n"
    "n concat 64 2 3\nn shl 64 0 1\nn xor 64 4 5\nn const 7 64\nn shr 64 1 7\nn add 64 6 8\nn slice 32 9 16\n"
    "next 0 9\nnext 1 10\nend\n",
]


@pytest.mark.parametrize("mode", ["lane_op", "lane_inst"])
def test_generated_code_compiles(mode):
    texts = [open(netgen.cached_netlist("tiny")).read()] + DEGENERATE
    texts += [random_tiny_circuit(s).to_text() for s in range(3)]
    texts.append(netgen.gen_flat(7, n_ops=3000, n_regs=200, depth=15, n_inputs=6, rams=((4, 64), (3, 16))).to_text())
    texts.append(netgen.gen_clocked().to_text())          # gated and divided clocks, lowered at load
    for text in texts:
        nl = sim.Netlist(text, mode=mode, lowering="generated")
        r = nl.compile_generated(mode)
        assert r["seconds"] >= 0
