"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/sim.h declares; netlist loading reports the paper's compile
errors (no GPU needed for the compiler)."""
import os
import re

import pytest

from paper_2403_04714_gb300 import sim
from paper_2403_04714_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(sim_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    L = sim.lib()
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(sim.EXPORTS)


def test_compile_errors():
    with pytest.raises(sim.SimError) as e:
        sim.Netlist("rtlnet 1\nreg 4 0\nn add 4 1 2\nn reg 4 0\nn add 4 0 1\nnext 0 0\nend\n")
    assert e.value.name == "SIM_ERR_COMB_LOOP"
    with pytest.raises(sim.SimError) as e:
        sim.Netlist("rtlnet 1\nreg 4 0\nn reg 4 0\nn concat 7 0 0\nnext 0 1\nend\n")
    assert e.value.name == "SIM_ERR_WIDTH"
    with pytest.raises(sim.SimError) as e:
        sim.Netlist("rtlnet 1\nreg 4 0\nn reg 4 0\nend\n")
    assert e.value.name == "SIM_ERR_PARSE"
    with pytest.raises(sim.SimError) as e:
        sim.Netlist("rtlnet 1\nreg 4 0\nn reg 4 0\nn slice 3 0 2\nnext 0 1\nend\n")
    assert e.value.name == "SIM_ERR_WIDTH"


def test_info_of_tiny_workload():
    from paper_2403_04714_gb300 import netgen
    nl = sim.Netlist.from_file(netgen.cached_netlist("tiny"))
    i = nl.info()
    assert i["n_regs"] == 70 and i["n_inputs"] == 8
    assert i["n_fibers"] == i["n_regs"]          # no memories in the tiny workload
    assert i["process_cost_max"] >= i["fiber_cost_max"]
    assert i["process_cost_sum"] <= i["fiber_cost_sum"]
