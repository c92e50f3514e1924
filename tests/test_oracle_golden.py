"""The oracle still reproduces its committed rank/phase fixtures."""
import os

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", ["ice_16x16x8_eps1e-2", "ice_16x16x8_eps1e-4"])
def test_golden(oracle_lib, name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, f"oracle_{name}.txt")) as fh:
        assert mg.compute(name) == fh.read()
