"""The oracle against its golden fixtures (tests/golden/oracle_small_cases.json,
written by tests/golden/make_golden.py from the oracle alone): the paper
prints no per-problem values, so these pin the oracle against unintended
change; the GPU is compared with them too."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2506_00263_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "oracle_small_cases.json")))

import importlib.util
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
_mg = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(_mg)


@pytest.mark.parametrize("name", sorted(GOLD["cases"]))
def test_oracle_reproduces_golden_histories(name):
    g = GOLD["cases"][name]
    make, n = _mg.CASES[name]
    r = oracle.run_fixed_source(make(), n, seed=GOLD["seed"])
    assert r["log_n"].tolist() == g["log_n"]
    assert r["log_cell"].tolist() == g["log_cell"]
    assert r["log_type"].tolist() == g["log_type"]
    assert [int(v) for v in r["events_by_type"]] == g["events_by_type"]
    assert [float.hex(float(v)) for v in r["scalars"]] == g["scalars"]


def test_oracle_log_golden():
    for xh, yh in zip(GOLD["log"]["x"], GOLD["log"]["y"]):
        assert float.hex(oracle.log(float.fromhex(xh))) == yh


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(GOLD["cases"]))
def test_gpu_reproduces_golden_histories(name):
    from paper_2506_00263_gb300 import binding as tb
    from paper_2506_00263_gb300 import build
    build.build()
    g = GOLD["cases"][name]
    make, n = _mg.CASES[name]
    prob = tb.Problem(make())
    prob.run_fixed_source(tb.RunOpts(n_histories=n, seed=GOLD["seed"], scheme=tb.SCHEME_ASYNC,
                                     want_event_log=True))
    a, b, c = prob.event_log(n)
    prob.close()
    assert a.tolist() == g["log_n"] and b.tolist() == g["log_cell"] and c.tolist() == g["log_type"]
