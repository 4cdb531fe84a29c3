"""Writes the golden fixtures of this directory from the oracle alone.

The paper prints no per-problem values (its figures are not available), so
these fixtures are the oracle's own outputs on small cases: they pin the
oracle against unintended change.  Any deliberate change to the oracle's
arithmetic regenerates them (python tests/golden/make_golden.py), and the
commit that does so names the passage or reading behind the change.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2506_00263_gb300 import inputs  # noqa: E402

CASES = {
    "cube": (inputs.cube_one_group, 64),
    "lattice": (inputs.c5g7_lattice, 64),
    "ce_pin_cell": (lambda: inputs.ce_pin_cell(n_points=2000, n_res=20, n_ebins=10), 32),
    "ce_timed": (lambda: inputs.ce_pin_cell(n_points=2000, n_res=20, n_ebins=10, source_energy=14e6)
                 .replace(t_census=2e-7, n_time_bins=8), 32),
}


def main():
    out = {"seed": 7, "cases": {}}
    for name, (make, n) in CASES.items():
        r = oracle.run_fixed_source(make(), n, seed=7)
        out["cases"][name] = {
            "n": n,
            "log_n": r["log_n"].tolist(), "log_cell": r["log_cell"].tolist(), "log_type": r["log_type"].tolist(),
            "events_by_type": [int(v) for v in r["events_by_type"]],
            "scalars": [float.hex(float(v)) for v in r["scalars"]],
        }
    xs = np.array([1e-300, 1e-9, 0.25, 0.5, 0.7071067811865476, 1.0 - 2.0 ** -53, 1.5, 2.0, 1e300])
    out["log"] = {"x": [float.hex(float(v)) for v in xs],
                  "y": [float.hex(oracle.log(float(v))) for v in xs]}
    with open(os.path.join(HERE, "oracle_small_cases.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
