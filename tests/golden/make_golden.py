"""Writes tests/golden/config1_dslash.json from the oracle alone.

The paper prints no worked example that fixes a value of D (its only numbers,
Table 1, are timings and operation counts of a configuration that is not
available).  This fixture is therefore a regression pin: D of the 8^4
workload (eps = 0.3 links with seed 1, Gaussian source with seed 2,
kappa = 0.12, c_sw = 1, antiperiodic time) at a few sites, as computed by the
oracle when the oracle's own pins pass.  It guards the input generator and the
oracle against silent change.  Run: python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

DIMS = (8, 8, 8, 8)
SITES = [0, 1, 7, 63, 511, 4095, 2222, 3000]


def compute():
    op = oracle.Op(DIMS, (1, 1, 1, -1), synth.gauge_field(DIMS, 0.3, 1), 0.12, 1.0)
    eta = synth.gaussian_source(DIMS, 2)
    out = op.dslash(eta)[SITES]
    U = op.U
    return {
        "dims": DIMS, "eps": 0.3, "gauge_seed": 1, "source_seed": 2, "kappa": 0.12, "c_sw": 1.0,
        "bc": [1, 1, 1, -1], "sites": SITES,
        "dslash_re": out.real.reshape(len(SITES), 12).tolist(),
        "dslash_im": out.imag.reshape(len(SITES), 12).tolist(),
        "link0_re": U[0, 0].real.tolist(), "link0_im": U[0, 0].imag.tolist(),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "config1_dslash.json"), "w") as f:
        json.dump(compute(), f, indent=1)
