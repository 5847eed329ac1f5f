"""Regression pin: the generator and the oracle still produce the stored values
(written by tests/golden/make_golden.py, which calls only the oracle)."""

import json
import os

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_config1_dslash_golden(oracle_mod):
    g = json.load(open(os.path.join(HERE, "golden", "config1_dslash.json")))
    dims = tuple(g["dims"])
    U = synth.gauge_field(dims, g["eps"], g["gauge_seed"])
    assert np.allclose(U[0, 0], np.array(g["link0_re"]) + 1j * np.array(g["link0_im"]), atol=1e-15, rtol=0)
    op = oracle_mod.Op(dims, g["bc"], U, g["kappa"], g["c_sw"], store_clover=False)
    eta = synth.gaussian_source(dims, g["source_seed"])
    got = op.dslash_sites(eta, g["sites"]).reshape(len(g["sites"]), 12)
    exp = np.array(g["dslash_re"]) + 1j * np.array(g["dslash_im"])
    assert np.abs(got - exp).max() < 1e-13
