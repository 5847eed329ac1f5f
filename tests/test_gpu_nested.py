"""The paper's outer solver on the GPU (outer_mode 1, Sec. 3): an FP64 BiCGStab
whose preconditioner is the FP32 / FP16 inner solve, restarted from the true
residual.  Every answer is checked with the oracle's FP64 D."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

DIMS, BC, KAPPA, CSW = (8, 8, 8, 16), (1, 1, 1, -1), 0.124, 1.0


def _system(seed, dims=DIMS):
    U = synth.gauge_field(dims, 0.3, seed)
    eta = synth.gaussian_source(dims, seed + 1)
    return U, eta


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("schwarz", ["ras", "sap", None])
@pytest.mark.parametrize("stream", [False, True])
def test_nested_solve_meets_tolerance(qdd, oracle_mod, prec, schwarz, stream):
    U, eta = _system(601)
    lat = qdd.create_lattice(DIMS, BC, stream=torch.cuda.Stream() if stream else None)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    d_eta = torch.from_numpy(eta).cuda()
    phi = torch.zeros_like(d_eta)
    kw = dict(use_ras=0) if schwarz is None else dict(block=(4, 4, 4, 4), n_ras=1, n_dominv=4, schwarz=schwarz)
    p = qdd.default_params(inner_prec=prec, outer_mode=1, inner_tol=1e-2, **kw)
    info = qdd.solve(lat, phi, d_eta, KAPPA, CSW, 1e-10, p)
    torch.cuda.synchronize()
    res = oracle_mod.Op(DIMS, BC, U, KAPPA, CSW).true_residual(eta, phi.cpu().numpy())
    assert res <= 1e-10
    assert abs(info["true_rel_residual"] - res) <= 1e-3 * res + 1e-14
    assert 1 <= info["outer_iters"] <= 30 and info["inner_iters"] > 0


def test_nested_accelerates_loose_inner_solves(qdd, oracle_mod):
    """Inner solves to 0.1: defect correction gains about a digit per step,
    the outer BiCGStab needs fewer outer iterations for the same tolerance."""
    U, eta = _system(611)
    lat = qdd.create_lattice(DIMS, BC)
    qdd.load_gauge(lat, U)
    out = {}
    for mode in (0, 1):
        phi = np.zeros_like(eta)
        p = qdd.default_params(inner_prec="f32", outer_mode=mode, inner_tol=0.1, n_ras=1, n_dominv=4)
        out[mode] = qdd.solve(lat, phi, eta, KAPPA, CSW, 1e-10, p)
        assert oracle_mod.Op(DIMS, BC, U, KAPPA, CSW).true_residual(eta, phi) <= 1e-10
    assert out[0]["outer_iters"] >= 9
    assert out[1]["outer_iters"] < 0.7 * out[0]["outer_iters"]


def test_nested_exact_preconditioner_ends_at_s(qdd, oracle_mod):
    """An inner solve to 1e-6 against a target of 1e-5: after one outer
    iteration |s| already meets the target, so the pass ends with
    e = alpha phat, without M(s)."""
    U, eta = _system(621)
    lat = qdd.create_lattice(DIMS, BC)
    qdd.load_gauge(lat, U)
    phi = np.zeros_like(eta)
    p = qdd.default_params(inner_prec="f32", outer_mode=1, inner_tol=1e-6, n_ras=1, n_dominv=4)
    info = qdd.solve(lat, phi, eta, KAPPA, CSW, 1e-5, p)
    assert info["outer_iters"] == 1
    assert oracle_mod.Op(DIMS, BC, U, KAPPA, CSW).true_residual(eta, phi) <= 1e-5


def test_nested_multi_rhs_and_batch(qdd, oracle_mod):
    """Three right-hand sides of one lattice, and two lattices in one batch,
    each with its own outer BiCGStab scalars."""
    U, _ = _system(631)
    etas = [synth.gaussian_source(DIMS, 632 + k) for k in range(3)]
    lat = qdd.create_lattice(DIMS, BC, n_rhs=3)
    qdd.load_gauge(lat, U)
    phi = np.zeros((3,) + etas[0].shape, dtype=np.complex128)
    p = qdd.default_params(inner_prec="f16", outer_mode=1, n_ras=1, n_dominv=4)
    infos = qdd.solve(lat, phi, np.stack(etas), KAPPA, CSW, 1e-10, p)
    op = oracle_mod.Op(DIMS, BC, U, KAPPA, CSW)
    for k in range(3):
        assert op.true_residual(etas[k], phi[k]) <= 1e-10 and infos[k]["status"] == 0
    dims2 = (8, 8, 8, 8)
    U2, eta2 = _system(641, dims2)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    la = qdd.create_lattice(DIMS, BC, stream=s1)
    lb = qdd.create_lattice(dims2, BC, stream=s2)
    qdd.load_gauge(la, U)
    qdd.load_gauge(lb, U2)
    pa, pb = np.zeros_like(etas[0]), np.zeros_like(eta2)
    qdd.solve_batch([la, lb], [pa, pb], [etas[0], eta2], [KAPPA, 0.12], [CSW, CSW], 1e-10, p)
    assert op.true_residual(etas[0], pa) <= 1e-10
    assert oracle_mod.Op(dims2, BC, U2, 0.12, CSW).true_residual(eta2, pb) <= 1e-10


def test_outer_mode_is_validated(qdd):
    U, eta = _system(651)
    lat = qdd.create_lattice(DIMS, BC)
    qdd.load_gauge(lat, U)
    with pytest.raises(qdd.QddError) as e:
        qdd.solve(lat, np.zeros_like(eta), eta, KAPPA, CSW, 1e-10, qdd.default_params(outer_mode=2))
    assert e.value.status == qdd.QDD_ERR_ARG
