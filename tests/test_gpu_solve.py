"""Every GPU solve meets |eta - D phi| / |eta| <= tol with the oracle's FP64 D."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def setup(qdd, oracle_mod, dims, eps, kappa, gseed=1, sseed=2):
    U = synth.gauge_field(dims, eps, gseed)
    eta = synth.gaussian_source(dims, sseed)
    op = oracle_mod.Op(dims, BC, U, kappa, 1.0, store_clover=int(np.prod(dims)) <= 65536)
    lat = qdd.create_lattice(dims, BC)
    qdd.load_gauge(lat, U)
    return op, lat, eta


def test_config1_plain_fp64(qdd, oracle_mod):
    """8^4, kappa = 0.12: plain FP64 BiCGStab to 1e-10; the solution agrees with
    the oracle's own plain solve to about cond * tol."""
    op, lat, eta = setup(qdd, oracle_mod, (8, 8, 8, 8), 0.3, 0.12)
    phi = np.empty_like(eta)
    info = qdd.solve(lat, phi, eta, 0.12, 1.0, 1e-10, qdd.default_params(inner_prec="f64", use_ras=0))
    assert info["status"] == 0 and info["inner_iters"] > 10
    assert op.true_residual(eta, phi) <= 1e-10
    ref, _ = op.solve(eta, 1e-12)
    assert rel(phi, ref) < 1e-8


@pytest.mark.parametrize("prec,use_ras", [("f32", 0), ("f32", 1), ("f16", 1), ("f16", 0)])
def test_config2_nested(qdd, oracle_mod, prec, use_ras):
    """16^4, kappa = 0.12: FP32/FP16 inner (RAS 4^4, s = 0, N_dominv = 4, inner tol
    1e-3) with FP64 defect correction to 1e-10."""
    op, lat, eta = setup(qdd, oracle_mod, (16, 16, 16, 16), 0.3, 0.12)
    d_eta = torch.from_numpy(eta).cuda()
    d_phi = torch.empty_like(d_eta)
    p = qdd.default_params(inner_prec=prec, use_ras=use_ras, block=(4, 4, 4, 4), overlap=0, n_dominv=4, n_ras=3)
    info = qdd.solve(lat, d_phi, d_eta, 0.12, 1.0, 1e-10, p)
    phi = d_phi.cpu().numpy()
    assert info["status"] == 0 and info["outer_iters"] >= 2
    assert op.true_residual(eta, phi) <= 1e-10
    assert abs(info["true_rel_residual"] - op.true_residual(eta, phi)) < 1e-11


@pytest.mark.parametrize("block,s", [((4, 4, 4, 4), 1), ((8, 4, 4, 4), 0), ((8, 8, 8, 8), 0)])
def test_nested_overlap_and_shapes(qdd, oracle_mod, block, s):
    op, lat, eta = setup(qdd, oracle_mod, (16, 16, 8, 8), 0.3, 0.12, 3, 4)
    phi = np.empty_like(eta)
    p = qdd.default_params(inner_prec="f32", block=block, overlap=s)
    info = qdd.solve(lat, phi, eta, 0.12, 1.0, 1e-10, p)
    assert info["status"] == 0
    assert op.true_residual(eta, phi) <= 1e-10


def test_zero_source_gives_zero(qdd, oracle_mod):
    op, lat, eta = setup(qdd, oracle_mod, (4, 4, 4, 4), 0.3, 0.12)
    z = np.zeros_like(eta)
    phi = np.ones_like(eta)
    info = qdd.solve(lat, phi, z, 0.12, 1.0, 1e-10)
    assert info["status"] == 0 and np.abs(phi).max() == 0


def test_point_source(qdd, oracle_mod):
    dims = (8, 8, 8, 8)
    op, lat, _ = setup(qdd, oracle_mod, dims, 0.25, 0.124)
    eta = synth.point_source(dims, 1, 2)
    phi = np.empty_like(eta)
    info = qdd.solve(lat, phi, eta, 0.124, 1.0, 1e-10, qdd.default_params(inner_prec="f16"))
    assert info["status"] == 0 and op.true_residual(eta, phi) <= 1e-10


def test_nonfinite_source_is_reported(qdd, oracle_mod):
    op, lat, eta = setup(qdd, oracle_mod, (4, 4, 4, 4), 0.3, 0.12)
    eta[3, 1, 1] = np.nan
    phi = np.empty_like(eta)
    with pytest.raises(qdd.QddError) as e:
        qdd.solve(lat, phi, eta, 0.12, 1.0, 1e-10)
    assert e.value.status == qdd.QDD_ERR_NONFINITE


def test_iteration_budget_returns_best_iterate(qdd, oracle_mod):
    op, lat, eta = setup(qdd, oracle_mod, (8, 8, 8, 8), 0.3, 0.12)
    phi = np.empty_like(eta)
    p = qdd.default_params(inner_prec="f32", max_outer=1)
    info = qdd.solve(lat, phi, eta, 0.12, 1.0, 1e-12, p, raise_on_failure=False)
    assert info["return_status"] == qdd.QDD_ERR_NOT_CONVERGED
    r = op.true_residual(eta, phi)
    assert r < 1e-2 and abs(r - info["true_rel_residual"]) < 1e-6


def test_autotune_returns_converging_parameters(qdd, oracle_mod):
    """The tuner's choice solves the system to the tolerance, and its reported
    time is that of a converged solve."""
    op, lat, eta = setup(qdd, oracle_mod, (8, 8, 8, 8), 0.3, 0.12)
    p, best = qdd.autotune(lat, eta, 0.12, 1.0, 1e-10, qdd.default_params(inner_prec="f16"), max_trials=12)
    assert best > 0 and p.n_dominv >= 1 and p.n_ras >= 1
    assert all(8 % b == 0 for b in p.block)
    phi = np.empty_like(eta)
    info = qdd.solve(lat, phi, eta, 0.12, 1.0, 1e-10, p)
    assert info["status"] == 0 and op.true_residual(eta, phi) <= 1e-10


def test_point_source_far_field_fp16(qdd, oracle_mod):
    """A point source on 16^4: the Krylov vectors decay like kappa^d away from
    the source and reach FP32 denormals, which the FP16 store must flush
    rather than turn into inf/NaN."""
    dims = (16, 16, 16, 16)
    op, lat, _ = setup(qdd, oracle_mod, dims, 0.25, 0.124)
    eta = synth.point_source(dims, 0, 0)
    phi = np.empty_like(eta)
    for prec in ("f16", "f32"):
        info = qdd.solve(lat, phi, eta, 0.124, 1.0, 1e-10, qdd.default_params(inner_prec=prec))
        assert info["status"] == 0 and op.true_residual(eta, phi) <= 1e-10


@pytest.mark.parametrize("stream", [False, True])
def test_back_to_back_host_solves(qdd, oracle_mod, stream):
    """Host sources are copied on the lattice's copy stream while the clover
    term is built: consecutive solves with different sources, kappas and a
    reloaded gauge field (host links, chunked copy and conversion at 16^4)
    must each see their own inputs."""
    dims = (16, 16, 16, 16)
    s = torch.cuda.Stream() if stream else None
    lat = qdd.create_lattice(dims, BC, stream=s)
    p = qdd.default_params(inner_prec="f16")
    for k, (gseed, sseed, kappa) in enumerate([(5, 6, 0.12), (5, 7, 0.121), (8, 9, 0.12)]):
        U = synth.gauge_field(dims, 0.3, gseed)
        eta = synth.gaussian_source(dims, sseed)
        if k != 1:
            qdd.load_gauge(lat, U)
        phi = np.empty_like(eta)
        info = qdd.solve(lat, phi, eta, kappa, 1.0, 1e-10, p)
        op = oracle_mod.Op(dims, BC, U, kappa, 1.0, store_clover=True)
        assert info["status"] == 0 and op.true_residual(eta, phi) <= 1e-10
