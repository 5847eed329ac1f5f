"""The TMA-staged RAS sweep: same result as the per-thread staging (and the
oracle) where it applies, with several right-hand sides, and a bounded wait
that gives up with QDD_ERR_TIMEOUT while the CUDA context stays usable."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import check_field, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

# FP32 arithmetic on identical inputs: the two stagings differ only in the
# order of nothing (same loads, same sums), so they agree to rounding noise.
TOL_SAME = {"f32": 1e-6, "f16": 1e-3}
TOL_ORACLE = {"f32": 1e-5, "f16": 1e-2}


def _ras(qdd, lat, eta, p):
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, 0.125, 1.0, p)
    return out


@pytest.mark.parametrize("dims,block", [((8, 8, 8, 8), (4, 4, 4, 4)), ((8, 8, 8, 16), (8, 4, 4, 2)),
                                        ((12, 8, 4, 8), (4, 4, 4, 4)), ((8, 8, 8, 8), (4, 4, 4, 2)),
                                        ((8, 4, 8, 8), (4, 2, 4, 4))])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_tma_staging_matches_per_thread_staging(qdd, oracle_mod, dims, block, prec):
    bc = (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 41)
    eta = synth.gaussian_source(dims, 42)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    tma = _ras(qdd, lat, eta, qdd.default_params(block=block, n_ras=2, n_dominv=3, inner_prec=prec, ras_kernel=0))
    per_thread = _ras(qdd, lat, eta, qdd.default_params(block=block, n_ras=2, n_dominv=3, inner_prec=prec,
                                                        ras_kernel=1))
    ref = oracle_mod.Op(dims, bc, U, 0.125, 1.0).ras(eta, block, s=0, n_ras=2, n_dominv=3)
    assert rel(tma, per_thread) <= TOL_SAME[prec]
    check_field(tma, ref, TOL_ORACLE[prec], dims, block)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_tma_staging_multi_rhs(qdd, oracle_mod, prec):
    """Right-hand side r of a multi-RHS field is the plane block r of the
    tensor map: each must get its own RAS."""
    dims, bc, block, n = (8, 8, 8, 8), (1, 1, 1, -1), (4, 4, 4, 4), 3
    U = synth.gauge_field(dims, 0.3, 43)
    etas = [synth.gaussian_source(dims, 44 + k) for k in range(n)]
    lat = qdd.create_lattice(dims, bc, n_rhs=n)
    qdd.load_gauge(lat, U)
    eta = np.stack(etas)
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, 0.125, 1.0, qdd.default_params(block=block, n_ras=1, n_dominv=4, inner_prec=prec))
    op = oracle_mod.Op(dims, bc, U, 0.125, 1.0)
    for k in range(n):
        ref = op.ras(etas[k], block, s=0, n_ras=1, n_dominv=4)
        check_field(out[k], ref, TOL_ORACLE[prec], dims, block)


def test_tma_wait_times_out_and_context_survives(qdd, oracle_mod):
    """A sweep whose mbarrier expects bytes that never arrive gives up after
    its bounded wait: the RAS call and a solve report QDD_ERR_TIMEOUT, and the
    next calls on the same lattice are correct."""
    dims, bc, block = (8, 8, 8, 8), (1, 1, 1, -1), (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 45)
    eta = synth.gaussian_source(dims, 46)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    p = qdd.default_params(block=block, n_ras=1, n_dominv=2, inner_prec="f16")
    d_eta = torch.from_numpy(eta).cuda()
    out = torch.empty_like(d_eta)
    try:
        qdd.test_ras_wait(extra_bytes=16, max_polls=4)
        with pytest.raises(qdd.QddError) as e:
            qdd.ras_apply(lat, out, d_eta, 0.125, 1.0, p)
        assert e.value.status == qdd.QDD_ERR_TIMEOUT
        phi = torch.zeros_like(d_eta)
        with pytest.raises(qdd.QddError) as e:
            qdd.solve(lat, phi, d_eta, 0.125, 1.0, 1e-10, p)
        assert e.value.status == qdd.QDD_ERR_TIMEOUT
    finally:
        qdd.test_ras_wait(0, 0)
    qdd.ras_apply(lat, out, d_eta, 0.125, 1.0, p)
    torch.cuda.synchronize()
    ref = oracle_mod.Op(dims, bc, U, 0.125, 1.0).ras(eta, block, s=0, n_ras=1, n_dominv=2)
    assert rel(out.cpu().numpy(), ref) <= TOL_ORACLE["f16"]
    phi = torch.zeros_like(d_eta)
    info = qdd.solve(lat, phi, d_eta, 0.125, 1.0, 1e-10, p)
    res = oracle_mod.Op(dims, bc, U, 0.125, 1.0).true_residual(eta, phi.cpu().numpy())
    assert res <= 1e-10 and info["true_rel_residual"] <= 1e-10
