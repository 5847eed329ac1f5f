"""The thread-block-cluster sweep (one cluster per extended domain, one CTA
per t-slice, t hops and the MR dot products through distributed shared
memory) against the oracle and against the general global-scratch kernel, for
the overlapping domains it serves: 6^4 (4^4 blocks, d = 2) and 8^4 (d = 4)
extended domains, a whole-lattice t direction that wraps across the cluster,
several right-hand sides, and the Schwarz variants."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import check_field, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f16": 1e-2}   # the RAS parity tolerances
# cluster and general kernel: same FP32 arithmetic, sums in another order
TOL_KERNELS = {"f32": 1e-5, "f16": 2e-3}

CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), 1),     # 6^4: six CTAs of 216 sites (224 threads)
    ((8, 8, 8, 8), (4, 4, 4, 4), 2),     # 8^4: eight CTAs of 512 sites, extension wraps
    ((8, 8, 8, 4), (4, 4, 4, 4), 1),     # t not decomposed: hops wrap from the last CTA to the first
    ((12, 8, 8, 8), (4, 4, 4, 4), 1),    # three blocks in x
    ((8, 8, 8, 8), (4, 2, 4, 4), 1),     # 6x4x6 slices of 144 sites
    ((16, 8, 8, 8), (8, 4, 4, 2), 1),    # 10x6x6 slices of 360 sites, four CTAs
]


def _ras(qdd, lat, eta, **kw):
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, 0.12, 1.0, qdd.default_params(**kw))
    return out


@pytest.mark.parametrize("dims,block,s", CASES)
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_cluster_sweep_matches_oracle_and_general_kernel(qdd, oracle_mod, dims, block, s, prec):
    bc = (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 501)
    eta = synth.gaussian_source(dims, 502)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    kw = dict(block=block, overlap=s, n_ras=2, n_dominv=4, inner_prec=prec)
    cl = _ras(qdd, lat, eta, **kw)
    gm = _ras(qdd, lat, eta, ras_kernel=3, **kw)
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=2, n_dominv=4)
    check_field(cl, ref, TOL[prec], dims, block)
    assert rel(cl, gm) <= TOL_KERNELS[prec]


@pytest.mark.parametrize("schwarz", ["sap", "as"])
def test_cluster_sweep_schwarz_variants(qdd, oracle_mod, schwarz):
    dims, bc, block, s = (8, 8, 8, 8), (1, 1, 1, -1), (4, 4, 4, 4), 2
    U = synth.gauge_field(dims, 0.3, 511)
    eta = synth.gaussian_source(dims, 512)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    out = _ras(qdd, lat, eta, block=block, overlap=s, n_ras=2, n_dominv=3, inner_prec="f32", schwarz=schwarz)
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=2, n_dominv=3, schwarz=schwarz)
    check_field(out, ref, TOL["f32"], dims, block)


def test_cluster_sweep_multi_rhs(qdd, oracle_mod):
    dims, bc, block, s, n = (8, 8, 8, 8), (1, 1, 1, -1), (4, 4, 4, 4), 1, 3
    U = synth.gauge_field(dims, 0.3, 521)
    etas = [synth.gaussian_source(dims, 522 + k) for k in range(n)]
    lat = qdd.create_lattice(dims, bc, n_rhs=n)
    qdd.load_gauge(lat, U)
    out = _ras(qdd, lat, np.stack(etas), block=block, overlap=s, n_ras=2, n_dominv=4, inner_prec="f16")
    op = oracle_mod.Op(dims, bc, U, 0.12, 1.0)
    for k in range(n):
        check_field(out[k], op.ras(etas[k], block, s=s, n_ras=2, n_dominv=4), TOL["f16"], dims, block)


def test_more_than_eight_slices_use_the_general_kernel(qdd, oracle_mod):
    """e_t = 10 exceeds the portable cluster size: the general kernel runs."""
    dims, bc, block, s = (8, 8, 8, 16), (1, 1, 1, -1), (4, 4, 4, 8), 1
    U = synth.gauge_field(dims, 0.3, 531)
    eta = synth.gaussian_source(dims, 532)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    out = _ras(qdd, lat, eta, block=block, overlap=s, n_ras=1, n_dominv=3, inner_prec="f32")
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=1, n_dominv=3)
    check_field(out, ref, TOL["f32"], dims, block)


@pytest.mark.parametrize("s", [1, 2])
def test_solve_with_cluster_sweeps(qdd, oracle_mod, s):
    dims, bc = (16, 16, 16, 16), (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 541)
    eta = synth.gaussian_source(dims, 542)
    lat = qdd.create_lattice(dims, bc, stream=torch.cuda.Stream())
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    d_eta = torch.from_numpy(eta).cuda()
    phi = torch.zeros_like(d_eta)
    p = qdd.default_params(block=(4, 4, 4, 4), overlap=s, n_ras=1, n_dominv=4, inner_prec="f16")
    info = qdd.solve(lat, phi, d_eta, 0.12, 1.0, 1e-10, p)
    torch.cuda.synchronize()
    res = oracle_mod.Op(dims, bc, U, 0.12, 1.0).true_residual(eta, phi.cpu().numpy())
    assert res <= 1e-10 and info["true_rel_residual"] <= 1e-10
