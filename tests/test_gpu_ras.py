"""K_RAS (Alg. 1) on the GPU against the oracle's RAS with the same blocking,
overlap, MR iteration count and sweep count."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import check_field, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

# The domain solves are MR in FP32 arithmetic; MR is a non-linear map of its
# input, and the FP32 rounding of ~N_dominv * NRAS steps is amplified by the
# conditioning of the domain operators; 1e-5 leaves a margin of ~10x over the
# observed error.  FP16 storage of the fields adds 2^-11 per stored vector.
TOL_RAS = {"f32": 1e-5, "f16": 1e-2}

CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), 0),    # the paper's best: no overlap (d = 0)
    ((8, 8, 8, 8), (8, 4, 4, 4), 0),    # 8x4^3 blocks, 512-site domains
    ((8, 8, 8, 8), (4, 4, 4, 4), 1),    # d = 2: 6^4 extended domains (general kernel)
    ((8, 8, 8, 8), (4, 4, 4, 4), 2),    # d = 4: extension wraps to the full extent
    ((8, 4, 4, 8), (4, 4, 4, 8), 0),    # t not decomposed: hops wrap inside the domain
    ((6, 4, 4, 8), (2, 2, 2, 2), 1),    # small blocks, ragged block count
    ((8, 8, 8, 8), (2, 4, 4, 4), 0),    # 128-site domains: expanded FP32 staging
    ((8, 8, 8, 8), (2, 2, 2, 2), 0),    # 16-site domains in 32-thread CTAs
    ((8, 4, 4, 8), (2, 2, 4, 4), 0),    # 64-site domains
    ((4, 4, 4, 8), (2, 2, 2, 8), 0),    # t not decomposed with expanded staging
]


@pytest.mark.parametrize("dims,block,s", CASES)
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_ras_matches_oracle(qdd, oracle_mod, dims, block, s, prec):
    bc, kappa, csw = (1, 1, 1, -1), 0.12, 1.0
    U = synth.gauge_field(dims, 0.3, 3)
    eta = synth.gaussian_source(dims, 4)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).ras(eta, block, s=s, n_ras=3, n_dominv=4)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, overlap=s, n_ras=3, n_dominv=4, inner_prec=prec)
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, kappa, csw, p)
    check_field(out, ref, TOL_RAS[prec], dims, block)


@pytest.mark.parametrize("n_ras,n_dominv", [(1, 1), (1, 5), (4, 2), (2, 0)])
def test_ras_parameters(qdd, oracle_mod, n_ras, n_dominv):
    dims, bc, kappa, csw = (8, 8, 8, 8), (1, 1, 1, -1), 0.125, 1.0
    U = synth.gauge_field(dims, 0.3, 7)
    eta = synth.gaussian_source(dims, 8)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).ras(eta, (4, 4, 4, 4), s=0, n_ras=n_ras, n_dominv=n_dominv)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    p = qdd.default_params(n_ras=n_ras, n_dominv=n_dominv, inner_prec="f32")
    d_eta = torch.from_numpy(eta).cuda()
    out = torch.empty_like(d_eta)
    qdd.ras_apply(lat, out, d_eta, kappa, csw, p)
    torch.cuda.synchronize()
    if n_dominv == 0:
        assert np.abs(out.cpu().numpy()).max() == 0
    else:
        check_field(out.cpu().numpy(), ref, TOL_RAS["f32"], dims, (4, 4, 4, 4))


def test_ras_rejects_bad_blocking(qdd):
    dims = (8, 8, 8, 8)
    lat = qdd.create_lattice(dims)
    qdd.load_gauge(lat, synth.gauge_field(dims, 0.3, 1))
    eta = synth.gaussian_source(dims, 2)
    for kw in (dict(block=(3, 4, 4, 4)), dict(block=(4, 4, 4, 4), overlap=3)):
        p = qdd.default_params(**kw)
        with pytest.raises(qdd.QddError) as e:
            qdd.ras_apply(lat, np.empty_like(eta), eta, 0.12, 1.0, p)
        assert e.value.status == qdd.QDD_ERR_ARG


@pytest.mark.parametrize("block", [(2, 2, 2, 2), (2, 2, 4, 4), (2, 4, 4, 4), (4, 4, 4, 4)])
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_ras_staging_variants(qdd, oracle_mod, block, variant, prec):
    """Compact (field-format) and expanded (FP32) staging of links and clover
    give the oracle's RAS at every domain size they apply to."""
    dims, bc, kappa, csw = (8, 8, 8, 8), (1, 1, 1, -1), 0.125, 1.0
    U = synth.gauge_field(dims, 0.3, 17)
    eta = synth.gaussian_source(dims, 18)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).ras(eta, block, s=0, n_ras=2, n_dominv=3)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, n_ras=2, n_dominv=3, inner_prec=prec, ras_kernel=variant)
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, kappa, csw, p)
    check_field(out, ref, TOL_RAS[prec], dims, block)
