"""The phased sweep: few large domains (the paper's x-slabs, or one domain
covering the lattice), each spread over many CTAs with one launch per MR
step, against the oracle and against the one-CTA-per-domain general kernel."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import check_field, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f16": 1e-2}
TOL_KERNELS = {"f32": 1e-5, "f16": 2e-3}

CASES = [
    ((16, 8, 8, 8), (8, 8, 8, 8), 0),     # two x-slabs
    ((16, 8, 8, 8), (8, 8, 8, 8), 1),     # two x-slabs, d = 2
    ((16, 8, 8, 8), (4, 8, 8, 8), 2),     # four x-slabs, d = 4
    ((16, 8, 8, 8), (2, 8, 8, 8), 1),     # eight x-slabs, d = 2
    ((8, 8, 8, 8), (8, 8, 8, 8), 0),      # one domain: the whole lattice
    ((12, 8, 8, 6), (6, 8, 8, 6), 1),     # ragged CTA tail (6 x 8 x 8 x 6 bulk)
]


def _ras(qdd, lat, eta, **kw):
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, 0.12, 1.0, qdd.default_params(**kw))
    return out


@pytest.mark.parametrize("dims,block,s", CASES)
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_phased_sweep_matches_oracle_and_general_kernel(qdd, oracle_mod, dims, block, s, prec):
    bc = (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 701)
    eta = synth.gaussian_source(dims, 702)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    kw = dict(block=block, overlap=s, n_ras=2, n_dominv=3, inner_prec=prec)
    ph = _ras(qdd, lat, eta, **kw)
    gm = _ras(qdd, lat, eta, ras_kernel=3, **kw)
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=2, n_dominv=3)
    check_field(ph, ref, TOL[prec], dims, block)
    assert rel(ph, gm) <= TOL_KERNELS[prec]


@pytest.mark.parametrize("schwarz", ["sap", "as"])
def test_phased_sweep_schwarz_variants(qdd, oracle_mod, schwarz):
    dims, bc, block, s = (16, 8, 8, 8), (1, 1, 1, -1), (4, 8, 8, 8), 1
    U = synth.gauge_field(dims, 0.3, 711)
    eta = synth.gaussian_source(dims, 712)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    out = _ras(qdd, lat, eta, block=block, overlap=s, n_ras=2, n_dominv=3, inner_prec="f32", schwarz=schwarz)
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=2, n_dominv=3, schwarz=schwarz)
    check_field(out, ref, TOL["f32"], dims, block)


def test_phased_sweep_multi_rhs(qdd, oracle_mod):
    dims, bc, block, s, n = (16, 8, 8, 8), (1, 1, 1, -1), (8, 8, 8, 8), 1, 3
    U = synth.gauge_field(dims, 0.3, 721)
    etas = [synth.gaussian_source(dims, 722 + k) for k in range(n)]
    lat = qdd.create_lattice(dims, bc, n_rhs=n)
    qdd.load_gauge(lat, U)
    out = _ras(qdd, lat, np.stack(etas), block=block, overlap=s, n_ras=2, n_dominv=3, inner_prec="f32")
    op = oracle_mod.Op(dims, bc, U, 0.12, 1.0)
    for k in range(n):
        check_field(out[k], op.ras(etas[k], block, s=s, n_ras=2, n_dominv=3), TOL["f32"], dims, block)


@pytest.mark.parametrize("s", [0, 1])
@pytest.mark.parametrize("stream", [False, True])
def test_slab_solve(qdd, oracle_mod, s, stream):
    """The paper's layout at a small size: four x-slab domains, NRAS 3,
    N_dominv 5, FP32 inner, solved to 1e-12 (eager and graph launches)."""
    dims, bc = (16, 8, 8, 8), (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 731)
    eta = synth.gaussian_source(dims, 732)
    lat = qdd.create_lattice(dims, bc, stream=torch.cuda.Stream() if stream else None)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    d_eta = torch.from_numpy(eta).cuda()
    phi = torch.zeros_like(d_eta)
    p = qdd.default_params(block=(4, 8, 8, 8), overlap=s, n_ras=3, n_dominv=5, inner_prec="f32")
    info = qdd.solve(lat, phi, d_eta, 0.124, 1.0, 1e-12, p)
    torch.cuda.synchronize()
    res = oracle_mod.Op(dims, bc, U, 0.124, 1.0).true_residual(eta, phi.cpu().numpy())
    assert res <= 1e-12 and info["status"] == 0
