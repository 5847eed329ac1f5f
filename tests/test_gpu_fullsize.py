"""The benchmark's 32^4 workload (the paper's lattice size, Sec. 5) in the
launch configuration that bench.py times: 4096 domains of 4^4 sites in one
TMA-staged sweep, reducing dslash epilogues whose resident grid strides over
the lattice several times, and the whole nested solve.

K_RAS with one sweep and no overlap is checked domain by domain: each
domain's bulk output depends only on the source inside that domain (Alg. 1
with NRAS = 1, d = 0), so the oracle's N_dominv MR domain solve of a sampled
domain gives K_RAS there exactly.  The solve is checked by the oracle's FP64
true residual |eta - D phi| / |eta| on the whole lattice."""

import numpy as np
import pytest
import torch

from gpu_common import check_field, qdd, workload_32  # noqa: F401

pytestmark = pytest.mark.gpu

DIMS, BC, KAPPA, CSW = (32, 32, 32, 32), (1, 1, 1, -1), 0.125, 1.0
BLOCK = (4, 4, 4, 4)
TOL_RAS = {"f32": 1e-5, "f16": 1e-2}


@pytest.fixture(scope="module")
def system(qdd, oracle_mod):
    U, eta = workload_32()
    lat = qdd.create_lattice(DIMS, BC)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    op = oracle_mod.Op(DIMS, BC, U, KAPPA, CSW, store_clover=False)
    return U, eta, lat, op


def _sample_domains(op):
    """Domains at every corner of the lattice (periodic x, y, z and the
    antiperiodic t boundary) and a random selection in between."""
    nb = [L // b for L, b in zip(DIMS, BLOCK)]
    doms = {kx + nb[0] * (ky + nb[1] * (kz + nb[2] * kt))
            for kx in (0, nb[0] - 1) for ky in (0, nb[1] - 1) for kz in (0, nb[2] - 1) for kt in (0, nb[3] - 1)}
    rng = np.random.default_rng(5)
    doms |= set(rng.integers(0, op.ndomains(BLOCK, 0), 8).tolist())
    return sorted(doms)


@pytest.mark.parametrize("prec", ["f16", "f32"])
def test_ras_full_size_sampled_domains(qdd, system, prec):
    U, eta, lat, op = system
    p = qdd.default_params(block=BLOCK, overlap=0, n_ras=1, n_dominv=4, inner_prec=prec)
    d_eta = torch.from_numpy(eta).cuda()
    out = torch.empty_like(d_eta)
    qdd.ras_apply(lat, out, d_eta, KAPPA, CSW, p)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    gs, rs = [], []
    for dom in _sample_domains(op):
        sites, bulk = op.domain_sites(BLOCK, 0, dom)
        assert bulk.all()
        ref = op.domain_solve(BLOCK, 0, dom, eta[sites], n_dominv=4)
        check_field(got[sites], ref, TOL_RAS[prec], what=f"domain {dom}")
        gs.append(got[sites])
        rs.append(ref)
    assert sum(len(g) for g in gs) >= 400
    check_field(np.concatenate(gs), np.concatenate(rs), TOL_RAS[prec], what="sampled domains")


@pytest.mark.parametrize("inner_prec", ["f16", "f32"])
def test_nested_solve_full_size(qdd, system, inner_prec):
    """The benchmark's solver configuration (4^4 blocks, d = 0, N_dominv 4,
    NRAS 1, inner tolerance 1e-3) on the benchmark's workload."""
    U, eta, lat, op = system
    d_eta = torch.from_numpy(eta).cuda()
    phi = torch.zeros_like(d_eta)
    p = qdd.default_params(block=BLOCK, overlap=0, n_ras=1, n_dominv=4, inner_prec=inner_prec, inner_tol=1e-3)
    info = qdd.solve(lat, phi, d_eta, KAPPA, CSW, 1e-10, p)
    torch.cuda.synchronize()
    res = op.true_residual(eta, phi.cpu().numpy())
    assert info["status"] == 0 and res <= 1e-10, (info, res)
    assert abs(info["true_rel_residual"] - res) < 1e-11
    assert info["ras_sweeps"] == 2 * info["inner_iters"]


def test_plain_fp64_solve_full_size(qdd, system):
    """The plain FP64 BiCGStab on the GPU (the comparison of the metric)."""
    U, eta, lat, op = system
    d_eta = torch.from_numpy(eta).cuda()
    phi = torch.zeros_like(d_eta)
    info = qdd.solve(lat, phi, d_eta, KAPPA, CSW, 1e-10, qdd.default_params(use_ras=0, inner_prec="f64"))
    torch.cuda.synchronize()
    res = op.true_residual(eta, phi.cpu().numpy())
    assert info["status"] == 0 and res <= 1e-10, (info, res)
