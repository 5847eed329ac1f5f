"""Wilson-clover D (Eq. 1) on the GPU against the FP64 oracle, element by
element, in all three precisions, through host and device pointers."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import TOL_D, max_elem, qdd, rel, workload_32  # noqa: F401

pytestmark = pytest.mark.gpu

SHAPES = [
    ((8, 8, 8, 8), (1, 1, 1, -1)),      # 16 blocks of 256 sites
    ((6, 4, 4, 10), (1, 1, 1, -1)),     # ragged tail: 960 sites
    ((5, 6, 3, 4), (-1, 1, 1, 1)),      # odd extents, antiperiodic x
    ((4, 1, 4, 2), (1, 1, -1, -1)),     # extent 1 and 2: both hops reach the same site
]


@pytest.mark.parametrize("dims,bc", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_dslash_matches_oracle(qdd, oracle_mod, dims, bc, prec):
    kappa, csw = 0.12, 1.0
    U = synth.gauge_field(dims, 0.3, 1)
    psi = synth.gaussian_source(dims, 2)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).dslash(psi)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    out = np.empty_like(psi)
    qdd.dslash(lat, out, psi, kappa, csw, prec)             # host buffers
    assert rel(out, ref) <= TOL_D[prec]
    assert max_elem(out, ref) <= 10 * TOL_D[prec]
    dpsi = torch.from_numpy(psi).cuda()
    dout = torch.empty_like(dpsi)
    qdd.dslash(lat, dout, dpsi, kappa, csw, prec)           # device buffers
    torch.cuda.synchronize()
    assert rel(dout.cpu().numpy(), ref) <= TOL_D[prec]


@pytest.mark.parametrize("kappa,csw", [(0.0, 1.0), (0.125, 0.0), (0.137, 1.9)])
def test_dslash_parameters(qdd, oracle_mod, kappa, csw):
    dims, bc = (4, 4, 4, 8), (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 5)
    psi = synth.gaussian_source(dims, 6)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).dslash(psi)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    for prec in ("f64", "f32"):
        out = np.empty_like(psi)
        qdd.dslash(lat, out, psi, kappa, csw, prec)
        assert rel(out, ref) <= TOL_D[prec]


def test_dslash_full_size_sampled(qdd, oracle_mod):
    """32^4 (the paper's lattice) in the launch configuration of the benchmark
    (internal fields, one dslash launch), checked at sampled sites, including
    the corners and every face, against the oracle computed site by site."""
    dims, bc, kappa, csw = (32, 32, 32, 32), (1, 1, 1, -1), 0.125, 1.0
    U, psi = workload_32()
    V = int(np.prod(dims))
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    rng = np.random.default_rng(0)
    corners = [x + 32 * (y + 32 * (z + 32 * t)) for x in (0, 31) for y in (0, 31) for z in (0, 31) for t in (0, 31)]
    sites = np.unique(np.concatenate([corners, rng.integers(0, V, 400)]))
    op = oracle_mod.Op(dims, bc, U, kappa, csw, store_clover=False)
    ref = op.dslash_sites(psi, sites)
    dpsi = torch.from_numpy(psi).cuda()
    for prec in ("f64", "f32", "f16"):
        fin = qdd.field_create(lat, prec)
        fout = qdd.field_create(lat, prec)
        qdd.field_import(fin, dpsi)
        qdd.dslash_field(lat, fout, fin, kappa, csw)
        dout = torch.empty_like(dpsi)
        qdd.field_export(fout, dout)
        torch.cuda.synchronize()
        got = dout.cpu().numpy()[sites]
        assert rel(got, ref) <= TOL_D[prec], prec
        assert max_elem(got, ref) <= 10 * TOL_D[prec], prec


def test_load_gauge_rejects_non_su3(qdd):
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1)
    U[17, 2] *= np.exp(0.1j)      # unitary but det != 1
    lat = qdd.create_lattice(dims)
    with pytest.raises(qdd.QddError) as e:
        qdd.load_gauge(lat, U)
    assert e.value.status == qdd.QDD_ERR_ARG
    U[17, 2] = 1.001 * np.eye(3)  # not unitary
    with pytest.raises(qdd.QddError):
        qdd.load_gauge(lat, U)
    psi = synth.gaussian_source(dims, 2)
    with pytest.raises(qdd.QddError) as e:
        qdd.dslash(lat, np.empty_like(psi), psi, 0.1, 1.0, "f32")
    assert e.value.status == qdd.QDD_ERR_STATE


def test_load_gauge_rejects_nan_links(qdd):
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1)
    U[5, 1, 2, 0] = np.nan
    lat = qdd.create_lattice(dims)
    with pytest.raises(qdd.QddError) as e:
        qdd.load_gauge(lat, U)
    assert e.value.status == qdd.QDD_ERR_ARG


@pytest.mark.parametrize("dims,host", [((16, 16, 8, 32), True), ((8, 8, 4, 16), True), ((8, 8, 4, 16), False), ((6, 4, 4, 10), True)])
def test_load_gauge_with_clover(qdd, oracle_mod, dims, host):
    """qdd_load_gauge_clover builds the clover term while the links load (for
    host links and Lt = 16 or 32, in 8 groups of t-slices as the neighbouring
    groups arrive; otherwise after the conversion): D equals the oracle's, and bit
    for bit the D of a lattice whose clover is built lazily by the first D."""
    bc, kappa, csw = (1, 1, 1, -1), 0.124, 1.3
    U = synth.gauge_field(dims, 0.3, 21)
    psi = synth.gaussian_source(dims, 22)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).dslash(psi)
    a = qdd.create_lattice(dims, bc)
    qdd.load_gauge(a, U if host else torch.from_numpy(U).cuda(), kappa, csw)
    b = qdd.create_lattice(dims, bc)
    qdd.load_gauge(b, U)
    for prec in ("f64", "f32", "f16"):
        oa, ob = np.empty_like(psi), np.empty_like(psi)
        qdd.dslash(a, oa, psi, kappa, csw, prec)
        qdd.dslash(b, ob, psi, kappa, csw, prec)
        assert np.array_equal(oa, ob), prec
        assert rel(oa, ref) <= TOL_D[prec] and max_elem(oa, ref) <= 10 * TOL_D[prec], prec


def test_load_gauge_with_clover_rejects_non_su3(qdd):
    dims = (8, 8, 4, 16)
    U = synth.gauge_field(dims, 0.3, 23)
    U[300, 1] *= np.exp(0.2j)
    lat = qdd.create_lattice(dims)
    with pytest.raises(qdd.QddError) as e:
        qdd.load_gauge(lat, U, 0.12, 1.0)
    assert e.value.status == qdd.QDD_ERR_ARG
    psi = synth.gaussian_source(dims, 24)
    with pytest.raises(qdd.QddError) as e:
        qdd.dslash(lat, np.empty_like(psi), psi, 0.12, 1.0, "f32")
    assert e.value.status == qdd.QDD_ERR_STATE
