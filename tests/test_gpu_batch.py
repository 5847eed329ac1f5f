"""Multi-RHS lattices and uneven batches (one captured graph) against the
oracle: every right-hand side of every system meets the FP64 residual."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import TOL_D, check_field, max_elem, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.mark.parametrize("prec,R", [("f64", 3), ("f32", 3), ("f16", 12), ("f16", 5), ("f16", 2)])
def test_multi_rhs_dslash(qdd, oracle_mod, prec, R):
    """Every right-hand side of a multi-RHS D against the oracle, element by
    element: FP16 lattices run the kernel that takes two right-hand sides per
    thread (R = 12 as in the point-source workload; an odd R leaves a last
    pair with one right-hand side)."""
    dims, kappa, csw = (4, 4, 6, 8), 0.124, 1.0
    U = synth.gauge_field(dims, 0.25, 1)
    src = np.stack([synth.gaussian_source(dims, 10 + r) for r in range(R)])
    op = oracle_mod.Op(dims, BC, U, kappa, csw)
    lat = qdd.create_lattice(dims, BC, n_rhs=R)
    qdd.load_gauge(lat, U)
    out = np.empty_like(src)
    qdd.dslash(lat, out, src, kappa, csw, prec)
    for r in range(R):
        ref = op.dslash(src[r])
        assert rel(out[r], ref) <= TOL_D[prec], r
        assert max_elem(out[r], ref) <= 10 * TOL_D[prec], r


def test_multi_rhs_residual_epilogue(qdd, oracle_mod):
    """K_RAS with two sweeps on a 4-right-hand-side FP16 lattice: between the
    sweeps the two-right-hand-side D runs its residual epilogue
    (r = r_in - D v) for every right-hand side; each result against the
    oracle's Alg. 1."""
    dims, R, kappa, csw, block = (8, 8, 4, 8), 4, 0.12, 1.0, (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 3)
    src = np.stack([synth.gaussian_source(dims, 30 + r) for r in range(R)])
    op = oracle_mod.Op(dims, BC, U, kappa, csw)
    lat = qdd.create_lattice(dims, BC, n_rhs=R)
    qdd.load_gauge(lat, U)
    out = np.empty_like(src)
    qdd.ras_apply(lat, out, src, kappa, csw, qdd.default_params(block=block, n_ras=2, n_dominv=3, inner_prec="f16"))
    for r in range(R):
        check_field(out[r], op.ras(src[r], block, s=0, n_ras=2, n_dominv=3), 1e-2, dims, block, what=f"rhs {r}")


@pytest.mark.parametrize("stream", [False, True])
def test_multi_rhs_point_sources(qdd, oracle_mod, stream):
    """12 unit point sources at the origin (one per spin-colour index) on one
    lattice: FP16 inner with RAS, FP64 outer; eager (default stream) and
    graph (own stream) execution."""
    dims, kappa, csw = (8, 8, 4, 8), 0.124, 1.0
    U = synth.gauge_field(dims, 0.25, 1)
    src = np.stack([synth.point_source(dims, s, c) for s in range(4) for c in range(3)])
    op = oracle_mod.Op(dims, BC, U, kappa, csw)
    st = torch.cuda.Stream() if stream else None
    lat = qdd.create_lattice(dims, BC, n_rhs=12, stream=st)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    d_src = torch.from_numpy(src).cuda()
    d_phi = torch.empty_like(d_src)
    infos = qdd.solve(lat, d_phi, d_src, kappa, csw, 1e-10, qdd.default_params(inner_prec="f16"))
    phi = d_phi.cpu().numpy()
    assert len(infos) == 12
    for r in range(12):
        assert infos[r]["status"] == 0
        assert op.true_residual(src[r], phi[r]) <= 1e-10


def test_uneven_batch_one_graph(qdd, oracle_mod):
    """Independent systems of different shapes, kappas and eps, solved in
    lockstep (one graph over the lattices' streams)."""
    draws = [((4, 4, 4, 4), 0.2, 0.11), ((6, 6, 6, 6), 0.35, 0.124), ((8, 4, 4, 8), 0.3, 0.12), ((4, 4, 4, 12), 0.25, 0.118)]
    lats, phis, etas, ops = [], [], [], []
    for k, (dims, eps, kappa) in enumerate(draws):
        U = synth.gauge_field(dims, eps, 100 + k)
        eta = synth.gaussian_source(dims, 200 + k)
        lat = qdd.create_lattice(dims, BC, stream=torch.cuda.Stream())
        qdd.load_gauge(lat, U)
        lats.append(lat)
        etas.append(torch.from_numpy(eta).cuda())
        phis.append(torch.empty_like(etas[-1]))
        ops.append((oracle_mod.Op(dims, BC, U, kappa, 1.0), eta))
    p = qdd.default_params(inner_prec="f16", block=(2, 2, 2, 2))
    infos = qdd.solve_batch(lats, phis, etas, [d[2] for d in draws], [1.0] * len(draws), 1e-10, p)
    for (op, eta), phi, info in zip(ops, phis, infos):
        assert info[0]["status"] == 0
        assert op.true_residual(eta, phi.cpu().numpy()) <= 1e-10


def test_batch_matches_single_solves(qdd, oracle_mod):
    """A batch gives each system the solution a separate solve gives (same
    unique D^{-1} eta to about cond * tol)."""
    dims = (4, 4, 4, 8)
    lats, phis, etas, singles = [], [], [], []
    for k in range(3):
        U = synth.gauge_field(dims, 0.3, 300 + k)
        eta = synth.gaussian_source(dims, 400 + k)
        lat = qdd.create_lattice(dims, BC, stream=torch.cuda.Stream())
        qdd.load_gauge(lat, U)
        one = np.empty_like(eta)
        qdd.solve(lat, one, eta, 0.12, 1.0, 1e-11)
        singles.append(one)
        lats.append(lat)
        etas.append(eta)
        phis.append(np.empty_like(eta))
    qdd.solve_batch(lats, phis, etas, [0.12] * 3, [1.0] * 3, 1e-11)
    for a, b in zip(phis, singles):
        assert rel(a, b) < 1e-8


@pytest.mark.parametrize("graph", [False, True])
def test_uneven_batch_per_lattice_parameters(qdd, oracle_mod, graph):
    """Each lattice of a batch solved with its own RAS blocking, n_ras,
    n_dominv and inner precision (qdd_solve_batch_each): every system meets
    the oracle's FP64 residual, and each lattice's sweep count follows its
    own n_ras."""
    draws = [((8, 8, 8, 8), 0.3, 0.12, dict(block=(4, 4, 4, 4), n_ras=1, n_dominv=4, inner_prec="f16")),
             ((8, 8, 4, 8), 0.25, 0.118, dict(block=(4, 4, 4, 2), n_ras=2, n_dominv=3, inner_prec="f32")),
             ((4, 4, 4, 12), 0.35, 0.12, dict(block=(2, 2, 2, 2), n_ras=3, n_dominv=2, inner_prec="f16"))]
    lats, phis, etas, ops, params = [], [], [], [], []
    for k, (dims, eps, kappa, kw) in enumerate(draws):
        U = synth.gauge_field(dims, eps, 300 + k)
        eta = synth.gaussian_source(dims, 400 + k)
        lat = qdd.create_lattice(dims, BC, stream=torch.cuda.Stream() if graph else None)
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        lats.append(lat)
        etas.append(torch.from_numpy(eta).cuda())
        phis.append(torch.zeros_like(etas[-1]))
        ops.append((oracle_mod.Op(dims, BC, U, kappa, 1.0), eta))
        params.append(qdd.default_params(**kw))
    infos = qdd.solve_batch(lats, phis, etas, [d[2] for d in draws], [1.0] * 3, 1e-10, params)
    torch.cuda.synchronize()
    for k in range(3):
        op, eta = ops[k]
        info = infos[k][0]
        assert info["status"] == 0 and op.true_residual(eta, phis[k].cpu().numpy()) <= 1e-10
        assert info["ras_sweeps"] == 2 * info["inner_iters"] * params[k].n_ras


def test_tuning_cache_feeds_the_batch(qdd, oracle_mod):
    """qdd_autotune keeps its choice per lattice shape; a batch entry without
    parameters takes it (and a shape never tuned takes the defaults)."""
    dims, kappa = (8, 8, 8, 8), 0.12
    U = synth.gauge_field(dims, 0.3, 311)
    eta = torch.from_numpy(synth.gaussian_source(dims, 312)).cuda()
    lat = qdd.create_lattice(dims, BC)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    p, _ = qdd.autotune(lat, eta, kappa, 1.0, 1e-10, qdd.default_params(inner_prec="f16"), max_trials=6)
    got = qdd.tuned_params(lat)
    assert got is not None and list(got.block) == list(p.block) and got.n_ras == p.n_ras
    assert got.n_dominv == p.n_dominv and got.inner_prec == p.inner_prec
    other = qdd.create_lattice((4, 4, 4, 8), BC)
    assert qdd.tuned_params(other) is None
    U2 = synth.gauge_field((4, 4, 4, 8), 0.3, 313)
    qdd.load_gauge(other, U2)
    eta2 = synth.gaussian_source((4, 4, 4, 8), 314)
    phi = torch.zeros_like(eta)
    phi2 = np.zeros_like(eta2)
    infos = qdd.solve_batch([lat, other], [phi, phi2], [eta, eta2], [kappa, kappa], [1.0, 1.0], 1e-10, [None, None])
    torch.cuda.synchronize()
    assert oracle_mod.Op(dims, BC, U, kappa, 1.0).true_residual(eta.cpu().numpy(), phi.cpu().numpy()) <= 1e-10
    assert oracle_mod.Op((4, 4, 4, 8), BC, U2, kappa, 1.0).true_residual(eta2, phi2) <= 1e-10
    assert infos[0][0]["ras_sweeps"] == 2 * infos[0][0]["inner_iters"] * p.n_ras


def _solve_batch_counted(qdd, lats, phis, etas, kappas, params, lists):
    prev = qdd.set_batch_lists(lists)
    try:
        torch.cuda.synchronize()
        n0 = qdd.kernel_launches()
        infos = qdd.solve_batch(lats, phis, etas, kappas, [1.0] * len(lats), 1e-10, params)
        torch.cuda.synchronize()
        return infos, qdd.kernel_launches() - n0
    finally:
        qdd.set_batch_lists(prev)


def test_batch_work_lists(qdd, oracle_mod):
    """Work lists (qdd_set_batch_lists): lattices with FP16 inner storage that
    share NRAS and the domain size run each step of their iteration as one
    launch over all of them -- every RAS sweep over all (lattice, domain)
    items, every D over the concatenated site ranges, the update.  Here two
    groups (256-site and 128-site domains, different shapes, blockings,
    N_dominv and kappa, so they converge after different iteration counts)
    and one lattice that keeps its own launches (FP32 storage).  Every
    system meets the oracle's FP64 residual with the lists on and off; the
    two give the same solution to about cond * tol, and the lists need
    fewer launches."""
    draws = [((8, 8, 8, 8), 0.3, 0.12, dict(block=(4, 4, 4, 4), n_dominv=3)),
             ((8, 8, 8, 16), 0.25, 0.118, dict(block=(4, 4, 4, 4), n_dominv=4)),
             ((12, 8, 8, 8), 0.35, 0.124, dict(block=(4, 4, 4, 4), n_dominv=2)),
             ((4, 4, 4, 12), 0.2, 0.11, dict(block=(4, 4, 4, 4), n_dominv=3)),
             ((8, 8, 4, 8), 0.3, 0.122, dict(block=(4, 4, 4, 2), n_dominv=3)),
             ((8, 4, 8, 8), 0.3, 0.12, dict(block=(4, 4, 2, 4), n_dominv=2)),
             ((8, 8, 8, 8), 0.3, 0.12, dict(block=(4, 4, 4, 4), n_dominv=3, inner_prec="f32"))]
    lats, etas, ops, params = [], [], [], []
    for k, (dims, eps, kappa, kw) in enumerate(draws):
        U = synth.gauge_field(dims, eps, 500 + k)
        eta = synth.gaussian_source(dims, 600 + k)
        lat = qdd.create_lattice(dims, BC, stream=torch.cuda.Stream())
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        lats.append(lat)
        etas.append(torch.from_numpy(eta).cuda())
        ops.append((oracle_mod.Op(dims, BC, U, kappa, 1.0), eta))
        params.append(qdd.default_params(**{"n_ras": 2, "inner_prec": "f16", **kw}))
    kappas = [d[2] for d in draws]
    out = {}
    for lists in (True, False):
        phis = [torch.zeros_like(e) for e in etas]
        infos, launches = _solve_batch_counted(qdd, lats, phis, etas, kappas, params, lists)
        for k, ((op, eta), phi, info) in enumerate(zip(ops, phis, infos)):
            assert info[0]["status"] == 0, (lists, k)
            assert op.true_residual(eta, phi.cpu().numpy()) <= 1e-10, (lists, k)
            assert info[0]["ras_sweeps"] == 2 * info[0]["inner_iters"] * 2
        out[lists] = ([p.cpu().numpy() for p in phis], launches, [i[0]["inner_iters"] for i in infos])
    for a, b in zip(out[True][0], out[False][0]):
        assert rel(a, b) < 1e-8
    assert len(set(out[True][2])) > 1          # the members stop at different iterations
    assert out[True][1] < 0.6 * out[False][1], (out[True][1], out[False][1])


def test_batch_work_lists_split_at_sixteen(qdd, oracle_mod):
    """17 compatible lattices: the first 16 share one group's launches (the
    largest list), the 17th keeps its own; every system meets the oracle's
    FP64 residual."""
    dims, n = (8, 8, 8, 8), 17
    lats, phis, etas, ops = [], [], [], []
    for k in range(n):
        U = synth.gauge_field(dims, 0.2 + 0.01 * k, 700 + k)
        eta = synth.gaussian_source(dims, 800 + k)
        kappa = 0.11 + 0.0008 * k
        lat = qdd.create_lattice(dims, BC, stream=torch.cuda.Stream())
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        lats.append(lat)
        etas.append(torch.from_numpy(eta).cuda())
        phis.append(torch.zeros_like(etas[-1]))
        ops.append((oracle_mod.Op(dims, BC, U, kappa, 1.0), eta, kappa))
    p = qdd.default_params(block=(4, 4, 4, 4), n_ras=2, n_dominv=3, inner_prec="f16")
    infos, _ = _solve_batch_counted(qdd, lats, phis, etas, [o[2] for o in ops], [p] * n, True)
    for (op, eta, _), phi, info in zip(ops, phis, infos):
        assert info[0]["status"] == 0
        assert op.true_residual(eta, phi.cpu().numpy()) <= 1e-10
