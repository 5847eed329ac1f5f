"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics, not by the oracle itself.

Every part of the oracle is checked by at least one of:
  * a closed form (free-field plane waves; a constant abelian field for the
    clover term; kappa = 0 making D site-local),
  * an invariant (gamma5-hermiticity, gauge covariance, the Clifford algebra,
    the restriction operators partitioning the lattice),
  * an independent library routine (numpy/LAPACK dense solves of the matrix
    assembled column by column),
  * a second definition from the paper (Eq. 2 against Alg. 1).
Tests are sized to finish in well under a minute on CPU.
"""

import numpy as np
import pytest

import synth

BC_AP = (1, 1, 1, -1)


def coords(dims):
    V = int(np.prod(dims))
    i = np.arange(V)
    c = np.empty((V, 4), dtype=np.int64)
    for mu in range(4):
        c[:, mu] = i % dims[mu]
        i = i // dims[mu]
    return c


def dense(apply, n):
    """Matrix of a linear map on C^n, assembled column by column."""
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[k] = 1.0
        M[:, k] = apply(e).reshape(-1)
        e[k] = 0.0
    return M


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ---------------------------------------------------------------- gammas
def test_gamma_clifford_algebra(oracle_mod):
    g = [oracle_mod.gamma(m) for m in range(4)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4), atol=0)
    g5 = oracle_mod.gamma(4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)
    # DeGrand-Rossi: gamma_4 couples the two chiral halves with the identity
    assert np.allclose(g[3][:2, 2:], np.eye(2)) and np.allclose(g[3][:2, :2], 0)


# ---------------------------------------------------------------- hopping
@pytest.mark.parametrize("dims,bc,n", [
    ((4, 4, 4, 6), BC_AP, (1, 2, 0, 1)),
    ((6, 4, 4, 4), BC_AP, (0, 0, 1, 0)),
    ((4, 6, 4, 4), (1, 1, 1, 1), (1, 3, 1, 2)),
    ((4, 4, 6, 4), (-1, 1, 1, 1), (2, 1, 1, 0)),
])
def test_free_field_plane_wave(oracle_mod, dims, bc, n):
    """U = 1: psi = exp(i p.x) u gives D psi = [1 - 2k sum cos p + 2ik sum gamma sin p] psi,
    with p_mu = 2 pi n / L (periodic) or (2n+1) pi / L (antiperiodic)."""
    kappa = 0.13
    op = oracle_mod.Op(dims, bc, synth.unit_gauge(dims), kappa, 1.7)
    L = np.array(dims, dtype=float)
    nn = np.array(n, dtype=float)
    p = np.where(np.array(bc) > 0, 2 * np.pi * nn / L, (2 * nn + 1) * np.pi / L)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    phase = np.exp(1j * coords(dims) @ p)
    psi = phase[:, None, None] * u[None]
    G = [np.array(oracle_mod.gamma(m)) for m in range(4)]
    M = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(G[m] * np.sin(p[m]) for m in range(4))
    expect = phase[:, None, None] * (M @ u)[None]
    assert np.abs(op.dslash(psi) - expect).max() < 1e-13


def test_gamma5_hermiticity(oracle_mod):
    """<x, g5 D g5 y> = <D x, y> on a random gauge field."""
    dims = (4, 4, 4, 4)
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 11), 0.125, 1.0)
    x = synth.gaussian_source(dims, 12)
    y = synth.gaussian_source(dims, 13)
    g5 = np.array([1, 1, -1, -1])[None, :, None]
    lhs = np.vdot(x, g5 * op.dslash(g5 * y))
    rhs = np.vdot(op.dslash(x), y)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13


def test_gauge_covariance(oracle_mod):
    """D[U^G](G psi) = G (D[U] psi), U^G_mu(x) = G(x) U_mu(x) G(x+mu)^dag."""
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, 0.3, 21)
    G = synth.random_su3(V, 22)
    c = coords(dims)
    UG = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        xf = cf[:, 0] + dims[0] * (cf[:, 1] + dims[1] * (cf[:, 2] + dims[2] * cf[:, 3]))
        UG[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(G[xf], -1, -2))
    psi = synth.gaussian_source(dims, 23)
    Gpsi = np.einsum("vab,vsb->vsa", G, psi)
    lhs = oracle_mod.Op(dims, BC_AP, UG, 0.12, 1.0).dslash(Gpsi)
    rhs = np.einsum("vab,vsb->vsa", G, oracle_mod.Op(dims, BC_AP, U, 0.12, 1.0).dslash(psi))
    assert rel(lhs, rhs) < 1e-13


def test_single_hop_placement(oracle_mod):
    """A point source at x0 reaches x0 -/+ mu only, with norm kappa |(1 -/+ gamma) u|
    (the links are unitary), and nothing else but A(x0) u at x0."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 31)
    kappa = 0.1
    op = oracle_mod.Op(dims, BC_AP, U, kappa, 0.0)
    x0 = 1 + 4 * (2 + 4 * (3 + 4 * 0))   # t = 0: the backward t hop crosses the boundary
    psi = np.zeros((op.V, 4, 3), complex)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi[x0] = u
    out = op.dslash(psi)
    nz = set(np.nonzero(np.abs(out).reshape(op.V, -1).max(axis=1) > 1e-14)[0].tolist())
    c0 = coords(dims)[x0]
    expect = {x0}
    for mu in range(4):
        for d in (-1, 1):
            cc = c0.copy()
            cc[mu] = (cc[mu] + d) % dims[mu]
            expect.add(int(cc[0] + 4 * (cc[1] + 4 * (cc[2] + 4 * cc[3]))))
    assert nz == expect
    assert np.allclose(out[x0], u, atol=1e-15)        # c_sw = 0: A = 1
    g = [oracle_mod.gamma(m) for m in range(4)]
    for mu in range(4):
        for d in (-1, 1):
            cc = c0.copy()
            cc[mu] = (cc[mu] + d) % dims[mu]
            y = int(cc[0] + 4 * (cc[1] + 4 * (cc[2] + 4 * cc[3])))
            # the site y = x0 - mu hops forward with (1 - gamma); y = x0 + mu hops back with (1 + gamma)
            proj = np.eye(4) - g[mu] if d < 0 else np.eye(4) + g[mu]
            assert abs(np.linalg.norm(out[y]) - kappa * np.linalg.norm(proj @ u)) < 1e-13


def test_antiperiodic_sign_flips_only_time_wrap(oracle_mod):
    """With U = 1 and a constant spinor, D psi differs between periodic and
    antiperiodic time only on the t = 0 and t = Lt-1 slices."""
    dims = (4, 4, 4, 4)
    U = synth.unit_gauge(dims)
    u = np.arange(12).reshape(4, 3) + 1j * np.arange(12, 0, -1).reshape(4, 3)
    psi = np.broadcast_to(u, (256, 4, 3)).copy()
    a = oracle_mod.Op(dims, (1, 1, 1, 1), U, 0.1, 0.0).dslash(psi)
    b = oracle_mod.Op(dims, BC_AP, U, 0.1, 0.0).dslash(psi)
    t = coords(dims)[:, 3]
    diff = np.abs(a - b).reshape(256, -1).max(axis=1)
    assert np.all(diff[(t > 0) & (t < 3)] == 0)
    assert np.all(diff[(t == 0) | (t == 3)] > 0.05)


# ---------------------------------------------------------------- clover
def abelian_field(dims, k):
    """U_y(x) = diag(e^{i th x}, e^{-i th x}, 1), th = 2 pi k / Lx; other links 1."""
    U = synth.unit_gauge(dims)
    th = 2 * np.pi * k / dims[0]
    x = coords(dims)[:, 0]
    U[:, 1, 0, 0] = np.exp(1j * th * x)
    U[:, 1, 1, 1] = np.exp(-1j * th * x)
    return U, th


def test_clover_constant_abelian_field(oracle_mod):
    """Every xy leaf is diag(e^{i th}, e^{-i th}, 1), so Fhat_xy = i diag(sin th, -sin th, 0)
    and A = 1 - kappa c_sw sin(th) sigma_xy (x) diag(1, -1, 0), with sigma_xy = diag(1,-1,1,-1)
    in the DeGrand-Rossi basis; the other planes vanish."""
    dims = (6, 4, 4, 4)
    U, th = abelian_field(dims, 1)
    kappa, csw = 0.12, 1.3
    F = oracle_mod.field_strength(dims, U, 37, 0, 1)
    assert np.allclose(F, 1j * np.diag([np.sin(th), -np.sin(th), 0]), atol=1e-15)
    for (mu, nu) in [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
        assert np.abs(oracle_mod.field_strength(dims, U, 37, mu, nu)).max() < 1e-15
    A = oracle_mod.clover(dims, U, kappa, csw)
    diag = 1 - kappa * csw * np.sin(th) * np.kron([1, -1, 1, -1], [1, -1, 0])
    assert np.abs(A - np.diag(diag)[None]).max() < 1e-15
    # the same A(x0) appears in D acting on a point source (hops leave x0)
    op = oracle_mod.Op(dims, BC_AP, U, kappa, csw)
    psi = np.zeros((op.V, 4, 3), complex)
    psi[5] = np.arange(12).reshape(4, 3) + 1j
    assert np.allclose(op.dslash(psi)[5].reshape(12), diag * psi[5].reshape(12), atol=1e-15)


def test_clover_structure(oracle_mod):
    """Off-chiral blocks vanish, the 6x6 blocks are Hermitian, c_sw = 0 gives A = 1,
    and A - 1 is linear in kappa c_sw."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 41)
    A = oracle_mod.clover(dims, U, 0.125, 1.0)
    assert np.abs(A[:, :6, 6:]).max() < 1e-15 and np.abs(A[:, 6:, :6]).max() < 1e-15
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-15
    assert np.abs(A[:, :6, :6] - np.eye(6)).max() > 1e-3
    assert np.abs(oracle_mod.clover(dims, U, 0.125, 0.0) - np.eye(12)).max() == 0
    A2 = oracle_mod.clover(dims, U, 0.25, 1.0)
    assert np.abs((A2 - np.eye(12)) - 2 * (A - np.eye(12))).max() < 1e-15


def test_field_strength_antihermitian(oracle_mod):
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 42)
    for (mu, nu) in [(0, 1), (1, 3), (2, 3)]:
        F = oracle_mod.field_strength(dims, U, 77, mu, nu)
        assert np.abs(F + F.conj().T).max() < 1e-15
        # orientation: Fhat_{nu mu} = -Fhat_{mu nu} needs the leaves traversed the other way;
        # a transposed plane must flip the sign
        Fr = oracle_mod.field_strength(dims, U, 77, nu, mu)
        assert np.abs(F + Fr).max() < 1e-14


# ---------------------------------------------------------------- dense solves
@pytest.fixture(scope="module")
def small_system(oracle_mod):
    dims = (4, 4, 2, 4)
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 51), 0.12, 1.0)
    n = op.V * 12
    Dm = dense(lambda v: op.dslash(v.reshape(op.V, 4, 3)), n)
    eta = synth.gaussian_source(dims, 52)
    x = np.linalg.solve(Dm, eta.reshape(-1))
    return op, Dm, eta, x.reshape(op.V, 4, 3)


def test_plain_bicgstab_matches_dense_solve(small_system):
    op, Dm, eta, x = small_system
    phi, st, it, _ = op.bicgstab(eta, 1e-12)
    assert st == 0 and it > 5
    assert rel(phi, x) < 1e-10
    assert op.true_residual(eta, phi) < 1e-12


def test_true_residual_matches_dense_residual(small_system):
    """The checker behind every solve's "<= 1e-10" (the Sec. 5 stopping rule
    |eta - D phi| / |eta|) against the residual of the dense matrix computed
    with numpy, for a random phi, a near-solution and the LAPACK solution;
    phi = 0 gives exactly 1 and the ratio is invariant under a common scale
    (a missing square root or a wrong normalisation fails here)."""
    op, Dm, eta, x = small_system
    rng = np.random.default_rng(53)
    e = eta.reshape(-1)
    rnd = (rng.standard_normal(e.size) + 1j * rng.standard_normal(e.size)).reshape(op.V, 4, 3)
    near = x + 1e-6 * rnd
    for phi in (rnd, near, x):
        want = np.linalg.norm(e - Dm @ phi.reshape(-1)) / np.linalg.norm(e)
        got = op.true_residual(eta, phi)
        assert abs(got - want) <= 1e-14 * max(want, 1e-300) + 1e-16, (got, want)
    assert 1e-9 < op.true_residual(eta, near) < 1e-4
    assert op.true_residual(eta, x) < 1e-13
    assert op.true_residual(eta, np.zeros_like(eta)) == pytest.approx(1.0, abs=1e-15)
    assert op.true_residual(3.0 * eta, 3.0 * near) == pytest.approx(op.true_residual(eta, near), rel=1e-12)


def test_nested_solve_matches_dense_solve(small_system):
    op, Dm, eta, x = small_system
    phi, info = op.solve(eta, 1e-11, inner_tol=1e-3, ras=dict(block=(2, 2, 2, 2), s=0, n_ras=3, n_dominv=4))
    assert info["status"] == 0 and info["outer_iters"] >= 2
    assert rel(phi, x) < 1e-9
    assert np.linalg.norm(Dm @ phi.reshape(-1) - eta.reshape(-1)) / np.linalg.norm(eta) < 1e-11


def test_ras_whole_lattice_block_is_exact_inverse(small_system):
    """One domain covering the lattice, exact domain solve, NRAS = 1: K_RAS = D^{-1}."""
    op, Dm, eta, x = small_system
    phi = op.ras(eta, op.dims, s=0, n_ras=1, exact=True)
    assert rel(phi, x) < 1e-11


# ---------------------------------------------------------------- domains
def test_restrictions_partition_the_lattice(oracle_mod):
    """sum_i R_i P_i = 1: every site is a bulk site of exactly one domain."""
    dims = (8, 4, 4, 8)
    op = oracle_mod.Op(dims, BC_AP, synth.unit_gauge(dims), 0.1, 0.0, store_clover=False)
    for block, s in [((4, 4, 4, 4), 0), ((2, 2, 4, 4), 1), ((4, 2, 2, 2), 1), ((2, 4, 4, 2), 2)]:
        count = np.zeros(op.V, int)
        nd = op.ndomains(block, s)
        assert nd == np.prod(np.array(dims) // np.array(block))
        for d in range(nd):
            sites, bulk = op.domain_sites(block, s, d)
            ext = [b if b == L else b + 2 * s for b, L in zip(block, dims)]
            assert sites.size == np.prod(ext) and bulk.sum() == np.prod(block)
            assert len(set(sites.tolist())) == sites.size
            np.add.at(count, sites[bulk], 1)
        assert np.all(count == 1)


@pytest.mark.parametrize("dims,block,s", [
    ((4, 4, 4, 4), (2, 2, 2, 2), 0),
    ((6, 6, 2, 2), (2, 2, 2, 2), 1),
    ((4, 8, 2, 2), (4, 2, 2, 2), 2),
])
def test_domain_operator_is_principal_submatrix(oracle_mod, dims, block, s):
    """Where the extended domain does not wrap onto itself, the Dirichlet operator
    D_Omega' is the principal submatrix of D on the domain's sites (hops that leave
    the domain are exactly the dropped columns)."""
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 61), 0.12, 1.0)
    Dm = dense(lambda v: op.dslash(v.reshape(op.V, 4, 3)), op.V * 12)
    for dom in range(min(op.ndomains(block, s), 4)):
        sites, _ = op.domain_sites(block, s, dom)
        idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
        sub = Dm[np.ix_(idx, idx)]
        Dd = dense(lambda v: op.domain_apply(block, s, dom, v.reshape(-1, 4, 3)), idx.size)
        assert np.abs(Dd - sub).max() < 1e-14
        # exact domain solve against LAPACK on the same submatrix
        r = synth.gaussian_source((idx.size // 12, 1, 1, 1), 62 + dom)
        v = op.domain_solve(block, s, dom, r, exact=True)
        assert rel(v.reshape(-1), np.linalg.solve(sub, r.reshape(-1))) < 1e-11


def test_mr_domain_solver_properties(oracle_mod):
    """MR: one step gives v = (<q,r>/<q,q>) r with q = D r; the residual
    |r - D v| never grows with the iteration count and tends to zero."""
    dims = (4, 4, 4, 4)
    block, s = (2, 2, 2, 2), 0
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 71), 0.12, 1.0)
    r = synth.gaussian_source((16, 1, 1, 1), 72)
    q = op.domain_apply(block, s, 3, r)
    v1 = op.domain_solve(block, s, 3, r, n_dominv=1)
    assert rel(v1, (np.vdot(q, r) / np.vdot(q, q)) * r) < 1e-14
    res = []
    for n in range(0, 30):
        v = op.domain_solve(block, s, 3, r, n_dominv=n)
        res.append(np.linalg.norm(r - op.domain_apply(block, s, 3, v)))
    assert all(res[k + 1] <= res[k] * (1 + 1e-12) for k in range(len(res) - 1))
    assert res[-1] < 1e-6 * res[0]


def test_mr_steps_minimise_the_residual_along_their_direction(oracle_mod):
    """Each MR step of the domain solve (Alg. 1 line 5 read as minimal
    residual) moves v along the current residual rho_k = r - D v_k with the
    complex step that minimises |rho_k - alpha D rho_k|: the step taken by
    the oracle is parallel to rho_k, and moving its coefficient by 1e-3 in
    the real or the imaginary direction makes the new residual larger (a
    conjugated or mis-normalised alpha fails).  No MR formula is restated."""
    dims, block, s, dom = (4, 4, 4, 4), (2, 2, 2, 2), 0, 5
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 73), 0.12, 1.0)
    r = synth.gaussian_source((16, 1, 1, 1), 74)
    v_prev = np.zeros_like(r)
    for k in range(4):
        v_next = op.domain_solve(block, s, dom, r, n_dominv=k + 1)
        rho = r - op.domain_apply(block, s, dom, v_prev)
        step = (v_next - v_prev).reshape(-1)
        rf = rho.reshape(-1)
        alpha = np.vdot(rf, step) / np.vdot(rf, rf)
        assert np.linalg.norm(step - alpha * rf) <= 1e-12 * np.linalg.norm(step)
        q = op.domain_apply(block, s, dom, rho).reshape(-1)
        best = np.linalg.norm(rf - alpha * q)
        assert best < np.linalg.norm(rf)
        for d in (1e-3, -1e-3, 1e-3j, -1e-3j):
            assert np.linalg.norm(rf - (alpha + d * abs(alpha)) * q) > best * (1 + 1e-9)
        # a conjugated coefficient is not the minimiser
        if abs(alpha.imag) > 1e-6 * abs(alpha):
            assert np.linalg.norm(rf - np.conj(alpha) * q) > best * (1 + 1e-9)
        v_prev = v_next


def test_ras_equals_eq2_with_exact_domain_solves(oracle_mod):
    """Alg. 1 computes K_RAS eta with K_RAS = S sum_{j<NRAS} (1 - D S)^j and
    S = sum_i R_i D_i'^{-1} P_i (Eq. 2); built here densely with LAPACK inverses
    of the principal submatrices."""
    dims = (6, 6, 2, 2)
    block, s = (2, 2, 2, 2), 1
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 81), 0.12, 1.0)
    n = op.V * 12
    Dm = dense(lambda v: op.dslash(v.reshape(op.V, 4, 3)), n)
    S = np.zeros((n, n), complex)
    for dom in range(op.ndomains(block, s)):
        sites, bulk = op.domain_sites(block, s, dom)
        idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
        inv = np.linalg.inv(Dm[np.ix_(idx, idx)])
        keep = np.repeat(bulk, 12)
        S[np.ix_(idx[keep], idx)] += inv[keep]
    eta = synth.gaussian_source(dims, 82)
    for nras in (1, 2, 3):
        K = np.zeros((n, n), complex)
        T = np.eye(n)
        for _ in range(nras):
            K += T
            T = T @ (np.eye(n) - Dm @ S)
        K = S @ K
        phi = op.ras(eta, block, s=s, n_ras=nras, exact=True)
        assert rel(phi.reshape(-1), K @ eta.reshape(-1)) < 1e-11


@pytest.mark.parametrize("block,s", [((2, 2, 2, 2), 0), ((2, 2, 2, 2), 1), ((4, 2, 2, 2), 1)])
def test_ras_kappa_zero_is_exact(oracle_mod, block, s):
    """kappa = 0 makes D = A site-local (and A = 1); more generally with a
    non-trivial clover and only the hopping switched off, RAS with exact domain
    solves inverts D in one sweep for any blocking."""
    dims = (8, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 91)
    A = oracle_mod.clover(dims, U, 0.12, 1.0)     # clover built with kappa = 0.12 ...
    op = oracle_mod.Op(dims, BC_AP, U, 0.0, 1.0, A=A)   # ... used with the hopping off
    eta = synth.gaussian_source(dims, 92)
    expect = np.linalg.solve(A, eta.reshape(op.V, 12)[..., None])[..., 0]
    phi = op.ras(eta, block, s=s, n_ras=1, exact=True)
    assert rel(phi.reshape(op.V, 12), expect) < 1e-12


def test_ras_sweeps_converge_to_inverse(small_system):
    """Exact domain solves: K_RAS eta -> D^{-1} eta as NRAS grows (Eq. 2 is a
    Neumann series in 1 - D S, which contracts for this blocking)."""
    op, Dm, eta, x = small_system
    errs = [rel(op.ras(eta, (2, 2, 2, 2), s=0, n_ras=k, exact=True), x) for k in (1, 4, 16)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


def mr_dense(M, r, n):
    """Minimal residual from zero on a dense matrix, n steps (the domain
    solver's definition written with numpy): q = M rho, alpha = <q, rho>/<q, q>,
    v += alpha rho, rho -= alpha q."""
    v = np.zeros_like(r)
    rho = r.copy()
    for _ in range(n):
        q = M @ rho
        qq = np.vdot(q, q).real
        if qq == 0:
            break
        a = np.vdot(q, rho) / qq
        v = v + a * rho
        rho = rho - a * q
    return v


def test_mr_domain_solver_matches_dense_mr(oracle_mod):
    """N_dominv MR steps of the oracle's domain solve equal the same steps on
    the dense Dirichlet matrix, for several step counts (an off-by-one in the
    iteration count or a swapped inner product fails)."""
    dims, block, s = (6, 6, 2, 2), (2, 2, 2, 2), 1
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 95), 0.12, 1.0)
    for dom in (0, 4):
        sites, _ = op.domain_sites(block, s, dom)
        n = sites.size * 12
        Dd = dense(lambda v: op.domain_apply(block, s, dom, v.reshape(-1, 4, 3)), n)
        r = synth.gaussian_source((sites.size, 1, 1, 1), 96 + dom)
        for k in (2, 3, 5):
            got = op.domain_solve(block, s, dom, r, n_dominv=k)
            assert rel(got.reshape(-1), mr_dense(Dd, r.reshape(-1), k)) < 1e-12


@pytest.mark.parametrize("s", [0, 1])
def test_ras_with_mr_domain_solves_matches_dense_alg1(oracle_mod, s):
    """Alg. 1 with the MR domain solver (a non-linear map, so Eq. 2 does not
    apply) written densely with numpy: per sweep, every domain's MR on its
    Dirichlet matrix, restricted to the bulk and summed, then phi += v and
    r -= D v."""
    dims, block = (6, 6, 2, 2), (2, 2, 2, 2)
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 97), 0.12, 1.0)
    Dm = dense(lambda v: op.dslash(v.reshape(op.V, 4, 3)), op.V * 12)
    doms = []
    for dom in range(op.ndomains(block, s)):
        sites, bulk = op.domain_sites(block, s, dom)
        idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
        doms.append((idx, np.repeat(bulk, 12), Dm[np.ix_(idx, idx)]))
    eta = synth.gaussian_source(dims, 98).reshape(-1)
    for n_ras, n_dominv in ((1, 3), (2, 3), (3, 2)):
        phi = np.zeros_like(eta)
        r = eta.copy()
        for _ in range(n_ras):
            v = np.zeros_like(eta)
            for idx, keep, M in doms:
                vl = mr_dense(M, r[idx], n_dominv)
                v[idx[keep]] += vl[keep]
            phi = phi + v
            r = r - Dm @ v
        got = op.ras(eta.reshape(op.V, 4, 3), block, s=s, n_ras=n_ras, n_dominv=n_dominv)
        assert rel(got.reshape(-1), phi) < 1e-12


# ---------------------------------------------------------------- Schwarz variants
def block_color(dims, block, dom):
    """Red/black colour of a domain: parity of the sum of its block coordinates."""
    nb = [L // b for L, b in zip(dims, block)]
    k, r = [], dom
    for mu in range(4):
        k.append(r % nb[mu])
        r //= nb[mu]
    return sum(k) % 2


def dense_domain_sweep(op, block, s, restrict, color=None):
    """S = sum_i Q_i D_i'^{-1} P_i' over the domains of one colour (all when
    colour is None): Q_i = R_i (bulk sites) for RAS and SAP, Q_i = P_i'^T (every
    extended site, overlaps summed) for AS; D_i' assembled column by column
    from the Dirichlet operator and inverted by LAPACK."""
    n = op.V * 12
    S = np.zeros((n, n), complex)
    for dom in range(op.ndomains(block, s)):
        if color is not None and block_color(op.dims, block, dom) != color:
            continue
        sites, bulk = op.domain_sites(block, s, dom)
        idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
        Dd = dense(lambda v: op.domain_apply(block, s, dom, v.reshape(-1, 4, 3)), idx.size)
        inv = np.linalg.inv(Dd)
        keep = np.repeat(bulk, 12) if restrict else np.ones(idx.size, bool)
        np.add.at(S, (idx[keep][:, None], idx[None, :]), inv[keep])
    return S


def stationary(Dm, sweeps, eta, ncycles):
    """x_0 = 0; each cycle applies x += S_c (eta - D x) for every S_c in turn."""
    x = np.zeros_like(eta)
    for _ in range(ncycles):
        for S in sweeps:
            x = x + S @ (eta - Dm @ x)
    return x


@pytest.fixture(scope="module")
def schwarz_system(oracle_mod):
    dims = (8, 4, 2, 2)
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 301), 0.12, 1.0)
    Dm = dense(lambda v: op.dslash(v.reshape(op.V, 4, 3)), op.V * 12)
    eta = synth.gaussian_source(dims, 302)
    return op, Dm, eta


def test_sap_without_overlap_is_block_gauss_seidel(schwarz_system):
    """Multiplicative Schwarz with exact domain solves and no overlap is block
    Gauss-Seidel over the red/black ordering: one cycle gives x = M^{-1} eta with
    M the block lower-triangular part [[D_RR, 0], [D_BR, D_BB]] of D (red
    blocks first), built here from the dense matrix by masking, not from the
    domains."""
    op, Dm, eta = schwarz_system
    block = (2, 2, 2, 2)
    c = coords(op.dims)
    red_site = ((c[:, 0] // 2 + c[:, 1] // 2) % 2) == 0
    red = np.repeat(red_site, 12)
    M = Dm.copy()
    M[np.ix_(red, ~red)] = 0.0
    e = eta.reshape(-1)
    x = np.zeros_like(e)
    for ncyc in (1, 2, 3):
        x = x + np.linalg.solve(M, e - Dm @ x)
        phi = op.ras(eta, block, s=0, n_ras=ncyc, exact=True, schwarz="sap")
        assert rel(phi.reshape(-1), x) < 1e-11
    # block Jacobi (the additive sweep) is a different operator
    assert rel(op.ras(eta, block, s=0, n_ras=1, exact=True).reshape(-1),
               np.linalg.solve(M, e)) > 1e-3


@pytest.mark.parametrize("s", [0, 1])
def test_sap_and_as_match_dense_schwarz_operators(schwarz_system, s):
    """SAP: x += S_red (eta - D x), then x += S_black (eta - D x) per cycle with
    the restricted colour sums; AS: x += S_AS (eta - D x) with the unrestricted
    sum over extended domains (Sec. 2)."""
    op, Dm, eta = schwarz_system
    block = (4, 2, 2, 2)
    e = eta.reshape(-1)
    S_red = dense_domain_sweep(op, block, s, True, 0)
    S_black = dense_domain_sweep(op, block, s, True, 1)
    S_as = dense_domain_sweep(op, block, s, False)
    for ncyc in (1, 2):
        sap = op.ras(eta, block, s=s, n_ras=ncyc, exact=True, schwarz="sap")
        assert rel(sap.reshape(-1), stationary(Dm, [S_red, S_black], e, ncyc)) < 1e-11
        add = op.ras(eta, block, s=s, n_ras=ncyc, exact=True, schwarz="as")
        assert rel(add.reshape(-1), stationary(Dm, [S_as], e, ncyc)) < 1e-11


def test_sap_with_an_odd_block_count(oracle_mod):
    """Three blocks in x: domains 0 and 2 have the same colour and touch across
    the periodic wrap; a half-sweep then solves them additively, which the
    colour sums S_c express."""
    dims, block = (6, 4, 2, 2), (2, 2, 2, 2)
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 305), 0.12, 1.0)
    Dm = dense(lambda v: op.dslash(v.reshape(op.V, 4, 3)), op.V * 12)
    eta = synth.gaussian_source(dims, 306)
    sweeps = [dense_domain_sweep(op, block, 0, True, c) for c in (0, 1)]
    for ncyc in (1, 2):
        sap = op.ras(eta, block, s=0, n_ras=ncyc, exact=True, schwarz="sap")
        assert rel(sap.reshape(-1), stationary(Dm, sweeps, eta.reshape(-1), ncyc)) < 1e-11


def test_as_without_overlap_is_ras(schwarz_system):
    """With d = 0 the extended domains are the bulk blocks: AS and RAS coincide
    (the restriction removes nothing)."""
    op, _, eta = schwarz_system
    for block in [(2, 2, 2, 2), (4, 2, 2, 2)]:
        a = op.ras(eta, block, s=0, n_ras=2, n_dominv=3, schwarz="as")
        r = op.ras(eta, block, s=0, n_ras=2, n_dominv=3)
        assert np.array_equal(a, r)


def test_sap_whole_lattice_block_is_exact_inverse(small_system):
    """One domain (red) covering the lattice with an exact solve: the black
    half-sweep has nothing to do and K_SAP = D^{-1}."""
    op, Dm, eta, x = small_system
    phi = op.ras(eta, op.dims, s=0, n_ras=1, exact=True, schwarz="sap")
    assert rel(phi, x) < 1e-11


@pytest.mark.parametrize("schwarz", ["sap", "as"])
def test_schwarz_kappa_zero_is_exact(oracle_mod, schwarz):
    """With the hopping off D = A is site-local and every member of the family
    inverts it in one cycle (AS sums overlapping copies: only without overlap)."""
    dims = (8, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 303)
    A = oracle_mod.clover(dims, U, 0.12, 1.0)
    op = oracle_mod.Op(dims, BC_AP, U, 0.0, 1.0, A=A)
    eta = synth.gaussian_source(dims, 304)
    expect = np.linalg.solve(A, eta.reshape(op.V, 12)[..., None])[..., 0]
    for block, s in [((2, 2, 2, 2), 0), ((4, 2, 2, 2), 1 if schwarz == "sap" else 0)]:
        phi = op.ras(eta, block, s=s, n_ras=1, exact=True, schwarz=schwarz)
        assert rel(phi.reshape(op.V, 12), expect) < 1e-12


def test_sap_converges_faster_than_ras_per_cycle(small_system):
    """The multiplicative sweep uses the red update before the black solve;
    on this system its cycles contract faster than the additive ones."""
    op, Dm, eta, x = small_system
    block = (2, 2, 2, 2)
    for k in (2, 4):
        sap = rel(op.ras(eta, block, s=0, n_ras=k, exact=True, schwarz="sap"), x)
        ras = rel(op.ras(eta, block, s=0, n_ras=k, exact=True), x)
        assert sap < ras


# ---------------------------------------------------------------- nested BiCGStab
@pytest.mark.parametrize("inner_tol", [1e-1, 1e-3])
@pytest.mark.parametrize("schwarz", [None, "ras", "sap"])
def test_nested_bicgstab_matches_dense_solve(small_system, inner_tol, schwarz):
    """The paper's outer BiCGStab around the inner solve reaches the dense
    LAPACK solution to the requested tolerance whatever the inner accuracy
    and preconditioner."""
    op, Dm, eta, x = small_system
    ras = None if schwarz is None else dict(block=(2, 2, 2, 2), s=0, n_ras=2, n_dominv=4, schwarz=schwarz)
    phi, info = op.solve_nested(eta, 1e-11, inner_tol=inner_tol, ras=ras)
    assert info["status"] == 0
    assert np.linalg.norm(Dm @ phi.reshape(-1) - eta.reshape(-1)) / np.linalg.norm(eta) <= 1e-11
    assert rel(phi, x) < 1e-9


def test_nested_bicgstab_with_exact_inner_solve_takes_one_iteration(small_system):
    """M = D^{-1} (inner solve to 1e-13): p = r, p_hat = D^{-1} r, v = r,
    alpha = 1 and s = 0, so one outer iteration solves the system."""
    op, Dm, eta, x = small_system
    phi, info = op.solve_nested(eta, 1e-11, inner_tol=1e-13,
                                ras=dict(block=(2, 2, 2, 2), s=0, n_ras=3, n_dominv=4))
    assert info["status"] == 0 and info["outer_iters"] == 1
    assert rel(phi, x) < 1e-11


def test_nested_outer_krylov_beats_defect_correction(small_system):
    """With a loose inner solve (1e-1, 0.5) defect correction gains at most
    that factor per outer step (a Richardson iteration); the outer BiCGStab
    builds a Krylov space from the same inner solves and needs fewer outer
    iterations."""
    op, Dm, eta, x = small_system
    ras = dict(block=(2, 2, 2, 2), s=0, n_ras=1, n_dominv=2)
    for inner_tol, min_dc in ((1e-1, 9), (0.5, 20)):
        _, dc = op.solve(eta, 1e-11, inner_tol=inner_tol, ras=ras)
        _, nb = op.solve_nested(eta, 1e-11, inner_tol=inner_tol, ras=ras)
        assert dc["status"] == 0 and nb["status"] == 0
        assert dc["outer_iters"] >= min_dc
        assert nb["outer_iters"] < 0.7 * dc["outer_iters"]


# ---------------------------------------------------------------- the config-1 contract
def test_config1_plain_fp64_solve(oracle_mod):
    """8^4, eps = 0.3 (seed 1), kappa = 0.12, c_sw = 1, Gaussian source (seed 2),
    FP64 plain BiCGStab to |r|/|eta| = 1e-10."""
    dims = (8, 8, 8, 8)
    op = oracle_mod.Op(dims, BC_AP, synth.gauge_field(dims, 0.3, 1), 0.12, 1.0)
    eta = synth.gaussian_source(dims, 2)
    phi, info = op.solve(eta, 1e-10)
    assert info["status"] == 0
    assert op.true_residual(eta, phi) <= 1e-10
    phi2, info2 = op.solve(eta, 1e-10, inner_tol=1e-3, ras=dict(block=(4, 4, 4, 4), s=0, n_ras=3, n_dominv=4))
    assert info2["status"] == 0 and op.true_residual(eta, phi2) <= 1e-10
    # the solution is unique: both methods agree to about cond * tol
    assert rel(phi2, phi) < 1e-8
    # RAS cuts the number of Krylov iterations (the paper's Table 1 trend)
    assert info2["inner_iters"] < info["inner_iters"]
