"""The other members of the Schwarz family on the GPU (Sec. 1, Sec. 2): the
multiplicative red/black SAP and plain additive Schwarz (AS) against the
oracle's sweeps with the same blocking, overlap, MR iteration count and cycle
count, through every staging of the sweep kernel, with several right-hand
sides, in the no-allocation entry point and as the preconditioner of a solve."""

import numpy as np
import pytest
import torch

import synth
from gpu_common import check_field, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

# As for RAS: MR in FP32 arithmetic, amplified by the domain operators'
# conditioning over N_dominv * cycles steps (~10x margin over the observed
# error); FP16 storage adds 2^-11 per stored vector.  AS sums overlapping
# copies with FP32 atomics: their order changes only the last bits.
TOL = {"f32": 1e-5, "f16": 1e-2}

SAP_CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), 0),    # 256-site domains: TMA staging
    ((8, 8, 8, 8), (2, 4, 4, 4), 0),    # 128-site domains: TMA staging
    ((8, 8, 8, 8), (2, 2, 2, 2), 0),    # 16-site domains in 32-thread CTAs
    ((8, 8, 8, 8), (8, 4, 4, 4), 0),    # 512-site domains, x not decomposed
    ((8, 8, 8, 8), (2, 2, 2, 2), 1),    # 256-site extended domains with overlap
    ((8, 8, 8, 8), (4, 4, 4, 4), 1),    # 6^4 extended domains: general kernel
    ((6, 4, 4, 8), (2, 2, 2, 2), 1),    # three blocks in x: an odd colouring
]

AS_CASES = [
    ((8, 8, 8, 8), (2, 2, 2, 2), 1),    # shared-memory kernel
    ((8, 8, 8, 8), (4, 4, 4, 4), 1),    # general kernel
    ((8, 8, 8, 8), (4, 4, 4, 4), 2),    # extension wraps to the full extent
    ((6, 4, 4, 8), (2, 2, 2, 2), 1),
    ((8, 4, 4, 8), (4, 2, 2, 8), 1),    # t not decomposed
]


def _setup(dims, seed):
    bc = (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, seed)
    eta = synth.gaussian_source(dims, seed + 1)
    return bc, U, eta


@pytest.mark.parametrize("dims,block,s", SAP_CASES)
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_sap_matches_oracle(qdd, oracle_mod, dims, block, s, prec):
    bc, U, eta = _setup(dims, 401)
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=2, n_dominv=4, schwarz="sap")
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, overlap=s, n_ras=2, n_dominv=4, inner_prec=prec, schwarz="sap")
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, 0.12, 1.0, p)
    check_field(out, ref, TOL[prec], dims, block)
    # the case separates SAP from RAS far beyond the FP32 tolerance
    ras = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=s, n_ras=2, n_dominv=4)
    assert rel(ref, ras) > 100 * TOL["f32"]


@pytest.mark.parametrize("dims,block,s", AS_CASES)
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_as_matches_oracle(qdd, oracle_mod, dims, block, s, prec):
    bc, U, eta = _setup(dims, 411)
    op = oracle_mod.Op(dims, bc, U, 0.12, 1.0)
    ref = op.ras(eta, block, s=s, n_ras=2, n_dominv=4, schwarz="as")
    assert rel(ref, op.ras(eta, block, s=s, n_ras=2, n_dominv=4)) > 100 * TOL["f32"]
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, overlap=s, n_ras=2, n_dominv=4, inner_prec=prec, schwarz="as")
    out = np.empty_like(eta)
    qdd.ras_apply(lat, out, eta, 0.12, 1.0, p)
    check_field(out, ref, TOL[prec], dims, block)


@pytest.mark.parametrize("block", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_as_without_overlap_is_ras_bit_for_bit(qdd, block):
    """d = 0: no site is covered twice, and the library runs the RAS sweep."""
    dims = (8, 8, 8, 8)
    bc, U, eta = _setup(dims, 421)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    outs = []
    for sch in ("ras", "as"):
        out = np.empty_like(eta)
        qdd.ras_apply(lat, out, eta, 0.12, 1.0, qdd.default_params(block=block, n_ras=2, schwarz=sch))
        outs.append(out)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_sap_stagings_agree(qdd, oracle_mod, prec):
    """TMA staging (auto) and per-thread staging run the same colour filter."""
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    bc, U, eta = _setup(dims, 431)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    outs = []
    for variant in (0, 1):
        out = np.empty_like(eta)
        p = qdd.default_params(block=block, n_ras=3, n_dominv=3, inner_prec=prec, schwarz="sap",
                               ras_kernel=variant)
        qdd.ras_apply(lat, out, eta, 0.12, 1.0, p)
        outs.append(out)
    assert rel(outs[0], outs[1]) <= {"f32": 1e-6, "f16": 1e-3}[prec]
    ref = oracle_mod.Op(dims, bc, U, 0.12, 1.0).ras(eta, block, s=0, n_ras=3, n_dominv=3, schwarz="sap")
    check_field(outs[0], ref, TOL[prec], dims, block)


@pytest.mark.parametrize("schwarz,s", [("sap", 0), ("sap", 1), ("as", 1)])
def test_schwarz_multi_rhs(qdd, oracle_mod, schwarz, s):
    """Every right-hand side of a multi-RHS field gets its own sweeps (and its
    own slice of the additive sum)."""
    dims, bc, block, n = (8, 8, 8, 8), (1, 1, 1, -1), (4, 4, 4, 4), 3
    U = synth.gauge_field(dims, 0.3, 441)
    etas = [synth.gaussian_source(dims, 442 + k) for k in range(n)]
    lat = qdd.create_lattice(dims, bc, n_rhs=n)
    qdd.load_gauge(lat, U)
    eta = np.stack(etas)
    out = np.empty_like(eta)
    p = qdd.default_params(block=block, overlap=s, n_ras=2, n_dominv=3, inner_prec="f32", schwarz=schwarz)
    qdd.ras_apply(lat, out, eta, 0.12, 1.0, p)
    op = oracle_mod.Op(dims, bc, U, 0.12, 1.0)
    for k in range(n):
        ref = op.ras(etas[k], block, s=s, n_ras=2, n_dominv=3, schwarz=schwarz)
        check_field(out[k], ref, TOL["f32"], dims, block)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_sap_noalloc_matches_ras_apply(qdd, prec):
    dims, block, s = (8, 8, 8, 8), (4, 4, 4, 4), 1
    bc, U, eta = _setup(dims, 451)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, overlap=s, n_ras=2, n_dominv=3, inner_prec=prec, schwarz="sap")
    ref = np.empty_like(eta)
    qdd.ras_apply(lat, ref, eta, 0.12, 1.0, p)
    f = [qdd.field_create(lat, prec) for _ in range(4)]
    try:
        qdd.field_import(f[1], eta)
        qdd.ras_field_noalloc(lat, f[0], f[1], f[2], f[3], 0.12, 1.0, p)
        out = np.empty_like(eta)
        qdd.field_export(f[0], out)
        assert rel(out, ref) <= {"f32": 1e-6, "f16": 1e-3}[prec]
        # the additive sum over overlapping domains needs a buffer: refused
        with pytest.raises(qdd.QddError) as e:
            qdd.ras_field_noalloc(lat, f[0], f[1], f[2], f[3], 0.12, 1.0,
                                  qdd.default_params(block=block, overlap=1, inner_prec=prec, schwarz="as"))
        assert e.value.status == qdd.QDD_ERR_ARG
    finally:
        for x in f:
            qdd.field_destroy(x)


def test_schwarz_rejects_unknown_variant(qdd):
    dims = (8, 8, 8, 8)
    bc, U, eta = _setup(dims, 461)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(schwarz=3)
    with pytest.raises(qdd.QddError) as e:
        qdd.ras_apply(lat, np.empty_like(eta), eta, 0.12, 1.0, p)
    assert e.value.status == qdd.QDD_ERR_ARG
    with pytest.raises(qdd.QddError) as e:
        qdd.solve(lat, np.empty_like(eta), eta, 0.12, 1.0, 1e-10, p)
    assert e.value.status == qdd.QDD_ERR_ARG


@pytest.mark.parametrize("schwarz,s,prec", [("sap", 0, "f16"), ("sap", 1, "f32"), ("as", 1, "f32"),
                                            ("as", 1, "f16")])
@pytest.mark.parametrize("stream", [False, True])
def test_solve_with_schwarz_preconditioner(qdd, oracle_mod, schwarz, s, prec, stream):
    """The nested solve reaches the FP64 tolerance with SAP or AS as K (eager
    launches, or CUDA graphs on a stream), and counts its sweeps and global D
    applications: per inner iteration two applications of K of n_ras cycles
    (two sweeps per SAP cycle), one D per sweep but the last, and two D of the
    BiCGStab itself.  AS runs one cycle: with overlap its Richardson
    iteration amplifies the residual (the doubly counted overlap), so more
    cycles make K a worse preconditioner, not a better one."""
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    n_ras = 1 if schwarz == "as" else 2
    bc, U, eta = _setup(dims, 471)
    st = torch.cuda.Stream() if stream else None
    lat = qdd.create_lattice(dims, bc, stream=st)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    d_eta = torch.from_numpy(eta).cuda()
    phi = torch.zeros_like(d_eta)
    p = qdd.default_params(block=block, overlap=s, n_ras=n_ras, n_dominv=4, inner_prec=prec, schwarz=schwarz)
    info = qdd.solve(lat, phi, d_eta, 0.12, 1.0, 1e-10, p)
    torch.cuda.synchronize()
    res = oracle_mod.Op(dims, bc, U, 0.12, 1.0).true_residual(eta, phi.cpu().numpy())
    assert res <= 1e-10 and info["true_rel_residual"] <= 1e-10
    nsweep = n_ras * (2 if schwarz == "sap" else 1)
    it = info["inner_iters"]
    assert info["ras_sweeps"] == 2 * it * nsweep
    assert info["dv_count"] == 2 * it + 2 * it * (nsweep - 1)
