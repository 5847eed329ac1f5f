"""Shared helpers of the GPU tests (the CUDA path through the C ABI)."""

import numpy as np
import pytest

# Relative L2 tolerances of one D application against the FP64 oracle.
# FP64: rounding of ~1900 flops per site (~1e-15) with margin.
# FP32: inputs rounded to 2^-24 and FP32 arithmetic, ~1e-7 observed scale.
# FP16: binary16 storage of spinor, links and clover (2^-11 relative to the
#       site norm), FP32 arithmetic.
TOL_D = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3}


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_elem(a, b):
    """Largest element-wise deviation, relative to the largest element of b."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="session")
def qdd():
    from paper_1011_3318_gb300 import build
    build.build()
    from paper_1011_3318_gb300 import qdd as q
    return q


def block_rel_max(a, b, dims, block):
    """Largest relative L2 deviation over the blocks of a blocking of the
    lattice (one RAS domain's bulk each): a single wrong domain shows here
    even when the whole-field norm hides it."""
    Lx, Ly, Lz, Lt = dims
    bx, by, bz, bt = block
    shape = (Lt // bt, bt, Lz // bz, bz, Ly // by, by, Lx // bx, bx, 12)
    a = np.asarray(a).reshape(shape)
    b = np.asarray(b).reshape(shape)
    num = (np.abs(a - b) ** 2).sum(axis=(1, 3, 5, 7, 8))
    den = (np.abs(b) ** 2).sum(axis=(1, 3, 5, 7, 8))
    return float(np.sqrt(num / den).max())


def check_field(out, ref, tol, dims=None, block=None, what=""):
    """A field against the oracle's: relative L2 <= tol over the field, the
    largest element deviation <= 10 tol (relative to the largest element), and,
    given a blocking, the relative L2 of every block <= 4 tol."""
    r = rel(out, ref)
    m = max_elem(out, ref)
    msg = f"{what} rel {r:.2e}, max element {m:.2e}"
    assert r <= tol, msg
    assert m <= 10 * tol, msg
    if dims is not None and block is not None:
        bm = block_rel_max(out, ref, dims, block)
        assert bm <= 4 * tol, msg + f", worst block {bm:.2e}"


_WORKLOAD_32 = {}


def workload_32():
    """The benchmark's 32^4 inputs (links eps = 0.3 seed 1, Gaussian source
    seed 2), generated once per test session (about 20 s of CPU)."""
    if not _WORKLOAD_32:
        import synth
        dims = (32, 32, 32, 32)
        _WORKLOAD_32["U"] = synth.gauge_field(dims, 0.3, 1)
        _WORKLOAD_32["eta"] = synth.gaussian_source(dims, 2)
    return _WORKLOAD_32["U"], _WORKLOAD_32["eta"]
