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
