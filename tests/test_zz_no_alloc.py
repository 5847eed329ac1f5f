"""The no-allocation K_RAS entry point (qdd_ras_field_noalloc) gives the same
result as qdd_ras_apply, on two calls in a row, through the C ABI.

It serves callers that cannot let the library allocate device memory when the
preconditioner runs (stream capture, caller-owned memory pools); its scratch
is a fixed array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process (the first call sets the scratch up).
"""

import ctypes

import numpy as np
import pytest

import synth
from gpu_common import qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

# the tolerances of the RAS parity tests
TOL = {"f32": 1e-5, "f16": 1e-2}


@pytest.mark.parametrize("block,s,prec", [((4, 4, 4, 4), 0, "f32"), ((4, 4, 4, 4), 1, "f32"),
                                          ((8, 4, 4, 4), 0, "f16"), ((4, 4, 4, 4), 2, "f16")])
def test_noalloc_matches_ras_apply_twice(qdd, block, s, prec):
    dims, bc, kappa, csw = (8, 8, 8, 8), (1, 1, 1, -1), 0.12, 1.0
    U = synth.gauge_field(dims, 0.3, 3)
    eta = synth.gaussian_source(dims, 4)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, overlap=s, n_ras=3, n_dominv=4, inner_prec=prec)
    ref = np.empty_like(eta)
    qdd.ras_apply(lat, ref, eta, kappa, csw, p)              # the existing entry point
    fin, fout, frho, fv = (qdd.field_create(lat, prec) for _ in range(4))
    qdd.field_import(fin, eta)
    for _ in range(2):
        st = qdd.lib().qdd_ras_field_noalloc(lat.handle, fout.handle, fin.handle, frho.handle, fv.handle,
                                             ctypes.c_double(kappa), ctypes.c_double(csw), ctypes.byref(p))
        assert st == qdd.QDD_OK, qdd.last_error()
        out = np.empty_like(eta)
        qdd.field_export(fout, out)
        assert rel(out, ref) <= TOL[prec]


def test_noalloc_rejects_oversized_domains(qdd):
    dims = (16, 16, 16, 16)
    lat = qdd.create_lattice(dims)
    qdd.load_gauge(lat, synth.gauge_field(dims, 0.3, 1))
    p = qdd.default_params(block=(16, 16, 16, 16), overlap=0, inner_prec="f32")   # 65536-site domain
    f = [qdd.field_create(lat, "f32") for _ in range(4)]
    with pytest.raises(qdd.QddError) as e:
        qdd.ras_field_noalloc(lat, f[0], f[1], f[2], f[3], 0.12, 1.0, p)
    assert e.value.status == qdd.QDD_ERR_ARG and "scratch" in str(e.value)
