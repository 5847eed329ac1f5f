"""The no-allocation K_RAS entry point (qdd_ras_field_noalloc), through the
C ABI: the oracle's K_RAS and the result of qdd_ras_apply on two calls in a
row, with the device's free memory unchanged by a call.

It serves callers that cannot let the library allocate device memory when the
preconditioner runs (programs whose device memory all comes from their own
pool, loops where an allocation would stall the GPU); its scratch is a fixed
array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process (the first call sets the scratch up).
"""

import ctypes

import numpy as np
import pytest
import torch

import synth
from gpu_common import check_field, qdd, rel  # noqa: F401

pytestmark = pytest.mark.gpu

# the tolerances of the RAS parity tests (against the oracle), and between
# two CUDA kernels of the same FP32 arithmetic on the same FP16/FP32 inputs
TOL = {"f32": 1e-5, "f16": 1e-2}
TOL_KERNELS = {"f32": 1e-5, "f16": 2e-3}


def _call(qdd, lat, fout, fin, frho, fv, kappa, csw, p):
    return qdd.lib().qdd_ras_field_noalloc(lat.handle, fout.handle, fin.handle, frho.handle, fv.handle,
                                           ctypes.c_double(kappa), ctypes.c_double(csw), ctypes.byref(p))


@pytest.mark.parametrize("block,s,prec", [((4, 4, 4, 4), 0, "f32"), ((4, 4, 4, 4), 1, "f32"),
                                          ((8, 4, 4, 4), 0, "f16"), ((4, 4, 4, 4), 2, "f16"),
                                          ((4, 4, 4, 4), 0, "f16")])
def test_noalloc_matches_oracle_and_ras_apply_twice(qdd, oracle_mod, block, s, prec):
    dims, bc, kappa, csw = (8, 8, 8, 8), (1, 1, 1, -1), 0.12, 1.0
    U = synth.gauge_field(dims, 0.3, 3)
    eta = synth.gaussian_source(dims, 4)
    ref = oracle_mod.Op(dims, bc, U, kappa, csw).ras(eta, block, s=s, n_ras=3, n_dominv=4)
    lat = qdd.create_lattice(dims, bc)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, overlap=s, n_ras=3, n_dominv=4, inner_prec=prec)
    lib_ref = np.empty_like(eta)
    qdd.ras_apply(lat, lib_ref, eta, kappa, csw, p)          # the existing entry point
    fin, fout, frho, fv = (qdd.field_create(lat, prec) for _ in range(4))
    qdd.field_import(fin, eta)
    for call in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call(qdd, lat, fout, fin, frho, fv, kappa, csw, p)
        assert st == qdd.QDD_OK, qdd.last_error()
        torch.cuda.synchronize()
        if call == 1:   # the first call may load kernel code; the second allocates nothing at all
            assert torch.cuda.mem_get_info()[0] == free0
        out = np.empty_like(eta)
        qdd.field_export(fout, out)
        check_field(out, ref, TOL[prec], dims, block, what=f"call {call}")
        assert rel(out, lib_ref) <= TOL_KERNELS[prec]


def test_noalloc_rejects_oversized_domains(qdd):
    dims = (16, 16, 16, 16)
    lat = qdd.create_lattice(dims)
    qdd.load_gauge(lat, synth.gauge_field(dims, 0.3, 1))
    p = qdd.default_params(block=(16, 16, 16, 16), overlap=0, inner_prec="f32")   # 65536-site domain
    f = [qdd.field_create(lat, "f32") for _ in range(4)]
    with pytest.raises(qdd.QddError) as e:
        qdd.ras_field_noalloc(lat, f[0], f[1], f[2], f[3], 0.12, 1.0, p)
    assert e.value.status == qdd.QDD_ERR_ARG and "scratch" in str(e.value)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_noalloc_refuses_an_unbuilt_clover_while_its_stream_is_captured(qdd, oracle_mod):
    """The clover term of a new (kappa, c_sw) cannot be built while the
    lattice's stream is being captured: the call returns QDD_ERR_STATE and
    leaves the clover cache as it was, so that the next eager call builds the
    right clover term."""
    dims, bc, block = (8, 8, 8, 8), (1, 1, 1, -1), (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 5)
    eta = synth.gaussian_source(dims, 6)
    st = torch.cuda.Stream()
    lat = qdd.create_lattice(dims, bc, stream=st)
    qdd.load_gauge(lat, U)
    p = qdd.default_params(block=block, n_ras=2, n_dominv=3, inner_prec="f32")
    f = [qdd.field_create(lat, "f32") for _ in range(4)]
    qdd.field_import(f[1], eta)
    assert _call(qdd, lat, f[0], f[1], f[2], f[3], 0.12, 1.0, p) == qdd.QDD_OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    status = []
    with torch.cuda.graph(g, stream=st):
        status.append(_call(qdd, lat, f[0], f[1], f[2], f[3], 0.13, 1.0, p))
    assert status[0] == qdd.QDD_ERR_STATE
    del g
    # eager again with the new kappa: the clover term is built now and is right
    assert _call(qdd, lat, f[0], f[1], f[2], f[3], 0.13, 1.0, p) == qdd.QDD_OK, qdd.last_error()
    out = np.empty_like(eta)
    qdd.field_export(f[0], out)
    ref = oracle_mod.Op(dims, bc, U, 0.13, 1.0).ras(eta, block, s=0, n_ras=2, n_dominv=3)
    check_field(out, ref, TOL["f32"], dims, block)
