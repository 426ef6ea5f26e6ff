"""gws_encode_noalloc: the encoding entry point for callers that cannot allocate device memory
(its scratch is a fixed array inside the library, not a caller workspace).

Collected last on purpose.  Called through the C ABI and compared with gws_encode, on two
calls in a row whose maxima differ (the shared scratch must be cleared between calls): both
entry points run the same kernels on the same input, so the phases must agree bit for bit.
A call must also leave the device's free memory unchanged."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2505_06582_gb300 import gws
from paper_2505_06582_gb300.scenes import SLM, random_field

pytestmark = pytest.mark.gpu


def _noalloc(field, slm, prec, out=None):
    lib = gws.load()
    opts = gws.make_opts(prec=prec)
    if out is None:
        out = torch.empty((slm.n_lambda, slm.H, slm.W), dtype=torch.float32, device="cuda")
    code = lib.gws_encode_noalloc(C.c_void_p(field.data_ptr()), C.byref(gws.Slm.of(slm)._c()), C.byref(opts),
                                  C.c_void_p(out.data_ptr()), C.c_float(0.0))
    assert code == 0, gws.STATUS.get(code, code)
    return out


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_noalloc_encode_matches_encode_on_two_calls(dtype):
    slm = SLM(96, 130, 8e-6, 8e-6, (638e-9, 520e-9, 450e-9))
    prec = gws.PREC_MIXED if dtype == np.complex64 else gws.PREC_FP64
    big = random_field(31, (3, 96, 130)).astype(dtype) * 4.0
    small = random_field(32, (3, 96, 130)).astype(dtype) * 0.25
    for f in (big, small):  # the second call has smaller maxima: stale scratch would show
        ft = torch.as_tensor(f, device="cuda")
        ref = gws.encode(ft, slm).cpu().numpy()
        got = _noalloc(ft, slm, prec).cpu().numpy()
        torch.cuda.synchronize()
        assert np.array_equal(got, ref)


def test_noalloc_encode_allocates_no_device_memory():
    slm = SLM(64, 96, 8e-6, 8e-6, (638e-9, 450e-9))
    ft = torch.as_tensor(random_field(33, (2, 64, 96)).astype(np.complex64), device="cuda")
    out = torch.empty((2, 64, 96), dtype=torch.float32, device="cuda")
    _noalloc(ft, slm, gws.PREC_MIXED, out)  # warm-up: module loading and the address look-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc(ft, slm, gws.PREC_MIXED, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_more_wavelengths_than_its_scratch():
    lib = gws.load()
    f = torch.zeros((1, 4, 4), dtype=torch.complex64, device="cuda")
    wl = (C.c_double * 17)(*([5e-7] * 17))
    s = gws._Slm(4, 4, 8e-6, 8e-6, 17, wl)
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    assert lib.gws_encode_noalloc(C.c_void_p(f.data_ptr()), C.byref(s), C.byref(gws.make_opts()),
                                  C.c_void_p(out.data_ptr()), C.c_float(0.0)) == 1
