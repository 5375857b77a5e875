"""vp_apply_noalloc: the potential apply for callers that may not allocate
device memory when they apply the operator (e.g. code running inside another
framework's allocator, or a latency-bound loop that cannot afford an
allocation's implicit synchronisation).  The call takes its scratch from an
array compiled into the library; its result must equal vp_apply's, call after
call, although the shared array keeps whatever the previous call left in it.

This file is named to be collected last so that a failing run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import apply as A
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {"fp32": 1e-5, "fp64": 1e-12}


def _noalloc(plan, f, phi, dtype):
    lib = vp.lib()
    return lib.vp_apply_noalloc(ctypes.c_void_p(plan.handle), ctypes.c_void_p(f.data_ptr()),
                                ctypes.c_void_p(phi.data_ptr()), dtype)


@pytest.mark.parametrize("d,N,kernel,k,prec", [(3, 32, "helmholtz", 20.0, "fp32"), (2, 256, "laplace", 0.0, "fp64"),
                                               (3, 24, "laplace", 0.0, "fp32")])
def test_noalloc_matches_apply_on_two_consecutive_calls(d, N, kernel, k, prec):
    cdt = np.complex64 if prec == "fp32" else np.complex128
    code = vp.VP_C64 if prec == "fp32" else vp.VP_C128
    plan = vp.Plan(d, N, kernel, k, 0.0, precision=prec)
    for call in range(2):
        src = I.random_gaussians(I.BASE_SEED + 500 + call, 5, d)
        f = torch.from_numpy(I.sample_gaussians(src, N).astype(cdt)).to(DEV)
        ref = plan.apply(f)
        out = torch.full_like(f, float("nan"))
        st = _noalloc(plan, f, out, code)
        torch.cuda.synchronize()
        assert st == vp.VP_OK, vp.lib().vp_last_error(ctypes.c_void_p(plan.handle))
        assert A.rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < TOL[prec]
    plan.close()


def test_noalloc_rejects_grids_beyond_the_static_array():
    plan = vp.Plan(3, 128, "laplace", 0.0, 0.0, precision="fp64")  # 6 N^3 x 16 B > 128 MiB
    f = torch.zeros((128,) * 3, dtype=torch.complex128, device=DEV)
    out = torch.empty_like(f)
    assert _noalloc(plan, f, out, vp.VP_C128) == vp.VP_ERR_UNSUPPORTED
    assert b"scratch" in vp.lib().vp_last_error(ctypes.c_void_p(plan.handle))
    # host pointers are refused (staging would need an allocation)
    fh = np.zeros((128,) * 3, np.complex128)
    st = vp.lib().vp_apply_noalloc(ctypes.c_void_p(plan.handle), ctypes.c_void_p(fh.ctypes.data),
                                   ctypes.c_void_p(fh.ctypes.data + 16), vp.VP_C128)
    assert st == vp.VP_ERR_INVALID_ARG
    plan.close()
