"""The C ABI library loads, exports every declared entry point, and rejects
bad arguments on the host before any device work (no GPU needed)."""
import os
import re

import pytest

from paper_1604_03155_gb300 import vp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return vp.lib(build_if_missing=True)


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as fh:
                text = fh.read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            # function declarations: "<return type> vp_name(" at the start of a line
            names |= set(re.findall(r"^\s*(?:vp_status|const char\*|int)\s+(vp_\w+)\s*\(", text, flags=re.M))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"vp_plan_create", "vp_apply", "vp_apply_grad", "vp_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name


def _create(d, N, kernel, k, L):
    import ctypes
    out = ctypes.c_void_p()
    st = vp.lib().vp_plan_create(ctypes.byref(out), d, N, kernel, k, L)
    return st, out.value


@pytest.mark.parametrize("args,status", [
    ((4, 16, vp.VP_LAPLACE, 0.0, 0.0), vp.VP_ERR_INVALID_ARG),       # d
    ((3, 15, vp.VP_LAPLACE, 0.0, 0.0), vp.VP_ERR_INVALID_ARG),       # odd N
    ((3, 2, vp.VP_LAPLACE, 0.0, 0.0), vp.VP_ERR_INVALID_ARG),        # N < 4
    ((3, 16, vp.VP_LAPLACE, 1.0, 0.0), vp.VP_ERR_INVALID_ARG),       # Laplace with k
    ((3, 16, vp.VP_HELMHOLTZ, 0.0, 0.0), vp.VP_ERR_INVALID_ARG),     # Helmholtz without k
    ((3, 16, vp.VP_HELMHOLTZ, float("nan"), 0.0), vp.VP_ERR_INVALID_ARG),
    ((3, 16, vp.VP_LAPLACE, 0.0, 1.7), vp.VP_ERR_INVALID_ARG),       # L <= sqrt(3)
    ((2, 16, vp.VP_LAPLACE, 0.0, 3.5), vp.VP_ERR_INVALID_ARG),       # L > 3
    ((3, 10, vp.VP_LAPLACE, 0.0, 0.0), vp.VP_ERR_UNSUPPORTED),       # 2N = 20 not built
    ((2, 9, 7, 0.0, 0.0), vp.VP_ERR_INVALID_ARG),                    # kernel enum
    ((3, 16, vp.VP_BIHARMONIC, 2.0, 0.0), vp.VP_ERR_INVALID_ARG),    # biharmonic with k
])
def test_plan_create_validation(lib, args, status):
    st, handle = _create(*args)
    assert st == status and not handle
    assert lib.vp_last_error(None)


def test_null_safety_and_strings(lib):
    assert lib.vp_destroy(None) == vp.VP_OK
    assert lib.vp_apply(None, None, None, vp.VP_C64) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_apply_pipeline(None, 1, None, None, None, vp.VP_C64) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_status_string(vp.VP_ERR_OOM) == b"VP_ERR_OOM"
    for n2 in (8, 12, 16, 24, 64, 96, 128, 192, 256, 512, 2048):
        assert lib.vp_fft_length_supported(n2) == 1
    for n2 in (10, 20, 100, 7):
        assert lib.vp_fft_length_supported(n2) == 0


def test_null_arguments_of_the_solver_network_and_batch_entry_points(lib):
    """Every entry point rejects a missing handle with VP_ERR_INVALID_ARG before
    touching the device."""
    import ctypes
    cnt = ctypes.c_int(0)
    assert lib.vp_plan_set_precision(None, vp.VP_FP32) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_plan_status(None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_operator(None, None, None, None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_rhs(None, None, None, None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_solve(None, None, None, None, None, None, None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_krylov_basis(None, None, None, 4, None, ctypes.byref(cnt)) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_flexible_basis(None, None, None, 4, None, None, None, ctypes.byref(cnt)) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_bicgstab(None, None, None, None, vp.VP_C128, 0, 1e-12, 10, None, None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_pb_gmres(None, None, None, None, None, 1e-12, 40, 10, None, None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_ls_last_error()
    assert lib.vp_kernel_entries(None, vp.VP_ARRAY_T, 0, None, 4, None, vp.VP_C128) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_matrix_block(None, vp.VP_ARRAY_T, 0, None, 2, None, 2, None, vp.VP_C128) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_unet_set_slope(None, 0.5) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_unet_destroy(None) == vp.VP_OK
    assert lib.vp_batch_apply(None, None, None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_batch_destroy(None) == vp.VP_OK
