"""The saved-plan file format (vp_plan_save / vp_plan_load), checked on the
host: the loader refuses a missing file, a wrong magic, version or size, a
truncated file, trailing bytes and a hash mismatch before any device work, and
accepts a well-formed file (on a machine without a GPU it then stops at the
device, with VP_ERR_CUDA).  The file is written here from the format's
definition: a 96-byte header and complex128 octants hashed by 64-bit FNV-1a
over 8-byte words."""
import ctypes
import struct

import numpy as np
import pytest

from paper_1604_03155_gb300 import vp

@pytest.fixture(scope="module")
def lib():
    return vp.lib()


def _fnv1a_words(payload: bytes) -> int:
    h = 14695981039346656037
    for (w,) in struct.iter_unpack("<Q", payload):
        h = ((h ^ w) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _plan_file(d=2, N=(4, 6), kernel=vp.VP_LAPLACE, k=0.0, L=1.5, grad=0, magic=b"VPPLAN01", version=1,
               checksum=None, extra=b"", cut=0):
    oct_ = int(np.prod([n + 1 for n in N]))
    narr = 2 + (2 * d if grad else 0)
    rng = np.random.default_rng(5)
    payload = rng.standard_normal(2 * oct_ * narr).astype("<f8").tobytes()
    h = _fnv1a_words(payload) if checksum is None else checksum
    Ns = list(N) + [0] * (3 - d)
    header = magic + struct.pack("<II", version, 96) + struct.pack("<5i", d, *Ns, kernel) + struct.pack("<i", grad)
    header += struct.pack("<dd", k, L) + struct.pack("<q", oct_) + struct.pack("<QQ", len(payload), h)
    header += bytes(16)
    assert len(header) == 96
    data = header + payload + extra
    return data[: len(data) - cut] if cut else data


def _load(lib, path):
    out = ctypes.c_void_p()
    st = lib.vp_plan_load(ctypes.byref(out), str(path).encode())
    if out.value:
        lib.vp_destroy(out)
    return st, (lib.vp_last_error(None) or b"").decode()


def test_null_and_missing(lib, tmp_path):
    out = ctypes.c_void_p()
    assert lib.vp_plan_load(None, b"x") == vp.VP_ERR_INVALID_ARG
    assert lib.vp_plan_load(ctypes.byref(out), None) == vp.VP_ERR_INVALID_ARG
    assert lib.vp_plan_save(None, b"x") == vp.VP_ERR_INVALID_ARG
    assert lib.vp_plan_kernel(None, None) == vp.VP_ERR_INVALID_ARG
    st, msg = _load(lib, tmp_path / "absent.vpplan")
    assert st == vp.VP_ERR_INVALID_ARG and "cannot open" in msg


@pytest.mark.parametrize("case,needle", [
    (dict(magic=b"VPPLAN02"), "magic"),
    (dict(version=2), "magic"),
    (dict(d=4, N=(4, 4, 4, 4)[:3]), "dimension"),
    (dict(N=(3, 6)), "grid size"),
    (dict(cut=8), "truncated"),
    (dict(extra=b"\0"), "trailing"),
    (dict(checksum=12345), "checksum"),
])
def test_malformed_files_are_refused(lib, tmp_path, case, needle):
    path = tmp_path / "bad.vpplan"
    if case.get("d") == 4:
        data = bytearray(_plan_file())
        data[16:20] = struct.pack("<i", 4)
    else:
        data = _plan_file(**case)
    path.write_bytes(bytes(data))
    st, msg = _load(lib, path)
    assert st == vp.VP_ERR_INVALID_ARG and needle in msg, (st, msg)


def test_size_mismatch_is_refused(lib, tmp_path):
    data = bytearray(_plan_file())
    data[56:64] = struct.pack("<q", 1)  # octant size that does not match the grid
    (tmp_path / "s.vpplan").write_bytes(bytes(data))
    st, msg = _load(lib, tmp_path / "s.vpplan")
    assert st == vp.VP_ERR_INVALID_ARG and "sizes" in msg


def test_well_formed_file_reaches_the_device(lib, tmp_path):
    import torch
    for kw in (dict(), dict(grad=1), dict(d=3, N=(4, 4, 6), L=1.8, kernel=vp.VP_HELMHOLTZ, k=3.0)):
        path = tmp_path / "ok.vpplan"
        path.write_bytes(_plan_file(**kw))
        st, msg = _load(lib, path)
        if torch.cuda.is_available():
            assert st == vp.VP_OK, msg
        else:
            assert st == vp.VP_ERR_CUDA, (st, msg)


def test_huge_announced_grid_with_a_short_file_is_refused_before_allocating(lib, tmp_path):
    """A header announcing a 60000^2 grid (two 58 GB octants) on a file of a
    few hundred bytes: refused as truncated from the file size, at once."""
    import time
    d, N = 2, (60000, 60000)
    oct_ = (N[0] + 1) * (N[1] + 1)
    header = b"VPPLAN01" + struct.pack("<II", 1, 96) + struct.pack("<5i", d, N[0], N[1], 0, vp.VP_LAPLACE)
    header += struct.pack("<i", 0) + struct.pack("<dd", 0.0, 1.5) + struct.pack("<q", oct_)
    header += struct.pack("<QQ", 2 * oct_ * 16, 0) + bytes(16)
    path = tmp_path / "huge.vpplan"
    path.write_bytes(header + bytes(256))
    t0 = time.perf_counter()
    st, msg = _load(lib, path)
    assert st == vp.VP_ERR_INVALID_ARG and "truncated" in msg, (st, msg)
    assert time.perf_counter() - t0 < 1.0
