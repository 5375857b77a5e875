"""Thin ctypes binding of the C ABI in include/vp.h (argument marshalling only).

Every step of the method runs in libvp.so's CUDA kernels; this module only
converts Python/torch/numpy arguments into pointers, sizes and enums.  It
raises ``VPError`` when the library is missing: there is no CPU fallback.

The module-level functions carry the C names (``vp_plan_create``,
``vp_apply``, ``vp_apply_grad``, ``vp_destroy`` ...); ``Plan`` wraps them.
Arrays may be CUDA torch tensors (device pointers; the call is asynchronous on
the plan's stream, by default torch's current stream) or host arrays (numpy or
CPU tensors; the library stages them and returns when the result is written).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VP_OK, VP_ERR_INVALID_ARG, VP_ERR_UNSUPPORTED, VP_ERR_OOM, VP_ERR_CUDA, VP_ERR_TIMEOUT, VP_ERR_NUMERICAL = range(7)
VP_LAPLACE, VP_HELMHOLTZ, VP_BIHARMONIC = 0, 1, 2
VP_FP32, VP_FP64 = 0, 1
VP_GRAD_EXACT, VP_GRAD_SPECTRAL2N = 0, 1
VP_R32, VP_C64, VP_R64, VP_C128 = 0, 1, 2, 3
VP_ARRAY_T, VP_ARRAY_GHAT, VP_ARRAY_TJ, VP_ARRAY_GHATJ = 0, 1, 2, 3

KERNELS = {"laplace": VP_LAPLACE, "helmholtz": VP_HELMHOLTZ, "biharmonic": VP_BIHARMONIC}
PRECISIONS = {"fp32": VP_FP32, "fp64": VP_FP64, "tc_bf16x2": 2, "tc_fp16x2": 3, "tc_bf16x3": 4}
GRAD_MODES = {"exact": VP_GRAD_EXACT, "spectral2n": VP_GRAD_SPECTRAL2N}


class VPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_STATUS_NAMES = {0: "VP_OK", 1: "VP_ERR_INVALID_ARG", 2: "VP_ERR_UNSUPPORTED", 3: "VP_ERR_OOM", 4: "VP_ERR_CUDA",
                 5: "VP_ERR_TIMEOUT", 6: "VP_ERR_NUMERICAL"}

_lib = None

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
c_char_p = ctypes.c_char_p

_SIGNATURES = {
    "vp_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_double, c_double]),
    "vp_plan_set_stream": (c_int, [c_void_p, c_void_p]),
    "vp_plan_set_precision": (c_int, [c_void_p, c_int]),
    "vp_plan_set_grad_mode": (c_int, [c_void_p, c_int]),
    "vp_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "vp_apply_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "vp_apply_pipeline": (c_int, [c_void_p, c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                  ctypes.POINTER(c_void_p), c_int]),
    "vp_plan_get_array": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(c_double), c_size_t]),
    "vp_plan_create_aniso": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_int), c_int, c_double,
                                     c_double]),
    "vp_plan_dims": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "vp_plan_save": (c_int, [c_void_p, c_char_p]),
    "vp_plan_load": (c_int, [ctypes.POINTER(c_void_p), c_char_p]),
    "vp_plan_kernel": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "vp_plan_set_host_access": (c_int, [c_void_p, c_int]),
    "vp_plan_autotune": (c_int, [c_void_p, c_int]),
    "vp_plan_pass_config": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_char_p, c_size_t]),
    "vp_plan_set_pass_config": (c_int, [c_void_p, c_int, c_int]),
    "vp_kernel_entries": (c_int, [c_void_p, c_int, c_int, c_void_p, ctypes.c_longlong, c_void_p, c_int]),
    "vp_matrix_block": (c_int, [c_void_p, c_int, c_int, c_void_p, ctypes.c_longlong, c_void_p, ctypes.c_longlong,
                                c_void_p, c_int]),
    "vp_plan_info": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_double),
                             ctypes.POINTER(c_double), ctypes.POINTER(c_size_t)]),
    "vp_plan_set_timing": (c_int, [c_void_p, c_int]),
    "vp_plan_get_timing": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_char_p),
                                   ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "vp_plan_launch_count": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "vp_plan_status": (c_int, [c_void_p]),
    "vp_last_error": (c_char_p, [c_void_p]),
    "vp_status_string": (c_char_p, [c_int]),
    "vp_destroy": (c_int, [c_void_p]),
    "vp_fft_length_supported": (c_int, [c_int]),
    "vp_apply_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "vp_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p)]),
    "vp_batch_set_stream": (c_int, [c_void_p, c_void_p]),
    "vp_batch_set_strategy": (c_int, [c_void_p, c_int]),
    "vp_batch_get_strategy": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "vp_batch_set_chunk": (c_int, [c_void_p, c_int]),
    "vp_batch_get_chunk": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "vp_batch_set_timeout": (c_int, [c_void_p, c_double]),
    "vp_batch_withhold": (c_int, [c_void_p, c_int, c_int]),
    "vp_batch_apply": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p)]),
    "vp_batch_status": (c_int, [c_void_p]),
    "vp_batch_info": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(c_int),
                              ctypes.POINTER(c_size_t)]),
    "vp_batch_last_error": (c_char_p, [c_void_p]),
    "vp_batch_destroy": (c_int, [c_void_p]),
    "vp_ls_operator": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "vp_ls_rhs": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "vp_ls_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "vp_ls_last_error": (c_char_p, []),
    "vp_ls_training_pair": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    ctypes.POINTER(c_double)]),
    "vp_ls_bicgstab": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_double, c_int, c_void_p,
                               c_void_p]),
    "vp_ls_bicgstab_mixed": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_int,
                                     c_void_p, c_void_p]),
    "vp_pb_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_void_p,
                            c_void_p]),
    "vp_pb_solve_mixed": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_int,
                                  c_void_p, c_void_p]),
    "vp_pb_gmres": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, c_void_p,
                            c_void_p]),
    "vp_ls_krylov_basis": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, ctypes.POINTER(c_int)]),
    "vp_ls_flexible_basis": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                     ctypes.POINTER(c_int)]),
    "vp_unet_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int]),
    "vp_unet_param_count": (c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "vp_unet_set_stream": (c_int, [c_void_p, c_void_p]),
    "vp_unet_set_weights": (c_int, [c_void_p, c_void_p, c_size_t]),
    "vp_unet_get_weights": (c_int, [c_void_p, c_int, c_void_p, c_size_t]),
    "vp_unet_forward": (c_int, [c_void_p, c_void_p, c_void_p]),
    "vp_unet_get_adam": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, ctypes.POINTER(ctypes.c_longlong)]),
    "vp_unet_set_adam": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, ctypes.c_longlong]),
    "vp_unet_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "vp_unet_adam_step": (c_int, [c_void_p, c_double]),
    "vp_unet_bind": (c_int, [c_void_p, c_void_p]),
    "vp_unet_set_slope": (c_int, [c_void_p, c_double]),
    "vp_unet_precond": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "vp_unet_status": (c_int, [c_void_p]),
    "vp_unet_set_timeout": (c_int, [c_void_p, c_double]),
    "vp_unet_withhold": (c_int, [c_void_p, c_int]),
    "vp_unet_last_error": (c_char_p, [c_void_p]),
    "vp_unet_destroy": (c_int, [c_void_p]),
}


def library_path() -> str:
    return _build.LIBPATH


def lib(build_if_missing: bool = False):
    """The loaded libvp.so; raises VPError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise VPError(VP_ERR_UNSUPPORTED, f"CUDA library not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, plan=None):
    if status != VP_OK:
        msg = lib().vp_last_error(plan)
        raise VPError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------

def vp_plan_create(d: int, N: int, kernel: int, k: float, L: float) -> int:
    out = c_void_p()
    _check(lib().vp_plan_create(ctypes.byref(out), d, N, kernel, float(k), float(L)))
    return out.value


def vp_plan_set_stream(plan: int, stream: int):
    _check(lib().vp_plan_set_stream(plan, stream), plan)


def vp_plan_set_precision(plan: int, precision: int):
    _check(lib().vp_plan_set_precision(plan, precision), plan)


def vp_plan_set_grad_mode(plan: int, mode: int):
    _check(lib().vp_plan_set_grad_mode(plan, mode), plan)


def vp_apply(plan: int, f_ptr: int, phi_ptr: int, dtype: int):
    _check(lib().vp_apply(plan, f_ptr, phi_ptr, dtype), plan)


def vp_apply_grad(plan: int, f_ptr: int, phi_ptr, grad_ptr: int, dtype: int):
    _check(lib().vp_apply_grad(plan, f_ptr, phi_ptr, grad_ptr, dtype), plan)


def vp_apply_noalloc(plan: int, f_ptr: int, phi_ptr: int, dtype: int):
    """vp_apply on the library's static scratch array (device pointers only);
    for callers that cannot allocate device memory at apply time."""
    _check(lib().vp_apply_noalloc(plan, f_ptr, phi_ptr, dtype), plan)


def vp_plan_status(plan: int):
    _check(lib().vp_plan_status(plan), plan)


def vp_destroy(plan: int):
    _check(lib().vp_destroy(plan))


def vp_fft_length_supported(n2: int) -> bool:
    return bool(lib().vp_fft_length_supported(n2))


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------

def _dtype_code(arr) -> int:
    name = str(arr.dtype).replace("torch.", "")
    table = {"float32": VP_R32, "complex64": VP_C64, "float64": VP_R64, "complex128": VP_C128}
    if name not in table:
        raise VPError(VP_ERR_INVALID_ARG, f"unsupported dtype {arr.dtype}")
    return table[name]


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> int:
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise VPError(VP_ERR_INVALID_ARG, "tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise VPError(VP_ERR_INVALID_ARG, "array must be C-contiguous")
        return x.ctypes.data
    raise VPError(VP_ERR_INVALID_ARG, f"unsupported array type {type(x)}")


def _empty_like(f, shape):
    if _is_torch(f):
        import torch
        return torch.empty(shape, dtype=f.dtype, device=f.device)
    return np.empty(shape, dtype=f.dtype)


class Plan:
    """A precomputed volume-potential operator (one d, N, kernel, k, L).  N is an
    int (N^d grid) or a tuple of d per-axis sizes (an N_0 x N_1 [x N_2] grid)."""

    def __init__(self, d: int, N, kernel: str = "laplace", k: float = 0.0, L: float = 0.0,
                 precision: str = "fp32", grad_mode: str = "exact", stream=None):
        self.d, self.N = d, N
        self.dims = tuple(N) if isinstance(N, (tuple, list)) else (N,) * d
        self.kernel = kernel
        if isinstance(N, (tuple, list)):
            if len(N) != d:
                raise VPError(VP_ERR_INVALID_ARG, "N needs d entries")
            out = c_void_p()
            arr = (c_int * d)(*N)
            _check(lib().vp_plan_create_aniso(ctypes.byref(out), d, arr, KERNELS[kernel], float(k), float(L)))
            self.handle = out.value
        else:
            self.handle = vp_plan_create(d, N, KERNELS[kernel], k, L)
        self.precision = precision
        vp_plan_set_precision(self.handle, PRECISIONS[precision])
        vp_plan_set_grad_mode(self.handle, GRAD_MODES[grad_mode])
        self._stream = stream
        if stream is not None:
            self.set_stream(stream)

    def save(self, path):
        """Write the plan's precompute results to `path` (vp_plan_save)."""
        _check(lib().vp_plan_save(self.handle, os.fsencode(path)), self.handle)

    @classmethod
    def load(cls, path, precision: str = "fp32", grad_mode: str = "exact", stream=None) -> "Plan":
        """A plan from a file written by save(), without the precompute."""
        out = c_void_p()
        _check(lib().vp_plan_load(ctypes.byref(out), os.fsencode(path)))
        self = cls.__new__(cls)
        self.handle = out.value
        d, kern = c_int(), c_int()
        _check(lib().vp_plan_info(self.handle, ctypes.byref(d), None, None, None, None), self.handle)
        dims = (c_int * 3)()
        _check(lib().vp_plan_dims(self.handle, dims), self.handle)
        _check(lib().vp_plan_kernel(self.handle, ctypes.byref(kern)), self.handle)
        self.d = d.value
        self.dims = tuple(dims[: self.d])
        self.N = self.dims[0] if len(set(self.dims)) == 1 else self.dims
        self.kernel = {v: name for name, v in KERNELS.items()}[kern.value]
        self.precision = precision
        vp_plan_set_precision(self.handle, PRECISIONS[precision])
        vp_plan_set_grad_mode(self.handle, GRAD_MODES[grad_mode])
        self._stream = stream
        if stream is not None:
            self.set_stream(stream)
        return self

    def set_stream(self, stream):
        """A torch.cuda.Stream, a raw cudaStream_t (int) or None (legacy default)."""
        raw = getattr(stream, "cuda_stream", stream)
        vp_plan_set_stream(self.handle, raw or 0)
        self._stream = stream

    def _sync_stream_to_torch(self, x):
        if self._stream is None and _is_torch(x) and x.is_cuda:
            import torch
            vp_plan_set_stream(self.handle, torch.cuda.current_stream(x.device).cuda_stream)

    def set_precision(self, precision: str):
        vp_plan_set_precision(self.handle, PRECISIONS[precision])
        self.precision = precision

    def set_host_access(self, direct: bool):
        """Pinned host buffers: access them in place (True) or stage them (False)."""
        _check(lib().vp_plan_set_host_access(self.handle, int(direct)), self.handle)

    PASS_NAMES = ("fwd_rows", "fwd_axis1", "fused_axis0", "inv_axis1", "inv_rows")

    def autotune(self, force: bool = False) -> dict:
        """Time the candidate tile shapes of each four-step pass; returns
        {pass name: chosen shape} for the passes that have candidates."""
        _check(lib().vp_plan_autotune(self.handle, 1 if force else 0), self.handle)
        return {name: cfg[2] for name, cfg in self.pass_configs().items() if cfg[1] > 0}

    def pass_config(self, pass_index: int):
        """(choice, number of candidates, name of the choice) of one pass."""
        cfg, count = c_int(), c_int()
        buf = ctypes.create_string_buffer(32)
        _check(lib().vp_plan_pass_config(self.handle, pass_index, ctypes.byref(cfg), ctypes.byref(count), buf, 32),
               self.handle)
        return cfg.value, count.value, buf.value.decode()

    def pass_configs(self) -> dict:
        return {name: self.pass_config(i) for i, name in enumerate(self.PASS_NAMES)
                if self.pass_config(i)[2] != "absent"}

    def set_pass_config(self, pass_index: int, cfg: int):
        _check(lib().vp_plan_set_pass_config(self.handle, pass_index, cfg), self.handle)

    def set_grad_mode(self, mode: str):
        vp_plan_set_grad_mode(self.handle, GRAD_MODES[mode])

    def apply(self, f, phi=None):
        if phi is None:
            phi = _empty_like(f, f.shape)
        self._sync_stream_to_torch(f)
        vp_apply(self.handle, _ptr(f), _ptr(phi), _dtype_code(f))
        return phi

    def apply_grad(self, f, phi=None, grad=None, with_phi: bool = True):
        if with_phi and phi is None:
            phi = _empty_like(f, f.shape)
        if grad is None:
            grad = _empty_like(f, (self.d,) + tuple(f.shape))
        self._sync_stream_to_torch(f)
        vp_apply_grad(self.handle, _ptr(f), _ptr(phi) if with_phi else None, _ptr(grad), _dtype_code(f))
        return (phi if with_phi else None), grad

    def apply_pipeline(self, fs, phis=None, grads=None, with_phi: bool = True, with_grad: bool = False):
        """phi_i = T * f_i (and grad_i when with_grad) for a list of host
        densities (pinned CPU tensors or numpy arrays), the transfers of one
        density overlapping the transform of the next; returns (phis, grads)."""
        fs = list(fs)
        if not fs:
            return [], []
        code = _dtype_code(fs[0])
        for f in fs:
            if _dtype_code(f) != code or tuple(f.shape) != tuple(fs[0].shape):
                raise VPError(VP_ERR_INVALID_ARG, "every density needs the same dtype and shape")
        if with_phi and phis is None:
            phis = [_empty_like(f, f.shape) for f in fs]
        if with_grad and grads is None:
            grads = [_empty_like(f, (self.d,) + tuple(f.shape)) for f in fs]
        self._sync_stream_to_torch(fs[0])

        def table(xs):
            if xs is None:
                return None
            if len(xs) != len(fs):
                raise VPError(VP_ERR_INVALID_ARG, "one output per density")
            return (c_void_p * len(xs))(*[_ptr(x) for x in xs])

        _check(lib().vp_apply_pipeline(self.handle, len(fs), table(fs), table(phis if with_phi else None),
                                       table(grads if with_grad else None), code), self.handle)
        return (phis if with_phi else None), (grads if with_grad else None)

    def get_array(self, which: str, axis: int = 0) -> np.ndarray:
        """An FP64 octant ((N+1)^d complex128): 'T', 'ghat', 'Tj', 'ghatj'."""
        code = {"T": VP_ARRAY_T, "ghat": VP_ARRAY_GHAT, "Tj": VP_ARRAY_TJ, "ghatj": VP_ARRAY_GHATJ}[which]
        shape = tuple(n + 1 for n in self.dims)
        buf = np.empty(2 * int(np.prod(shape)), dtype=np.float64)
        _check(lib().vp_plan_get_array(self.handle, code, axis,
                                       buf.ctypes.data_as(ctypes.POINTER(c_double)), buf.size), self.handle)
        return buf.view(np.complex128).reshape(shape)

    def kernel_entries(self, offsets, which: str = "T", axis: int = 0, dtype=None):
        """Nystrom entries T(n) for a (count, d) int32 device tensor of offsets
        (|n_j| <= N); which 'T' or 'Tj' (derivative along `axis`).  Returns a
        complex128 (or `dtype`) device tensor of length count."""
        import torch
        dtype = torch.complex128 if dtype is None else dtype
        out = torch.empty(offsets.shape[0], dtype=dtype, device=offsets.device)
        code = {"T": VP_ARRAY_T, "Tj": VP_ARRAY_TJ}[which]
        self._sync_stream_to_torch(offsets)
        _check(lib().vp_kernel_entries(self.handle, code, axis, _ptr(offsets), offsets.shape[0], _ptr(out),
                                       _dtype_code(out)), self.handle)
        return out

    def matrix_block(self, rows, cols, which: str = "T", axis: int = 0, dtype=None):
        """The (len(rows), len(cols)) block of the Nystrom matrix, T(p(row) - p(col)),
        for int64 device tensors of flat grid indices."""
        import torch
        dtype = torch.complex128 if dtype is None else dtype
        out = torch.empty((rows.shape[0], cols.shape[0]), dtype=dtype, device=rows.device)
        code = {"T": VP_ARRAY_T, "Tj": VP_ARRAY_TJ}[which]
        self._sync_stream_to_torch(rows)
        _check(lib().vp_matrix_block(self.handle, code, axis, _ptr(rows), rows.shape[0], _ptr(cols), cols.shape[0],
                                     _ptr(out), _dtype_code(out)), self.handle)
        return out

    def kernel_line(self, axis: int = 0, which: str = "T"):
        """T along one grid axis through the origin, offsets -N+1 .. N-1 (the
        paper's Fig. 2 view of the kernel), as a complex128 device tensor."""
        import torch
        Na = self.dims[axis]
        n = torch.arange(-Na + 1, Na, dtype=torch.int32, device="cuda")
        off = torch.zeros((n.shape[0], self.d), dtype=torch.int32, device="cuda")
        off[:, axis] = n
        return self.kernel_entries(off, which, axis)

    def info(self) -> dict:
        d, N, k, L, b = c_int(), c_int(), c_double(), c_double(), c_size_t()
        _check(lib().vp_plan_info(self.handle, ctypes.byref(d), ctypes.byref(N), ctypes.byref(k), ctypes.byref(L),
                                  ctypes.byref(b)), self.handle)
        return {"d": d.value, "N": N.value, "k": k.value, "L": L.value, "device_bytes": b.value}

    def set_timing(self, enable: bool):
        _check(lib().vp_plan_set_timing(self.handle, int(enable)), self.handle)

    def get_timing(self) -> dict:
        cap = 8
        npass = c_int()
        names = (c_char_p * cap)()
        launches = (c_int * cap)()
        ms = (c_double * cap)()
        _check(lib().vp_plan_get_timing(self.handle, cap, ctypes.byref(npass), names, launches, ms), self.handle)
        return {names[i].decode(): (launches[i], ms[i]) for i in range(min(cap, npass.value))}

    def launch_count(self, grad: bool) -> int:
        out = c_int()
        _check(lib().vp_plan_launch_count(self.handle, int(grad), ctypes.byref(out)), self.handle)
        return out.value

    def status(self):
        vp_plan_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            vp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


VP_BATCH_AUTO, VP_BATCH_PERSISTENT, VP_BATCH_PERSISTENT_ONE_PER_SM, VP_BATCH_PER_DENSITY = 0, 1, 2, 3
VP_BATCH_GRAPH_STREAMS = 4


def _bcheck(status: int, batch):
    if status != VP_OK:
        msg = lib().vp_batch_last_error(batch)
        raise VPError(status, msg.decode() if msg else "")


class Batch:
    """Many FP32 plans applied in one persistent launch (vp_batch_* of the C ABI)."""

    def __init__(self, plans, stream=None):
        self.plans = list(plans)  # borrowed: keep them alive
        arr = (c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        out = c_void_p()
        _bcheck(lib().vp_batch_create(ctypes.byref(out), len(self.plans), arr), None)
        self.handle = out.value
        self._stream = stream
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        raw = getattr(stream, "cuda_stream", stream)
        _bcheck(lib().vp_batch_set_stream(self.handle, raw or 0), self.handle)
        self._stream = stream

    def set_strategy(self, strategy: int):
        _bcheck(lib().vp_batch_set_strategy(self.handle, strategy), self.handle)

    def strategy(self) -> int:
        s = c_int()
        _bcheck(lib().vp_batch_get_strategy(self.handle, ctypes.byref(s)), self.handle)
        return s.value

    def set_chunk(self, chunk: int):
        """Tiles per work item of the persistent kernel (0: the autotuner's choice)."""
        _bcheck(lib().vp_batch_set_chunk(self.handle, chunk), self.handle)

    def chunk(self) -> int:
        s = c_int()
        _bcheck(lib().vp_batch_get_chunk(self.handle, ctypes.byref(s)), self.handle)
        return s.value

    def set_timeout(self, seconds: float):
        _bcheck(lib().vp_batch_set_timeout(self.handle, seconds), self.handle)

    def withhold(self, density: int, pass_index: int):
        _bcheck(lib().vp_batch_withhold(self.handle, density, pass_index), self.handle)

    def apply(self, fs, phis=None):
        if phis is None:
            phis = [_empty_like(f, f.shape) for f in fs]
        if self._stream is None and fs and _is_torch(fs[0]) and fs[0].is_cuda:
            import torch
            lib().vp_batch_set_stream(self.handle, torch.cuda.current_stream(fs[0].device).cuda_stream)
        fa = (c_void_p * len(fs))(*[_ptr(f) for f in fs])
        pa = (c_void_p * len(phis))(*[_ptr(p) for p in phis])
        _bcheck(lib().vp_batch_apply(self.handle, fa, pa), self.handle)
        return phis

    def status(self):
        """Synchronises; raises VPError (VP_ERR_TIMEOUT) if a bounded wait gave up."""
        _bcheck(lib().vp_batch_status(self.handle), self.handle)

    def info(self) -> dict:
        items, passes, b = ctypes.c_longlong(), c_int(), c_size_t()
        _bcheck(lib().vp_batch_info(self.handle, ctypes.byref(items), ctypes.byref(passes), ctypes.byref(b)),
                self.handle)
        return {"items": items.value, "passes": passes.value, "device_bytes": b.value}

    def close(self):
        if getattr(self, "handle", None):
            lib().vp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Lippmann-Schwinger solve and the learned preconditioner
# ---------------------------------------------------------------------------

PRECOND_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, c_void_p, c_void_p)


class LSOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("maxit", c_int), ("restart", c_int), ("use_initial_guess", c_int),
                ("precond", c_void_p), ("precond_ctx", c_void_p)]


class LSStats(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("matvecs", c_int), ("restarts", c_int), ("used_fallback", c_int),
                ("estimated_residual", c_double), ("true_residual", c_double), ("seconds", c_double)]


def _lscheck(status: int):
    if status != VP_OK:
        msg = lib().vp_ls_last_error()
        raise VPError(status, msg.decode() if msg else "")


def ls_operator(plan: Plan, q, u, out=None):
    """out = u - k^2 V[q u] (device tensors: q float32, u complex64)."""
    out = _empty_like(u, u.shape) if out is None else out
    plan._sync_stream_to_torch(u)
    _lscheck(lib().vp_ls_operator(plan.handle, _ptr(q), _ptr(u), _ptr(out)))
    return out


def ls_rhs(plan: Plan, q, u_inc, b=None):
    """b = k^2 V[q u_inc]."""
    b = _empty_like(u_inc, u_inc.shape) if b is None else b
    plan._sync_stream_to_torch(u_inc)
    _lscheck(lib().vp_ls_rhs(plan.handle, _ptr(q), _ptr(u_inc), _ptr(b)))
    return b


def ls_solve(plan: Plan, q, b, u, u_inc=None, tol=1e-6, maxit=1000, restart=30, precond=None,
             initial_guess=False) -> dict:
    """Flexible GMRES on u - k^2 V[q u] = b; precond is a UNet (bound to q) or None."""
    opts = LSOpts(tol, maxit, restart, int(initial_guess), None, None)
    if precond is not None:
        opts.precond = ctypes.cast(lib().vp_unet_precond, c_void_p)
        opts.precond_ctx = precond.handle
    st = LSStats()
    plan._sync_stream_to_torch(b)
    _lscheck(lib().vp_ls_solve(plan.handle, _ptr(q), _ptr(b), _ptr(u_inc) if u_inc is not None else None, _ptr(u),
                               ctypes.byref(opts), ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in LSStats._fields_}


LS_FORMS = {"field": 0, "density": 1}


def ls_bicgstab(plan: Plan, q, u_inc, u=None, form: str = "field", tol: float = 1e-12, maxit: int = 10000,
                history: bool = False):
    """The paper's solver: Bi-CGStab on the field form u - k^2 V[q u] = k^2 V[q u_inc]
    or the density form s - k^2 q V[s] = k^2 q u_inc, u = V[s].  Device tensors:
    complex64 u_inc with float32 q (plan in fp32) or complex128 with float64 q (plan
    in fp64).  Returns (u, stats) or (u, stats, residual history) with history=True."""
    if form not in LS_FORMS:
        raise VPError(VP_ERR_INVALID_ARG, f"form must be one of {sorted(LS_FORMS)}")
    u = _empty_like(u_inc, u_inc.shape) if u is None else u
    st = LSStats()
    hist = np.zeros(maxit + 1) if history else None
    plan._sync_stream_to_torch(u_inc)
    _lscheck(lib().vp_ls_bicgstab(plan.handle, _ptr(q), _ptr(u_inc), _ptr(u), _dtype_code(u_inc), LS_FORMS[form],
                                  tol, maxit, _ptr(hist) if history else None, ctypes.byref(st)))
    stats = {k: getattr(st, k) for k, _ in LSStats._fields_}
    if history:
        return u, stats, hist[:stats["iterations"] + 1]
    return u, stats


def ls_bicgstab_mixed(plan: Plan, q, u_inc, u=None, form: str = "field", tol: float = 1e-12, delta: float = 1e-2,
                      maxit: int = 10000, history: bool = False):
    """Bi-CGStab with FP32 iterations and FP64 reliable updates: FP64 accuracy
    (complex128 u_inc/u, float64 q) at mostly FP32 cost.  Returns (u, stats) or
    (u, stats, history); stats["restarts"] counts the FP64 updates, and
    stats["used_fallback"] is 1 when the FP32 phase gave up (after maxit
    iterations or a stall) and FP64 Bi-CGStab finished the solve from the
    mixed iterate (on the correction equation M e = b - M x)."""
    if form not in LS_FORMS:
        raise VPError(VP_ERR_INVALID_ARG, f"form must be one of {sorted(LS_FORMS)}")
    u = _empty_like(u_inc, u_inc.shape) if u is None else u
    st = LSStats()
    hist = np.zeros(maxit + 1) if history else None
    plan._sync_stream_to_torch(u_inc)
    _lscheck(lib().vp_ls_bicgstab_mixed(plan.handle, _ptr(q), _ptr(u_inc), _ptr(u), LS_FORMS[form], tol, delta,
                                        maxit, _ptr(hist) if history else None, ctypes.byref(st)))
    stats = {k: getattr(st, k) for k, _ in LSStats._fields_}
    if history:
        return u, stats, hist[:stats["iterations"] + 1]
    return u, stats


def pb_solve(plan: Plan, eps, grad_eps, rho, sigma=None, tol: float = 1e-12, maxit: int = 1000,
             mixed: bool = False, delta: float = 1e-2, history: bool = False):
    """-eps sigma + grad(eps) . grad V[sigma] = rho on a Laplace plan (Section 5.2).
    eps (N^d), grad_eps (d, N^d...) real and rho complex device tensors of the
    plan's precision (mixed=True: FP64 data, FP32 iterations with FP64 reliable
    updates).  Returns (sigma, stats) or (sigma, stats, history)."""
    sigma = _empty_like(rho, rho.shape) if sigma is None else sigma
    st = LSStats()
    hist = np.zeros(maxit + 1) if history else None
    plan._sync_stream_to_torch(rho)
    hp = _ptr(hist) if history else None
    if mixed:
        code = lib().vp_pb_solve_mixed(plan.handle, _ptr(eps), _ptr(grad_eps), _ptr(rho), _ptr(sigma), tol, delta,
                                       maxit, hp, ctypes.byref(st))
    else:
        code = lib().vp_pb_solve(plan.handle, _ptr(eps), _ptr(grad_eps), _ptr(rho), _ptr(sigma), _dtype_code(rho),
                                 tol, maxit, hp, ctypes.byref(st))
    _lscheck(code)
    stats = {k: getattr(st, k) for k, _ in LSStats._fields_}
    if history:
        return sigma, stats, hist[:stats["iterations"] + 1]
    return sigma, stats


def pb_gmres(plan: Plan, eps, grad_eps, rho, sigma=None, tol: float = 1e-12, restart: int = 40,
             maxit: int = 1000, history: bool = False):
    """The Section 5.2 equation with restarted GMRES(restart), the paper's
    solver for it, in FP64 (an FP64 plan; float64 eps and grad_eps, complex128
    rho).  Returns (sigma, stats) or (sigma, stats, history); history[j] is the
    GMRES residual estimate after step j (the explicit residual at a restart)."""
    sigma = _empty_like(rho, rho.shape) if sigma is None else sigma
    st = LSStats()
    hist = np.zeros(maxit + 1) if history else None
    plan._sync_stream_to_torch(rho)
    _lscheck(lib().vp_pb_gmres(plan.handle, _ptr(eps), _ptr(grad_eps), _ptr(rho), _ptr(sigma), tol, restart, maxit,
                               _ptr(hist) if history else None, ctypes.byref(st)))
    stats = {k: getattr(st, k) for k, _ in LSStats._fields_}
    if history:
        return sigma, stats, hist[:stats["iterations"] + 1]
    return sigma, stats


def ls_training_pair(plan: Plan, q, b, u_s, u_star, x_out, t_out) -> float:
    """Network input/target of one (residual, correction) pair; returns ||r||."""
    rn = c_double()
    _lscheck(lib().vp_ls_training_pair(plan.handle, _ptr(q), _ptr(b), _ptr(u_s) if u_s is not None else None,
                                       _ptr(u_star), _ptr(x_out), _ptr(t_out), ctypes.byref(rn)))
    return rn.value


def ls_krylov_basis(plan: Plan, q, b, m: int):
    """Orthonormal Krylov basis v_0..v_m of the plain operator from b, as an
    (m+1, *b.shape) complex64 tensor (fewer rows only at an exact breakdown)."""
    import torch
    V = torch.empty((m + 1,) + tuple(b.shape), dtype=torch.complex64, device=b.device)
    cnt = c_int()
    plan._sync_stream_to_torch(b)
    _lscheck(lib().vp_ls_krylov_basis(plan.handle, _ptr(q), _ptr(b), m, _ptr(V), ctypes.byref(cnt)))
    return V[:cnt.value]


def ls_flexible_basis(plan: Plan, q, b, m: int, precond):
    """Preconditioned directions z_0..z_{m-1} of one flexible GMRES cycle from b
    with the network `precond` (bound to q), as an (m, *b.shape) complex64 tensor."""
    import torch
    Z = torch.empty((m,) + tuple(b.shape), dtype=torch.complex64, device=b.device)
    cnt = c_int()
    plan._sync_stream_to_torch(b)
    _lscheck(lib().vp_ls_flexible_basis(plan.handle, _ptr(q), _ptr(b), m, ctypes.cast(lib().vp_unet_precond, c_void_p),
                                        precond.handle, _ptr(Z), ctypes.byref(cnt)))
    return Z[:cnt.value]


class UNet:
    """The learned preconditioner network (vp_unet_*)."""

    def __init__(self, S: int, C: int = 16, weights=None, slope: float = 0.1):
        out = c_void_p()
        st = lib().vp_unet_create(ctypes.byref(out), S, C)
        if st != VP_OK:
            raise VPError(st, "vp_unet_create failed")
        self.handle, self.S, self.C = out.value, S, C
        n = c_size_t()
        lib().vp_unet_param_count(self.handle, ctypes.byref(n))
        self.nparams = n.value
        self._check(lib().vp_unet_set_slope(self.handle, slope))
        if weights is not None:
            self.set_weights(weights)

    def _check(self, st):
        if st != VP_OK:
            msg = lib().vp_unet_last_error(self.handle)
            raise VPError(st, msg.decode() if msg else "")

    def set_stream(self, stream):
        self._check(lib().vp_unet_set_stream(self.handle, getattr(stream, "cuda_stream", stream) or 0))

    def set_weights(self, layers):
        """layers: list of (w [Co][Ci][27], b [Co]) arrays, or a flat float32 array."""
        if isinstance(layers, np.ndarray):
            flat = np.ascontiguousarray(layers, dtype=np.float32)
        else:
            flat = np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                                   for w, b in layers])
        assert flat.size == self.nparams
        self._check(lib().vp_unet_set_weights(self.handle, flat.ctypes.data, flat.size))

    def get(self, which: int = 0) -> np.ndarray:
        buf = np.empty(self.nparams, np.float32)
        self._check(lib().vp_unet_get_weights(self.handle, which, buf.ctypes.data, buf.size))
        return buf

    def forward(self, x, out=None):
        import torch
        out = torch.empty((2,) + tuple(x.shape[1:]), dtype=torch.float32, device=x.device) if out is None else out
        self._check(lib().vp_unet_forward(self.handle, _ptr(x), _ptr(out)))
        return out

    def loss_grad(self, x, target) -> float:
        loss = c_double()
        self._check(lib().vp_unet_loss_grad(self.handle, _ptr(x), _ptr(target), ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr: float):
        self._check(lib().vp_unet_adam_step(self.handle, lr))

    def get_adam(self):
        """(first moments, second moments, step count) of the optimiser."""
        m, v = np.empty(self.nparams, np.float32), np.empty(self.nparams, np.float32)
        step = ctypes.c_longlong()
        self._check(lib().vp_unet_get_adam(self.handle, m.ctypes.data, v.ctypes.data, self.nparams, ctypes.byref(step)))
        return m, v, step.value

    def set_adam(self, m, v, step: int):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        if m.size != self.nparams or v.size != self.nparams:
            raise VPError(VP_ERR_INVALID_ARG, "Adam state: one value per parameter")
        self._check(lib().vp_unet_set_adam(self.handle, m.ctypes.data, v.ctypes.data, self.nparams, int(step)))

    def status(self):
        """Synchronises the network's stream; raises on a timed-out convolution."""
        self._check(lib().vp_unet_status(self.handle))

    def set_timeout(self, seconds: float):
        self._check(lib().vp_unet_set_timeout(self.handle, seconds))

    def withhold(self, on: bool):
        """Test hook: the tensor-core kernels issue no MMAs, so their bounded waits run out."""
        self._check(lib().vp_unet_withhold(self.handle, int(on)))

    def bind(self, q):
        self._q = q
        self._check(lib().vp_unet_bind(self.handle, _ptr(q)))

    def close(self):
        if getattr(self, "handle", None):
            lib().vp_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
