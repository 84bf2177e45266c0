"""Python binding of the GB300 primed-PCA library (``include/ppca.h``).

Argument marshalling only: every function has the name of its C entry point,
turns torch tensors into device pointers and sizes, calls the shared library
and raises ``PPCAError`` on a non-OK status.  All arithmetic runs in the CUDA
kernels of ``libppca_gb300.so``; there is no CPU path.  If the library has not
been built, importing works but the first call raises.

Layouts (as in the header): X is n x d row-major; bases and eigenvectors are
d x m column-major FP32, i.e. torch tensors of shape (m, d) whose row j is
direction j (``V.T`` is the d x m matrix).
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "PPCAError", "load_library", "library_path",
    "PPCA_OK", "PPCA_ERR_INVALID", "PPCA_ERR_OOM", "PPCA_ERR_CUDA", "PPCA_ERR_STATE", "PPCA_ERR_NUMERICAL",
    "PPCA_ERR_TIMEOUT", "PPCA_ERR_UNSUPPORTED", "PPCA_F32", "PPCA_BF16", "PPCA_FP8_E4M3", "PPCA_POWER", "PPCA_OJA", "PPCA_EIGENGAME", "PPCA_POWER_SEQ",
    "PPCA_PREC_AUTO", "PPCA_PREC_FAST", "PPCA_PREC_ACCURATE", "ppca_prime_params",
    "ppca_version", "ppca_last_error", "ppca_prime_params_default", "ppca_create", "ppca_set_refine",
    "ppca_set_workspace_limit", "ppca_prime", "ppca_prime_continue", "ppca_finalize", "ppca_get_basis",
    "ppca_sync", "ppca_get_state", "ppca_set_state", "ppca_destroy", "ppca_xpass", "ppca_orthonormalize",
    "ppca_projected_gram", "ppca_autotune", "ppca_batch_autotune",
    "ppca_eigh", "ppca_quantize_bf16", "ppca_quantize_fp8", "ppca_set_timing", "ppca_get_timing",
    "ppca_timing", "ppca_eigh_noalloc", "ppca_schedule", "ppca_set_schedule", "ppca_instance_desc",
    "ppca_batch_create", "ppca_batch_run", "ppca_batch_sync", "ppca_batch_destroy", "ppca_batch_kernel_count",
    "ppca_upload", "ppca_finalize_host", "ppca_finalize_sampled", "ppca_variance_captured", "ppca_set_wait_limit",
    "ppca_set_allreduce", "TorchAllReduce", "ppca_batch_set_priming", "ppca_batch_set_lockstep",
    "ppca_batch_lockstep", "ppca_set_step_graphs", "EXPORTED_SYMBOLS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "_lib", "libppca_gb300.so")

PPCA_OK = 0
(PPCA_ERR_INVALID, PPCA_ERR_OOM, PPCA_ERR_CUDA, PPCA_ERR_STATE, PPCA_ERR_NUMERICAL, PPCA_ERR_TIMEOUT,
 PPCA_ERR_UNSUPPORTED) = range(1, 8)
PPCA_F32, PPCA_BF16, PPCA_FP8_E4M3 = 0, 1, 2
PPCA_POWER, PPCA_OJA, PPCA_EIGENGAME, PPCA_POWER_SEQ = 0, 1, 2, 3
PPCA_PREC_AUTO, PPCA_PREC_FAST, PPCA_PREC_ACCURATE = 0, 1, 2

_STATUS = {0: "PPCA_OK", 1: "PPCA_ERR_INVALID", 2: "PPCA_ERR_OOM", 3: "PPCA_ERR_CUDA", 4: "PPCA_ERR_STATE",
           5: "PPCA_ERR_NUMERICAL", 6: "PPCA_ERR_TIMEOUT", 7: "PPCA_ERR_UNSUPPORTED"}

EXPORTED_SYMBOLS = [
    "ppca_version", "ppca_last_error", "ppca_prime_params_default", "ppca_create", "ppca_set_refine",
    "ppca_set_workspace_limit", "ppca_prime", "ppca_prime_continue", "ppca_finalize", "ppca_get_basis",
    "ppca_sync", "ppca_get_state", "ppca_set_state", "ppca_destroy", "ppca_xpass", "ppca_orthonormalize",
    "ppca_eigh", "ppca_quantize_bf16", "ppca_quantize_fp8", "ppca_set_timing", "ppca_get_timing",
    "ppca_eigh_noalloc", "ppca_set_schedule", "ppca_projected_gram", "ppca_autotune", "ppca_batch_autotune",
    "ppca_batch_create", "ppca_batch_run", "ppca_batch_sync", "ppca_batch_destroy", "ppca_batch_kernel_count",
    "ppca_upload", "ppca_finalize_host", "ppca_finalize_sampled", "ppca_variance_captured",
    "ppca_set_wait_limit", "ppca_set_allreduce", "ppca_batch_set_priming", "ppca_batch_set_lockstep",
    "ppca_batch_lockstep", "ppca_set_step_graphs",
]


class PPCAError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        self.status = status
        self.status_name = _STATUS.get(status, str(status))
        super().__init__(f"{func}: {self.status_name}: {message}")


class ppca_prime_params(ctypes.Structure):
    _fields_ = [
        ("V0", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
        ("batch", ctypes.c_int64),
        ("lr", ctypes.c_double),
        ("lr_offset", ctypes.c_double),
        ("momentum", ctypes.c_double),
        ("t0", ctypes.c_int64),
        ("precision", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("eps", ctypes.c_double),
    ]


class ppca_timing(ctypes.Structure):
    _fields_ = [
        ("pass_ms", ctypes.c_double * 3),
        ("passes", ctypes.c_int64 * 3),
        ("pass_rows", ctypes.c_int64 * 3),
        ("launches", ctypes.c_int64),
    ]


class ppca_schedule(ctypes.Structure):
    _fields_ = [
        ("fused", ctypes.c_int32),
        ("producers", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("flush", ctypes.c_int32),
        ("engine", ctypes.c_int32),
        ("kparts", ctypes.c_int32),
        ("l2_keep", ctypes.c_int32),
        ("fp8_mma", ctypes.c_int32),
    ]


class ppca_instance_desc(ctypes.Structure):
    _fields_ = [
        ("X", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int64),
        ("ld", ctypes.c_int64),
        ("dtype", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("row_scales", ctypes.c_void_p),
        ("V0", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
        ("E", ctypes.c_void_p),
        ("lambda_", ctypes.c_void_p),
        ("V_out", ctypes.c_void_p),
    ]


_lib = None
_lock = threading.Lock()

_c_status = ctypes.c_int
_vp, _i64, _i32, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double

_SIGS = {
    "ppca_version": (_i32, []),
    "ppca_last_error": (ctypes.c_char_p, []),
    "ppca_prime_params_default": (_c_status, [ctypes.POINTER(ppca_prime_params), ctypes.c_int]),
    "ppca_create": (_c_status, [ctypes.POINTER(_vp), _vp, _i64, _i64, _i64, ctypes.c_int, _vp, _vp]),
    "ppca_set_refine": (_c_status, [_vp, _vp, _i64, ctypes.c_int]),
    "ppca_set_workspace_limit": (_c_status, [_vp, _i64]),
    "ppca_prime": (_c_status, [_vp, ctypes.c_int, _i32, _i64, ctypes.POINTER(ppca_prime_params)]),
    "ppca_prime_continue": (_c_status, [_vp, _i64]),
    "ppca_finalize": (_c_status, [_vp, _i32, _vp, _vp, ctypes.c_int]),
    "ppca_upload": (_c_status, [_vp, _vp, _i64, _vp]),
    "ppca_finalize_host": (_c_status, [_vp, _i32, _vp, _vp, ctypes.c_int]),
    "ppca_finalize_sampled": (_c_status, [_vp, _i32, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                          ctypes.POINTER(_i64)]),
    "ppca_variance_captured": (_c_status, [_vp, _vp, _i32, _vp, ctypes.c_int]),
    "ppca_get_basis": (_c_status, [_vp, _vp]),
    "ppca_sync": (_c_status, [_vp]),
    "ppca_get_state": (_c_status, [_vp, _vp, ctypes.POINTER(_i64)]),
    "ppca_set_state": (_c_status, [_vp, _vp, _i64]),
    "ppca_destroy": (_c_status, [_vp]),
    "ppca_xpass": (_c_status, [_vp, _vp, _i32, _i64, _i64, _vp, ctypes.c_int]),
    "ppca_orthonormalize": (_c_status, [_vp, _vp, _vp, _i32]),
    "ppca_projected_gram": (_c_status, [_vp, _vp, _i32, _i64, _i64, _vp, ctypes.c_int]),
    "ppca_eigh": (_c_status, [_vp, _vp, _i32, _vp, _vp]),
    "ppca_quantize_bf16": (_c_status, [_vp, _i64, _i64, _i64, _vp, _i64, _vp]),
    "ppca_quantize_fp8": (_c_status, [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp]),
    "ppca_set_timing": (_c_status, [_vp, _i32]),
    "ppca_get_timing": (_c_status, [_vp, ctypes.POINTER(ppca_timing)]),
    "ppca_eigh_noalloc": (_c_status, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "ppca_set_schedule": (_c_status, [_vp, ctypes.POINTER(ppca_schedule)]),
    "ppca_set_wait_limit": (_c_status, [ctypes.c_uint64]),
    "ppca_set_allreduce": (_c_status, [_vp, _vp, _vp, _i64, _vp, _i64]),
    "ppca_batch_set_priming": (_c_status, [_vp, _i32]),
    "ppca_batch_set_lockstep": (_c_status, [_vp, _i32]),
    "ppca_set_step_graphs": (_c_status, [_vp, _i32]),
    "ppca_batch_lockstep": (_c_status, [_vp, ctypes.POINTER(_i32)]),
    "ppca_autotune": (_c_status, [_vp, _i32, _i64, _i32, ctypes.POINTER(ppca_schedule)]),
    "ppca_batch_autotune": (_c_status, [_vp, _i32, ctypes.POINTER(_i32)]),
    "ppca_batch_create": (_c_status, [ctypes.POINTER(_vp), ctypes.POINTER(ppca_instance_desc), _i32, _i32, _vp]),
    "ppca_batch_run": (_c_status, [_vp]),
    "ppca_batch_sync": (_c_status, [_vp]),
    "ppca_batch_destroy": (_c_status, [_vp]),
    "ppca_batch_kernel_count": (_c_status, [_vp, ctypes.POINTER(_i64)]),
}


def library_path() -> str:
    return _LIBPATH


def load_library(path: str | None = None):
    """Load libppca_gb300.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _LIBPATH
        if not os.path.exists(p):
            raise RuntimeError(f"the pPCA CUDA library is not built ({p} missing); "
                               "run `python -m paper_2109_03709_gb300.build`")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status: int, func: str):
    if status != PPCA_OK:
        msg = load_library().ppca_last_error()
        raise PPCAError(status, func, msg.decode() if msg else "")


def _arg(t, what: str, on_device: bool, itemsize: int | None, contiguous: bool) -> int | None:
    """Address of a tensor argument, refused here if it cannot be what the library
    reads or writes there: memory on the wrong side (a host tensor where a kernel
    would write through the address, or the reverse), the wrong element size, or
    a non-contiguous layout where the call takes no leading dimension.  None and
    integer addresses are passed through unchecked."""
    if t is None or isinstance(t, int):
        return t
    if bool(t.is_cuda) != on_device:
        raise ValueError(f"{what} must be in {'device' if on_device else 'host'} memory "
                         f"({'a CUDA' if on_device else 'a CPU'} tensor)")
    if itemsize is not None and t.element_size() != itemsize:
        raise TypeError(f"{what} must have {itemsize}-byte elements, not {t.dtype}")
    if contiguous and not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def _dev(t, what: str, itemsize: int | None = None, contiguous: bool = True) -> int | None:
    return _arg(t, what, True, itemsize, contiguous)


def _host(t, what: str, itemsize: int | None = None, contiguous: bool = True) -> int | None:
    return _arg(t, what, False, itemsize, contiguous)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return PPCA_F32
    if t.dtype == torch.bfloat16:
        return PPCA_BF16
    if t.dtype == torch.uint8 or (hasattr(torch, "float8_e4m3fn") and t.dtype == torch.float8_e4m3fn):
        return PPCA_FP8_E4M3
    raise TypeError(f"unsupported X dtype {t.dtype}")


class Handle:
    """Owns a ppca_handle* and keeps the borrowed tensors alive."""

    def __init__(self, ptr: int, keep: list):
        self.ptr = ptr
        self._keep = keep

    def __del__(self):
        try:
            if self.ptr:
                load_library().ppca_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


# --------------------------------------------------------------------------- C ABI mirror

def ppca_version() -> int:
    return load_library().ppca_version()


def ppca_last_error() -> str:
    return load_library().ppca_last_error().decode()


def ppca_prime_params_default(method: int) -> ppca_prime_params:
    p = ppca_prime_params()
    _check(load_library().ppca_prime_params_default(ctypes.byref(p), method), "ppca_prime_params_default")
    return p


def ppca_create(X, row_scales=None, stream=None, *, n=None, d=None, ld=None, dtype=None) -> Handle:
    """Create a handle over X (a 2-D CUDA tensor, row-major; strides give ld)."""
    lib = load_library()
    if n is None:
        n, d = X.shape
        ld = X.stride(0)
        if X.stride(1) != 1:
            raise ValueError("X must be row-major (unit column stride)")
        dtype = _dtype_code(X)
    out = ctypes.c_void_p()
    _check(lib.ppca_create(ctypes.byref(out), _dev(X, "X", contiguous=False), n, d, ld, dtype,
                           _dev(row_scales, "row_scales", 4), _stream_ptr(stream)), "ppca_create")
    return Handle(out.value, [X, row_scales])


def ppca_set_refine(h: Handle, X_refine, ld=None, dtype=None):
    if X_refine is None:
        _check(load_library().ppca_set_refine(h.ptr, None, 0, 0), "ppca_set_refine")
        return
    ld = X_refine.stride(0) if ld is None else ld
    dtype = _dtype_code(X_refine) if dtype is None else dtype
    _check(load_library().ppca_set_refine(h.ptr, _dev(X_refine, "X_refine", contiguous=False), ld, dtype),
           "ppca_set_refine")
    h._keep.append(X_refine)


def ppca_set_workspace_limit(h: Handle, nbytes: int):
    _check(load_library().ppca_set_workspace_limit(h.ptr, nbytes), "ppca_set_workspace_limit")


def ppca_prime(h: Handle, method: int, m: int, T: int, params: ppca_prime_params | None = None, V0=None):
    if params is None:
        params = ppca_prime_params_default(method)
    if V0 is not None:
        params.V0 = _dev(V0, "V0", 4)
    _check(load_library().ppca_prime(h.ptr, method, m, T, ctypes.byref(params)), "ppca_prime")


def ppca_prime_continue(h: Handle, T: int):
    _check(load_library().ppca_prime_continue(h.ptr, T), "ppca_prime_continue")


def ppca_finalize(h: Handle, k: int, E, lam, precision: int = PPCA_PREC_AUTO):
    _check(load_library().ppca_finalize(h.ptr, k, _dev(E, "E", 4), _dev(lam, "lam", 8), precision),
           "ppca_finalize")


def ppca_upload(h: Handle, X_host, row_scales_host=None, ld_host: int | None = None):
    """Copy host X (a CPU tensor or array pointer of the handle's dtype) into the handle's device X."""
    if ld_host is None:
        ld_host = X_host.stride(0)
    _check(load_library().ppca_upload(h.ptr, _host(X_host, "X_host", contiguous=False), ld_host,
                                      _host(row_scales_host, "row_scales_host", 4)), "ppca_upload")


def ppca_finalize_host(h: Handle, k: int, E_host, lam_host, precision: int = PPCA_PREC_AUTO):
    """pPCA step with E (k x d row-major = d x k column-major FP32) and lambda (k FP64) written to host memory."""
    _check(load_library().ppca_finalize_host(h.ptr, k, _host(E_host, "E_host", 4), _host(lam_host, "lam_host", 8),
                                             precision), "ppca_finalize_host")


def ppca_finalize_sampled(h: Handle, k: int, E, lam, precision: int = PPCA_PREC_AUTO, fraction: float = 0.1,
                          seed: int = 0) -> int:
    """pPCA step over a seeded sample of 128-row blocks; returns the number of sampled rows."""
    rows = ctypes.c_int64(0)
    _check(load_library().ppca_finalize_sampled(h.ptr, k, _dev(E, "E", 4), _dev(lam, "lam", 8), precision, fraction,
                                                seed, ctypes.byref(rows)), "ppca_finalize_sampled")
    return rows.value


def ppca_variance_captured(h: Handle, E, k: int, var, precision: int = PPCA_PREC_AUTO):
    """var[j] = e_j^T X^T X e_j for the k columns of E (device (k, d) tensor = d x k column-major)."""
    _check(load_library().ppca_variance_captured(h.ptr, _dev(E, "E", 4), k, _dev(var, "var", 8), precision),
           "ppca_variance_captured")


def ppca_get_basis(h: Handle, V_out):
    _check(load_library().ppca_get_basis(h.ptr, _dev(V_out, "V_out", 4)), "ppca_get_basis")


def ppca_sync(h: Handle):
    _check(load_library().ppca_sync(h.ptr), "ppca_sync")


def ppca_get_state(h: Handle) -> bytes:
    lib = load_library()
    nbytes = ctypes.c_int64(0)
    _check(lib.ppca_get_state(h.ptr, None, ctypes.byref(nbytes)), "ppca_get_state")
    buf = ctypes.create_string_buffer(nbytes.value)
    _check(lib.ppca_get_state(h.ptr, buf, ctypes.byref(nbytes)), "ppca_get_state")
    return buf.raw[:nbytes.value]


def ppca_set_state(h: Handle, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load_library().ppca_set_state(h.ptr, buf, len(state)), "ppca_set_state")


def ppca_destroy(h: Handle):
    if h.ptr:
        _check(load_library().ppca_destroy(h.ptr), "ppca_destroy")
        h.ptr = None


def ppca_xpass(h: Handle, V, m: int, r0: int, r1: int, Z, precision: int = PPCA_PREC_AUTO):
    _check(load_library().ppca_xpass(h.ptr, _dev(V, "V", 4), m, r0, r1, _dev(Z, "Z", 4), precision), "ppca_xpass")


def ppca_projected_gram(h: Handle, Q, m: int, r0: int, r1: int, G, precision: int = PPCA_PREC_AUTO):
    """G (m x m FP64, device) = (X[r0:r1] Q)^T (X[r0:r1] Q) over the data the pPCA step reads."""
    _check(load_library().ppca_projected_gram(h.ptr, _dev(Q, "Q", 4), m, r0, r1, _dev(G, "G", 8), precision),
           "ppca_projected_gram")


def ppca_orthonormalize(h: Handle, V, Q, m: int):
    _check(load_library().ppca_orthonormalize(h.ptr, _dev(V, "V", 4), _dev(Q, "Q", 4), m), "ppca_orthonormalize")


def _need(t, count: int, what: str):
    """Refuse a tensor holding fewer than `count` elements (a kernel would run past its end)."""
    if t is not None and not isinstance(t, int) and t.numel() < count:
        raise ValueError(f"{what} holds {t.numel()} elements, the call needs {count}")


def _on_current_device(t, what: str):
    """Refuse a CUDA tensor that lives on another GPU than the current one."""
    if t is not None and not isinstance(t, int) and t.is_cuda:
        import torch
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{what} is on cuda:{t.device.index}, the current device is "
                             f"cuda:{torch.cuda.current_device()}")


def ppca_eigh(h: Handle, G, m: int, w, U):
    for t, c, what in ((G, m * m, "G"), (U, m * m, "U"), (w, m, "w")):
        _need(t, c, what)
    _check(load_library().ppca_eigh(h.ptr, _dev(G, "G", 8), m, _dev(w, "w", 8), _dev(U, "U", 8)), "ppca_eigh")


class Batch:
    """Owns a ppca_batch* and keeps the instances' tensors alive."""

    def __init__(self, ptr: int, keep: list):
        self.ptr = ptr
        self._keep = keep

    def __del__(self):
        try:
            if self.ptr:
                load_library().ppca_batch_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


def ppca_batch_create(instances, slots: int = 0, stream=None) -> Batch:
    """instances: list of dicts with X (CUDA tensor), k, m, T, E ((k, d) tensor), lam ((k,) float64 tensor),
    optional V0 ((m, d) tensor), seed, row_scales."""
    arr = (ppca_instance_desc * len(instances))()
    keep = []
    for i, ins in enumerate(instances):
        X = ins["X"]
        arr[i].X = _dev(X, f"instance {i} X", contiguous=False)
        arr[i].n, arr[i].d = X.shape
        arr[i].ld = X.stride(0)
        arr[i].dtype = _dtype_code(X)
        arr[i].k, arr[i].m, arr[i].T = ins["k"], ins["m"], ins["T"]
        arr[i].row_scales = _dev(ins.get("row_scales"), f"instance {i} row_scales", 4)
        arr[i].V0 = _dev(ins.get("V0"), f"instance {i} V0", 4)
        arr[i].seed = ins.get("seed", 0)
        arr[i].E = _dev(ins["E"], f"instance {i} E", 4)
        arr[i].lambda_ = _dev(ins["lam"], f"instance {i} lam", 8)
        arr[i].V_out = _dev(ins.get("V_out"), f"instance {i} V_out", 4)
        keep.append(ins)
    out = ctypes.c_void_p()
    _check(load_library().ppca_batch_create(ctypes.byref(out), arr, len(instances), slots, _stream_ptr(stream)),
           "ppca_batch_create")
    return Batch(out.value, keep)


def ppca_batch_run(b: Batch):
    _check(load_library().ppca_batch_run(b.ptr), "ppca_batch_run")


def ppca_batch_set_priming(b: Batch, dtype: int):
    """PPCA_BF16: prime FP32 instances on their BF16 rounding (pPCA step on the FP32 data); PPCA_F32: as given."""
    _check(load_library().ppca_batch_set_priming(b.ptr, dtype), "ppca_batch_set_priming")


def ppca_batch_set_lockstep(b: Batch, enable: bool):
    """Allow (default) or forbid priming every instance in lockstep (grouped launches) at the first run."""
    _check(load_library().ppca_batch_set_lockstep(b.ptr, 1 if enable else 0), "ppca_batch_set_lockstep")


def ppca_batch_lockstep(b: Batch) -> bool:
    """True if the captured graph primes the instances in lockstep."""
    a = _i32(0)
    _check(load_library().ppca_batch_lockstep(b.ptr, ctypes.byref(a)), "ppca_batch_lockstep")
    return bool(a.value)


def ppca_batch_autotune(b: Batch, reps: int = 2) -> int:
    """Tune every (dtype, d, m, n bucket) group of the batch before its first run; returns the group count."""
    g = _i32(0)
    _check(load_library().ppca_batch_autotune(b.ptr, reps, ctypes.byref(g)), "ppca_batch_autotune")
    return int(g.value)


def ppca_batch_kernel_count(b: Batch) -> int:
    """Kernel launches one ppca_batch_run performs (0 before the first run)."""
    c = _i64(0)
    _check(load_library().ppca_batch_kernel_count(b.ptr, ctypes.byref(c)), "ppca_batch_kernel_count")
    return int(c.value)


def ppca_batch_sync(b: Batch):
    _check(load_library().ppca_batch_sync(b.ptr), "ppca_batch_sync")


def ppca_batch_destroy(b: Batch):
    if b.ptr:
        _check(load_library().ppca_batch_destroy(b.ptr), "ppca_batch_destroy")
        b.ptr = None


def ppca_set_schedule(h: Handle, fused: int = -1, producers: int = 0, window: int = 0, flush: int = 0,
                      engine: int = 0, kparts: int = 0, l2_keep: int = 0, fp8_mma: int = 0):
    s = ppca_schedule(fused, producers, window, flush, engine, kparts, l2_keep, fp8_mma)
    _check(load_library().ppca_set_schedule(h.ptr, ctypes.byref(s)), "ppca_set_schedule")


def ppca_set_step_graphs(h: Handle, enable: bool):
    """Run full-minibatch Oja / EigenGame steps from a captured CUDA graph (default) or step by step."""
    _check(load_library().ppca_set_step_graphs(h.ptr, 1 if enable else 0), "ppca_set_step_graphs")


def ppca_set_wait_limit(ns: int = 0):
    """Limit (ns) of the bounded waits in the tensor-core kernels on the current device; 0 restores 2 s."""
    _check(load_library().ppca_set_wait_limit(int(ns)), "ppca_set_wait_limit")


# ppca_allreduce_fn: (buf, count, elem_bytes, stream, ctx) -> ppca_status
_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_void_p)


class TorchAllReduce:
    """The sum across ranks for ppca_set_allreduce, done by torch.distributed.

    Owns a staging tensor of `max_bytes` on `device`: the library copies each
    sum's operand into it and calls back; the callback sums the first `count`
    elements over `group` with dist.all_reduce (NCCL: on the device; gloo:
    through a host copy), after synchronising the device so that the library's
    copy has landed.  An exception inside the callback is kept in `error` and
    reported to the library as PPCA_ERR_CUDA.
    """

    def __init__(self, max_bytes: int, device, group=None):
        import torch
        self.group = group
        self.staging = torch.zeros(int(max_bytes), dtype=torch.uint8, device=device)
        self.error = None
        self.calls = 0
        self._cb = _ALLREDUCE_FN(self._call)

    def _call(self, buf, count, elem_bytes, stream, ctx):
        try:
            import torch
            import torch.distributed as dist
            dt = {4: torch.float32, 8: torch.float64}[int(elem_bytes)]
            t = self.staging[: int(count) * int(elem_bytes)].view(dt)
            if t.is_cuda:
                torch.cuda.synchronize(t.device)
            if t.is_cuda and dist.get_backend(self.group) == "nccl":
                dist.all_reduce(t, group=self.group)
            else:
                c = t.cpu()
                dist.all_reduce(c, group=self.group)
                t.copy_(c)
            if t.is_cuda:
                torch.cuda.synchronize(t.device)
            self.calls += 1
            return PPCA_OK
        except Exception as e:          # no exception may cross the C ABI
            self.error = e
            return PPCA_ERR_CUDA


def ppca_set_allreduce(h: Handle, reducer: "TorchAllReduce | None", n_total: int = 0):
    """Shard the rows of X over ranks: every pass's sum goes through `reducer` (None: one process)."""
    if reducer is None:
        _check(load_library().ppca_set_allreduce(h.ptr, None, None, 0, None, 0), "ppca_set_allreduce")
        return
    _check(load_library().ppca_set_allreduce(h.ptr, ctypes.cast(reducer._cb, ctypes.c_void_p), None, int(n_total),
                                             _dev(reducer.staging, "staging"), reducer.staging.numel()),
           "ppca_set_allreduce")
    h._keep.append(reducer)


def ppca_autotune(h: Handle, m: int, rows: int = 0, reps: int = 3) -> ppca_schedule:
    """Time the candidate fast-pass schedules on the handle's data; the fastest is set and returned."""
    best = ppca_schedule()
    _check(load_library().ppca_autotune(h.ptr, m, rows, reps, ctypes.byref(best)), "ppca_autotune")
    return best


def ppca_eigh_noalloc(G, m: int, w, U, status=None, stream=None):
    """Eigensolve without any device allocation (fixed library scratch, m <= 128).

    For callers that cannot allocate device memory at the point where they
    solve (a host program whose device memory is handed out by its own
    allocator, or a latency-critical path where cudaMalloc may synchronise the
    device); calls that overlap on the same GPU race on the shared scratch and
    must be ordered by the caller.  Tensor arguments are refused here when they
    are too small for m or live on another GPU than the current one (the
    scratch array used is the current device's).
    """
    for t, c, what in ((G, m * m, "G"), (U, m * m, "U"), (w, m, "w"), (status, 1, "status")):
        _need(t, c, what)
    for t, what in ((G, "G"), (w, "w"), (U, "U"), (status, "status")):
        _on_current_device(t, what)
    _check(load_library().ppca_eigh_noalloc(_dev(G, "G", 8), m, _dev(w, "w", 8), _dev(U, "U", 8),
                                            _dev(status, "status", 4), _stream_ptr(stream)),
           "ppca_eigh_noalloc")


def ppca_quantize_bf16(X, out, stream=None):
    n, d = X.shape
    _check(load_library().ppca_quantize_bf16(_dev(X, "X", 4, contiguous=False), n, d, X.stride(0),
                                             _dev(out, "out", 2, contiguous=False), out.stride(0),
                                             _stream_ptr(stream)), "ppca_quantize_bf16")


def ppca_quantize_fp8(X, out, scales, stream=None):
    n, d = X.shape
    _check(load_library().ppca_quantize_fp8(_dev(X, "X", 4, contiguous=False), n, d, X.stride(0),
                                            _dev(out, "out", 1, contiguous=False), out.stride(0),
                                            _dev(scales, "scales", 4), _stream_ptr(stream)), "ppca_quantize_fp8")


def ppca_set_timing(h: Handle, enable: bool = True):
    _check(load_library().ppca_set_timing(h.ptr, 1 if enable else 0), "ppca_set_timing")


def ppca_get_timing(h: Handle) -> ppca_timing:
    t = ppca_timing()
    _check(load_library().ppca_get_timing(h.ptr, ctypes.byref(t)), "ppca_get_timing")
    return t
