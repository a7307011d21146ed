"""Python binding of libmoa — the GB300 generalized inner / outer product of
arbitrary-rank arrays (Raynolds & Mullin, A Mathematics of Arrays).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libmoa.so`` behind the C ABI of ``include/moa.h``.  PyTorch
supplies device memory and the current stream.  There is no CPU fallback:
if the library has not been built, importing the binding's functions raises.

Low-level calls mirror the C ABI one to one (``moa_inner``, ``moa_outer``,
``moa_inner_shape`` ...).  ``inner`` / ``outer`` are conveniences that take
torch tensors, read rho A / rho B from their shapes and allocate the result.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

__all__ = [
    "MoaError", "lib", "moa_inner", "moa_outer", "moa_inner_shape", "moa_outer_shape", "moa_status_string",
    "moa_device_status", "moa_release_workspace", "moa_version", "inner", "outer", "OPS", "DTYPES", "FORMS",
    "moa_batch_plan_create", "moa_batch_execute", "moa_batch_plan_destroy", "moa_batch_plan_info", "MoaProblem",
    "moa_inner_bf16x3_noalloc", "NOALLOC_SCRATCH_BYTES", "make_problems", "moa_selftest_wait_timeout",
    "moa_inner_host", "moa_kernel_timing", "moa_kernel_timing_read", "moa_inner_e4m3_scaled", "moa_ozaki_slices",
]

# size of the fixed device buffer behind moa_inner_bf16x3_noalloc (MOA_NOALLOC_SCRATCH_BYTES)
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024

OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "min": 4, "max": 5, "or": 6, "and": 7}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "fp8e4m3": 3, "i32": 4, "b1": 5, "f16": 6}
FORMS = {"native": 0, "bf16": 1, "fp8_t128": 2, "bf16x3": 3, "ozaki": 4, "f16": 5}
STATUS = {0: "MOA_OK", 1: "MOA_ERR_NULL", 2: "MOA_ERR_RANK", 3: "MOA_ERR_SHAPE_MISMATCH", 4: "MOA_ERR_OVERFLOW",
          5: "MOA_ERR_UNSUPPORTED", 6: "MOA_ERR_WORKSPACE", 7: "MOA_ERR_CUDA", 8: "MOA_ERR_TIMEOUT",
          9: "MOA_ERR_INTERNAL", 10: "MOA_ERR_ALIGNMENT", 11: "MOA_ERR_INVALID", 12: "MOA_ERR_SCRATCH_LIMIT",
          13: "MOA_ERR_NOT_DEVICE"}

_lib = None
_I64P = C.POINTER(C.c_int64)


class MoaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {STATUS.get(self.status, self.status)} ({_status_text(self.status)})")


class MoaProblem(C.Structure):
    """One problem of a batch (moa_problem in include/moa.h)."""
    _fields_ = [("kind", C.c_int32), ("reduce", C.c_int32), ("combine", C.c_int32), ("dtype", C.c_int32),
                ("form", C.c_int32), ("out_dtype", C.c_int32), ("rankA", C.c_int32), ("rankB", C.c_int32),
                ("shapeA", _I64P), ("shapeB", _I64P), ("A", C.c_void_p), ("B", C.c_void_p), ("out", C.c_void_p)]


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded libmoa.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmoa.so is not built ({path}); run __graft_entry__.build() first")
        L = C.CDLL(path)
        V, I, P, I64 = C.c_void_p, C.c_int, C.c_void_p, C.c_int64
        L.moa_inner.argtypes = [I, I, I, I, I, _I64P, P, I, _I64P, P, P, I, V]
        L.moa_outer.argtypes = [I, I, I, _I64P, P, I, _I64P, P, P, I, V]
        L.moa_inner_axes.argtypes = [I, I, I, I, I, _I64P, P, I, I, _I64P, P, I, P, I, V]
        L.moa_inner_host.argtypes = [I, I, I, I, I, _I64P, P, I, _I64P, P, P, I, V]
        L.moa_inner_e4m3_scaled.argtypes = [I, _I64P, P, P, I, _I64P, P, P, P, V]
        L.moa_kernel_timing.argtypes = [I]
        L.moa_kernel_timing_read.argtypes = [C.POINTER(I64), C.POINTER(C.c_double)]
        L.moa_ozaki_slices.argtypes = [I64]
        L.moa_ozaki_slices.restype = C.c_int
        L.moa_transpose.argtypes = [I, I, _I64P, C.POINTER(C.c_int), P, P, V]
        L.moa_inner_shape.argtypes = [I, _I64P, I, _I64P, C.POINTER(C.c_int), _I64P]
        L.moa_outer_shape.argtypes = [I, _I64P, I, _I64P, C.POINTER(C.c_int), _I64P]
        L.moa_status_string.argtypes = [I]
        L.moa_status_string.restype = C.c_char_p
        L.moa_device_status.argtypes = [V]
        L.moa_batch_plan_create.argtypes = [I, C.POINTER(MoaProblem), C.POINTER(C.c_void_p), C.POINTER(C.c_int)]
        L.moa_batch_execute.argtypes = [V, V]
        L.moa_batch_plan_destroy.argtypes = [V]
        L.moa_batch_plan_destroy.restype = None
        L.moa_batch_plan_info.argtypes = [V, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(C.c_double)]
        L.moa_inner_bf16x3_noalloc.argtypes = [I, _I64P, P, I, _I64P, P, P, V]
        L.moa_selftest_wait_timeout.argtypes = [C.c_uint32, V]
        _lib = L
    return _lib


def _status_text(st: int) -> str:
    try:
        return lib().moa_status_string(int(st)).decode()
    except Exception:
        return "?"


def _shape(shape):
    arr = (C.c_int64 * max(1, len(shape)))(*[int(s) for s in shape])
    return C.cast(arr, _I64P), arr


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _hptr(x):
    """Host address of a CPU tensor, a numpy array or an int."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _enum(table, v):
    return table[v] if isinstance(v, str) else int(v)


def _check(st, what):
    if st != 0:
        raise MoaError(st, what)


# ------------------------------------------------------------------ raw ABI
def moa_inner(reduce, combine, dtype, form, shapeA, A, shapeB, B, out, out_dtype, stream=None, check=True):
    """C ABI moa_inner: Eq. (2) D = reduce_p (A[..., p] combine B[p, ...])."""
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    st = lib().moa_inner(_enum(OPS, reduce), _enum(OPS, combine), _enum(DTYPES, dtype), _enum(FORMS, form),
                         len(shapeA), sa, _ptr(A), len(shapeB), sb, _ptr(B), _ptr(out), _enum(DTYPES, out_dtype),
                         _stream(stream))
    if check:
        _check(st, "moa_inner")
    return st


def moa_inner_host(reduce, combine, dtype, form, shapeA, A, shapeB, B, out, out_dtype, stream=None, check=True):
    """C ABI moa_inner_host: Eq. (2) on arrays in host memory (copies in and
    out inside the call, ordered on `stream`).  A, B, out: host addresses or
    CPU tensors / numpy arrays (page-locked memory keeps the copies async)."""
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    st = lib().moa_inner_host(_enum(OPS, reduce), _enum(OPS, combine), _enum(DTYPES, dtype), _enum(FORMS, form),
                              len(shapeA), sa, _hptr(A), len(shapeB), sb, _hptr(B), _hptr(out),
                              _enum(DTYPES, out_dtype), _stream(stream))
    if check:
        _check(st, "moa_inner_host")
    return st


def moa_inner_e4m3_scaled(shapeA, A, scale_a, shapeB, B, scale_b, out, stream=None, check=True):
    """C ABI moa_inner_e4m3_scaled: Eq. (2) (+,*) on E4M3 arrays with per-128 power-of-two block scales."""
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    st = lib().moa_inner_e4m3_scaled(len(shapeA), sa, _ptr(A), _ptr(scale_a), len(shapeB), sb, _ptr(B), _ptr(scale_b),
                                     _ptr(out), _stream(stream))
    if check:
        _check(st, "moa_inner_e4m3_scaled")
    return st


def moa_kernel_timing(enable: bool):
    """Start (True) or stop (False) CUDA-event timing of the library's GEMM launches."""
    _check(lib().moa_kernel_timing(1 if enable else 0), "moa_kernel_timing")


def moa_ozaki_slices(K: int) -> int:
    """Digit slices per operand the Ozaki form takes for a contraction of length K."""
    return int(lib().moa_ozaki_slices(int(K)))


def moa_kernel_timing_read():
    """(launches, total device milliseconds) of the GEMM launches recorded since the last start."""
    n, ms = C.c_int64(0), C.c_double(0.0)
    _check(lib().moa_kernel_timing_read(C.byref(n), C.byref(ms)), "moa_kernel_timing_read")
    return int(n.value), float(ms.value)


def moa_inner_axes(reduce, combine, dtype, form, shapeA, A, axisA, shapeB, B, axisB, out, out_dtype, stream=None,
                   check=True):
    """C ABI moa_inner_axes: Eq. (2) contracting axis axisA of A with axis axisB of B."""
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    st = lib().moa_inner_axes(_enum(OPS, reduce), _enum(OPS, combine), _enum(DTYPES, dtype), _enum(FORMS, form),
                              len(shapeA), sa, _ptr(A), int(axisA), len(shapeB), sb, _ptr(B), int(axisB), _ptr(out),
                              _enum(DTYPES, out_dtype), _stream(stream))
    if check:
        _check(st, "moa_inner_axes")
    return st


def moa_transpose(dtype, shape, A, perm, out, stream=None, check=True):
    """C ABI moa_transpose: output axis k is input axis perm[k]."""
    sa, _ka = _shape(shape)
    pm = (C.c_int * max(1, len(perm)))(*[int(p) for p in perm])
    st = lib().moa_transpose(_enum(DTYPES, dtype), len(shape), sa, pm, _ptr(A), _ptr(out), _stream(stream))
    if check:
        _check(st, "moa_transpose")
    return st


def moa_outer(op, dtype, shapeA, A, shapeB, B, out, out_dtype, stream=None, check=True):
    """C ABI moa_outer: Eq. (1) C = A op B, rho C = rho A ++ rho B."""
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    st = lib().moa_outer(_enum(OPS, op), _enum(DTYPES, dtype), len(shapeA), sa, _ptr(A), len(shapeB), sb, _ptr(B),
                         _ptr(out), _enum(DTYPES, out_dtype), _stream(stream))
    if check:
        _check(st, "moa_outer")
    return st


def moa_inner_bf16x3_noalloc(shapeA, A, shapeB, B, out, stream=None, check=True):
    """C ABI moa_inner_bf16x3_noalloc: the FP32 split-BF16x3 inner product
    with its scratch in a fixed device buffer, for callers that must not
    allocate device memory (see include/moa.h)."""
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    st = lib().moa_inner_bf16x3_noalloc(len(shapeA), sa, _ptr(A), len(shapeB), sb, _ptr(B), _ptr(out),
                                        _stream(stream))
    if check:
        _check(st, "moa_inner_bf16x3_noalloc")
    return st


def moa_inner_shape(shapeA, shapeB):
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    rd = C.c_int(0)
    out = (C.c_int64 * 16)()
    _check(lib().moa_inner_shape(len(shapeA), sa, len(shapeB), sb, C.byref(rd), C.cast(out, _I64P)),
           "moa_inner_shape")
    return tuple(out[i] for i in range(rd.value))


def moa_outer_shape(shapeA, shapeB):
    sa, _ka = _shape(shapeA)
    sb, _kb = _shape(shapeB)
    rc = C.c_int(0)
    out = (C.c_int64 * 16)()
    _check(lib().moa_outer_shape(len(shapeA), sa, len(shapeB), sb, C.byref(rc), C.cast(out, _I64P)),
           "moa_outer_shape")
    return tuple(out[i] for i in range(rc.value))


def moa_status_string(st: int) -> str:
    return _status_text(st)


def moa_device_status(stream=None) -> int:
    return int(lib().moa_device_status(_stream(stream)))


def moa_selftest_wait_timeout(limit_us: int, stream=None) -> int:
    return int(lib().moa_selftest_wait_timeout(int(limit_us), _stream(stream)))


def moa_release_workspace() -> int:
    return int(lib().moa_release_workspace())


def moa_version() -> int:
    return int(lib().moa_version())


def make_problems(specs):
    """Build a ctypes array of MoaProblem from dicts with keys kind ("inner" |
    "outer"), reduce, combine, dtype, form, out_dtype, shapeA, shapeB, A, B,
    out (tensors or device addresses).  Returns (array, keep-alive list)."""
    arr = (MoaProblem * len(specs))()
    keep = []
    for i, sp in enumerate(specs):
        sa, ka = _shape(sp["shapeA"])
        sb, kb = _shape(sp["shapeB"])
        keep += [ka, kb]
        q = arr[i]
        q.kind = 0 if sp["kind"] == "inner" else 1
        q.reduce = _enum(OPS, sp.get("reduce", "add"))
        q.combine = _enum(OPS, sp.get("combine", "mul"))
        q.dtype = _enum(DTYPES, sp.get("dtype", "f32"))
        q.form = _enum(FORMS, sp.get("form", "native"))
        q.out_dtype = _enum(DTYPES, sp.get("out_dtype", "f32"))
        q.rankA, q.rankB = len(sp["shapeA"]), len(sp["shapeB"])
        q.shapeA, q.shapeB = sa, sb
        q.A, q.B, q.out = _ptr(sp["A"]), _ptr(sp["B"]), _ptr(sp["out"])
    return arr, keep


def moa_batch_plan_create(problems):
    """problems: a ctypes array of MoaProblem.  Returns the plan handle."""
    plan = C.c_void_p()
    bad = C.c_int(-1)
    st = lib().moa_batch_plan_create(len(problems), problems, C.byref(plan), C.byref(bad))
    if st != 0:
        raise MoaError(st, f"moa_batch_plan_create (problem {bad.value})")
    return plan


def moa_batch_execute(plan, stream=None):
    _check(lib().moa_batch_execute(plan, _stream(stream)), "moa_batch_execute")


def moa_batch_plan_info(plan):
    a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
    _check(lib().moa_batch_plan_info(plan, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "moa_batch_plan_info")
    return {"problems": a.value, "launches": b.value, "tiles": c.value, "work_flops": d.value}


def moa_batch_plan_destroy(plan):
    lib().moa_batch_plan_destroy(plan)


# ------------------------------------------------------------ conveniences
def _dtype_of(t):
    import torch
    table = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16",
             torch.int32: "i32"}
    if hasattr(torch, "float8_e4m3fn"):
        table[torch.float8_e4m3fn] = "fp8e4m3"
    return table[t.dtype]


def inner(A, B, reduce="add", combine="mul", form="native", out=None, out_dtype=None, stream=None):
    """Eq. (2) on torch CUDA tensors (rho A = A.shape, rho B = B.shape)."""
    import torch
    dt = _dtype_of(A)
    if out_dtype is None:
        out_dtype = "f32" if dt in ("bf16", "f16", "fp8e4m3") else dt
    shD = tuple(A.shape[:-1]) + tuple(B.shape[1:])
    if out is None:
        tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32}[out_dtype]
        out = torch.empty(shD, dtype=tdt, device=A.device)
    moa_inner(reduce, combine, dt, form, tuple(A.shape), A.contiguous(), tuple(B.shape), B.contiguous(), out,
              out_dtype, stream)
    return out


def outer(A, B, op="mul", out=None, out_dtype=None, stream=None):
    """Eq. (1) on torch CUDA tensors; rho C = rho A ++ rho B."""
    import torch
    dt = _dtype_of(A)
    out_dtype = out_dtype or dt
    shC = tuple(A.shape) + tuple(B.shape)
    if out is None:
        tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "i32": torch.int32}[out_dtype]
        out = torch.empty(shC, dtype=tdt, device=A.device)
    moa_outer(op, dt, tuple(A.shape), A.contiguous(), tuple(B.shape), B.contiguous(), out, out_dtype, stream)
    return out
