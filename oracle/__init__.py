"""Python access to the CPU oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU legs
of ``bench.py`` may import this package; the library under
``paper_0907_0792_gb300/`` never does.  The oracle shares no code with the
CUDA path.  ``build()`` compiles it with gcc (no FMA contraction, no fast
math) into ``oracle/_build/liboracle.so``.

Every function takes numpy arrays whose ``.shape`` is the MoA shape vector
(rho) and whose C-order ravel is the element vector.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "min": 4, "max": 5, "or": 6, "and": 7}
_ERR = {1: "rank", 2: "shape mismatch (rho A[-1] != rho B[0])", 3: "unsupported operator", 4: "output index"}


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than oracle.c."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
    return _lib


def _sh(x: np.ndarray):
    s = np.asarray(x.shape if isinstance(x, np.ndarray) else x, dtype=np.int64)
    return s.ctypes.data_as(C.POINTER(C.c_int64)), s


def _c(a, dtype):
    """C-contiguous copy that keeps rank 0 (np.ascontiguousarray would not)."""
    return np.array(a, dtype=dtype, order="C")


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(st):
    if st != 0:
        raise ValueError(f"oracle error: {_ERR.get(st, st)}")


def inner_shape(shape_a, shape_b):
    """rho D for Eq. (2): rho A without its last axis ++ rho B without its first."""
    sa = np.asarray(shape_a, dtype=np.int64)
    sb = np.asarray(shape_b, dtype=np.int64)
    rd = C.c_int(0)
    out = np.zeros(16, dtype=np.int64)
    _check(lib().oracle_inner_shape(len(sa), _p(sa), len(sb), _p(sb), C.byref(rd), _p(out)))
    return tuple(int(v) for v in out[: rd.value])


def outer_shape(shape_a, shape_b):
    """rho C for Eq. (1): rho A ++ rho B."""
    return tuple(shape_a) + tuple(shape_b)


def _outidx(n_total, idx):
    if idx is None:
        return n_total, None, None
    idx = np.ascontiguousarray(idx, dtype=np.int64).ravel()
    return idx.size, idx, _p(idx)


def inner_dot2(A, B, out_idx=None):
    """(+,*) inner product by Dot2 in FP64; returns (D, sum_p |A||B|).

    With ``out_idx`` (flat offsets into D) only those elements are computed
    and 1-D arrays are returned; otherwise arrays of shape rho D."""
    A = _c(A, dtype=np.float64)
    B = _c(B, dtype=np.float64)
    shD = inner_shape(A.shape, B.shape)
    n, idx, pidx = _outidx(int(np.prod(shD, dtype=np.int64)), out_idx)
    D = np.empty(n, dtype=np.float64)
    S = np.empty(n, dtype=np.float64)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_inner_dot2(A.ndim, sa, _p(A), B.ndim, sb, _p(B), C.c_int64(n), pidx, _p(D), _p(S)))
    if out_idx is None:
        return D.reshape(shD), S.reshape(shD)
    return D, S


def inner_f32(reduce: str, combine: str, A, B, out_idx=None):
    """reduce min or max, combine +, -, *, min or max, over FP32: the bit-exact definition."""
    A = _c(A, dtype=np.float32)
    B = _c(B, dtype=np.float32)
    shD = inner_shape(A.shape, B.shape)
    n, idx, pidx = _outidx(int(np.prod(shD, dtype=np.int64)), out_idx)
    D = np.empty(n, dtype=np.float32)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_inner_f32(OPS[reduce], OPS[combine], A.ndim, sa, _p(A), B.ndim, sb, _p(B), C.c_int64(n),
                                  pidx, _p(D)))
    return D.reshape(shD) if out_idx is None else D


def inner_i32(A, B, out_idx=None):
    """(+,*) over int32 with wraparound."""
    A = _c(A, dtype=np.int32)
    B = _c(B, dtype=np.int32)
    shD = inner_shape(A.shape, B.shape)
    n, idx, pidx = _outidx(int(np.prod(shD, dtype=np.int64)), out_idx)
    D = np.empty(n, dtype=np.int32)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_inner_i32(A.ndim, sa, _p(A), B.ndim, sb, _p(B), C.c_int64(n), pidx, _p(D)))
    return D.reshape(shD) if out_idx is None else D


def inner_bool(A, B, out_idx=None):
    """(or,and) over Booleans (unpacked bool arrays in, bool out)."""
    A = _c(A, dtype=np.uint8)
    B = _c(B, dtype=np.uint8)
    shD = inner_shape(A.shape, B.shape)
    n, idx, pidx = _outidx(int(np.prod(shD, dtype=np.int64)), out_idx)
    D = np.empty(n, dtype=np.uint8)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_inner_bool(A.ndim, sa, _p(A), B.ndim, sb, _p(B), C.c_int64(n), pidx, _p(D)))
    D = D.astype(bool)
    return D.reshape(shD) if out_idx is None else D


_OUT_KIND = {"f64": (0, np.float64), "f32": (1, np.float32), "bf16": (2, np.uint16)}


def move_axes(A, B, axis_a: int, axis_b: int):
    """The operands of a contraction over axis_a of A and axis_b of B in the
    form Eq. (2) contracts: axis_a moved last in A, axis_b moved first in B,
    the other axes keeping their order (numpy's moveaxis as the transpose).
    Any inner_* function then gives D with rho D = (rho A without axis_a) ++
    (rho B without axis_b)."""
    return np.ascontiguousarray(np.moveaxis(A, axis_a, -1)), np.ascontiguousarray(np.moveaxis(B, axis_b, 0))


def outer_f(op: str, A, B, out: str = "f64", out_idx=None):
    """Eq. (1) over floating operands given exactly as float64.

    out "f64": the op in binary64; "f32": correctly rounded to FP32; "bf16":
    the FP32 result rounded to bfloat16 (RNE), returned as uint16 bits."""
    A = _c(A, dtype=np.float64)
    B = _c(B, dtype=np.float64)
    shC = outer_shape(A.shape, B.shape)
    kind, dt = _OUT_KIND[out]
    n, idx, pidx = _outidx(int(np.prod(shC, dtype=np.int64)), out_idx)
    Cout = np.empty(n, dtype=dt)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_outer_f(OPS[op], A.ndim, sa, _p(A), B.ndim, sb, _p(B), kind, C.c_int64(n), pidx, _p(Cout)))
    return Cout.reshape(shC) if out_idx is None else Cout


def outer_i32(op: str, A, B, out_idx=None):
    A = _c(A, dtype=np.int32)
    B = _c(B, dtype=np.int32)
    shC = outer_shape(A.shape, B.shape)
    n, idx, pidx = _outidx(int(np.prod(shC, dtype=np.int64)), out_idx)
    Cout = np.empty(n, dtype=np.int32)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_outer_i32(OPS[op], A.ndim, sa, _p(A), B.ndim, sb, _p(B), C.c_int64(n), pidx, _p(Cout)))
    return Cout.reshape(shC) if out_idx is None else Cout


_ROW_KIND = {"f64": (0, np.float64), "f32": (1, np.float32), "i32": (2, np.int32), "bool": (3, np.uint8)}


def rowwise(kind: str, A, B, reduce: str = "add", combine: str = "mul", threads: int = 1):
    """The appendix-order loop (row i; l over the contraction; j along the
    row), with rows dealt cyclically to ``threads`` OpenMP threads.  Plain
    recursive summation; returns D with shape rho D."""
    k, dt = _ROW_KIND[kind]
    A = _c(A, dtype=dt)
    B = _c(B, dtype=dt)
    shD = inner_shape(A.shape, B.shape)
    D = np.empty(shD, dtype=dt)
    sa, _ka = _sh(A)
    sb, _kb = _sh(B)
    _check(lib().oracle_rowwise(k, OPS[reduce], OPS[combine], A.ndim, sa, _p(A), B.ndim, sb, _p(B), _p(D),
                                int(threads)))
    return D.astype(bool) if kind == "bool" else D


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def normalised_error(D, D_ref, abs_sum):
    """max |D - D_ref| / sum_p |A||B|; elements with a zero normaliser must match exactly."""
    D = np.asarray(D, dtype=np.float64).ravel()
    R = np.asarray(D_ref, dtype=np.float64).ravel()
    S = np.asarray(abs_sum, dtype=np.float64).ravel()
    zero = S == 0
    if np.any(D[zero] != R[zero]):
        return float("inf")
    if np.all(zero):
        return 0.0
    return float(np.max(np.abs(D[~zero] - R[~zero]) / S[~zero]))
