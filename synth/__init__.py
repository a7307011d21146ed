"""Seeded synthetic inputs for the MoA generalized inner / outer product.

This module is shared by the CPU oracle (``oracle/``), the tests and
``bench.py``.  It holds no arithmetic of the method itself: it only draws
numbers, rounds them to the storage type an operand is given in, and packs
Boolean arrays into the bit layout of the C ABI.

Generator
---------
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) is counter based: its i-th output is
``mix(key + (i + 1) * GAMMA)``.  That lets numpy draw any slice of a stream
in one vectorised pass, and gives the same bytes on x86-64 and aarch64
(integer arithmetic plus IEEE float ops only, no libm transcendental).
Each (seed, stream) pair selects an independent key.

Workload recipes follow the five benchmark configurations of the method's
inner product (Eq. 2) and outer product (Eq. 1); the shapes, value
distributions and structure are stated beside each function.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = _mix(np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(int(stream) & 0xFFFFFFFF) + np.uint64(1))
        return np.uint64(_mix(k ^ np.uint64(0xD1B54A32D192ED03)))


def u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream (seed, stream)."""
    key = _key(seed, stream)
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + idx * GAMMA)


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each output."""
    return (u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, stream: int, shape, lo: float, hi: float) -> np.ndarray:
    n = int(np.prod(shape, dtype=np.int64))
    return (lo + (hi - lo) * uniform01(seed, stream, n)).reshape(shape)


def uniform_at(seed: int, stream: int, idx, lo: float, hi: float) -> np.ndarray:
    """The elements of ``uniform(seed, stream, shape, lo, hi)`` at the given
    flat (row-major) positions, without drawing the rest of the stream."""
    key = _key(seed, stream)
    i = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        z = _mix(key + i * GAMMA)
    return lo + (hi - lo) * ((z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53))


def u64_at(seed: int, stream: int, idx) -> np.ndarray:
    """The elements of ``u64(seed, stream, n)`` at the given positions."""
    key = _key(seed, stream)
    i = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        return _mix(key + i * GAMMA)


def _i64(u: int) -> int:
    """A 64-bit pattern as the signed integer torch stores it as."""
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


def device_uniform(seed: int, stream: int, shape, lo: float, hi: float, device, dtype=None, chunk: int = 1 << 26):
    """``uniform(seed, stream, shape, lo, hi)`` drawn directly in device memory
    with torch integer ops (int64 arithmetic wraps modulo 2^64; logical
    shifts by masking), then cast to ``dtype`` (RNE, as ``to_f32``).  For
    operands too large to draw on the host; the values are identical."""
    import torch
    dtype = dtype or torch.float64
    n = int(np.prod(shape, dtype=np.int64))
    out = torch.empty(n, dtype=dtype, device=device)
    key = _i64(int(_key(seed, stream)))
    g, m1, m2 = _i64(int(GAMMA)), _i64(int(_M1)), _i64(int(_M2))

    def lsr(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    for o in range(0, n, chunk):
        c = min(chunk, n - o)
        z = torch.arange(o + 1, o + c + 1, dtype=torch.int64, device=device) * g + key
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        u = lsr(z, 11).to(torch.float64) * (2.0 ** -53)
        out[o:o + c] = (lo + (hi - lo) * u).to(dtype)
        del z, u
    return out.view(*shape)


def int_uniform(seed: int, stream: int, shape, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) as int32; modulo bias < 2^-40."""
    n = int(np.prod(shape, dtype=np.int64))
    span = np.uint64(hi - lo + 1)
    v = (u64(seed, stream, n) % span).astype(np.int64) + lo
    return v.astype(np.int32).reshape(shape)


def bernoulli(seed: int, stream: int, shape, p: float) -> np.ndarray:
    return uniform01(seed, stream, int(np.prod(shape, dtype=np.int64))).reshape(shape) < p


def _log_uniform_from(r: np.ndarray, lo_exp2: int, hi_exp2: int) -> np.ndarray:
    e = (r % np.uint64(hi_exp2 - lo_exp2)).astype(np.int64) + lo_exp2
    f = 1.0 + ((r >> np.uint64(11)) & np.uint64((1 << 52) - 1)).astype(np.float64) * (2.0 ** -52)
    s = np.where((r >> np.uint64(10)) & np.uint64(1), -1.0, 1.0)
    return s * np.ldexp(f, e)


def log_uniform_at(seed: int, stream: int, idx, lo_exp2: int = -13, hi_exp2: int = 13) -> np.ndarray:
    """The elements of ``log_uniform_signed`` at the given flat positions."""
    return _log_uniform_from(u64_at(seed, stream, idx), lo_exp2, hi_exp2)


def log_uniform_signed(seed: int, stream: int, shape, lo_exp2: int = -13, hi_exp2: int = 13) -> np.ndarray:
    """Random sign times a magnitude spread evenly over octaves.

    Stand-in for ``sign * 10**U(-4, 4)``: the binary exponent is uniform over
    the integers in [lo_exp2, hi_exp2) and the significand uniform in [1, 2),
    so magnitudes cover 2^-13 .. 2^13 (1.2e-4 .. 8.2e3), every octave equally
    likely.  Built with ``ldexp`` only, so it is bit-identical across hosts.
    """
    n = int(np.prod(shape, dtype=np.int64))
    return _log_uniform_from(u64(seed, stream, n), lo_exp2, hi_exp2).reshape(shape)


# ---------------------------------------------------------------- rounding
def to_f32(x: np.ndarray) -> np.ndarray:
    """Round to FP32 (IEEE round-to-nearest-even, numpy's cast)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """FP32 -> bfloat16 bit patterns, round-to-nearest-even (finite inputs and inf)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = (u & np.uint64(0x7FFFFFFF)) > np.uint64(0x7F800000)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    r = np.where(nan, (u >> np.uint64(16)) | np.uint64(0x40), r)
    return r.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def to_bf16(x: np.ndarray):
    """Round to bfloat16 via FP32 (f64 -> f32 RNE -> bf16 RNE).

    Returns (bits as uint16, the exact values as float64)."""
    b = f32_to_bf16_bits(to_f32(x))
    return b, bf16_bits_to_f64(b)


def to_f16(x: np.ndarray):
    """Round to IEEE binary16 (RNE, numpy's conversion from float64).

    Returns (bits as uint16, the exact values as float64)."""
    h = np.asarray(x, dtype=np.float64).astype(np.float16)
    return h.view(np.uint16), h.astype(np.float64)


def e4m3_decode_table() -> np.ndarray:
    """The value of every FP8 E4M3 code (OCP 8-bit floating point, E4M3):
    bit 7 sign, bits 3-6 exponent with bias 7, bits 0-2 mantissa; exponent
    field 0 encodes subnormals m/8 * 2^-6; codes 0x7F and 0xFF are NaN; no
    infinities (the all-ones exponent with mantissa < 7 is a normal number)."""
    out = np.empty(256, dtype=np.float64)
    for c in range(256):
        sgn = -1.0 if c & 0x80 else 1.0
        e, m = (c >> 3) & 0xF, c & 0x7
        if e == 0xF and m == 0x7:
            out[c] = np.nan
        elif e == 0:
            out[c] = sgn * (m / 8.0) * 2.0 ** -6
        else:
            out[c] = sgn * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return out


def e4m3_codes(seed: int, stream: int, shape, max_exp: int = 15):
    """FP8 E4M3 operands as stored: codes drawn uniformly over the finite
    codes whose exponent field is at most max_exp (NaN never drawn).

    Returns (codes as uint8, the exact values as float64)."""
    table = e4m3_decode_table()
    finite = np.array([c for c in range(256) if not np.isnan(table[c]) and ((c >> 3) & 0xF) <= max_exp],
                      dtype=np.uint8)
    n = int(np.prod(shape, dtype=np.int64))
    codes = finite[(u64(seed, stream, n) % np.uint64(len(finite))).astype(np.int64)].reshape(shape)
    return codes, table[codes]


# ---------------------------------------------------------------- bit packing
def pack_bits(x: np.ndarray) -> np.ndarray:
    """Row-major ravel packed as a bit stream: element e -> word e//32, bit e%32
    (LSB first); the last word is zero-padded.  Matches the MOA_B1_U32 layout."""
    flat = np.ascontiguousarray(x, dtype=bool).ravel()
    nw = (flat.size + 31) // 32
    pad = np.zeros(nw * 32, dtype=np.uint64)
    pad[: flat.size] = flat
    w = pad.reshape(nw, 32) << np.arange(32, dtype=np.uint64)
    return w.sum(axis=1).astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint32).astype(np.uint64)
    bits = (w[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return bits.ravel()[:n].astype(bool)


# ---------------------------------------------------------------- workloads
# Inner product (Eq. 2), FP64, rank 4 x rank 3.
C1_SHAPE_A = (16, 12, 8, 64)
C1_SHAPE_B = (64, 24, 20)
C1_SHAPE_B_OUTER = (4, 5)
# Semirings, rank 3 x rank 3.
C3_SHAPE_A = (32, 128, 512)
C3_SHAPE_B = (512, 64, 64)
# Memory-bound outer product (Eq. 1): 128*64*32 x 32*64 = 536,870,912 outputs.
C4_SHAPE_A = (128, 64, 32)
C4_SHAPE_B = (32, 64)
C2_SIZES = (256, 512, 1024, 2048, 4096, 8192)
# the method's own measurement (Sec. IV): an m x 128 array times a 128 x n
# array, m = 1..4, n = 2^10 .. 2^26; values unstated there, U(-1, 1) here
SKINNY_K = 128
SKINNY_M = (1, 2, 3, 4)
SKINNY_N_MAX = 1 << 26
SKINNY_SEED = 6


def rank4x3_f64(seed: int = 1, shape_a=C1_SHAPE_A, shape_b=C1_SHAPE_B):
    """Plain-method inner product inputs: U(-1, 1) FP64, A <16,12,8,64>, B <64,24,20>."""
    return uniform(seed, 0, shape_a, -1.0, 1.0), uniform(seed, 1, shape_b, -1.0, 1.0)


def outer_second_f64(seed: int = 1, shape=C1_SHAPE_B_OUTER):
    """Second outer-product operand for the plain method: U(-1, 1), shape <4,5>."""
    return uniform(seed, 2, shape, -1.0, 1.0)


def square(n: int, dist: str = "uniform", seed: int = 2, m: int | None = None, k: int | None = None):
    """Square (or m x k . k x n) matrix-multiply operands as FP64.

    dist = "uniform": U(-1, 1); dist = "loguniform": random sign times an
    octave-uniform magnitude over 2^-13 .. 2^13 (see ``log_uniform_signed``)."""
    m = n if m is None else m
    k = n if k is None else k
    tag = 0 if dist == "uniform" else 10
    if dist == "uniform":
        return uniform(seed, tag, (m, k), -1.0, 1.0), uniform(seed, tag + 1, (k, n), -1.0, 1.0)
    if dist == "loguniform":
        return log_uniform_signed(seed, tag, (m, k)), log_uniform_signed(seed, tag + 1, (k, n))
    raise ValueError(dist)


SWEEP_N = (256, 512, 1024, 2048, 4096, 8192)


def square_leading(n: int, dist: str = "uniform", n_full: int = 8192, seed: int = 2):
    """The leading n x n blocks of the operands ``square(n_full, dist)``,
    drawn positionally (the square sweep's smaller sizes are sub-blocks of
    its largest case; n = n_full gives ``square(n_full, dist)`` itself)."""
    if n == n_full:
        return square(n_full, dist, seed)
    idx = (np.arange(n, dtype=np.int64)[:, None] * n_full + np.arange(n, dtype=np.int64)[None, :]).reshape(-1)
    tag = 0 if dist == "uniform" else 10
    if dist == "uniform":
        A, B = uniform_at(seed, tag, idx, -1.0, 1.0), uniform_at(seed, tag + 1, idx, -1.0, 1.0)
    elif dist == "loguniform":
        A, B = log_uniform_at(seed, tag, idx), log_uniform_at(seed, tag + 1, idx)
    else:
        raise ValueError(dist)
    return A.reshape(n, n), B.reshape(n, n)


def skinny_shapes(m: int, n: int, k: int = SKINNY_K):
    return (m, k), (k, n)


def skinny(m: int, n: int, k: int = SKINNY_K, seed: int = SKINNY_SEED):
    """A (m x k) and B (k x n), U(-1, 1) FP64: streams 0 and 1 of the seed."""
    sa, sb = skinny_shapes(m, n, k)
    return uniform(seed, 0, sa, -1.0, 1.0), uniform(seed, 1, sb, -1.0, 1.0)


def skinny_columns(cols, n: int, k: int = SKINNY_K, seed: int = SKINNY_SEED) -> np.ndarray:
    """Columns ``cols`` of the k x n operand B of ``skinny`` (k x len(cols))."""
    cols = np.asarray(cols, dtype=np.int64)
    idx = np.arange(k, dtype=np.int64)[:, None] * n + cols[None, :]
    return uniform_at(seed, 1, idx.reshape(-1), -1.0, 1.0).reshape(k, len(cols))


def semiring_inputs(kind: str, seed: int = 3, shape_a=C3_SHAPE_A, shape_b=C3_SHAPE_B):
    """Operands of the semiring workloads.

    kind: "tropical" ((min,+) and (max,+)): U(0, 100) FP32 with 5% +inf;
          "tropical_finite": U(0, 100) FP32, no inf;
          "maxmul": U(0, 1) FP32;
          "int32": integers uniform in [-128, 127];
          "bool": Bernoulli(0.05) (returned unpacked, as bool arrays).
    """
    if kind == "tropical":
        a = to_f32(uniform(seed, 20, shape_a, 0.0, 100.0))
        b = to_f32(uniform(seed, 21, shape_b, 0.0, 100.0))
        a[bernoulli(seed, 22, shape_a, 0.05)] = np.inf
        b[bernoulli(seed, 23, shape_b, 0.05)] = np.inf
        return a, b
    if kind == "tropical_finite":
        return to_f32(uniform(seed, 24, shape_a, 0.0, 100.0)), to_f32(uniform(seed, 25, shape_b, 0.0, 100.0))
    if kind == "maxmul":
        return to_f32(uniform(seed, 26, shape_a, 0.0, 1.0)), to_f32(uniform(seed, 27, shape_b, 0.0, 1.0))
    if kind == "int32":
        return int_uniform(seed, 28, shape_a, -128, 127), int_uniform(seed, 29, shape_b, -128, 127)
    if kind == "bool":
        return bernoulli(seed, 30, shape_a, 0.05), bernoulli(seed, 31, shape_b, 0.05)
    raise ValueError(kind)


def outer_inputs(op: str, dtype: str, seed: int = 4, shape_a=C4_SHAPE_A, shape_b=C4_SHAPE_B):
    """Outer-product operands: U(-1, 1); for "/" the divisor is U(-1, 1)
    conditioned on |b| >= 0.1 (drawn directly as sign * U(0.1, 1)).
    dtype "f32" -> float32 arrays; "bf16" -> (uint16 bits, float64 values)
    pairs; "i32" -> integers uniform in [-1000, 1000]; "f64" -> float64."""
    if dtype == "i32":
        return int_uniform(seed, 40, shape_a, -1000, 1000), int_uniform(seed, 41, shape_b, -1000, 1000)
    a = uniform(seed, 42, shape_a, -1.0, 1.0)
    if op == "div":
        mag = uniform(seed, 43, shape_b, 0.1, 1.0)
        sgn = np.where(bernoulli(seed, 44, shape_b, 0.5), -1.0, 1.0)
        b = sgn * mag
    else:
        b = uniform(seed, 43, shape_b, -1.0, 1.0)
    if dtype == "f64":
        return a, b
    if dtype == "f32":
        return to_f32(a), to_f32(b)
    if dtype == "bf16":
        return to_bf16(a), to_bf16(b)
    raise ValueError(dtype)


# ---------------------------------------------------------------- batched workload
def _octave_int(u, lo_exp2: int, octaves: int) -> np.ndarray:
    """Integers spread evenly over octaves: 2^(lo + k) * (1 + f) with k uniform in
    [0, octaves) and f from the fractional part of the draw, rounded; an
    exp()-free stand-in for round(2^U(lo, lo + octaves))."""
    x = np.asarray(u, dtype=np.float64) * octaves
    k = np.floor(x)
    f = x - k
    return np.rint(np.ldexp(1.0 + f, (k + lo_exp2).astype(np.int64))).astype(np.int64)


def _split_axes(total: int, rank: int, draws) -> list:
    """Factor `total` into `rank` axes by successive random divisors."""
    axes = []
    rem = int(total)
    for r in range(rank - 1):
        divs = [d for d in range(1, rem + 1) if rem % d == 0]
        d = divs[min(len(divs) - 1, int(draws[r] * len(divs)))]
        axes.append(d)
        rem //= d
    axes.append(rem)
    return axes


def batched_problems(count: int = 10000, seed: int = 5, mn_octaves: int = 11, p_lo: int = 3, p_octaves: int = 6):
    """The uneven batch: `count` problems, ranks 1..5 per operand, contraction
    length p octave-uniform in [8, 512], flattened M and N octave-uniform in
    [1, 2048]; 70% (+,*) split-BF16x3 FP32, 20% (min,+) FP32, 10% outer
    product (*) FP32.  A rank-1 left operand of an inner product forces M = 1.

    Returns a list of dicts with keys kind ("bf16x3" | "minplus" | "outer"),
    shapeA, shapeB, M, K, N."""
    u = uniform01(seed, 50, count * 6).reshape(count, 6)
    ax = uniform01(seed, 51, count * 8).reshape(count, 8)
    probs = []
    for i in range(count):
        t = u[i, 0]
        kind = "bf16x3" if t < 0.7 else ("minplus" if t < 0.9 else "outer")
        ra = 1 + int(u[i, 1] * 5)
        rb = 1 + int(u[i, 2] * 5)
        p = int(_octave_int(u[i, 3], p_lo, p_octaves))
        M = int(np.clip(_octave_int(u[i, 4], 0, mn_octaves), 1, 2 ** mn_octaves))
        N = int(np.clip(_octave_int(u[i, 5], 0, mn_octaves), 1, 2 ** mn_octaves))
        p = int(np.clip(p, 2 ** p_lo, 2 ** (p_lo + p_octaves)))
        if kind == "outer":
            sa = _split_axes(M, ra, ax[i, :4])
            sb = _split_axes(N, rb, ax[i, 4:])
            probs.append({"kind": kind, "shapeA": tuple(sa), "shapeB": tuple(sb), "M": M, "K": 0, "N": N})
        else:
            if ra == 1:
                M = 1
            sa = (_split_axes(M, ra - 1, ax[i, :4]) if ra > 1 else []) + [p]
            sb = [p] + (_split_axes(N, rb - 1, ax[i, 4:]) if rb > 1 else [])
            if rb == 1:
                N = 1
            probs.append({"kind": kind, "shapeA": tuple(sa), "shapeB": tuple(sb), "M": M, "K": p, "N": N})
    return probs


def batched_inputs(probs, seed: int = 5):
    """Element pools for a batch: every operand is a slice of one FP32 pool
    (element e of the pool is U(-1,1) draw e for bf16x3 and outer problems,
    and U(0,100) draw e with a 5% chance of +inf for (min,+) problems).
    Returns (pool, offsets_A, offsets_B, out_offsets, out_total); offsets are
    in elements, 4-aligned."""
    sizes_a = [int(np.prod(p["shapeA"])) for p in probs]
    sizes_b = [int(np.prod(p["shapeB"])) for p in probs]
    offs_a, offs_b, offs_d = [], [], []
    pos = 0
    for sa, sb in zip(sizes_a, sizes_b):
        pos = (pos + 3) // 4 * 4
        offs_a.append(pos)
        pos += sa
        pos = (pos + 3) // 4 * 4
        offs_b.append(pos)
        pos += sb
    total = pos
    pool = np.empty(total, dtype=np.float32)
    chunk = 1 << 24
    for s0 in range(0, total, chunk):
        n = min(chunk, total - s0)
        pool[s0:s0 + n] = (-1.0 + 2.0 * uniform01(seed, 52, n, s0)).astype(np.float32)
    for p, oa, ob, sa, sb in zip(probs, offs_a, offs_b, sizes_a, sizes_b):
        if p["kind"] != "minplus":
            continue
        for o, n in ((oa, sa), (ob, sb)):
            v = (100.0 * uniform01(seed, 53, n, o)).astype(np.float32)
            v[uniform01(seed, 54, n, o) < 0.05] = np.inf
            pool[o:o + n] = v
    dpos = 0
    for p in probs:
        dpos = (dpos + 3) // 4 * 4
        offs_d.append(dpos)
        dpos += p["M"] * p["N"]
    return pool, offs_a, offs_b, offs_d, dpos
