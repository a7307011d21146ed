"""GPU parity of the generalized outer product (Eq. 1) against the oracle:
bit-exact for every op and type, at small ragged sizes (whole result) and at
the memory-bound 128x64x32 (x) 32x64 workload (sampled elements)."""
import numpy as np
import pytest

import oracle
import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import bf16_dev, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

OPS = ["mul", "add", "sub", "div", "min", "max"]


def _run(op, dt, A, B, out_dt, shA, shB):
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "i32": torch.int32}[out_dt]
    out = empty(tuple(shA) + tuple(shB), tdt)
    moa.moa_outer(op, dt, shA, A, shB, B, out, out_dt)
    return out


def _host(t):
    import torch
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def test_plain_method_outer_f64():
    """Rank-4 A <16,12,8,64> (x) B <4,5>, FP64, the whole result."""
    A, _ = synth.rank4x3_f64()
    B = synth.outer_second_f64()
    C = _run("mul", "f64", to_dev(A), to_dev(B), "f64", A.shape, B.shape)
    assert C.shape == (16, 12, 8, 64, 4, 5)
    assert np.array_equal(_host(C), oracle.outer_f("mul", A, B))
    check_status()


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("shA,shB", [((5, 7, 3), (3, 21)), ((2, 33), (64,)), ((1,), (1000,)), ((300,), (8, 4))])
def test_small_ragged_f32_bf16(op, shA, shB):
    A, B = synth.outer_inputs(op, "f32", shape_a=shA, shape_b=shB)
    C = _run(op, "f32", to_dev(A), to_dev(B), "f32", shA, shB)
    assert np.array_equal(_host(C), oracle.outer_f(op, A, B, out="f32"))
    (ab, av), (bb, bv) = synth.outer_inputs(op, "bf16", shape_a=shA, shape_b=shB)
    Cb = _run(op, "bf16", bf16_dev(ab), bf16_dev(bb), "bf16", shA, shB)
    assert np.array_equal(_host(Cb), oracle.outer_f(op, av, bv, out="bf16"))
    Cf = _run(op, "bf16", bf16_dev(ab), bf16_dev(bb), "f32", shA, shB)
    assert np.array_equal(_host(Cf), oracle.outer_f(op, av, bv, out="f32"))
    check_status()


def _bf16_values(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _same_bf16(got, want):
    """Equal bit patterns, except that any NaN matches any NaN."""
    nan_w = (want & 0x7F80) == 0x7F80
    nan_w &= (want & 0x7F) != 0
    nan_g = ((got & 0x7F80) == 0x7F80) & ((got & 0x7F) != 0)
    return np.array_equal(nan_g, nan_w) and np.array_equal(got[~nan_w], want[~nan_w])


def test_bf16_division_every_divisor_and_dividend():
    """bf16 / bf16 -> bf16 (reciprocal multiply where it is exact, division
    elsewhere) against the FP32 quotient rounded once to bf16: every one of
    the 65536 bit patterns as divisor, and as dividend, against 48 values
    that cover zeros, subnormals, normals of all sizes, the largest
    finite, infinities and NaN."""
    every = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    pick = np.array([0x0000, 0x8000, 0x0001, 0x8001, 0x007F, 0x0080, 0x8080, 0x00FF, 0x3F80, 0xBF80, 0x3F81, 0x4049,
                     0xC0A0, 0x7F7F, 0xFF7F, 0x7F80, 0xFF80, 0x7FC0, 0x0100, 0x3C00, 0x4300, 0x5F00, 0x7E80, 0x0200,
                     0x3E4D, 0x3DCD, 0xBDCD, 0x41FF, 0x42C8, 0x7F00, 0x00A0, 0x8055, 0x1234, 0x9234, 0x2F00, 0x6F00,
                     0x3F00, 0x3FFF, 0x407F, 0xC0FF, 0x4B7F, 0x0C00, 0x7300, 0x0080 | 0x8000, 0x3F7F, 0x7F7E, 0x0040,
                     0x4F7F], dtype=np.uint16)
    for a_bits, b_bits in ((pick, every), (every, pick)):
        C = _run("div", "bf16", bf16_dev(a_bits), bf16_dev(b_bits), "bf16", a_bits.shape, b_bits.shape)
        want = oracle.outer_f("div", _bf16_values(a_bits), _bf16_values(b_bits), out="bf16")
        assert _same_bf16(_host(C), want)
    check_status()


@pytest.mark.parametrize("op", ["mul", "add", "sub"])
def test_small_i32(op):
    A, B = synth.outer_inputs(op, "i32", shape_a=(7, 9), shape_b=(5, 13))
    C = _run(op, "i32", to_dev(A), to_dev(B), "i32", A.shape, B.shape)
    assert np.array_equal(_host(C), oracle.outer_i32(op, A, B))
    big = np.array([2 ** 31 - 1, -(2 ** 31), 65537, -3], dtype=np.int32)
    C = _run(op, "i32", to_dev(big), to_dev(big), "i32", big.shape, big.shape)
    assert np.array_equal(_host(C), oracle.outer_i32(op, big, big))


def test_rank0_and_empty():
    import torch
    s = np.array(2.5, dtype=np.float32)
    B = synth.to_f32(synth.uniform(3, 3, (17,), -1, 1))
    C = _run("mul", "f32", to_dev(s), to_dev(B), "f32", (), (17,))
    assert np.array_equal(_host(C), oracle.outer_f("mul", s, B, out="f32"))
    out = empty((0, 17), torch.float32)
    moa.moa_outer("mul", "f32", (0,), 0, (17,), to_dev(B), out, "f32")
    check_status()


@pytest.mark.parametrize("op,dt", [("mul", "f32"), ("add", "f32"), ("sub", "f32"), ("div", "f32"),
                                   ("mul", "bf16"), ("div", "bf16"), ("mul", "i32")])
def test_full_size_sampled(op, dt):
    """A <128,64,32> (x) B <32,64>: 536,870,912 outputs; 200,000 sampled."""
    import torch
    shA, shB = synth.C4_SHAPE_A, synth.C4_SHAPE_B
    if dt == "i32":
        A, B = synth.outer_inputs(op, "i32")
        C = _run(op, "i32", to_dev(A), to_dev(B), "i32", shA, shB)
        idx = sample_idx(C.numel(), 200000)
        got = C.view(-1)[torch.from_numpy(idx).to(C.device)].cpu().numpy()
        assert np.array_equal(got, oracle.outer_i32(op, A, B, out_idx=idx))
        slab = C.view(-1)[: 8 * B.size].cpu().numpy()
        want = oracle.outer_i32(op, A.ravel()[:8], B.ravel())
    elif dt == "f32":
        A, B = synth.outer_inputs(op, "f32")
        C = _run(op, "f32", to_dev(A), to_dev(B), "f32", shA, shB)
        idx = sample_idx(C.numel(), 200000)
        got = C.view(-1)[torch.from_numpy(idx).to(C.device)].cpu().numpy()
        assert np.array_equal(got, oracle.outer_f(op, A, B, out="f32", out_idx=idx))
        slab = C.view(-1)[: 8 * B.size].cpu().numpy()
        want = oracle.outer_f(op, A.ravel()[:8], B.ravel(), out="f32")
    else:
        (ab, av), (bb, bv) = synth.outer_inputs(op, "bf16")
        C = _run(op, "bf16", bf16_dev(ab), bf16_dev(bb), "bf16", shA, shB)
        idx = sample_idx(C.numel(), 200000)
        got = C.view(torch.int16).view(-1)[torch.from_numpy(idx).to(C.device)].cpu().numpy().view(np.uint16)
        assert np.array_equal(got, oracle.outer_f(op, av, bv, out="bf16", out_idx=idx))
        slab = C.view(torch.int16).view(-1)[: 8 * bv.size].cpu().numpy().view(np.uint16)
        want = oracle.outer_f(op, av.ravel()[:8], bv.ravel(), out="bf16")
    # the first eight rows of the flattened result whole: row i is A[i] op B
    assert np.array_equal(slab.ravel(), np.asarray(want).ravel())
    check_status()
    del C
    torch.cuda.empty_cache()
