"""GPU parity of the pair-MMA (cta_group::2) kernels at tile edges: results
of just over one 256-row pair tile (the peer CTA holding 1..127 live rows),
column counts one past a 256- or 224-wide tile, contractions of 1, of one
past a k-block and of several exact chunks, for every form that runs on the
pair kernel (bf16 operands, BF16 and split-BF16x3 forms, FP8 block-scaled,
Ozaki).  Tolerances as in the per-form tests."""
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, bf16_dev, check_status, empty, to_dev

pytestmark = pytest.mark.gpu

BF16_SHAPES = [((129, 64), (64, 129)), ((257, 72), (72, 513)), ((300, 1), (1, 300)), ((260, 65), (65, 257)),
               ((513, 1030), (1030, 300))]


@pytest.mark.parametrize("shA,shB", BF16_SHAPES)
def test_pair_bf16_operands(shA, shB):
    import torch
    a_bits, a = synth.to_bf16(synth.uniform(61, 0, shA, -1, 1))
    b_bits, b = synth.to_bf16(synth.uniform(61, 1, shB, -1, 1))
    D = empty((shA[0], shB[1]), torch.float32)
    moa.moa_inner("add", "mul", "bf16", "native", shA, bf16_dev(a_bits), shB, bf16_dev(b_bits), D, "f32")
    assert_norm_err(D.cpu().numpy(), a, b, 2e-6)
    check_status()


@pytest.mark.parametrize("form,tol", [("bf16x3", 2e-6), ("bf16", 1e-2)])
@pytest.mark.parametrize("shA,shB", [((257, 100), (100, 300)), ((300, 1029), (1029, 257))])
def test_pair_f32_forms(form, tol, shA, shB):
    import torch
    A = synth.to_f32(synth.log_uniform_signed(62, 0, shA))
    B = synth.to_f32(synth.log_uniform_signed(62, 1, shB))
    D = empty((shA[0], shB[1]), torch.float32)
    moa.moa_inner("add", "mul", "f32", form, shA, to_dev(A), shB, to_dev(B), D, "f32")
    assert_norm_err(D.cpu().numpy(), A, B, tol)
    check_status()


@pytest.mark.parametrize("shA,shB", [((129, 300), (300, 225)), ((300, 1024), (1024, 449)), ((257, 129), (129, 224)),
                                     ((260, 2000), (2000, 500))])
def test_pair_fp8(shA, shB):
    """Block-scaled FP8 on 256 x 224 tiles: columns one past a tile, K not a
    multiple of the 128-deep scale block (uniform data, K >= 256 -> 6e-2;
    K = 129 -> the two-rounding bound 0.129)."""
    import torch
    A = synth.to_f32(synth.uniform(63, 0, shA, -1, 1))
    B = synth.to_f32(synth.uniform(63, 1, shB, -1, 1))
    D = empty((shA[0], shB[1]), torch.float32)
    moa.moa_inner("add", "mul", "f32", "fp8_t128", shA, to_dev(A), shB, to_dev(B), D, "f32")
    tol = 6e-2 if shA[-1] >= 256 else 2 * 2.0 ** -4 + 2.0 ** -8
    assert_norm_err(D.cpu().numpy(), A, B, tol)
    check_status()


@pytest.mark.parametrize("shA,shB", [((129, 64), (64, 129)), ((300, 3000), (3000, 260)), ((257, 1), (1, 257))])
def test_pair_ozaki(shA, shB):
    """Ozaki on the pair kernel: one row past a pair tile, a contraction of
    three exact chunks (S = 8), and a contraction of 1."""
    import torch
    A = synth.log_uniform_signed(64, 0, shA)
    B = synth.log_uniform_signed(64, 1, shB)
    D = empty((shA[0], shB[1]), torch.float64)
    moa.moa_inner("add", "mul", "f64", "ozaki", shA, to_dev(A), shB, to_dev(B), D, "f64")
    assert_norm_err(D.cpu().numpy(), A, B, 1e-12)
    check_status()
