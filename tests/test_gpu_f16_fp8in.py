"""GPU parity of the (+,*) inner product (Eq. 2, matrix multiply as its
special case, Sec. I) on fp16 and FP8 E4M3 operands: fp16 or e4m3 operands
as given (tensor cores, one FP32 accumulator over the whole contraction),
and the FP16 form of FP32 operands (rounded to fp16, then the same kernels).

Bars (normalised error against the oracle's Dot2 of the operands as the
form receives them): operands as given max(2e-6, (K/16) 2^-23) (products
are exact in FP32; the accumulator is truncated at most once per 16-deep
MMA step); FP16 form 2e-3 (each product carries at most two fp16
roundings, 2u + u^2 with u = 2^-11, plus the accumulation)."""
import numpy as np
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

# ragged tiles (more and fewer than 128 rows / 256 columns, tails), contractions not a multiple of 8 or 16
SHAPES = [((300, 136), (136, 200)), ((2, 64, 72), (72, 5, 80)), ((129, 8), (8, 257)), ((1, 64), (64, 8)),
          ((520, 1000), (1000, 700)), ((37, 61), (61, 45)), ((130, 13), (13, 131)), ((260, 300), (300, 140))]


def _acc_tol(K):
    return max(2e-6, (K / 16) * 2.0 ** -23)


def _dev_bits(bits, torch_dtype):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(bits).view(np.int16 if bits.dtype == np.uint16 else np.uint8))
    return t.view(torch_dtype).to("cuda:0")


@pytest.mark.parametrize("shA,shB", SHAPES)
def test_f16_operands_native(shA, shB):
    import torch
    (ab, a), (bb, b) = synth.to_f16(synth.uniform(71, 0, shA, -1, 1)), synth.to_f16(synth.uniform(71, 1, shB, -1, 1))
    D = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner("add", "mul", "f16", "native", shA, _dev_bits(ab, torch.float16), shB, _dev_bits(bb, torch.float16), D,
                  "f32")
    assert_norm_err(D.cpu().numpy(), a, b, _acc_tol(shA[-1]))
    check_status()


@pytest.mark.parametrize("shA,shB", SHAPES)
@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
def test_f16_form(shA, shB, dist):
    import torch
    if dist == "uniform":
        A, B = synth.to_f32(synth.uniform(72, 0, shA, -1, 1)), synth.to_f32(synth.uniform(72, 1, shB, -1, 1))
    else:
        A, B = synth.to_f32(synth.log_uniform_signed(72, 0, shA)), synth.to_f32(synth.log_uniform_signed(72, 1, shB))
    D = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner("add", "mul", "f32", "f16", shA, to_dev(A), shB, to_dev(B), D, "f32")
    assert_norm_err(D.cpu().numpy(), A, B, 2e-3)
    check_status()


def test_f16_form_holds_large_magnitudes():
    """Magnitudes beyond fp16's largest finite value are held at 65504: the
    result stays finite (the form's accuracy statement covers fp16's range)."""
    import torch
    A = synth.to_f32(synth.uniform(73, 0, (200, 64), -1, 1))
    A[:, 0] = 1e6
    B = synth.to_f32(synth.uniform(73, 1, (64, 300), -1, 1))
    D = empty((200, 300), torch.float32)
    moa.moa_inner("add", "mul", "f32", "f16", (200, 64), to_dev(A), (64, 300), to_dev(B), D, "f32")
    assert np.isfinite(D.cpu().numpy()).all()
    check_status()


@pytest.mark.parametrize("shA,shB", SHAPES)
@pytest.mark.parametrize("max_exp", [9, 15])
def test_e4m3_operands_native(shA, shB, max_exp):
    """Codes drawn over every finite E4M3 code (max_exp 15: magnitudes up
    to 448, subnormals included) or a narrower range."""
    import torch
    (ac, a), (bc, b) = synth.e4m3_codes(74, 0, shA, max_exp), synth.e4m3_codes(74, 1, shB, max_exp)
    D = empty(shA[:-1] + shB[1:], torch.float32)
    dA = torch.from_numpy(np.ascontiguousarray(ac)).to("cuda:0")
    dB = torch.from_numpy(np.ascontiguousarray(bc)).to("cuda:0")
    moa.moa_inner("add", "mul", "fp8e4m3", "native", shA, dA, shB, dB, D, "f32")
    assert_norm_err(D.cpu().numpy(), a, b, _acc_tol(shA[-1]))
    check_status()


@pytest.mark.parametrize("n", [2048, 8192])
def test_f16_and_e4m3_square_sampled(n):
    import torch
    idx = sample_idx(n * n, 1500, seed=n + 1)
    (ab, a), (bb, b) = synth.to_f16(synth.uniform(75, 0, (n, n), -1, 1)), synth.to_f16(synth.uniform(75, 1, (n, n), -1, 1))
    D = empty((n, n), torch.float32)
    moa.moa_inner("add", "mul", "f16", "native", (n, n), _dev_bits(ab, torch.float16), (n, n),
                  _dev_bits(bb, torch.float16), D, "f32")
    got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
    assert_norm_err(got, a, b, _acc_tol(n), out_idx=idx)
    (ac, a8), (bc, b8) = synth.e4m3_codes(76, 0, (n, n), 11), synth.e4m3_codes(76, 1, (n, n), 11)
    moa.moa_inner("add", "mul", "fp8e4m3", "native", (n, n), torch.from_numpy(ac).to("cuda:0"), (n, n),
                  torch.from_numpy(bc).to("cuda:0"), D, "f32")
    got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
    assert_norm_err(got, a8, b8, _acc_tol(n), out_idx=idx)
    check_status()
    del D
    torch.cuda.empty_cache()


def _pow2_scales(seed, stream, shape, lo=-20, hi=20):
    return np.ldexp(1.0, synth.int_uniform(seed, stream, shape, lo, hi)).astype(np.float32)


@pytest.mark.parametrize("shA,shB", [((300, 136), (136, 200)), ((2, 64, 300), (300, 5, 80)), ((260, 700), (700, 390)),
                                     ((37, 61), (61, 45)), ((129, 8), (8, 257))])
def test_e4m3_with_block_scales(shA, shB):
    """moa_inner_e4m3_scaled: e4m3 codes times per-block powers of two (A per
    row and 128-block of the contraction, B per 128 x 128 block) against the
    oracle's Dot2 of the scaled operands (exact in FP64)."""
    import torch
    M, K = int(np.prod(shA[:-1])), shA[-1]
    N = int(np.prod(shB[1:]))
    KB, NB = (K + 127) // 128, (N + 127) // 128
    (ac, a), (bc, b) = synth.e4m3_codes(77, 0, shA, 12), synth.e4m3_codes(77, 1, shB, 12)
    sa, sb = _pow2_scales(77, 2, (M, KB)), _pow2_scales(77, 3, (KB, NB))
    kb = np.arange(K) // 128
    As = a.reshape(M, K) * sa.astype(np.float64)[:, kb]
    Bs = b.reshape(K, N) * sb.astype(np.float64)[kb][:, np.arange(N) // 128]
    D = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner_e4m3_scaled(shA, torch.from_numpy(np.ascontiguousarray(ac)).to("cuda:0"), to_dev(sa), shB,
                              torch.from_numpy(np.ascontiguousarray(bc)).to("cuda:0"), to_dev(sb), D)
    assert_norm_err(D.cpu().numpy().reshape(M, N), As, Bs, _acc_tol(K))
    check_status()
