"""GPU parity of the tensor-core (tcgen05) forms of the (+,*) inner product
against the oracle (Dot2 FP64 reference of the operands as given), within
the normalised tolerance of each form: bf16 operands as given and the
split-BF16x3 form <= 2e-6, the BF16 form <= 1e-2."""
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, bf16_dev, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

# ragged tiles: 128-row and 128/256-column tiles with tails, odd contraction
SHAPES = [((300, 136), (136, 200)), ((2, 64, 72), (72, 5, 80)), ((129, 8), (8, 257)), ((1, 64), (64, 8)),
          ((520, 1000), (1000, 700))]
UNALIGNED = [((37, 61), (61, 45)), ((130, 13), (13, 131))]


def _bf16_inputs(shA, shB, seed=21):
    a_bits, a = synth.to_bf16(synth.uniform(seed, 0, shA, -1, 1))
    b_bits, b = synth.to_bf16(synth.uniform(seed, 1, shB, -1, 1))
    return a_bits, a, b_bits, b


@pytest.mark.parametrize("shA,shB", SHAPES + UNALIGNED)
def test_bf16_operands_native(shA, shB):
    import torch
    a_bits, a, b_bits, b = _bf16_inputs(shA, shB)
    D = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner("add", "mul", "bf16", "native", shA, bf16_dev(a_bits), shB, bf16_dev(b_bits), D, "f32")
    assert_norm_err(D.cpu().numpy(), a, b, 2e-6)
    check_status()


@pytest.mark.parametrize("form,tol", [("bf16x3", 2e-6), ("bf16", 1e-2)])
@pytest.mark.parametrize("shA,shB", SHAPES + UNALIGNED)
@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
def test_f32_forms(form, tol, shA, shB, dist):
    import torch
    if dist == "uniform":
        A = synth.to_f32(synth.uniform(22, 0, shA, -1, 1))
        B = synth.to_f32(synth.uniform(22, 1, shB, -1, 1))
    else:
        A = synth.to_f32(synth.log_uniform_signed(22, 0, shA))
        B = synth.to_f32(synth.log_uniform_signed(22, 1, shB))
    D = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner("add", "mul", "f32", form, shA, to_dev(A), shB, to_dev(B), D, "f32")
    assert_norm_err(D.cpu().numpy(), A, B, tol)
    check_status()


@pytest.mark.parametrize("n", [256, 512])
def test_square_sweep_small_whole(n):
    """The square matrix-multiply sweep at sizes the oracle finishes whole."""
    import torch
    A64, B64 = synth.square(n, "uniform")
    A, B = synth.to_f32(A64), synth.to_f32(B64)
    for form, tol in (("bf16x3", 2e-6), ("bf16", 1e-2)):
        D = empty((n, n), torch.float32)
        moa.moa_inner("add", "mul", "f32", form, (n, n), to_dev(A), (n, n), to_dev(B), D, "f32")
        assert_norm_err(D.cpu().numpy(), A, B, tol)
    check_status()


@pytest.mark.parametrize("n", [4096, 8192])
def test_square_sweep_large_sampled(n):
    """n = 4096 and 8192 in the launch configuration the benchmark times;
    2,000 outputs checked against the oracle."""
    import torch
    A64, B64 = synth.square(n, "uniform")
    A, B = synth.to_f32(A64), synth.to_f32(B64)
    idx = sample_idx(n * n, 2000)
    for form, tol in (("bf16x3", 2e-6), ("bf16", 1e-2)):
        D = empty((n, n), torch.float32)
        moa.moa_inner("add", "mul", "f32", form, (n, n), to_dev(A), (n, n), to_dev(B), D, "f32")
        got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
        assert_norm_err(got, A, B, tol, out_idx=idx)
        del D
    a_bits, a = synth.to_bf16(A64)
    b_bits, b = synth.to_bf16(B64)
    D = empty((n, n), torch.float32)
    moa.moa_inner("add", "mul", "bf16", "native", (n, n), bf16_dev(a_bits), (n, n), bf16_dev(b_bits), D, "f32")
    got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
    assert_norm_err(got, a, b, 2e-6, out_idx=idx)
    check_status()
    torch.cuda.empty_cache()
