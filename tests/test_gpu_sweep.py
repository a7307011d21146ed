"""GPU parity of every configuration of the square matrix-multiply sweep that
bench.py times: each form of the (+,*) inner product (Eq. 2, matrix multiply
as its special case, Sec. I) at n = 256 .. 8192 with uniform and log-uniform
values, on the sweep's own operands (leading blocks of the n = 8192 arrays,
synth.square_leading), in the launch configuration the benchmark times.
Whole results at n <= 512, 1,500 sampled outputs above, against the
oracle's Dot2 reference of the operands as the form receives them.

Bars (normalised error |D - D_exact| / sum_p |A||B|): Ozaki and plain FP64
1e-12; FP32 native and split-BF16x3 2e-6; bf16 operands as given
max(2e-6, (K/16) 2^-23) (one FP32 accumulator over the whole contraction,
truncated at most once per 16-deep MMA step); BF16 form 1e-2; FP16 form
2e-3; FP8 form 6e-2, except log-uniform contractions below 512, held to the
two-rounding bound 2u + u^2 = 0.129 of e4m3 (u = 2^-4): such sums are
dominated by a few products whose e4m3 rounding does not average out
(measured 8.2e-2 over the whole 256 x 256 result)."""
import numpy as np
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, bf16_dev, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

FORMS = [("ozaki", "f64", 1e-12), ("native", "f64", 1e-12), ("native", "f32", 2e-6), ("bf16x3", "f32", 2e-6),
         ("bf16", "f32", 1e-2), ("f16", "f32", 2e-3), ("fp8_t128", "f32", 6e-2), ("native", "bf16", None)]


def _tol(form, dtype, tol, n, dist):
    if tol is None:  # one FP32 tensor-core accumulator over the whole contraction
        return max(2e-6, (n / 16) * 2.0 ** -23)
    if form == "fp8_t128" and dist == "loguniform" and n < 512:
        return 2 * 2.0 ** -4 + 2.0 ** -8
    return tol
_FULL = {}


def _operands(n, dist):
    if dist not in _FULL:
        _FULL[dist] = synth.square(max(synth.SWEEP_N), dist)
    A, B = _FULL[dist]
    return np.ascontiguousarray(A[:n, :n]), np.ascontiguousarray(B[:n, :n])


@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
@pytest.mark.parametrize("n", list(synth.SWEEP_N))
def test_sweep_configuration(n, dist):
    import torch
    A64, B64 = _operands(n, dist)
    assert np.array_equal(A64[:64, :64], synth.square_leading(64, dist)[0])  # the sweep's own operands
    idx = None if n <= 512 else sample_idx(n * n, 1500, seed=n)
    for form, dtype, tol in FORMS:
        if dtype == "f64":
            a, b, A, B = A64, B64, to_dev(A64), to_dev(B64)
        elif dtype == "f32":
            a, b = synth.to_f32(A64), synth.to_f32(B64)
            A, B = to_dev(a), to_dev(b)
        else:
            (abits, a), (bbits, b) = synth.to_bf16(A64), synth.to_bf16(B64)
            A, B = bf16_dev(abits), bf16_dev(bbits)
        D = empty((n, n), torch.float64 if dtype == "f64" else torch.float32)
        moa.moa_inner("add", "mul", dtype, form, (n, n), A, (n, n), B, D, "f64" if dtype == "f64" else "f32")
        got = D.cpu().numpy() if idx is None else D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
        try:
            assert_norm_err(got, a, b, _tol(form, dtype, tol, n, dist), out_idx=idx)
        except AssertionError as e:
            raise AssertionError(f"{form}:{dtype} n={n} {dist}: {e}") from None
        del A, B, D
    check_status()
    torch.cuda.empty_cache()
