"""GPU parity of the Ozaki-sliced FP64 (+,*) inner product (tensor cores,
FP64-accurate) against the oracle's Dot2 reference: normalised error
<= 1e-12, the bound the plain FP64 form is held to."""
import numpy as np
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12
# contractions on both sides of each slice-count change (10 slices up to K = 64, 8 up to K = 256, 7 below
# K = 4096, 6 from there)
SHAPES = [((300, 136), (136, 200)), ((2, 64, 72), (72, 5, 80)), ((129, 8), (8, 257)), ((1, 1), (1, 1)),
          ((37, 61), (61, 45)), ((130, 1500), (1500, 131)), ((16, 12, 8, 64), (64, 24, 20)),
          ((140, 256), (256, 150)), ((140, 257), (257, 150)), ((260, 3000), (3000, 270)),
          ((96, 4095), (4095, 70)), ((96, 4096), (4096, 70))]


def _ozaki(A, B):
    import torch
    D = empty(A.shape[:-1] + B.shape[1:], torch.float64)
    moa.moa_inner("add", "mul", "f64", "ozaki", A.shape, to_dev(A), B.shape, to_dev(B), D, "f64")
    return D


@pytest.mark.parametrize("shA,shB", SHAPES)
@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
def test_ozaki_small(shA, shB, dist):
    if dist == "uniform":
        A, B = synth.uniform(41, 0, shA, -1, 1), synth.uniform(41, 1, shB, -1, 1)
    else:
        A, B = synth.log_uniform_signed(41, 0, shA), synth.log_uniform_signed(41, 1, shB)
    D = _ozaki(A, B)
    assert_norm_err(D.cpu().numpy(), A, B, TOL)
    check_status()


@pytest.mark.parametrize("K", [90, 300, 4100])
def test_ozaki_zero_rows_columns_and_wide_range(K):
    """Zero rows and columns, scales 1e+-200, a subnormal, and digits that
    carry into the top one, at 8 slices (K = 90), 7 (K = 300) and 6
    (K = 4100; A's rows then take the single-pass row kernel)."""
    A = synth.uniform(42, 0, (70, K), -1, 1)
    B = synth.uniform(42, 1, (K, 50), -1, 1)
    A[3] = 0.0
    B[:, 7] = 0.0
    A[5] *= 1e200
    B[:, 9] *= 1e-200
    A[6, 4] = 5e-310  # subnormal entry
    # entries just below a power of two: every lower digit of the scaled value is all ones, so the
    # balanced digits carry into the top one (which becomes 2^(beta-1))
    A[8] = np.nextafter(1.0, 0.0) * np.where(np.arange(K) % 2, 1.0, -1.0)
    B[:, 11] = np.nextafter(0.5, 0.0)
    A[9, :] = np.nextafter(np.ldexp(1.0, -3), 0.0)
    D = _ozaki(A, B).cpu().numpy()
    assert np.all(D[3] == 0) and np.all(D[:, 7] == 0)
    assert_norm_err(D, A, B, TOL)


@pytest.mark.parametrize("n", [512])
def test_ozaki_square_whole(n):
    for dist in ("uniform", "loguniform"):
        A, B = synth.square(n, dist)
        assert_norm_err(_ozaki(A, B).cpu().numpy(), A, B, TOL)
    check_status()


def test_ozaki_longest_contraction_sampled():
    """K = 21845, the longest contraction the form takes (6 slices: a class
    sum of 6 slice pairs of K products of at most 2^14 stays below 2^31)."""
    import torch
    for dist in ("uniform", "loguniform"):
        A, B = synth.square(300, dist, m=300, k=21845)
        D = _ozaki(A, B)
        idx = sample_idx(300 * 300, 2000)
        got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
        assert_norm_err(got, A, B, TOL, out_idx=idx)
    check_status()


def test_ozaki_contraction_past_the_limit_is_refused():
    """K = 21846: a class sum could reach 2^31, so the call is refused before any launch."""
    A, B = synth.uniform(43, 0, (4, 21846), -1, 1), synth.uniform(43, 1, (21846, 3), -1, 1)
    import torch
    D = empty((4, 3), torch.float64)
    with pytest.raises(moa.MoaError) as e:
        moa.moa_inner("add", "mul", "f64", "ozaki", A.shape, to_dev(A), B.shape, to_dev(B), D, "f64")
    assert moa.STATUS[e.value.status] == "MOA_ERR_UNSUPPORTED"
    check_status()


@pytest.mark.parametrize("n", [4096, 8192])
def test_ozaki_square_large_sampled(n):
    import torch
    idx = sample_idx(n * n, 1000)
    for dist in ("uniform", "loguniform"):
        A, B = synth.square(n, dist)
        D = _ozaki(A, B)
        got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
        assert_norm_err(got, A, B, TOL, out_idx=idx)
        del D
    check_status()
    torch.cuda.empty_cache()
