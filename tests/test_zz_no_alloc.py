"""moa_inner_bf16x3_noalloc: the split-BF16x3 inner product for callers that
cannot allocate device memory (graph capture, fixed-budget serving loops,
callbacks that may not re-enter an allocator).  Its scratch is a fixed
device array inside the library instead of the allocated workspace.

Checked through the C ABI against the allocating entry point moa_inner
(MOA_FORM_BF16X3) on two calls in a row with different shapes and values —
the second call runs on the array the first one left behind — within the
tolerance the other bf16x3 tests use, plus the oracle's bound.  This file is
collected last so a failure here stops a -x run only after every other test.
"""
import numpy as np
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, empty, to_dev

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _allocating(shA, A, shB, B):
    import torch
    D = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner("add", "mul", "f32", "bf16x3", shA, A, shB, B, D, "f32")
    return D


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    # the third problem has fewer than 128 rows and a contraction that is not a multiple of 8, so A's and B's
    # planes carry padding columns; it runs on the array the two earlier calls left behind
    cases = [((3, 100, 72), (72, 5, 60), 31), ((300, 1000), (1000, 200), 32), ((5, 7, 37), (37, 9), 33)]
    for shA, shB, seed in cases:  # two calls in a row, different problems
        A = synth.to_f32(synth.uniform(seed, 0, shA, -1, 1))
        B = synth.to_f32(synth.uniform(seed, 1, shB, -1, 1))
        dA, dB = to_dev(A), to_dev(B)
        D = torch.full(shA[:-1] + shB[1:], float("nan"), dtype=torch.float32, device="cuda:0")
        moa.moa_inner_bf16x3_noalloc(shA, dA, shB, dB, D)
        ref = _allocating(shA, dA, shB, dB)
        got = D.cpu().numpy()
        want = ref.cpu().numpy()
        S = np.abs(A.reshape(-1, shA[-1]).astype(np.float64)) @ np.abs(B.reshape(shB[0], -1).astype(np.float64))
        assert np.max(np.abs(got - want).reshape(S.shape) / S) <= TOL
        assert_norm_err(got, A, B, TOL)
    check_status()


def test_noalloc_rejects_problems_beyond_its_buffer():
    # 6 * (M*Kp + K*Np) bytes must fit in the fixed buffer; this needs ~384 MiB
    st = moa.moa_inner_bf16x3_noalloc((8192, 4096), 0x1000, (4096, 8192), 0x2000, 0x3000, stream=0, check=False)
    assert st == 12  # MOA_ERR_SCRATCH_LIMIT, returned before any launch
    assert moa.NOALLOC_SCRATCH_BYTES == 32 * 1024 * 1024
