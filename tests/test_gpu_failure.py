"""Failure detection without faulting the GPU: a device wait that can only
run out (a barrier nothing completes) gives up after its limit, the host
reads MOA_ERR_TIMEOUT from the status word, and the context stays usable.
Host-side failures (bad arguments, a failing workspace allocation) return
their status before any launch."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import empty, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    assert moa.moa_device_status() == 0
    assert moa.moa_selftest_wait_timeout(50_000) == 0  # 50 ms
    assert moa.moa_device_status() == 8  # MOA_ERR_TIMEOUT, read and cleared
    assert moa.moa_device_status() == 0
    A, B = synth.semiring_inputs("tropical", seed=3, shape_a=(40, 30), shape_b=(30, 20))
    D = empty((40, 20), torch.float32)
    moa.moa_inner("min", "add", "f32", "native", A.shape, to_dev(A), B.shape, to_dev(B), D, "f32")
    assert np.array_equal(D.cpu().numpy(), oracle.inner_f32("min", "add", A, B))
    assert moa.moa_selftest_wait_timeout(0) == 11  # limit out of range: MOA_ERR_INVALID, no launch


def test_workspace_allocation_failure_is_reported():
    code = (
        "import sys; sys.path.insert(0, %r); import torch, paper_0907_0792_gb300 as moa;"
        "A = torch.ones(64, 64, device='cuda'); D = torch.empty(64, 64, device='cuda');"
        "st = moa.moa_inner('add', 'mul', 'f32', 'bf16x3', (64, 64), A, (64, 64), A, D, 'f32', check=False);"
        "print(st)" % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    env = dict(os.environ, MOA_FAULT_INJECT="workspace")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.stdout.strip().splitlines()[-1] == "6", out.stderr  # MOA_ERR_WORKSPACE
