"""GPU tests of moa_inner_host (Eq. 2 on arrays held in host memory: copies
in and out inside the call, row blocks overlapped) and of the GEMM timing
hook.  Results are compared with the oracle at each form's bar, and with
moa_inner on device copies of the same operands: the row blocks of
moa_inner_host each hold more than 128 rows, so every output takes the
same arithmetic and the two agree bit for bit."""
import numpy as np
import pytest

import oracle
import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, empty, to_dev

pytestmark = pytest.mark.gpu


def _host_vs_device(reduce, combine, dtype, form, A, B, out_np_dtype, pinned):
    import torch
    shD = A.shape[:-1] + B.shape[1:]
    tA, tB = torch.from_numpy(np.ascontiguousarray(A)), torch.from_numpy(np.ascontiguousarray(B))
    hD = torch.empty(shD, dtype=torch.from_numpy(np.zeros(1, out_np_dtype)).dtype)
    if pinned:
        tA, tB, hD = tA.pin_memory(), tB.pin_memory(), hD.pin_memory()
    odt = {np.float64: "f64", np.float32: "f32", np.int32: "i32"}[out_np_dtype]
    moa.moa_inner_host(reduce, combine, dtype, form, A.shape, tA, B.shape, tB, hD, odt)
    torch.cuda.synchronize()
    Dd = empty(shD, hD.dtype)
    moa.moa_inner(reduce, combine, dtype, form, A.shape, to_dev(A), B.shape, to_dev(B), Dd, odt)
    check_status()
    return hD.numpy(), Dd.cpu().numpy()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_ozaki_row_blocks(pinned):
    """2100 result rows: four row blocks of 525, overlapped with the copies."""
    A = synth.uniform(61, 0, (2100, 700), -1, 1)
    B = synth.log_uniform_signed(61, 1, (700, 300))
    h, d = _host_vs_device("add", "mul", "f64", "ozaki", A, B, np.float64, pinned)
    assert np.array_equal(h, d)
    assert_norm_err(h, A, B, 1e-12)


def test_host_f32_forms_and_semirings():
    A = synth.to_f32(synth.uniform(62, 0, (3, 700, 130), -1, 1))
    B = synth.to_f32(synth.uniform(62, 1, (130, 5, 77), -1, 1))
    for form, tol in (("bf16x3", 2e-6), ("native", 2e-6), ("fp8_t128", 0.129)):
        h, d = _host_vs_device("add", "mul", "f32", form, A, B, np.float32, True)
        assert np.array_equal(h, d), form
        assert_norm_err(h, A, B, tol)
    T, U = synth.semiring_inputs("tropical", seed=63, shape_a=(1300, 90), shape_b=(90, 140))
    h, d = _host_vs_device("min", "add", "f32", "native", T, U, np.float32, True)
    assert np.array_equal(h, oracle.inner_f32("min", "add", T, U)) and np.array_equal(h, d)
    I = synth.int_uniform(64, 0, (1100, 77), -128, 127)
    J = synth.int_uniform(64, 1, (77, 150), -128, 127)
    h, d = _host_vs_device("add", "mul", "i32", "native", I, J, np.int32, True)
    assert np.array_equal(h, oracle.inner_i32(I, J))


def test_host_packed_bits_and_edges():
    import torch
    A = synth.bernoulli(65, 0, (40, 64), 0.2)
    B = synth.bernoulli(65, 1, (64, 96), 0.2)
    pa = torch.from_numpy(synth.pack_bits(A).view(np.int32)).pin_memory()
    pb = torch.from_numpy(synth.pack_bits(B).view(np.int32)).pin_memory()
    hD = torch.zeros(((40 * 96 + 31) // 32,), dtype=torch.int32).pin_memory()
    moa.moa_inner_host("or", "and", "b1", "native", A.shape, pa, B.shape, pb, hD, "b1")
    torch.cuda.synchronize()
    got = synth.unpack_bits(hD.numpy().view(np.uint32), 40 * 96).reshape(40, 96)
    assert np.array_equal(got, oracle.inner_bool(A, B))
    # empty contraction: the identity of the reduce, written into host memory
    hE = torch.full((5, 6), 3.0, dtype=torch.float32).pin_memory()
    moa.moa_inner_host("min", "add", "f32", "native", (5, 0), 0, (0, 6), 0, hE, "f32")
    torch.cuda.synchronize()
    assert np.all(hE.numpy() == np.inf)
    # device memory is not host memory
    dA = empty((4, 5), torch.float32)
    st = moa.moa_inner_host("add", "mul", "f32", "native", (4, 5), dA.data_ptr(), (5, 3),
                            np.zeros((5, 3), np.float32), np.zeros((4, 3), np.float32), "f32", check=False)
    assert st == 11
    check_status()


def test_gemm_timing_hook():
    """moa_kernel_timing brackets each tensor-core GEMM launch with events."""
    import torch
    A = to_dev(synth.to_f32(synth.uniform(66, 0, (512, 512), -1, 1)))
    B = to_dev(synth.to_f32(synth.uniform(66, 1, (512, 512), -1, 1)))
    D = empty((512, 512), torch.float32)
    moa.moa_kernel_timing(True)
    for _ in range(3):
        moa.moa_inner("add", "mul", "f32", "bf16x3", (512, 512), A, (512, 512), B, D, "f32")
    moa.moa_inner("min", "add", "f32", "native", (512, 512), A, (512, 512), B, D, "f32")  # no GEMM: not recorded
    moa.moa_kernel_timing(False)
    moa.moa_inner("add", "mul", "f32", "bf16x3", (512, 512), A, (512, 512), B, D, "f32")  # after stop
    n, ms = moa.moa_kernel_timing_read()
    assert n == 3 and 0.0 < ms < 1000.0
    moa.moa_kernel_timing(True)  # a new start clears the record
    moa.moa_kernel_timing(False)
    assert moa.moa_kernel_timing_read() == (0, 0.0)
    check_status()
