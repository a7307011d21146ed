"""GPU parity of the CUDA-core inner products (Eq. 2 with a general
(reduce, combine)) against the oracle.  Min/max, integer and Boolean results
are bit-exact; FP64 / FP32 (+,*) within the normalised tolerance."""
import numpy as np
import pytest

import oracle
import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

SEMIRINGS = [("min", "add", "tropical"), ("max", "add", "tropical"), ("max", "mul", "maxmul"),
             ("min", "mul", "maxmul"), ("max", "add", "tropical_finite"), ("min", "add", "tropical_finite"),
             # widest and minimax paths, differences, and the idempotent pairs
             ("max", "min", "tropical"), ("min", "max", "tropical"), ("min", "sub", "tropical_finite"),
             ("max", "sub", "tropical_finite"), ("min", "min", "tropical"), ("max", "max", "maxmul")]
# several 128 x 128 tiles, ragged M, N and a contraction tail
RAGGED = [((3, 100, 77), (77, 5, 53)), ((1, 129), (129, 1)), ((257, 16), (16, 129)), ((7, 33), (33, 300))]


def _f32(reduce, combine, A, B):
    import torch
    D = empty(A.shape[:-1] + B.shape[1:], torch.float32)
    moa.moa_inner(reduce, combine, "f32", "native", A.shape, to_dev(A), B.shape, to_dev(B), D, "f32")
    return D


@pytest.mark.parametrize("reduce,combine,kind", SEMIRINGS)
@pytest.mark.parametrize("shA,shB", RAGGED)
def test_f32_semirings_small(reduce, combine, kind, shA, shB):
    A, B = synth.semiring_inputs(kind, seed=5, shape_a=shA, shape_b=shB)
    D = _f32(reduce, combine, A, B)
    assert np.array_equal(D.cpu().numpy(), oracle.inner_f32(reduce, combine, A, B))
    check_status()


@pytest.mark.parametrize("reduce,combine,kind", SEMIRINGS[:3] + SEMIRINGS[6:9])
def test_f32_semirings_full_size_sampled(reduce, combine, kind):
    """A <32,128,512>, B <512,64,64>: 16.8M outputs, 20,000 sampled."""
    import torch
    A, B = synth.semiring_inputs(kind)
    D = _f32(reduce, combine, A, B)
    idx = sample_idx(D.numel(), 20000)
    got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
    assert np.array_equal(got, oracle.inner_f32(reduce, combine, A, B, out_idx=idx))
    if kind == "tropical" and reduce == "min":
        assert np.isfinite(got).all()  # (min,+) outputs are finite at 5% inf
    check_status()


def test_i32_small_and_wrap():
    import torch
    for shA, shB in RAGGED:
        A, B = synth.semiring_inputs("int32", seed=6, shape_a=shA, shape_b=shB)
        D = empty(A.shape[:-1] + B.shape[1:], torch.int32)
        moa.moa_inner("add", "mul", "i32", "native", shA, to_dev(A), shB, to_dev(B), D, "i32")
        assert np.array_equal(D.cpu().numpy(), oracle.inner_i32(A, B))
    A = synth.int_uniform(8, 0, (70, 45), -(2 ** 31), 2 ** 31 - 1)
    B = synth.int_uniform(8, 1, (45, 90), -(2 ** 31), 2 ** 31 - 1)
    D = empty((70, 90), torch.int32)
    moa.moa_inner("add", "mul", "i32", "native", A.shape, to_dev(A), B.shape, to_dev(B), D, "i32")
    assert np.array_equal(D.cpu().numpy(), oracle.inner_i32(A, B))
    check_status()


def test_i32_full_size_sampled():
    import torch
    A, B = synth.semiring_inputs("int32")
    D = empty((32, 128, 64, 64), torch.int32)
    moa.moa_inner("add", "mul", "i32", "native", A.shape, to_dev(A), B.shape, to_dev(B), D, "i32")
    idx = sample_idx(D.numel(), 20000)
    got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
    assert np.array_equal(got, oracle.inner_i32(A, B, out_idx=idx))


def _i32(A, B):
    import torch
    D = empty(A.shape[:-1] + B.shape[1:], torch.int32)
    moa.moa_inner("add", "mul", "i32", "native", A.shape, to_dev(A), B.shape, to_dev(B), D, "i32")
    return D.cpu().numpy()


# more than 128 rows and columns and K <= 1024: the bf16 tensor-core path
# when the values are int8-range; ragged tiles and contraction tails
I8_SHAPES = [((300, 77), (77, 260)), ((129, 1024), (1024, 136)), ((4, 64, 33), (33, 3, 100)), ((257, 8), (8, 129)),
             ((520, 1), (1, 515))]


@pytest.mark.parametrize("shA,shB", I8_SHAPES)
def test_i32_int8_range_tensor_core_path(shA, shB):
    A = synth.int_uniform(21, 0, shA, -128, 127)
    B = synth.int_uniform(21, 1, shB, -128, 127)
    assert np.array_equal(_i32(A, B), oracle.inner_i32(A, B))
    check_status()


@pytest.mark.parametrize("K", [1024, 1025])
def test_i32_int8_range_largest_sums(K):
    """Every value -128: each sum is 2^14 K, at K = 1024 exactly 2^24, the
    largest the FP32 accumulation has to hold; K = 1025 runs on CUDA cores.
    Alternating signs in B give sums of both signs."""
    A = np.full((130, K), -128, np.int32)
    B = np.full((K, 200), -128, np.int32)
    B[:, 1::2] = 127
    got = _i32(A, B)
    assert np.array_equal(got, oracle.inner_i32(A, B))
    assert got[0, 0] == 16384 * K
    check_status()


@pytest.mark.parametrize("where,value", [("A", 128), ("A", -129), ("B", 2 ** 31 - 1), ("B", -(2 ** 31))])
def test_i32_out_of_range_value_recomputed_on_cuda_cores(where, value):
    """One value outside [-128, 127] anywhere: the range flag sends the whole
    product to the CUDA-core kernel, with wrap-around where it occurs."""
    A = synth.int_uniform(22, 0, (200, 300), -128, 127)
    B = synth.int_uniform(22, 1, (300, 180), -128, 127)
    if where == "A":
        A[199, 299] = value
    else:
        B[0, 90] = value
    assert np.array_equal(_i32(A, B), oracle.inner_i32(A, B))
    check_status()


def _bool(A, B):
    import torch
    shD = A.shape[:-1] + B.shape[1:]
    nD = int(np.prod(shD))
    D = torch.full(((nD + 31) // 32,), -1, dtype=torch.int32, device="cuda:0")
    moa.moa_inner("or", "and", "b1", "native", A.shape, to_dev(synth.pack_bits(A).view(np.int32)), B.shape,
                  to_dev(synth.pack_bits(B).view(np.int32)), D, "b1")
    words = D.cpu().numpy().view(np.uint32)
    if nD % 32:
        assert words[-1] >> np.uint32(nD % 32) == 0  # padding bits written as zero
    return synth.unpack_bits(words, nD).reshape(shD)


@pytest.mark.parametrize("shA,shB", [((64, 96), (96, 64)), ((3, 50, 77), (77, 5, 13)), ((100, 32), (32, 33)),
                                     ((1, 1), (1, 1)), ((65, 1000), (1000, 64))])
def test_bool_small(shA, shB):
    A, B = synth.semiring_inputs("bool", seed=9, shape_a=shA, shape_b=shB)
    assert np.array_equal(_bool(A, B), oracle.inner_bool(A, B))
    check_status()


@pytest.mark.parametrize("shA,shB,dens", [((300, 100), (100, 320), 0.05), ((129, 16), (16, 160), 0.5),
                                          ((257, 1000), (1000, 256), 0.002), ((4, 130, 77), (77, 8, 32), 0.05),
                                          ((300, 48), (48, 448), 0.0)])
def test_bool_tensor_core_path(shA, shB, dens):
    """(or, and) by exact counting on the tensor cores (results with more
    than 128 rows and a multiple of 32 columns): bit-exact, at densities from
    none to half, K not a multiple of 32 or of 128."""
    A = synth.bernoulli(19, 0, shA, dens)
    B = synth.bernoulli(19, 1, shB, dens)
    assert np.array_equal(_bool(A, B), oracle.inner_bool(A, B))
    check_status()


def test_bool_full_size_sampled():
    A, B = synth.semiring_inputs("bool")
    D = _bool(A, B)
    idx = sample_idx(D.size, 50000)
    assert np.array_equal(D.ravel()[idx], oracle.inner_bool(A, B, out_idx=idx))


def test_f64_plain_method_rank4x3():
    """The plain method: FP64 (+,*), A <16,12,8,64> . B <64,24,20>, whole result."""
    import torch
    A, B = synth.rank4x3_f64()
    D = empty((16, 12, 8, 24, 20), torch.float64)
    moa.moa_inner("add", "mul", "f64", "native", A.shape, to_dev(A), B.shape, to_dev(B), D, "f64")
    assert_norm_err(D.cpu().numpy(), A, B, 1e-12)
    check_status()


@pytest.mark.parametrize("shA,shB", RAGGED + [((256, 256), (256, 256))])
def test_f32_f64_plus_times_small(shA, shB):
    import torch
    A = synth.uniform(10, 0, shA, -1, 1)
    B = synth.uniform(10, 1, shB, -1, 1)
    D = empty(shA[:-1] + shB[1:], torch.float64)
    moa.moa_inner("add", "mul", "f64", "native", shA, to_dev(A), shB, to_dev(B), D, "f64")
    assert_norm_err(D.cpu().numpy(), A, B, 1e-12)
    A32, B32 = synth.to_f32(A), synth.to_f32(B)
    D32 = empty(shA[:-1] + shB[1:], torch.float32)
    moa.moa_inner("add", "mul", "f32", "native", shA, to_dev(A32), shB, to_dev(B32), D32, "f32")
    assert_norm_err(D32.cpu().numpy(), A32, B32, 2e-6)
    check_status()


def test_empty_contraction_fills_identity():
    import torch
    for reduce, combine, want in (("min", "add", np.inf), ("max", "mul", -np.inf)):
        D = empty((4, 6), torch.float32)
        moa.moa_inner(reduce, combine, "f32", "native", (4, 0), 0, (0, 6), 0, D, "f32")
        assert np.all(D.cpu().numpy() == want)
    D = torch.full((3, 5), 7.0, dtype=torch.float64, device="cuda:0")
    moa.moa_inner("add", "mul", "f64", "native", (3, 0), 0, (0, 5), 0, D, "f64")
    assert np.all(D.cpu().numpy() == 0)
    check_status()
