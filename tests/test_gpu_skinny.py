"""GPU parity of the skinny (add, mul) path -- a result of at most 8 rows,
the shape of the method's own measurement in Sec. IV (m x 128 times 128 x n,
m <= 4, n up to 2^26) -- against the oracle: FP64 within 1e-12 and FP32
within 2e-6 normalised error (Dot2 reference of the operands as given).
Covers the vector and scalar column paths (N not a multiple of the vector
width, operands off 16-byte alignment), K shorter than, equal to and longer
than one staged chunk of A, and the full-size n = 2^26 operand drawn on the
device by the same counter-based generator, checked on sampled columns."""
import numpy as np
import pytest

import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, dev, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


def _run(dt, A, B, offset=0):
    """D = A . B through the C ABI; `offset` elements shift the device
    copies of B and D off 16-byte alignment."""
    import torch
    tdt = torch.float64 if dt == "f64" else torch.float32
    a = to_dev(A, tdt)
    bflat = torch.zeros(B.size + offset, dtype=tdt, device=dev())
    bflat[offset:] = to_dev(B.ravel(), tdt)
    b = bflat[offset:].view(B.shape)
    dflat = torch.full((A.shape[0] * B.shape[1] + offset,), float("nan"), dtype=tdt, device=dev())
    d = dflat[offset:].view(A.shape[0], B.shape[1])
    moa.moa_inner("add", "mul", dt, "native", A.shape, a, B.shape, b, d, dt)
    return d.cpu().numpy()


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("k,n", [(128, 1024), (1, 37), (7, 4099), (300, 2050), (128, 1)])
def test_skinny_whole(dt, m, k, n):
    A, B = synth.skinny(m, n, k)
    if dt == "f32":
        A, B = synth.to_f32(A), synth.to_f32(B)
    D = _run(dt, A, B)
    assert_norm_err(D, A, B, TOL[dt])
    check_status()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_skinny_unaligned_scalar_path(dt):
    A, B = synth.skinny(3, 1000, 128)
    if dt == "f32":
        A, B = synth.to_f32(A), synth.to_f32(B)
    D = _run(dt, A, B, offset=1)
    assert_norm_err(D, A, B, TOL[dt])
    check_status()


def test_skinny_loguniform_f64():
    A = synth.log_uniform_signed(6, 2, (4, 128))
    B = synth.log_uniform_signed(6, 3, (128, 8192))
    D = _run("f64", A, B)
    assert_norm_err(D, A, B, 1e-12)
    check_status()


@pytest.mark.parametrize("dt,m", [("f64", 4), ("f32", 1)])
def test_skinny_full_size_sampled(dt, m):
    """n = 2^26 (B of 64 GiB in FP64): B drawn on the device, 512 sampled
    outputs checked against the oracle on the same values drawn on the host."""
    import torch
    n, k = synth.SKINNY_N_MAX, synth.SKINNY_K
    tdt = torch.float64 if dt == "f64" else torch.float32
    A64, _ = synth.skinny(m, 1, k)  # A depends only on (m, k)
    B = synth.device_uniform(synth.SKINNY_SEED, 1, (k, n), -1.0, 1.0, dev(), dtype=tdt)
    D = empty((m, n), tdt)
    a = to_dev(A64, tdt)
    moa.moa_inner("add", "mul", dt, "native", (m, k), a, (k, n), B, D, dt)
    idx = sample_idx(m * n, 512, seed=11)
    rows, cols = idx // n, idx % n
    got = D.view(-1)[torch.from_numpy(idx).to(dev())].cpu().numpy()
    del B, D
    torch.cuda.empty_cache()
    Bc = synth.skinny_columns(cols, n, k)
    A = A64 if dt == "f64" else synth.to_f32(A64)
    if dt == "f32":
        Bc = synth.to_f32(Bc)
    # output e = (row r, column c): the row of A times the column drawn for it
    for e in range(len(idx)):
        assert_norm_err(got[e:e + 1], A[rows[e]:rows[e] + 1], Bc[:, e:e + 1], TOL[dt])
    check_status()


def test_device_generator_matches_host():
    import torch
    a = synth.uniform(6, 1, (128, 3000), -1.0, 1.0)
    b = synth.device_uniform(6, 1, (128, 3000), -1.0, 1.0, dev(), chunk=5000).cpu().numpy()
    assert np.array_equal(a, b)
    b32 = synth.device_uniform(6, 1, (128, 3000), -1.0, 1.0, dev(), dtype=torch.float32).cpu().numpy()
    assert np.array_equal(synth.to_f32(a), b32)
