"""GPU parity of moa_transpose and moa_inner_axes (Eq. 2 over any pair of
axes of equal length) against numpy's transpose and the oracle on the
moved operands: bit-exact for data movement, integers and min/max; the
floating (+,*) forms within their normalised tolerances."""
import numpy as np
import pytest

import oracle
import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import assert_norm_err, check_status, empty, sample_idx, to_dev

pytestmark = pytest.mark.gpu

TORCH_DT = {"f64": "float64", "f32": "float32", "i32": "int32", "bf16": "bfloat16"}

# (shape, perm): both kernels (innermost axis kept / 32 x 32 tiles), ragged
# tiles, extent-1 axes, merged runs, rank 0, 1 and 8
TRANSPOSES = [((), ()), ((5,), (0,)), ((3, 4), (1, 0)), ((37, 65), (1, 0)), ((3, 37, 65), (2, 0, 1)),
              ((3, 37, 65), (1, 0, 2)), ((2, 1, 33, 1, 40), (4, 3, 2, 1, 0)), ((4, 5, 6, 7), (0, 2, 3, 1)),
              ((2, 3, 2, 3, 2, 3, 2, 3), (7, 0, 6, 1, 5, 2, 4, 3)), ((64, 1000), (1, 0)), ((1000, 3), (1, 0)),
              ((3, 1000), (1, 0)), ((1, 1, 1), (2, 0, 1)),
              # rows copied as 16-byte vectors; more rows than one grid dimension holds
              ((6, 5, 64), (1, 0, 2)), ((70000, 2, 8), (1, 0, 2)), ((3, 70000, 5), (2, 1, 0))]


def _dev(x, dt):
    import torch
    if dt == "bf16":
        return torch.from_numpy(x.view(np.int16)).view(torch.bfloat16).cuda()
    return to_dev(x)


@pytest.mark.parametrize("shape,perm", TRANSPOSES)
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16", "i32"])
def test_transpose_bit_exact(shape, perm, dt):
    import torch
    n = int(np.prod(shape, dtype=np.int64))
    bits = {"f64": np.uint64, "f32": np.uint32, "i32": np.uint32, "bf16": np.uint16}[dt]
    x = (synth.u64(24, 0, n) >> np.uint64(64 - 8 * np.dtype(bits).itemsize)).astype(bits).reshape(shape)
    src = {"f64": np.float64, "f32": np.float32, "i32": np.int32, "bf16": np.uint16}[dt]
    x = x.view(src)
    out = empty(tuple(shape[a] for a in perm), getattr(torch, TORCH_DT[dt]))
    moa.moa_transpose(dt, shape, _dev(x, dt), perm, out)
    got = out.cpu()
    got = got.view(torch.int16).numpy().view(np.uint16) if dt == "bf16" else got.numpy()
    assert np.array_equal(got.view(bits), np.transpose(x, perm).view(bits))
    check_status()


def _axes_case(sa, ax_a, sb, ax_b):
    sb = list(sb)
    sb[ax_b] = sa[ax_a]
    return tuple(sb)


# moved problems (M, K, N): (30, 40, 21), (780, 300, 4), (21000, 33, 145), (420, 4, 66)
AXES = [((6, 40, 5), 1, (7, 40, 3), 1), ((300, 3, 260), 0, (4, 300), 1), ((150, 33, 140), 1, (145, 33), 1),
        ((2, 3, 4, 70), 2, (4, 2, 33), 0)]


@pytest.mark.parametrize("sa,ax_a,sb,ax_b", AXES)
def test_inner_axes_exact_semirings(sa, ax_a, sb, ax_b):
    """int32 (+,*) (tensor-core path where the moved problem has more than 128
    rows and columns) and (min,+), (max,min) FP32: bit-exact."""
    import torch
    sb = _axes_case(sa, ax_a, sb, ax_b)
    A = synth.int_uniform(25, 0, sa, -128, 127)
    B = synth.int_uniform(25, 1, sb, -128, 127)
    Am, Bm = oracle.move_axes(A, B, ax_a, ax_b)
    want = oracle.inner_i32(Am, Bm)
    D = empty(want.shape, torch.int32)
    moa.moa_inner_axes("add", "mul", "i32", "native", sa, to_dev(A), ax_a, sb, to_dev(B), ax_b, D, "i32")
    assert np.array_equal(D.cpu().numpy(), want)
    Af, Bf = synth.semiring_inputs("tropical", seed=25, shape_a=sa, shape_b=sb)
    for reduce, combine in (("min", "add"), ("max", "min")):
        want = oracle.inner_f32(reduce, combine, *oracle.move_axes(Af, Bf, ax_a, ax_b))
        D = empty(want.shape, torch.float32)
        moa.moa_inner_axes(reduce, combine, "f32", "native", sa, to_dev(Af), ax_a, sb, to_dev(Bf), ax_b, D, "f32")
        assert np.array_equal(D.cpu().numpy(), want)
    check_status()


@pytest.mark.parametrize("sa,ax_a,sb,ax_b", AXES)
def test_inner_axes_floating_forms(sa, ax_a, sb, ax_b):
    import torch
    sb = _axes_case(sa, ax_a, sb, ax_b)
    A = synth.uniform(26, 0, sa, -1, 1)
    B = synth.uniform(26, 1, sb, -1, 1)
    Am, Bm = oracle.move_axes(A, B, ax_a, ax_b)
    shD = oracle.inner_shape(Am.shape, Bm.shape)
    D = empty(shD, torch.float64)
    moa.moa_inner_axes("add", "mul", "f64", "native", sa, to_dev(A), ax_a, sb, to_dev(B), ax_b, D, "f64")
    assert_norm_err(D.cpu().numpy(), Am, Bm, 1e-12)
    D = empty(shD, torch.float64)
    moa.moa_inner_axes("add", "mul", "f64", "ozaki", sa, to_dev(A), ax_a, sb, to_dev(B), ax_b, D, "f64")
    assert_norm_err(D.cpu().numpy(), Am, Bm, 1e-12)
    A32, B32 = synth.to_f32(A), synth.to_f32(B)
    Am32, Bm32 = oracle.move_axes(A32, B32, ax_a, ax_b)
    D = empty(shD, torch.float32)
    moa.moa_inner_axes("add", "mul", "f32", "bf16x3", sa, to_dev(A32), ax_a, sb, to_dev(B32), ax_b, D, "f32")
    assert_norm_err(D.cpu().numpy(), Am32, Bm32, 2e-6)
    check_status()


def test_inner_axes_without_transpose_is_moa_inner():
    """axisA last and axisB first: the plain call, packed Booleans included."""
    import torch
    A, B = synth.semiring_inputs("bool", seed=27, shape_a=(200, 70), shape_b=(70, 160))
    a = torch.from_numpy(synth.pack_bits(A).view(np.int32)).cuda()
    b = torch.from_numpy(synth.pack_bits(B).view(np.int32)).cuda()
    D = torch.zeros(((200 * 160 + 31) // 32,), dtype=torch.int32, device="cuda")
    moa.moa_inner_axes("or", "and", "b1", "native", A.shape, a, 1, B.shape, b, 0, D, "b1")
    got = np.unpackbits(D.cpu().numpy().view(np.uint8), bitorder="little")[:200 * 160].reshape(200, 160)
    assert np.array_equal(got.astype(bool), oracle.inner_bool(A, B))
    check_status()


def test_inner_axes_full_size_sampled():
    """The bench's configuration: the semiring shapes with the contracted axes
    inside the operands, A <32,512,128> over axis 1 and B <64,64,512> over
    axis 2, (min,+) with 5% +inf; 20,000 outputs sampled."""
    import torch
    A, B = synth.semiring_inputs("tropical")  # <32,128,512> x <512,64,64>
    Am = np.ascontiguousarray(np.moveaxis(A, 2, 1))
    Bm = np.ascontiguousarray(np.moveaxis(B, 0, 2))
    D = empty((32, 128, 64, 64), torch.float32)
    moa.moa_inner_axes("min", "add", "f32", "native", Am.shape, to_dev(Am), 1, Bm.shape, to_dev(Bm), 2, D, "f32")
    idx = sample_idx(D.numel(), 20000)
    got = D.view(-1)[torch.from_numpy(idx).to(D.device)].cpu().numpy()
    want = oracle.inner_f32("min", "add", *oracle.move_axes(Am, Bm, 1, 2), out_idx=idx)
    assert np.array_equal(got, want)
    assert np.array_equal(want, oracle.inner_f32("min", "add", A, B, out_idx=idx))  # the moves undo each other
    check_status()
