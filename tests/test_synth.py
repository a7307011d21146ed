"""The seeded input generators: published test vectors, determinism, the
stated distributions, the bf16 rounding and the bit-packing layout."""
import numpy as np
import pytest

import synth


def test_splitmix64_published_vector():
    # SplitMix64 with state 1234567: the first five outputs of the reference C
    # implementation (Vigna, splitmix64.c).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    with np.errstate(over="ignore"):
        got = [int(synth._mix(np.uint64(1234567) + np.uint64(i + 1) * synth.GAMMA)) for i in range(5)]
    assert got == want


def test_streams_are_deterministic_and_sliceable():
    a = synth.u64(5, 3, 1000)
    assert np.array_equal(a, synth.u64(5, 3, 1000))
    assert np.array_equal(a[400:700], synth.u64(5, 3, 300, offset=400))
    assert not np.array_equal(a, synth.u64(5, 4, 1000))
    assert not np.array_equal(a, synth.u64(6, 3, 1000))


def test_distributions():
    u = synth.uniform(1, 0, (200000,), -1, 1)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.01
    t, _ = synth.semiring_inputs("tropical", shape_a=(64, 512), shape_b=(512, 8))
    frac = np.isinf(t).mean()
    assert 0.04 < frac < 0.06 and np.nanmin(t) >= 0 and t[np.isfinite(t)].max() < 100
    i, _ = synth.semiring_inputs("int32", shape_a=(64, 512), shape_b=(512, 8))
    assert i.min() == -128 and i.max() == 127
    lg = synth.log_uniform_signed(2, 0, (100000,))
    m = np.abs(lg)
    assert m.min() >= 2.0 ** -13 and m.max() < 2.0 ** 13
    assert 0.45 < (lg < 0).mean() < 0.55
    _, b = synth.outer_inputs("div", "f32")
    assert np.abs(b).min() >= np.float32(0.1)
    bb, _ = synth.semiring_inputs("bool", shape_a=(64, 512), shape_b=(512, 8))
    assert 0.04 < bb.mean() < 0.06


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([synth.uniform(3, 0, (5000,), -1, 1), synth.log_uniform_signed(3, 1, (5000,), -120, 120),
                        np.array([0.0, -0.0, np.inf, -np.inf, 1.00390625, 1.01171875])]).astype(np.float32)
    ours = synth.f32_to_bf16_bits(x).view(np.int16)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(ours, ref)


def test_bit_packing_layout():
    x = np.zeros((3, 40), dtype=bool)
    x[0, 0] = x[0, 33] = x[2, 39] = True  # elements 0, 33, 119
    w = synth.pack_bits(x)
    assert w.dtype == np.uint32 and w.size == 4
    assert w[0] == 1 and w[1] == 2 and w[2] == 0 and w[3] == (1 << (119 - 96))
    y = synth.semiring_inputs("bool", shape_a=(7, 96), shape_b=(96, 3))[0]
    assert np.array_equal(synth.unpack_bits(synth.pack_bits(y), y.size).reshape(y.shape), y)


def test_positional_and_torch_draws_match_the_stream():
    """uniform_at (any positions) and device_uniform (torch integer ops, here
    on the CPU) reproduce uniform() exactly, including across chunk edges."""
    import torch
    a = synth.uniform(6, 1, (16, 1000), -1.0, 1.0)
    idx = np.array([0, 1, 999, 1000, 15999, 7777], dtype=np.int64)
    assert np.array_equal(synth.uniform_at(6, 1, idx, -1.0, 1.0), a.ravel()[idx])
    b = synth.device_uniform(6, 1, (16, 1000), -1.0, 1.0, "cpu", chunk=333).numpy()
    assert np.array_equal(a, b)
    b32 = synth.device_uniform(6, 1, (16, 1000), -1.0, 1.0, "cpu", dtype=torch.float32).numpy()
    assert np.array_equal(synth.to_f32(a), b32)
    cols = synth.skinny_columns([3, 500, 999], 1000, k=16)
    assert np.array_equal(cols, a[:, [3, 500, 999]])


def test_batched_workload_matches_its_recipe():
    """The 10,000-problem batch: kinds in the stated mix, ranks 1..5 per
    operand, contraction 8..512, flattened M and N within 1..2048 and equal to
    the products of the shape vectors (rho of the operands), octave-uniform
    sizes (each octave of M holds a similar share)."""
    probs = synth.batched_problems()
    assert len(probs) == 10000
    kinds = [p["kind"] for p in probs]
    share = {k: kinds.count(k) / len(kinds) for k in ("bf16x3", "minplus", "outer")}
    assert abs(share["bf16x3"] - 0.7) < 0.02 and abs(share["minplus"] - 0.2) < 0.02 and abs(share["outer"] - 0.1) < 0.02
    octaves = np.zeros(12)
    for p in probs:
        sa, sb = p["shapeA"], p["shapeB"]
        assert 1 <= len(sa) <= 5 and 1 <= len(sb) <= 5 and all(e >= 1 for e in sa + sb)
        if p["kind"] == "outer":
            assert int(np.prod(sa)) == p["M"] and int(np.prod(sb)) == p["N"] and p["K"] == 0
        else:
            assert sa[-1] == sb[0] == p["K"] and 8 <= p["K"] <= 512
            assert int(np.prod(sa[:-1])) == p["M"] and int(np.prod(sb[1:])) == p["N"]
        assert 1 <= p["M"] <= 2048 and 1 <= p["N"] <= 2048
        if p["kind"] == "outer" or len(sa) > 1:
            octaves[int(np.log2(p["M"]))] += 1
    share = octaves[:11] / octaves[:11].sum()
    # about 1/11 per octave; rounding 2^0 (1 + f) sends half of the first octave to M = 2
    assert 0.07 < share[1:].min() and share[1:].max() < 0.13 and 0.02 < share[0] < 0.08



def test_square_leading_is_the_leading_block():
    """The sweep's smaller sizes are the leading blocks of the largest case's
    operands, drawn positionally."""
    for dist in ("uniform", "loguniform"):
        A, B = synth.square(512, dist)
        a, b = synth.square_leading(64, dist, n_full=512)
        assert np.array_equal(a, A[:64, :64]) and np.array_equal(b, B[:64, :64])
        a, b = synth.square_leading(512, dist, n_full=512)
        assert np.array_equal(a, A) and np.array_equal(b, B)


def test_f16_rounding_and_e4m3_table():
    """fp16 rounding is numpy's binary16 conversion (a library routine) and
    keeps its range ends; the E4M3 decode table written from the format's
    definition agrees with torch's float8_e4m3fn for every code, and with
    values worked by hand."""
    bits, vals = synth.to_f16(np.array([1.0, 65504.0, 2.0 ** -24, 1.0 + 2.0 ** -11, -0.1]))
    assert list(bits[:3]) == [0x3C00, 0x7BFF, 0x0001] and vals[3] == 1.0  # a tie rounds to even
    assert vals[4] == np.float64(np.float16(-0.1))
    t = synth.e4m3_decode_table()
    assert t[0x00] == 0.0 and t[0x38] == 1.0 and t[0xB8] == -1.0 and t[0x7E] == 448.0 and t[0x01] == 2.0 ** -9
    assert t[0x08] == 2.0 ** -6 and np.isnan(t[0x7F]) and np.isnan(t[0xFF]) and t[0x77] == 240.0
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    ref = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(t, ref, equal_nan=True)
    codes, vals = synth.e4m3_codes(3, 0, (1000,), max_exp=9)
    assert not np.isnan(vals).any() and np.abs(vals).max() <= 2.0 ** 3 * 1.875
    assert np.array_equal(vals, t[codes])
