"""Pins for the CPU oracle: each check compares it with something other than
itself — a library routine, exact rational arithmetic, a closed form, a
hand-computed fixture, or a second formulation of the same definition.

Eq. (1) (outer product) and Eq. (2) (inner product) of Sec. I define what is
checked; the Fig. 1 example fixes the shape rule.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _num(v):
    return {"inf": np.inf, "-inf": -np.inf}.get(v, v) if isinstance(v, str) else v


# ------------------------------------------------------------------ shapes
def test_shape_rule_fig1_example():
    # Fig. 1: rho A = <2 3>, rho B = <3 4>; the inner product is 2 x 4.
    assert oracle.inner_shape((2, 3), (3, 4)) == (2, 4)
    # Eq. (2) index list: D_{ijklm} from A_{ijkp}, B_{plm}.
    assert oracle.inner_shape(synth.C1_SHAPE_A, synth.C1_SHAPE_B) == (16, 12, 8, 24, 20)
    assert oracle.inner_shape((32, 128, 512), (512, 64, 64)) == (32, 128, 64, 64)
    # Eq. (1) index list: C_{ijkpqlm} from A_{ijkp}, B_{qlm}.
    assert oracle.outer_shape((16, 12, 8, 64), (4, 5)) == (16, 12, 8, 64, 4, 5)
    with pytest.raises(ValueError):
        oracle.inner_shape((2, 3), (4, 3))


# ------------------------------------------------------------------ (+,*)
@pytest.mark.parametrize("sa,sb", [((2, 3), (3, 4)), ((3, 4, 5, 7), (7, 2, 6)), ((9,), (9,)), ((5, 1), (1, 3)),
                                   ((4, 3, 33), (33, 5))])
def test_dot2_matches_tensordot(sa, sb):
    """Eq. (2) for (+,*) is numpy's tensordot over one axis (library special case)."""
    A = synth.uniform(7, 0, sa, -1, 1)
    B = synth.uniform(7, 1, sb, -1, 1)
    D, S = oracle.inner_dot2(A, B)
    R = np.tensordot(A, B, axes=1)
    assert D.shape == R.shape
    k = sa[-1]
    assert np.all(np.abs(D - R) <= 2 * k * U64 * S + 1e-300)


def test_dot2_matches_matmul_square():
    A, B = synth.square(40, "loguniform", seed=9)
    D, S = oracle.inner_dot2(A, B)
    assert np.all(np.abs(D - A @ B) <= 2 * 40 * U64 * S)


def test_dot2_against_exact_rationals():
    """Dot2 is within one rounding of the exact sum, checked with Fractions on
    ill-conditioned dot products where plain summation loses every digit."""
    small_a = synth.log_uniform_signed(11, 0, (6, 24), -30, -10)
    small_b = synth.log_uniform_signed(11, 1, (24, 5), -3, 3)
    big_a = synth.log_uniform_signed(11, 2, (6, 1), 28, 30)
    big_b = synth.log_uniform_signed(11, 3, (1, 5), -3, 3)
    # the first and last products cancel exactly, leaving only the small terms
    A = np.concatenate([big_a, small_a, -big_a], axis=1)
    B = np.concatenate([big_b, small_b, big_b], axis=0)
    D, S = oracle.inner_dot2(A, B)
    plain_fail = 0
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[:, j]))
            ex = float(exact)
            assert abs(Fraction(float(D[i, j])) - exact) <= Fraction(U64) * abs(exact) + Fraction(1e-25) * Fraction(S[i, j])
            if abs(float(np.dot(A[i], B[:, j])) - ex) > 1e-3 * abs(ex):
                plain_fail += 1
    assert plain_fail > 0  # the inputs really are ill-conditioned


def test_identity_and_ones_operands():
    A = synth.uniform(5, 0, (6, 7, 9), -1, 1)
    D, _ = oracle.inner_dot2(A, np.eye(9))
    assert np.array_equal(D, A)  # A . I = A exactly
    Dr, _ = oracle.inner_dot2(A, np.ones((9, 1)))
    rows = np.array([[math.fsum(A[i, j]) for j in range(7)] for i in range(6)])
    assert np.array_equal(Dr[..., 0], rows)  # A . 1 = correctly rounded row sums


def test_inner_equals_reduced_outer_f64():
    """Sec. I: the inner product is the outer product reduced along the matched
    axes: D[i,j] = sum_p C[i,p,p,j] with C = A (x) B."""
    A = synth.uniform(6, 0, (3, 2, 5), -1, 1)
    B = synth.uniform(6, 1, (5, 4), -1, 1)
    Cm = oracle.outer_f("mul", A, B)  # shape (3,2,5,5,4)
    diag = np.einsum("ijppk->ijpk", Cm)
    D, S = oracle.inner_dot2(A, B)
    ref = np.array([[[math.fsum(diag[i, j, :, k]) for k in range(4)] for j in range(2)] for i in range(3)])
    assert np.all(np.abs(D - ref) <= 5 * U64 * S)


# -------------------------------------------------------------- semirings
@pytest.mark.parametrize("reduce,combine,kind", [("min", "add", "tropical"), ("max", "add", "tropical"),
                                                 ("max", "mul", "maxmul"), ("min", "add", "tropical_finite")])
def test_f32_semiring_matches_numpy_broadcast(reduce, combine, kind):
    A, B = synth.semiring_inputs(kind, seed=12, shape_a=(3, 7, 37), shape_b=(37, 2, 9))
    D = oracle.inner_f32(reduce, combine, A, B)
    a2, b2 = A.reshape(-1, 37), B.reshape(37, -1)
    t = (a2[:, :, None] + b2[None]) if combine == "add" else (a2[:, :, None] * b2[None])
    assert t.dtype == np.float32
    R = (t.min(axis=1) if reduce == "min" else t.max(axis=1)).reshape(D.shape)
    assert np.array_equal(D, R)


def test_i32_matches_numpy_with_wraparound():
    A, B = synth.semiring_inputs("int32", seed=13, shape_a=(5, 4, 19), shape_b=(19, 6))
    D = oracle.inner_i32(A, B)
    R = np.tensordot(A.astype(np.int64), B.astype(np.int64), axes=1)
    assert np.array_equal(D, R.astype(np.int32))
    # large values: the products and sums wrap modulo 2^32
    A = synth.int_uniform(14, 0, (4, 23), -(2 ** 31), 2 ** 31 - 1)
    B = synth.int_uniform(14, 1, (23, 3), -(2 ** 31), 2 ** 31 - 1)
    D = oracle.inner_i32(A, B)
    R = np.array([[sum(int(a) * int(b) for a, b in zip(A[i], B[:, j])) for j in range(3)] for i in range(4)])
    R = ((R + 2 ** 31) % 2 ** 32 - 2 ** 31).astype(np.int64)
    assert np.array_equal(D.astype(np.int64), R)
    assert np.any(np.abs(R) > 0) and np.max(np.abs(np.abs(R) - 2 ** 30)) < 2 ** 31


def test_bool_matches_counting_matmul():
    A, B = synth.semiring_inputs("bool", seed=15, shape_a=(4, 8, 70), shape_b=(70, 3, 11))
    D = oracle.inner_bool(A, B)
    R = np.tensordot(A.astype(np.int64), B.astype(np.int64), axes=1) > 0
    assert np.array_equal(D, R)


def test_inner_equals_reduced_outer_exact_semirings():
    """The outer/inner identity of Sec. I, bit-exact for min/max and integers."""
    A, B = synth.semiring_inputs("tropical", seed=16, shape_a=(3, 11), shape_b=(11, 2, 3))
    C = oracle.outer_f("add", A.astype(np.float64), B.astype(np.float64), out="f32")  # (3,11,11,2,3)
    diag = np.einsum("ippjk->ipjk", C)
    assert np.array_equal(oracle.inner_f32("min", "add", A, B), diag.min(axis=1))
    assert np.array_equal(oracle.inner_f32("max", "add", A, B), diag.max(axis=1))
    Ai, Bi = synth.semiring_inputs("int32", seed=16, shape_a=(3, 11), shape_b=(11, 2, 3))
    Ci = oracle.outer_i32("mul", Ai, Bi)
    di = np.einsum("ippjk->ipjk", Ci).astype(np.int64).sum(axis=1)
    assert np.array_equal(oracle.inner_i32(Ai, Bi), di.astype(np.int32))


def test_rowwise_agrees_with_definition():
    """The appendix-order loop and the psi-index definition loop are two
    formulations of Eq. (2); they agree bit for bit where the result is exact."""
    A, B = synth.semiring_inputs("tropical", seed=17, shape_a=(3, 5, 29), shape_b=(29, 4, 3))
    for red in ("min", "max"):
        assert np.array_equal(oracle.rowwise("f32", A, B, red, "add", threads=3), oracle.inner_f32(red, "add", A, B))
    Am, Bm = synth.semiring_inputs("maxmul", seed=17, shape_a=(6, 29), shape_b=(29, 7))
    assert np.array_equal(oracle.rowwise("f32", Am, Bm, "max", "mul"), oracle.inner_f32("max", "mul", Am, Bm))
    Ai, Bi = synth.semiring_inputs("int32", seed=17, shape_a=(3, 5, 29), shape_b=(29, 4, 3))
    assert np.array_equal(oracle.rowwise("i32", Ai, Bi, threads=2), oracle.inner_i32(Ai, Bi))
    Ab, Bb = synth.semiring_inputs("bool", seed=17, shape_a=(3, 5, 29), shape_b=(29, 4, 3))
    assert np.array_equal(oracle.rowwise("bool", Ab, Bb, "or", "and"), oracle.inner_bool(Ab, Bb))
    A64 = synth.uniform(17, 5, (4, 6, 31), -1, 1)
    B64 = synth.uniform(17, 6, (31, 5), -1, 1)
    D, S = oracle.inner_dot2(A64, B64)
    assert np.all(np.abs(oracle.rowwise("f64", A64, B64, threads=4) - D) <= 31 * U64 * S)


@pytest.mark.parametrize("reduce", ["min", "max"])
@pytest.mark.parametrize("combine", ["add", "sub", "mul", "min", "max"])
def test_rowwise_agrees_with_definition_every_fp32_pair(reduce, combine):
    """The appendix-order loop and the definition loop, bit for bit, for
    every FP32 (reduce, combine) the library supports."""
    kind = "tropical_finite" if combine == "sub" else "tropical"
    A, B = synth.semiring_inputs(kind, seed=24, shape_a=(3, 4, 27), shape_b=(27, 5, 2))
    assert np.array_equal(oracle.rowwise("f32", A, B, reduce, combine, threads=2),
                          oracle.inner_f32(reduce, combine, A, B))


def _closure(semiring, w, squarings=3):
    red, comb = semiring
    x = w
    for _ in range(squarings):
        if red == "or":
            x = oracle.inner_bool(x, x)
        else:
            x = oracle.inner_f32(red, comb, x, x)
    return x


@pytest.mark.parametrize("name", ["minplus_apsp", "maxplus_dag_longest", "maxmul_reliability", "maxmin_widest",
                                  "minmax_minimax", "orand_reachability"])
def test_path_closures_hand_computed(name):
    g = _gold("semiring_paths.json")[name]
    if g["semiring"][0] == "or":
        w = np.array(g["w"], dtype=bool)
        want = np.array(g["closure"], dtype=bool)
    else:
        w = np.array([[_num(v) for v in r] for r in g["w"]], dtype=np.float32)
        want = np.array([[_num(v) for v in r] for r in g["closure"]], dtype=np.float32)
    got = _closure(g["semiring"], w)
    assert np.array_equal(got, want), got


def test_minmax_combines_on_booleans_reduce_to_or_and():
    """On {0, 1} values (max, min) is (or, and), and (min, max) is its De
    Morgan dual: min_p max(a, b) = not or_p (not a and not b)."""
    Ab, Bb = synth.semiring_inputs("bool", seed=20, shape_a=(4, 3, 45), shape_b=(45, 7))
    Ab = Ab | synth.bernoulli(20, 9, Ab.shape, 0.3)  # denser, so that both outcomes occur
    A, B = Ab.astype(np.float32), Bb.astype(np.float32)
    ref = oracle.inner_bool(Ab, Bb)
    assert ref.any() and not ref.all()
    assert np.array_equal(oracle.inner_f32("max", "min", A, B), ref.astype(np.float32))
    dual = ~oracle.inner_bool(~Ab, ~Bb)
    assert np.array_equal(oracle.inner_f32("min", "max", A, B), dual.astype(np.float32))


def test_sub_combine_is_add_of_the_negation():
    """a - b and a + (-b) are the same IEEE operation, so (min|max, -) with B
    equals (min|max, +) with -B bit for bit."""
    A, B = synth.semiring_inputs("tropical_finite", seed=21, shape_a=(5, 33), shape_b=(33, 6))
    for red in ("min", "max"):
        assert np.array_equal(oracle.inner_f32(red, "sub", A, B), oracle.inner_f32(red, "add", A, -B))


def test_idempotent_combines_against_closed_forms():
    """(max, max) and (min, min) split into reductions of each operand:
    max_p max(a, b) = max(max_p a, max_p b); (max, min) with a constant row
    of A is that constant capped by each column maximum of B."""
    A, B = synth.semiring_inputs("tropical", seed=22, shape_a=(6, 40), shape_b=(40, 5))
    want = np.maximum(A.max(axis=1)[:, None], B.max(axis=0)[None, :])
    assert np.array_equal(oracle.inner_f32("max", "max", A, B), want)
    want = np.minimum(A.min(axis=1)[:, None], B.min(axis=0)[None, :])
    assert np.array_equal(oracle.inner_f32("min", "min", A, B), want)
    c = np.float32(37.5)
    got = oracle.inner_f32("max", "min", np.full((2, 40), c, np.float32), B)
    assert np.array_equal(got, np.minimum(c, B.max(axis=0))[None, :].repeat(2, axis=0))


@pytest.mark.parametrize("sa,sb,ax_a,ax_b", [((4, 9, 3), (5, 9, 2), 1, 1), ((7, 2, 3), (3, 4), 0, 1),
                                              ((6,), (2, 6, 3), 0, 1), ((3, 5), (5, 2), 1, 0)])
def test_move_axes_matches_tensordot(sa, sb, ax_a, ax_b):
    """Contraction over arbitrary axes: move_axes then the definition equals
    numpy's tensordot over the same pair of axes (exact for integers)."""
    sb = list(sb)
    sb[ax_b] = sa[ax_a]  # the contracted axes have equal length
    A = synth.int_uniform(23, 0, sa, -1000, 1000)
    B = synth.int_uniform(23, 1, tuple(sb), -1000, 1000)
    D = oracle.inner_i32(*oracle.move_axes(A, B, ax_a, ax_b))
    R = np.tensordot(A.astype(np.int64), B.astype(np.int64), axes=([ax_a], [ax_b]))
    assert D.shape == R.shape and np.array_equal(D, R.astype(np.int32))


def test_tropical_identity_operand():
    A = synth.semiring_inputs("tropical", seed=18, shape_a=(5, 8), shape_b=(8, 2))[0]
    E = np.full((8, 8), np.inf, dtype=np.float32)
    np.fill_diagonal(E, 0)
    assert np.array_equal(oracle.inner_f32("min", "add", A, E), A)
    Ab = synth.semiring_inputs("bool", seed=18, shape_a=(5, 8), shape_b=(8, 2))[0]
    assert np.array_equal(oracle.inner_bool(Ab, np.eye(8, dtype=bool)), Ab)
    Ai = synth.int_uniform(18, 3, (5, 8), -1000, 1000)
    assert np.array_equal(oracle.inner_i32(Ai, np.eye(8, dtype=np.int32)), Ai)


def test_empty_contraction_gives_identity():
    A = np.zeros((3, 0), dtype=np.float32)
    B = np.zeros((0, 4), dtype=np.float32)
    assert np.all(oracle.inner_f32("min", "add", A, B) == np.inf)
    assert np.all(oracle.inner_f32("max", "add", A, B) == -np.inf)
    D, S = oracle.inner_dot2(A, B)
    assert np.all(D == 0) and np.all(S == 0)
    assert not oracle.inner_bool(A.astype(bool), B.astype(bool)).any()


def test_sampled_outputs_match_full():
    A, B = synth.semiring_inputs("tropical", seed=19, shape_a=(4, 6, 13), shape_b=(13, 5, 2))
    full = oracle.inner_f32("min", "add", A, B)
    idx = np.array([0, 7, 239, 100, 3], dtype=np.int64)
    assert np.array_equal(oracle.inner_f32("min", "add", A, B, out_idx=idx), full.ravel()[idx])
    A64, B64 = synth.rank4x3_f64()
    D, S = oracle.inner_dot2(A64, B64, out_idx=idx * 150)
    Df, Sf = oracle.inner_dot2(A64[:1], B64)  # the first 46,080 outputs cover these offsets
    assert np.array_equal(D, Df.ravel()[idx * 150])


# ------------------------------------------------------------------ outer
@pytest.mark.parametrize("op,uf", [("mul", np.multiply), ("add", np.add), ("sub", np.subtract), ("div", np.divide),
                                   ("min", np.minimum), ("max", np.maximum)])
def test_outer_matches_numpy_ufunc_outer(op, uf):
    A, B = synth.outer_inputs(op, "f64", shape_a=(3, 4, 5), shape_b=(2, 7))
    assert np.array_equal(oracle.outer_f(op, A, B), uf.outer(A, B))
    A32, B32 = synth.outer_inputs(op, "f32", shape_a=(3, 4, 5), shape_b=(2, 7))
    got = oracle.outer_f(op, A32, B32, out="f32")
    assert np.array_equal(got, uf.outer(A32, B32))  # numpy float32 ops are IEEE RNE
    torch = pytest.importorskip("torch")
    (ab, av), (bb, bv) = synth.outer_inputs(op, "bf16", shape_a=(3, 4, 5), shape_b=(2, 7))
    gb = oracle.outer_f(op, av, bv, out="bf16")
    ta = torch.from_numpy(av.astype(np.float32))
    tb = torch.from_numpy(bv.astype(np.float32))
    t = {"mul": torch.mul, "add": torch.add, "sub": torch.sub, "div": torch.div, "min": torch.minimum,
         "max": torch.maximum}[op]
    ref = t(ta.reshape(3, 4, 5, 1, 1), tb.reshape(1, 1, 1, 2, 7)).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(gb.view(np.int16), ref)


def _wrap32(x):
    """int64 values reduced to int32 two's complement (modulo 2^32)."""
    x = np.asarray(x, dtype=np.int64) % 2 ** 32
    return np.where(x >= 2 ** 31, x - 2 ** 32, x).astype(np.int32)


@pytest.mark.parametrize("op,uf", [("add", np.add), ("sub", np.subtract), ("mul", np.multiply)])
def test_outer_i32_and_rank0(op, uf):
    """Eq. (1) over int32 for every operator: numpy's ufunc.outer in int64,
    reduced modulo 2^32, on ordinary and on wrapping operands (sub is
    A - B, not B - A)."""
    A, B = synth.outer_inputs("mul", "i32", shape_a=(4, 3), shape_b=(5,))
    assert np.array_equal(oracle.outer_i32(op, A, B), _wrap32(uf.outer(A.astype(np.int64), B.astype(np.int64))))
    big = np.array([2 ** 31 - 1, -(2 ** 31), -1, 7], dtype=np.int32)
    small = np.array([1, -2, 2 ** 30], dtype=np.int32)
    assert np.array_equal(oracle.outer_i32(op, big, small),
                          _wrap32(uf.outer(big.astype(np.int64), small.astype(np.int64))))
    assert np.array_equal(oracle.outer_i32(op, big, big), _wrap32(uf.outer(big.astype(np.int64), big.astype(np.int64))))
    # one element by hand: 2^31 - 1 + 1 wraps to -2^31; -2^31 - 1 wraps to 2^31 - 1; 3 - 5 = -2
    assert oracle.outer_i32("add", big[:1], small[:1])[0, 0] == -(2 ** 31)
    assert oracle.outer_i32("sub", big[1:2], small[:1])[0, 0] == 2 ** 31 - 1
    assert oracle.outer_i32("sub", np.array([3], np.int32), np.array([5], np.int32))[0, 0] == -2
    # rank 0 operand: rho C = rho B
    s = np.array(3.0)
    assert np.array_equal(oracle.outer_f("mul", s, np.arange(4.0)), 3.0 * np.arange(4.0))


def test_outer_sampled():
    A, B = synth.outer_inputs("div", "f32")  # the full 128x64x32 (x) 32x64 shapes
    idx = synth.int_uniform(1, 1, (50,), 0, A.size * B.size - 1).astype(np.int64)
    got = oracle.outer_f("div", A, B, out="f32", out_idx=idx)
    ia, ib = np.divmod(idx, B.size)
    assert np.array_equal(got, (A.ravel()[ia] / B.ravel()[ib]).astype(np.float32))


def test_normalised_error_measure():
    assert oracle.normalised_error([1.0, 2.0], [1.0, 2.5], [1.0, 5.0]) == 0.1
    assert oracle.normalised_error([0.0], [0.0], [0.0]) == 0.0
    assert oracle.normalised_error([1e-300], [0.0], [0.0]) == float("inf")
