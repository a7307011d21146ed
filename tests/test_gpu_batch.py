"""GPU parity of the batched path (many uneven inner / outer products in one
grouped launch inside a CUDA graph) against the oracle, problem by problem:
split-BF16x3 (+,*) within 2e-6 normalised error, (min,+) and outer products
bit-exact.  The first execute tunes and captures, the second replays the
graph; both must give the same results."""
import numpy as np
import pytest

import oracle
import paper_0907_0792_gb300 as moa
import synth
from gpu_helpers import check_status, sample_idx

pytestmark = pytest.mark.gpu


def _build(probs, seed=5):
    import torch
    pool, oa, ob, od, dtot = synth.batched_inputs(probs, seed)
    dpool = torch.from_numpy(pool).cuda()
    dout = torch.full((max(1, dtot),), float("nan"), dtype=torch.float32, device="cuda")
    base, obase = dpool.data_ptr(), dout.data_ptr()
    specs = []
    for p, a, b, d in zip(probs, oa, ob, od):
        if p["kind"] == "outer":
            specs.append(dict(kind="outer", combine="mul", shapeA=p["shapeA"], shapeB=p["shapeB"], A=base + 4 * a,
                              B=base + 4 * b, out=obase + 4 * d))
        elif p["kind"] == "minplus":
            specs.append(dict(kind="inner", reduce="min", combine="add", shapeA=p["shapeA"], shapeB=p["shapeB"],
                              A=base + 4 * a, B=base + 4 * b, out=obase + 4 * d))
        else:
            specs.append(dict(kind="inner", form="bf16x3", shapeA=p["shapeA"], shapeB=p["shapeB"], A=base + 4 * a,
                              B=base + 4 * b, out=obase + 4 * d))
    return pool, oa, ob, od, dpool, dout, specs


def _check(probs, pool, oa, ob, od, out, which, max_out=4096):
    for i in which:
        p = probs[i]
        A = pool[oa[i]:oa[i] + int(np.prod(p["shapeA"]))].reshape(p["shapeA"])
        B = pool[ob[i]:ob[i] + int(np.prod(p["shapeB"]))].reshape(p["shapeB"])
        n = p["M"] * p["N"]
        D = out[od[i]:od[i] + n]
        idx = sample_idx(n, max_out, seed=i)
        if p["kind"] == "outer":
            assert np.array_equal(D[idx], oracle.outer_f("mul", A, B, out="f32", out_idx=idx)), i
        elif p["kind"] == "minplus":
            assert np.array_equal(D[idx], oracle.inner_f32("min", "add", A, B, out_idx=idx)), i
        else:
            ref, S = oracle.inner_dot2(A.astype(np.float64), B.astype(np.float64), out_idx=idx)
            err = oracle.normalised_error(D[idx], ref, S)
            assert err <= 2e-6, (i, err)


def test_batch_small_all_problems():
    import torch
    probs = synth.batched_problems(400, seed=7, mn_octaves=8)
    pool, oa, ob, od, dpool, dout, specs = _build(probs, seed=7)
    arr, keep = moa.make_problems(specs)
    plan = moa.moa_batch_plan_create(arr)
    try:
        info = moa.moa_batch_plan_info(plan)
        # split, grouped, matrix-vector, (min,+) by tile halves
        assert info["problems"] == 400 and info["launches"] <= 3 + 4
        moa.moa_batch_execute(plan)
        torch.cuda.synchronize()
        first = dout.cpu().numpy()
        _check(probs, pool, oa, ob, od, first, range(len(probs)))
        dout.fill_(float("nan"))
        moa.moa_batch_execute(plan)  # graph replay
        torch.cuda.synchronize()
        assert np.array_equal(dout.cpu().numpy(), first, equal_nan=True)
    finally:
        moa.moa_batch_plan_destroy(plan)
    check_status()


def test_batch_full_10000_sampled():
    """The full uneven batch: 10,000 problems, ranks 1-5, M and N up to 2048,
    contraction 8-512; 60 problems checked on up to 4,096 outputs each."""
    import torch
    probs = synth.batched_problems()
    pool, oa, ob, od, dpool, dout, specs = _build(probs)
    arr, keep = moa.make_problems(specs)
    plan = moa.moa_batch_plan_create(arr)
    try:
        moa.moa_batch_execute(plan)
        moa.moa_batch_execute(plan)
        torch.cuda.synchronize()
        out = dout.cpu().numpy()
    finally:
        moa.moa_batch_plan_destroy(plan)
    which = list(sample_idx(len(probs), 60, seed=3))
    kinds = [probs[i]["kind"] for i in which]
    assert "outer" in kinds and "minplus" in kinds and "bf16x3" in kinds
    _check(probs, pool, oa, ob, od, out, which)
    check_status()


@pytest.mark.parametrize("schedule", ["0", "8", "13"])
def test_batch_outer_and_fill_items_every_schedule(schedule, monkeypatch):
    """Outer products and empty contractions (identity fills) beside tensor-core
    and CUDA-core problems, with those items on the grouped kernel's epilogue
    warps (schedules without bit 3) or in the thin-item kernel (with it);
    every output checked."""
    import torch
    monkeypatch.setenv("MOA_BATCH_SCHEDULE", schedule)
    probs = [p for p in synth.batched_problems(200, seed=13, mn_octaves=8)][:120]
    pool, oa, ob, od, dpool, dout, specs = _build(probs, seed=13)
    # two empty contractions: (+,*) fills 0, (min,+) fills +inf
    n_out = dout.numel()
    dfill = torch.full((2 * 35,), float("nan"), dtype=torch.float32, device="cuda")
    specs.append(dict(kind="inner", form="bf16x3", shapeA=(5, 0), shapeB=(0, 7), A=dpool.data_ptr(),
                      B=dpool.data_ptr(), out=dfill.data_ptr()))
    specs.append(dict(kind="inner", reduce="min", combine="add", shapeA=(5, 0), shapeB=(0, 7), A=dpool.data_ptr(),
                      B=dpool.data_ptr(), out=dfill.data_ptr() + 4 * 35))
    arr, keep = moa.make_problems(specs)
    plan = moa.moa_batch_plan_create(arr)
    try:
        moa.moa_batch_execute(plan)
        torch.cuda.synchronize()
        _check(probs, pool, oa, ob, od, dout.cpu().numpy(), range(len(probs)), max_out=1 << 30)
        fills = dfill.cpu().numpy()
        assert np.all(fills[:35] == 0.0) and np.all(fills[35:] == np.inf)
    finally:
        moa.moa_batch_plan_destroy(plan)
    assert n_out > 0
    check_status()


@pytest.mark.parametrize("schedule", ["0", "1", "2", "3", "4", "7"])
def test_batch_tensor_core_tiles_every_schedule(schedule, monkeypatch):
    """Split-BF16x3 tiles under each schedule: ragged M, N and K (K % 32 != 0,
    K < 32, K = 1), M = 1 and N = 1 problems (matrix-vector items with one to
    32 lanes per row and one to 128 columns per item), narrow last column
    tiles, K past one promotion block; every output checked."""
    import torch
    monkeypatch.setenv("MOA_BATCH_SCHEDULE", schedule)
    shapes = [(1, 1, 1), (1, 37, 200), (130, 8, 1), (129, 45, 64), (257, 300, 190), (64, 129, 65), (200, 97, 33),
              (3, 513, 7), (140, 31, 250), (128, 128, 128),
              # matrix-vector items: many column blocks, one-lane and eight-lane rows, a one-column last block
              (1, 512, 2048), (2048, 8, 1), (500, 100, 1), (1, 3, 129), (1, 1000, 33)]
    probs = []
    for M, K, N in shapes:
        probs.append({"kind": "bf16x3", "shapeA": (M, K), "shapeB": (K, N), "M": M, "K": K, "N": N})
    probs += [p for p in synth.batched_problems(120, seed=9, mn_octaves=8) if p["kind"] != "outer"][:60]
    pool, oa, ob, od, dpool, dout, specs = _build(probs, seed=9)
    arr, keep = moa.make_problems(specs)
    plan = moa.moa_batch_plan_create(arr)
    try:
        moa.moa_batch_execute(plan)
        torch.cuda.synchronize()
        _check(probs, pool, oa, ob, od, dout.cpu().numpy(), range(len(probs)), max_out=1 << 30)
    finally:
        moa.moa_batch_plan_destroy(plan)
    check_status()


@pytest.mark.parametrize("schedule", ["0", "1", "2", "3", "4", "7"])
def test_batch_every_cuda_core_operator_and_schedule(schedule, monkeypatch):
    """Every CUDA-core (reduce, combine) of the batch, tiles with one, two or
    four occupied halves and several tiles per problem, and M = 1 / N = 1
    problems (matrix-vector items), under each schedule."""
    import torch
    monkeypatch.setenv("MOA_BATCH_SCHEDULE", schedule)
    ops = [("min", "add", "tropical"), ("max", "add", "tropical"), ("min", "mul", "maxmul"), ("max", "mul", "maxmul"),
           ("add", "mul", "maxmul")]
    shapes = [((40, 33), (33, 50)), ((100, 70), (70, 30)), ((20, 90), (90, 200)), ((300, 17), (17, 140)),
              ((1, 5), (5, 1)), ((1, 300), (300, 70)), ((90, 40), (40, 1))]
    cases, chunks, off = [], [], 0
    for t, (red, comb, kind) in enumerate(ops):
        for u, (sa, sb) in enumerate(shapes):
            A, B = synth.semiring_inputs(kind, seed=40 + 5 * t + u, shape_a=sa, shape_b=sb)
            cases.append((red, comb, A, B, off))
            chunks += [A.ravel(), B.ravel()]
            off += A.size + B.size
    pool = np.concatenate(chunks).astype(np.float32)
    dpool = torch.from_numpy(pool).cuda()
    n_out = sum(c[2].shape[0] * c[3].shape[1] for c in cases)
    dout = torch.full((n_out,), float("nan"), dtype=torch.float32, device="cuda")
    specs, outs, o = [], [], 0
    for red, comb, A, B, a_off in cases:
        base = dpool.data_ptr()
        specs.append(dict(kind="inner", reduce=red, combine=comb, shapeA=A.shape, shapeB=B.shape, A=base + 4 * a_off,
                          B=base + 4 * (a_off + A.size), out=dout.data_ptr() + 4 * o))
        outs.append(o)
        o += A.shape[0] * B.shape[1]
    arr, keep = moa.make_problems(specs)
    plan = moa.moa_batch_plan_create(arr)
    try:
        moa.moa_batch_execute(plan)
        torch.cuda.synchronize()
        got = dout.cpu().numpy()
    finally:
        moa.moa_batch_plan_destroy(plan)
    for (red, comb, A, B, _), o in zip(cases, outs):
        D = got[o:o + A.shape[0] * B.shape[1]].reshape(A.shape[0], B.shape[1])
        if red == "add":
            ref, S = oracle.inner_dot2(A.astype(np.float64), B.astype(np.float64))
            assert oracle.normalised_error(D, ref, S) <= 2e-6, (red, comb, A.shape, B.shape)
        else:
            assert np.array_equal(D, oracle.inner_f32(red, comb, A, B)), (red, comb, A.shape, B.shape)
    check_status()


def test_batch_rejects_bad_problem_and_reports_index():
    import ctypes as C
    specs = [dict(kind="inner", reduce="min", combine="add", shapeA=(4, 5), shapeB=(5, 3), A=0x1000, B=0x2000,
                  out=0x3000)] * 3
    specs = specs + [dict(kind="inner", shapeA=(4, 5), shapeB=(6, 3), A=0x1000, B=0x2000, out=0x3000, form="bf16x3")]
    arr, keep = moa.make_problems(specs)
    plan = C.c_void_p()
    bad = C.c_int(-1)
    st = moa.lib().moa_batch_plan_create(len(arr), arr, C.byref(plan), C.byref(bad))
    assert st == 3 and bad.value == 3 and not plan.value
