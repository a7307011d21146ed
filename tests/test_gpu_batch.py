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
        assert info["problems"] == 400 and info["launches"] <= 2
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
