"""Host logic of the transpose behind moa_transpose / moa_inner_axes, on the
CPU: the plan (extent-1 axes dropped, adjacent in-order axes merged, input
and output strides, the two axes the kernels walk) must reproduce numpy's
transpose element for element, for random shapes and permutations."""
import itertools
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_0907_0792_gb300", "csrc")


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("plan") / "plan")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "transpose_plan_main.cpp"), "-o", exe],
                   check=True)

    def run(cases):
        text = "".join(f"{len(s)} {' '.join(map(str, s))} {' '.join(map(str, p))}\n" for s, p in cases)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
        assert len(out) == len(cases)
        return out
    return run


def _cases():
    rnd = random.Random(7)
    cases = [((), ()), ((5,), (0,)), ((1, 1, 1), (2, 0, 1)), ((3, 4), (1, 0)), ((2, 0, 3), (2, 0, 1)),
             ((2, 3, 4, 5), (0, 1, 2, 3)), ((2, 3, 4, 5), (1, 0, 2, 3)), ((2, 3, 4, 5), (3, 2, 1, 0)),
             ((2, 1, 33, 1, 40), (4, 3, 2, 1, 0)), ((2, 3, 2, 3, 2, 3, 2, 3), (7, 0, 6, 1, 5, 2, 4, 3))]
    for _ in range(400):
        r = rnd.randint(1, 6)
        shape = tuple(rnd.choice([1, 1, 2, 3, 4, 5]) for _ in range(r))
        perm = list(range(r))
        rnd.shuffle(perm)
        cases.append((shape, tuple(perm)))
    return cases


def test_plan_reproduces_numpy_transpose(planner):
    cases = _cases()
    for (shape, perm), line in zip(cases, planner(cases)):
        f = line.split()
        total, n, xin, yout, rows = map(int, f[:5])
        ext = [int(v) for v in f[5::3]]
        ist = [int(v) for v in f[6::3]]
        ost = [int(v) for v in f[7::3]]
        assert total == int(np.prod(shape, dtype=np.int64))
        if total == 0:
            continue
        assert n == len(ext) <= len(shape) and int(np.prod(ext, dtype=np.int64)) == total
        x = np.arange(total).reshape(shape)
        want = np.transpose(x, perm).ravel()
        if n <= 1:  # a plain copy
            assert np.array_equal(want, x.ravel()), (shape, perm)
            continue
        assert ist[xin] == 1 and ost[yout] == 1 and rows == (xin == yout)
        got = np.full(total, -1)
        src = x.ravel()
        for idx in itertools.product(*[range(e) for e in ext]):
            got[sum(i * s for i, s in zip(idx, ost))] = src[sum(i * s for i, s in zip(idx, ist))]
        assert np.array_equal(got, want), (shape, perm)


def test_plan_merges_what_stays_in_order(planner):
    """Axes that keep their input order collapse to one axis: an identity
    permutation is a plain copy; swapping two outer axes leaves three merged
    axes with the innermost kept (rows); moving the innermost axis makes
    tiles."""
    out = planner([((4, 5, 6, 7), (0, 1, 2, 3)), ((4, 5, 6, 7), (1, 0, 2, 3)), ((4, 5, 6, 7), (0, 1, 3, 2)),
                   ((4, 5, 6, 7), (0, 1, 2, 3)[::-1])])
    n = [int(l.split()[1]) for l in out]
    rows = [int(l.split()[4]) for l in out]
    assert n == [1, 3, 3, 4]
    assert rows[1] == 1 and rows[2] == 0 and rows[3] == 0
