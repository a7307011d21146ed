"""The C ABI library without a GPU: it loads, exports every function that
include/moa.h declares, and its host-side validation rejects bad calls
before any launch (these calls never reach CUDA)."""
import ctypes as C
import os
import re

import pytest

import paper_0907_0792_gb300 as moa
from paper_0907_0792_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return moa.lib()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(moa_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(L):
    names = _declared()
    assert "moa_inner" in names and "moa_outer" in names and len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_inner_shape_fig1_example(L):
    assert moa.moa_inner_shape((2, 3), (3, 4)) == (2, 4)
    assert moa.moa_inner_shape((16, 12, 8, 64), (64, 24, 20)) == (16, 12, 8, 24, 20)
    assert moa.moa_outer_shape((16, 12, 8, 64), (4, 5)) == (16, 12, 8, 64, 4, 5)
    assert moa.moa_outer_shape((), (3,)) == (3,)
    with pytest.raises(moa.MoaError) as e:
        moa.moa_inner_shape((2, 3), (4, 3))
    assert e.value.status == 3


def _inner_status(reduce, combine, dtype, form, sa, sb, out_dtype, A=0x1000, B=0x2000, out=0x3000):
    return moa.moa_inner(reduce, combine, dtype, form, sa, A, sb, B, out, out_dtype, stream=0, check=False)


def test_validation_before_launch(L):
    # shape mismatch (Eq. 2 needs rho A[-1] == rho B[0])
    assert _inner_status("add", "mul", "f64", "native", (4, 5), (6, 7), "f64") == 3
    # ranks
    assert _inner_status("add", "mul", "f64", "native", (), (6, 7), "f64") == 2
    assert _inner_status("add", "mul", "f64", "native", (1,) * 9, (1, 2), "f64") == 2
    # unsupported tuples
    assert _inner_status("add", "mul", "f64", "bf16x3", (4, 5), (5, 7), "f64") == 5
    assert _inner_status("min", "add", "f64", "native", (4, 5), (5, 7), "f64") == 5
    assert _inner_status("or", "and", "f32", "native", (4, 5), (5, 7), "f32") == 5
    assert _inner_status("add", "mul", "i32", "native", (4, 5), (5, 7), "f32") == 5
    assert _inner_status("min", "div", "f32", "native", (4, 5), (5, 7), "f32") == 5
    assert _inner_status("add", "min", "f32", "native", (4, 5), (5, 7), "f32") == 5
    # negative extent, overflow
    assert _inner_status("add", "mul", "f32", "native", (-1, 5), (5, 7), "f32") == 4
    assert _inner_status("add", "mul", "f32", "native", (2 ** 40, 5), (5, 2 ** 40), "f32") == 4
    # null pointers
    assert _inner_status("add", "mul", "f32", "native", (4, 5), (5, 7), "f32", out=0) == 1
    assert _inner_status("add", "mul", "f32", "native", (4, 5), (5, 7), "f32", A=0) == 1
    # misaligned
    assert _inner_status("add", "mul", "f64", "native", (4, 5), (5, 7), "f64", A=0x1004) == 10
    # bad enum
    assert _inner_status(99, "mul", "f32", "native", (4, 5), (5, 7), "f32") == 11
    # empty result: a no-op that succeeds without touching the device
    assert _inner_status("add", "mul", "f32", "native", (0, 5), (5, 7), "f32", A=0, out=0) == 0


def test_operands_must_be_device_memory(L):
    """A well-formed call whose A, B or out is not memory of the current
    device (here: host memory, with no GPU at all) is rejected before any
    launch with MOA_ERR_NOT_DEVICE, for every entry point that reads caller
    memory; a call that touches no memory still succeeds."""
    import numpy as np
    a = np.zeros((4, 5), np.float32)
    b = np.zeros((5, 7), np.float32)
    d = np.zeros((4, 7), np.float32)
    pa, pb, pd = a.ctypes.data, b.ctypes.data, d.ctypes.data
    assert _inner_status("add", "mul", "f32", "native", (4, 5), (5, 7), "f32", A=pa, B=pb, out=pd) == 13
    assert _inner_status("min", "add", "f32", "native", (4, 5), (5, 7), "f32", A=pa, B=pb, out=pd) == 13
    assert moa.moa_outer("mul", "f32", (4, 5), pa, (5, 7), pb, np.zeros(4 * 5 * 5 * 7, np.float32).ctypes.data,
                         "f32", stream=0, check=False) == 13
    assert moa.moa_transpose("f32", (4, 5), pa, (1, 0), pd, stream=0, check=False) == 13
    assert moa.moa_inner_bf16x3_noalloc((4, 5), pa, (5, 7), pb, pd, stream=0, check=False) == 13
    # empty contraction on host memory: out is still written, so it is still rejected
    assert _inner_status("add", "mul", "f32", "native", (4, 0), (0, 7), "f32", A=0, B=0, out=pd) == 13
    assert moa.moa_status_string(13) == "pointer is not device memory of the current device"


def test_axes_and_transpose_validation(L):
    def ax(sa, a, sb, b, dt="f32", A=0x1000, B=0x2000, out=0x3000):
        return moa.moa_inner_axes("add", "mul", dt, "native", sa, A, a, sb, B, b, out, dt, stream=0, check=False)
    assert ax((4, 5), 2, (5, 7), 0) == 11  # axis out of range
    assert ax((4, 5), 0, (5, 7), -1) == 11
    assert ax((4, 5), 0, (5, 7), 0) == 3  # contracted lengths 4 and 5 differ
    assert ax((0, 5), 1, (5, 7), 0, A=0, out=0) == 0  # empty result
    assert moa.moa_inner_axes("or", "and", "b1", "native", (4, 5), 0x1000, 0, (4, 7), 0x2000, 0, 0x3000, "b1",
                              stream=0, check=False) == 5  # bit streams are not transposed

    def tr(shape, perm, dt="f32", A=0x1000, out=0x2000):
        return moa.moa_transpose(dt, shape, A, perm, out, stream=0, check=False)
    assert tr((2, 3), (0, 0)) == 11
    assert tr((2, 3), (0, 2)) == 11
    assert tr((1,) * 9, tuple(range(9))) == 2
    assert tr((2, 3), (1, 0), dt="b1") == 5
    assert tr((2, 0, 3), (2, 1, 0), A=0, out=0) == 0
    assert tr((2, 3), (1, 0), A=0x1000, out=0x1000) == 11
    assert tr((2, 3), (1, 0), dt="f64", A=0x1004) == 10


def test_batch_plan_validation(L):
    """moa_batch_plan_create validates every problem as its single call would,
    before touching the device, and reports the first bad one by index."""
    import ctypes as C
    good = dict(kind="inner", reduce="min", combine="add", shapeA=(4, 5), shapeB=(5, 3), A=0x1000, B=0x2000,
                out=0x3000)

    def create(bad_spec, at=2, n=4):
        specs = [dict(good) for _ in range(n)]
        specs[at] = dict(good, **bad_spec)
        arr, keep = moa.make_problems(specs)
        plan, bad = C.c_void_p(), C.c_int(-1)
        st = moa.lib().moa_batch_plan_create(len(arr), arr, C.byref(plan), C.byref(bad))
        assert not plan.value
        return st, bad.value

    assert create(dict(shapeB=(6, 3))) == (3, 2)  # contracted lengths differ (Eq. 2)
    assert create(dict(shapeA=(1,) * 9)) == (2, 2)  # rank above 8
    assert create(dict(shapeA=(-1, 5))) == (4, 2)  # negative extent
    assert create(dict(dtype="f64", out_dtype="f64")) == (5, 2)  # the batch is FP32
    assert create(dict(form="bf16x3")) == (5, 2)  # a form only (add, mul) has
    assert create(dict(reduce="or", combine="and")) == (5, 2)
    assert create(dict(kind="outer", combine="or", shapeA=(4,), shapeB=(3,))) == (5, 2)
    assert create(dict(out=0)) == (1, 2)
    assert create(dict(A=0x1002)) == (10, 2)  # not FP32-aligned
    assert create(dict(kind="outer", shapeA=(4,), shapeB=(3,), out=0x3001)) == (10, 2)
    assert create(dict(shapeA=(4, 5), shapeB=(6, 3)), at=0, n=1) == (3, 0)
    # every problem well formed, but their pointers are not device memory: the first one is reported
    assert create(dict()) == (13, 0)
    plan, bad = C.c_void_p(), C.c_int(-1)
    assert moa.lib().moa_batch_plan_create(-1, None, C.byref(plan), C.byref(bad)) == 11
    assert moa.lib().moa_batch_plan_create(2, None, C.byref(plan), C.byref(bad)) == 1


def test_outer_validation(L):
    def st(op, dt, sa, sb, odt, A=0x1000, B=0x2000, out=0x3000):
        return moa.moa_outer(op, dt, sa, A, sb, B, out, odt, stream=0, check=False)
    assert st("mul", "f32", (1,) * 9, (2,), "f32") == 2
    assert st("div", "i32", (3,), (2,), "i32") == 5
    assert st("mul", "f32", (3,), (2,), "f64") == 5
    assert st("mul", "f32", (2 ** 32,), (2 ** 32,), "f32") == 4
    assert st("mul", "f32", (3,), (2,), "f32", out=0) == 1
    assert st("mul", "f32", (0,), (2,), "f32", A=0, out=0) == 0


def test_noalloc_and_selftest_validation(L):
    """Host checks of the fixed-scratch entry point and of the wait self-test,
    all answered before any device work."""
    def na(sa, sb, A=0x1000, B=0x2000, out=0x3000):
        return moa.moa_inner_bf16x3_noalloc(sa, A, sb, B, out, stream=0, check=False)
    assert na((4, 5), (6, 3)) == 3
    assert na((), (5, 3)) == 2
    assert na((4, 5), (5, 3), out=0) == 1
    assert na((4, 5), (5, 3), A=0x1002) == 10
    assert na((0, 5), (5, 3), A=0, B=0, out=0) == 0  # empty result
    # 6 (M Kp + K Np) bytes of planes must fit the 32 MiB buffer: 4096 x 1024 . 1024 x 1024 needs 30 MiB, 4096 x 2048
    # . 2048 x 1024 needs 60 MiB
    assert na((4096, 2048), (2048, 1024)) == 12
    st = moa.lib().moa_selftest_wait_timeout(0, None)
    assert st == 11
    assert moa.lib().moa_selftest_wait_timeout(2000000, None) == 11
    for code in range(14):
        assert moa.moa_status_string(code) != "unknown status"


def test_problem_struct_layout_matches_header(tmp_path):
    """The binding's ctypes moa_problem has the size and field offsets the C
    compiler gives the header's struct (a plain C program built with gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    fields = [f for f, _ in moa.MoaProblem._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"moa.h\"\nint main(void) {\n"
                    '    printf("%zu\\n", sizeof(moa_problem));\n' +
                    "".join(f'    printf("%zu\\n", offsetof(moa_problem, {f}));\n' for f in fields) + "    return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == C.sizeof(moa.MoaProblem)
    assert got[1:] == [getattr(moa.MoaProblem, f).offset for f in fields]


def test_host_entry_and_timing_validation(L):
    """moa_inner_host validates shapes, types and null pointers before any
    copy; the timing read rejects null outputs."""
    def h(sa, sb, dt="f32", form="native", A=0x1000, B=0x2000, out=0x3000, odt="f32"):
        return moa.moa_inner_host("add", "mul", dt, form, sa, A, sb, B, out, odt, stream=0, check=False)
    assert h((4, 5), (6, 7)) == 3
    assert h((), (5, 7)) == 2
    assert h((4, 5), (5, 7), dt="f64", form="bf16x3", odt="f64") == 5
    assert h((4, 5), (5, 7), out=0) == 1
    assert h((0, 5), (5, 7), A=0, out=0) == 0
    assert moa.lib().moa_kernel_timing_read(None, None) == 1
    # the scaled e4m3 call: shape and null checks before any device work
    def e4(sa, sb, A=0x1000, B=0x2000, out=0x3000, scA=0x4000, scB=0x5000):
        return moa.moa_inner_e4m3_scaled(sa, A, scA, sb, B, scB, out, stream=0, check=False)
    assert e4((4, 5), (6, 7)) == 3
    assert e4((4, 5), (5, 7), out=0) == 1
    assert e4((0, 5), (5, 7), A=0, out=0) == 0


def test_ozaki_slice_count_matches_the_bench(L, monkeypatch):
    """The slice count the library's Ozaki form takes (a host-side query) is
    the one bench.py's roofline counts slice products with, at every
    threshold of the rule; and the int32 class-sum bound S K 2^14 < 2^31 holds
    up to the longest contraction the form accepts."""
    monkeypatch.delenv("MOA_OZAKI_SLICES", raising=False)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_for_abi", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for K in (1, 2, 63, 64, 65, 255, 256, 257, 1024, 4095, 4096, 4097, 8192, 16384, 21845):
        assert moa.moa_ozaki_slices(K) == bench.ozaki_slices(K), K
        S = moa.moa_ozaki_slices(K)
        assert S * K * 16384 < 2 ** 31 or K > 21845
    assert moa.moa_ozaki_slices(-1) == 0


def test_status_strings(L):
    assert moa.moa_status_string(0) == "ok"
    assert "shape" in moa.moa_status_string(3)
    assert moa.moa_version() >= 0x000100


def test_header_cites_the_paper():
    txt = open(os.path.join(ROOT, "include", "moa.h")).read()
    assert "Eq. (1)" in txt and "Eq. (2)" in txt
