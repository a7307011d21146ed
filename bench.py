"""Benchmark of the MoA generalized inner / outer product on GB300.

Headline workload: the square matrix-multiply sweep's largest case at the
paper's precision: the FP64 (+,*) inner product (Eq. 2, matrix multiply as
its special case, Sec. I; the paper measures FP64 matrix multiply, Sec. II.B)
of two 8192 x 8192 arrays of U(-1,1) values, through ``moa_inner`` in the
Ozaki-sliced form (FP64 in and out, normalised error <= 1e-12).  One step =
one such product (2 n^3 flops of the FP64 product); inputs (2 x 512 MiB) are
larger than L2, so no flush is needed between steps.

Also measured in the same run, each in its own timed loop (keys "rows",
with a compact "summary" as the line's last key): every form of the square
sweep (plain FP64, FP32, BF16 / FP8 / split-BF16x3 from FP32 operands, bf16
operands, Ozaki) at n = 256 .. 8192 for uniform and log-uniform values, the
generalized semirings on the <32,128,512> x <512,64,64> arrays, the
memory-bound outer products of <128,64,32> x <32,64>, the plain-method FP64
rank-4 x rank-3 product, the transposes, the paper's own m x 128 . 128 x n
shape, and the batch of 10,000 uneven products.

``--impl reference`` times the CPU oracle (the appendix-order loop, FP64,
OpenMP over result rows) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_HEAD = 8192
METRIC = "MoA inner-product TFLOP/s (% peak) & outer-product GB/s; mixed vs FP64 form"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def kernel_source_hash() -> str:
    """SHA-256 over the sources the headline kernel (tc_gemm_pair.cu) is compiled from and over
    ozaki_plan.cu, which sets the slice count and chunk length and so the work of each of its launches."""
    import hashlib
    h = hashlib.sha256()
    for f in ("tc_gemm_pair.cu", "tc_ptx.cuh", "common.cuh", "ozaki_epi.cuh", "ozaki_plan.cu"):
        with open(os.path.join(ROOT, "paper_0907_0792_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _ncu_traffic(kernel: str, n: int, path=None):
    """DRAM bytes per launch of `kernel` on the n x n x n product from the
    committed ncu summary, or None when there is none for that size or the
    kernel's sources changed since it was taken."""
    p = path or os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("n") != n or rec.get("source_sha256") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; each line
    is stamped with the host time it arrived so only samples inside the timed
    window are summarised."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        import threading
        self.stamped = []
        self.window = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        if self.proc is not None:
            def reader():
                for line in self.proc.stdout:
                    if line.strip():
                        self.stamped.append((time.time(), line))
            self.thread = threading.Thread(target=reader, daemon=True)
            self.thread.start()
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window if self.window else (0.0, float("inf"))
        lines = [l for t, l in self.stamped if t0 <= t <= t1 + 0.06]
        for l in lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm), "window_s": round(t1 - t0, 3) if self.window else None}


# ---------------------------------------------------------------- helpers
def _bind_near_gpu(index: int):
    """Run the host side on the CPUs of the GPU's own NUMA node (from sysfs),
    so the page-locked buffers of the end-to-end leg are allocated in the
    memory nearest to the GPU's host link.  Returns the CPU list used, or None
    when the node is unknown (the affinity is then left alone)."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(index)
        dev = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{dev}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
            return spec
    except Exception:
        return None
    return None



def _events_time(fn, iters, stream):
    """Average ms per call of fn over `iters` calls, CUDA events on `stream`."""
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(iters):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / iters


def _flushed_time(fn, stream, flush):
    """ms of one call of fn from a cold L2: the flush (a 256 MiB write, tens
    of microseconds) is enqueued first and the start event behind it, so the
    host's marshalling and launch of the call overlap the flush and the time
    is the device's, as it is between the back-to-back calls of a step."""
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    flush()
    s.record(stream)
    fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e)


def _flush_l2(buf):
    buf.add_(1)  # writes 256 MiB, larger than L2


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if os.environ.get("MOA_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)  # before the process group, so its communicator lands on this rank's GPU
    dist.init_process_group(backend)
    return dist.get_rank(), ws, local


def _max_over_ranks(x, ws, device="cuda"):
    """The slowest rank's time (the job is done when the last rank is)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(work_per_rank, ms_max, ws):
    """Whole-job throughput of `ws` replicas that each did `work_per_rank`,
    timed by the slowest rank: units per second."""
    return ws * work_per_rank / (ms_max * 1e-3)


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- rows
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal peak
# FP32 FFMA issue bound: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (unit counts and maximum clock)
FP32_FFMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# (form, operand dtype): the square sweep's forms
SWEEP_FORMS = (("ozaki", "f64"), ("native", "f64"), ("native", "f32"), ("bf16x3", "f32"), ("bf16", "f32"),
               ("f16", "f32"), ("fp8_t128", "f32"), ("native", "bf16"))


def ozaki_slices(k: int) -> int:
    """Digit slices per operand the library's Ozaki form takes for a contraction of length k."""
    return 10 if k <= 64 else (8 if k <= 256 else (7 if k < 4096 else 6))


def ozaki_kernels_per_call(n: int) -> int:
    """Kernels of one n x n x n Ozaki call: A's row maxima and digit planes in one pass where
    its rows fit (6 or 7 slices, n % 4 == 0, n <= 8192; the pass also zeroes the column
    maxima), else a maxima pass and a slicing pass; |B| column maxima; B's digit planes;
    the slice-pair GEMM."""
    fused = ozaki_slices(n) in (6, 7) and n % 4 == 0 and (n + 7) // 8 * 8 <= 8192
    return 4 if fused else 5


def sweep_work(form: str, dtype: str, n: int, peaks: dict, sustained: bool = False):
    """(flop the underlying units execute per product, their peak TFLOP/s, bound, peak label)."""
    f = 2.0 * n ** 3
    bf16 = peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"]
    if form == "ozaki":
        s = ozaki_slices(n)
        return f * s * (s + 1) // 2, bf16, "tensor", "bf16 dense"
    if form == "bf16x3":
        return 6 * f, bf16, "tensor", "bf16 dense"
    if form == "fp8_t128":
        return f, 2 * bf16, "tensor", "e4m3 dense (2x measured bf16)"
    if form in ("bf16", "f16") or dtype == "bf16":
        return f, bf16, "tensor", "bf16 dense" if form != "f16" else "fp16 dense (= bf16 measured)"
    if dtype == "f32":
        return f, FP32_FFMA_TFLOPS, "alu", "FP32 FFMA issue bound"
    return f, FP64_NOMINAL_TFLOPS, "fp64", "FP64 nominal"


class SweepInputs:
    """The square sweep's operands: leading blocks of the n = 8192 arrays
    (synth.square_leading), per distribution, generated once."""

    def __init__(self):
        self.full = {}

    def get(self, n: int, dist: str):
        import numpy as np

        import synth
        if dist not in self.full:
            self.full[dist] = synth.square(max(synth.SWEEP_N), dist)
        A, B = self.full[dist]
        return np.ascontiguousarray(A[:n, :n]), np.ascontiguousarray(B[:n, :n])


def _row_sweep(moa, torch, inputs, n, dist, stream, peaks, flush, forms=SWEEP_FORMS):
    import numpy as np

    import synth
    A64, B64 = inputs.get(n, dist)
    out = []
    dev = {}
    for form, dtype in forms:
        if dtype not in dev:
            if dtype == "f64":
                dev[dtype] = (torch.from_numpy(A64).cuda(), torch.from_numpy(B64).cuda())
            elif dtype == "f32":
                dev[dtype] = (torch.from_numpy(synth.to_f32(A64)).cuda(), torch.from_numpy(synth.to_f32(B64)).cuda())
            else:
                dev[dtype] = tuple(torch.from_numpy(synth.to_bf16(X)[0].view(np.int16)).view(torch.bfloat16).cuda()
                                   for X in (A64, B64))
        A, B = dev[dtype]
        odt = "f64" if dtype == "f64" else "f32"
        D = torch.empty((n, n), dtype=torch.float64 if odt == "f64" else torch.float32, device="cuda")
        call = lambda: moa.moa_inner("add", "mul", dtype, form, (n, n), A, (n, n), B, D, odt, stream)
        call()
        torch.cuda.synchronize()
        reps = 1 if (form, dtype) == ("native", "f64") and n >= 4096 else (3 if n >= 4096 else 5)
        times = []
        for _ in range(reps):
            times.append(_flushed_time(call, stream, flush))
        ms = statistics.median(times)
        work, peak, bound, plabel = sweep_work(form, dtype, n, peaks)
        row = {"form": form, "dtype": dtype, "n": n, "dist": dist, "ms": round(ms, 4),
               "tflops_effective": round(2.0 * n ** 3 / (ms * 1e-3) / 1e12, 2),
               "frac_of_peak": round(work / (ms * 1e-3) / 1e12 / peak, 3), "bound": bound, "peak": plabel}
        if form == "ozaki":
            row["slices"] = ozaki_slices(n)
        out.append(row)
        del D
    del dev
    torch.cuda.empty_cache()
    return out


def _row_semiring(moa, torch, kind, reduce, combine, reps, stream, flush):
    import numpy as np

    import synth
    A, B = synth.semiring_inputs(kind)
    M, K, N = 32 * 128, 512, 64 * 64
    if kind == "bool":
        a = torch.from_numpy(synth.pack_bits(A).view(np.int32)).cuda()
        b = torch.from_numpy(synth.pack_bits(B).view(np.int32)).cuda()
        D = torch.empty(((M * N + 31) // 32,), dtype=torch.int32, device="cuda")
        dt = odt = "b1"
    else:
        a, b = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        D = torch.empty((32, 128, 64, 64), dtype=a.dtype, device="cuda")
        dt = odt = "i32" if kind == "int32" else "f32"
    call = lambda: moa.moa_inner(reduce, combine, dt, "native", A.shape, a, B.shape, b, D, odt, stream)
    call()
    times = []
    for _ in range(reps):
        times.append(_flushed_time(call, stream, flush))
    ms = statistics.median(times)
    path = {"bool": "tensor cores, e4m3 exact count", "int32": "tensor cores, bf16 exact (int8-range values)"}
    return {"semiring": f"({reduce},{combine})", "dtype": dt, "shape": "<32,128,512>x<512,64,64>", "ms": round(ms, 4),
            "gops": round(M * N * K / (ms * 1e-3) / 1e9, 1), "path": path.get(kind, "CUDA cores")}


def _row_outer(moa, torch, op, dt, reps, stream, peaks):
    import numpy as np

    import synth
    shA, shB = synth.C4_SHAPE_A, synth.C4_SHAPE_B
    if dt == "bf16":
        (ab, _), (bb, _) = synth.outer_inputs(op, "bf16")
        A = torch.from_numpy(ab.view(np.int16)).view(torch.bfloat16).cuda()
        B = torch.from_numpy(bb.view(np.int16)).view(torch.bfloat16).cuda()
        C = torch.empty(shA + shB, dtype=torch.bfloat16, device="cuda")
    else:
        A, B = (torch.from_numpy(x).cuda() for x in synth.outer_inputs(op, dt))
        C = torch.empty(shA + shB, dtype=A.dtype, device="cuda")
    call = lambda: moa.moa_outer(op, dt, shA, A, shB, B, C, dt, stream)
    call()
    ms = _events_time(call, reps, stream)  # output (>= 1 GiB) is far larger than L2
    nbytes = C.numel() * C.element_size() + (A.numel() + B.numel()) * A.element_size()
    gbs = nbytes / (ms * 1e-3) / 1e9
    row = {"op": op, "dtype": dt, "shape": "<128,64,32>x<32,64>", "ms": round(ms, 4), "gbs": round(gbs, 1),
           "frac_hbm": round(gbs / peaks["hbm_gbs"], 3)}
    del A, B, C
    torch.cuda.empty_cache()
    return row


def _row_axes(moa, torch, reps, stream, peaks, flush):
    """Contraction over non-adjacent axes: the transpose pre-pass alone
    (GB/s of read + write against the copy bandwidth, both kernels) and
    moa_inner_axes on the semiring shapes with the contracted axes moved
    inside the operands, next to moa_inner on the adjacent layout."""
    import numpy as np

    import synth
    out = []
    for shape, perm in (((1024, 512, 512), (2, 0, 1)), ((512, 1024, 512), (1, 0, 2))):
        x = torch.empty(shape, dtype=torch.float32, device="cuda").uniform_()
        y = torch.empty(tuple(shape[a] for a in perm), dtype=torch.float32, device="cuda")
        call = lambda: moa.moa_transpose("f32", shape, x, perm, y, stream)
        call()
        ms = _events_time(call, reps, stream)  # 2 GiB moved per call, far above L2
        gbs = 2 * x.numel() * 4 / (ms * 1e-3) / 1e9
        out.append({"op": "transpose", "shape": list(shape), "perm": list(perm), "ms": round(ms, 4),
                    "gbs": round(gbs, 1), "frac_hbm": round(gbs / peaks["hbm_gbs"], 3)})
        del x, y
    A, B = synth.semiring_inputs("tropical")  # <32,128,512> x <512,64,64>
    Am = np.ascontiguousarray(np.moveaxis(A, 2, 1))  # <32,512,128>: contract axis 1
    Bm = np.ascontiguousarray(np.moveaxis(B, 0, 2))  # <64,64,512>: contract axis 2
    a, b, am, bm = (torch.from_numpy(v).cuda() for v in (A, B, Am, Bm))
    D = torch.empty((32, 128, 64, 64), dtype=torch.float32, device="cuda")
    for label, call in (("adjacent (moa_inner)",
                         lambda: moa.moa_inner("min", "add", "f32", "native", A.shape, a, B.shape, b, D, "f32", stream)),
                        ("axes 1 and 2 (moa_inner_axes)",
                         lambda: moa.moa_inner_axes("min", "add", "f32", "native", Am.shape, am, 1, Bm.shape, bm, 2, D,
                                                    "f32", stream))):
        call()
        times = []
        for _ in range(reps):
            times.append(_flushed_time(call, stream, flush))
        out.append({"op": "(min,add) " + label, "ms": round(statistics.median(times), 4)})
    del a, b, am, bm, D
    torch.cuda.empty_cache()
    return out


def _row_plain_method(moa, torch, reps, stream):
    import synth
    A, B = synth.rank4x3_f64()
    Ob = synth.outer_second_f64()
    a, b, ob = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), torch.from_numpy(Ob).cuda()
    D = torch.empty((16, 12, 8, 24, 20), dtype=torch.float64, device="cuda")
    C = torch.empty((16, 12, 8, 64, 4, 5), dtype=torch.float64, device="cuda")
    ci = lambda: moa.moa_inner("add", "mul", "f64", "native", A.shape, a, B.shape, b, D, "f64", stream)
    co = lambda: moa.moa_outer("mul", "f64", A.shape, a, Ob.shape, ob, C, "f64", stream)
    ci(), co()
    ms_i = _events_time(ci, reps, stream)
    ms_o = _events_time(co, reps, stream)
    return {"inner_ms": round(ms_i, 4), "inner_gflops": round(2 * 1536 * 480 * 64 / (ms_i * 1e-3) / 1e9, 1),
            "outer_ms": round(ms_o, 4), "outer_gbs": round((C.numel() + A.size) * 8 / (ms_o * 1e-3) / 1e9, 1)}


def _row_skinny(moa, torch, reps, stream, peaks, n=None, cpu=True):
    """The method's own measurement (Sec. IV): D (m x n) = A (m x 128) .
    B (128 x n), m = 1..4, n = 2^26, FP64 and FP32.  B (up to 64 GiB) is
    drawn on the device by the seeded generator; it is read once per call,
    far larger than L2."""
    import oracle
    import synth
    n = n or synth.SKINNY_N_MAX
    k = synth.SKINNY_K
    out = []
    for dt in ("f64", "f32"):
        tdt = torch.float64 if dt == "f64" else torch.float32
        esz = 8 if dt == "f64" else 4
        B = synth.device_uniform(synth.SKINNY_SEED, 1, (k, n), -1.0, 1.0, "cuda", dtype=tdt)
        for m in synth.SKINNY_M:
            A64, _ = synth.skinny(m, 1, k)
            A = torch.from_numpy(A64).to(tdt).cuda()
            D = torch.empty((m, n), dtype=tdt, device="cuda")
            call = lambda: moa.moa_inner("add", "mul", dt, "native", (m, k), A, (k, n), B, D, dt, stream)
            call()
            ms = _events_time(call, reps, stream)
            nbytes = (m * k + k * n + m * n) * esz
            flops = 2.0 * m * k * n
            row = {"dtype": dt, "m": m, "k": k, "n": n, "ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                   "gflops": round(flops / (ms * 1e-3) / 1e9, 1),
                   "frac_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 3)}
            if dt == "f64":
                row["frac_fp64_nominal"] = round(flops / (ms * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS, 3)
                row["bound"] = "fp64" if flops / (FP64_NOMINAL_TFLOPS * 1e12) > nbytes / (peaks["hbm_gbs"] * 1e9) \
                    else "hbm"
            else:
                row["bound"] = "hbm"
            out.append(row)
            del A, D
        del B
        torch.cuda.empty_cache()
    res = {"rows": out}
    if cpu:  # the appendix-order loop on a column sample of the m = 4 FP64 product
        ns = 1 << 18
        A64, B64 = synth.skinny(4, ns, k)
        cpu_rows = []
        for th in sorted({1, oracle.max_threads()}):
            t0 = time.perf_counter()
            oracle.rowwise("f64", A64, B64, threads=th)
            dt_s = time.perf_counter() - t0
            cpu_rows.append({"threads": th, "gflops": round(2.0 * 4 * k * ns / dt_s / 1e9, 2),
                             "sample": f"m=4, n={ns} columns, FP64"})
        res["cpu_oracle"] = cpu_rows
    return res


def _row_batched(moa, torch, reps, stream, compare=True, count=10000):
    """The uneven batch: 10,000 problems (70% split-BF16x3, 20% (min,+),
    10% outer) through one plan (grouped persistent kernel in a CUDA graph),
    against one call per problem of the same forms."""
    import synth
    probs = synth.batched_problems(count)
    pool, oa, ob, od, dtot = synth.batched_inputs(probs)
    dpool = torch.from_numpy(pool).cuda()
    dout = torch.empty((dtot,), dtype=torch.float32, device="cuda")
    base, obase = dpool.data_ptr(), dout.data_ptr()
    specs = []
    for p, a, b, d in zip(probs, oa, ob, od):
        common = dict(shapeA=p["shapeA"], shapeB=p["shapeB"], A=base + 4 * a, B=base + 4 * b, out=obase + 4 * d)
        if p["kind"] == "outer":
            specs.append(dict(kind="outer", combine="mul", **common))
        elif p["kind"] == "minplus":
            specs.append(dict(kind="inner", reduce="min", combine="add", **common))
        else:
            specs.append(dict(kind="inner", form="bf16x3", **common))
    arr, keep = moa.make_problems(specs)
    plan = moa.moa_batch_plan_create(arr)
    info = moa.moa_batch_plan_info(plan)
    t0 = time.perf_counter()
    moa.moa_batch_execute(plan, stream)  # tunes (first use) and captures the graph
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    moa.moa_batch_execute(plan, stream)
    ms = _events_time(lambda: moa.moa_batch_execute(plan, stream), reps, stream)

    def per_problem():
        for sp in specs:
            if sp["kind"] == "outer":
                moa.moa_outer("mul", "f32", sp["shapeA"], sp["A"], sp["shapeB"], sp["B"], sp["out"], "f32", stream)
            elif sp.get("reduce") == "min":
                moa.moa_inner("min", "add", "f32", "native", sp["shapeA"], sp["A"], sp["shapeB"], sp["B"], sp["out"],
                              "f32", stream)
            else:
                moa.moa_inner("add", "mul", "f32", "bf16x3", sp["shapeA"], sp["A"], sp["shapeB"], sp["B"], sp["out"],
                              "f32", stream)
    ms_single = None
    if compare:
        per_problem()
        ms_single = _events_time(per_problem, 1, stream)
    moa.moa_batch_plan_destroy(plan)
    n = len(probs)
    return {"problems": n, "items": info["items"] if "items" in info else info["tiles"],
            "grouped_launches_per_execute": info["launches"], "ms": round(ms, 3),
            "problems_per_s": round(n / (ms * 1e-3), 1),
            "effective_tflops": round(info["work_flops"] / (ms * 1e-3) / 1e12, 2),
            "one_call_per_problem_ms": round(ms_single, 3) if ms_single else None,
            "speedup_vs_one_call_per_problem": round(ms_single / ms, 2) if ms_single else None,
            "first_execute_s_incl_tuning": round(first_s, 3)}


# ---------------------------------------------------------------- CPU oracle
class OracleSampler:
    """The oracle's appendix-order loop (FP64, OpenMP over rows) on leading
    rows of the n = 8192 headline product: the operands are the headline's
    (U(-1,1) FP64), made once; the rate is calibrated once so that each
    sample can be sized in seconds."""

    def __init__(self, threads: int | None = None):
        import oracle
        import synth
        self.n = N_HEAD
        self.threads = threads or oracle.max_threads()
        self.A, self.B = synth.square(self.n, "uniform")
        rows = max(self.threads, 16)
        t0 = time.perf_counter()
        oracle.rowwise("f64", self.A[:rows], self.B, threads=self.threads)
        self.s_per_row = max(time.perf_counter() - t0, 1e-4) / rows

    def rows_for(self, seconds: float) -> int:
        R = int(min(self.n, max(self.threads, seconds / self.s_per_row)))
        return max(self.threads, R // self.threads * self.threads)

    def run(self, rows: int) -> dict:
        import oracle
        t0 = time.perf_counter()
        oracle.rowwise("f64", self.A[:rows], self.B, threads=self.threads)
        dt = time.perf_counter() - t0
        flop = 2.0 * rows * self.n * self.n
        return {"value": flop / dt / 1e12, "unit": "TFLOP/s", "cores": self.threads, "kind": "oracle", "flop": flop,
                "seconds": dt,
                "sample": f"appendix-order FP64 loop, first {rows} of {self.n} result rows of the {self.n}x{self.n} "
                          f"product ({flop / 1e9:.1f} GFLOP in {dt:.2f} s)"}


def cpu_oracle_sample(seconds: float = 12.0, threads: int | None = None):
    """One sample of about `seconds` of oracle work (the GPU arm's cpu_baseline)."""
    smp = OracleSampler(threads)
    r = smp.run(smp.rows_for(seconds))
    r.pop("flop"), r.pop("seconds")
    return r


def headline_config(ws: int, n: int = N_HEAD) -> dict:
    """The workload both arms report (the reference arm samples its rows)."""
    return {"workload": f"square (+,*) inner product n={n}, FP64 in/out, Ozaki-sliced form (normalised error <= 1e-12)",
            "M": n, "K": n, "N": n, "seed": 2, "values": "U(-1,1) FP64",
            "l2": "inputs 2 x 512 MiB > L2, no flush",
            "parallelism": "single GPU" if ws == 1 else f"row partition x{ws} (B broadcast once, {ws} x {n} rows)"}


def run_reference(args, rank, ws):
    """The reference arm: the oracle timed on the host cores.  Every step is
    a sample of the headline product (its leading rows), sized so that the
    W warm-up and K timed steps together take about two minutes; value =
    flop of the K timed samples / their time."""
    if rank != 0:
        return
    smp = OracleSampler()
    rows = smp.rows_for(120.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        smp.run(rows)
    runs = [smp.run(rows) for _ in range(max(1, args.steps))]
    flop, sec = sum(r["flop"] for r in runs), sum(r["seconds"] for r in runs)
    v = flop / sec / 1e12
    full_ms = 2.0 * smp.n ** 3 / (v * 1e12) * 1e3  # the whole 8192^3 product at the sampled rate
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(full_ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(ws),
            "cpu_baseline": {"kind": "oracle", "cores": smp.threads, "value": v,
                             "sample": f"each step: {runs[0]['sample'].split(' (')[0]}; ms_per_step is the whole "
                                       f"product at that rate"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- main
SHORT_FORM = {("ozaki", "f64"): "oz", ("native", "f64"): "f64", ("native", "f32"): "f32", ("bf16x3", "f32"): "x3",
              ("bf16", "f32"): "bf16", ("f16", "f32"): "f16", ("fp8_t128", "f32"): "fp8", ("native", "bf16"): "bf16in"}


def _summary(rows: dict) -> dict:
    """Compact digest of the rows (kept short: it ends the JSON line).  Sweep
    keys: form (oz Ozaki, f64 / f32 native, x3 split-BF16x3, bf16 / f16 / fp8
    forms from FP32, bf16in bf16 operands) : distribution (u uniform, l
    log-uniform);
    values per sweep size."""
    out = {}
    sw = rows.get("square_sweep") or []
    if sw:
        eff, frac = {}, {}
        for r in sw:
            key = f"{SHORT_FORM.get((r['form'], r['dtype']), r['form'])}:{r['dist'][0]}"
            v = r["tflops_effective"]
            eff.setdefault(key, []).append(round(v) if v >= 100 else (round(v, 1) if v >= 10 else round(v, 2)))
            if r["n"] >= 4096:
                frac.setdefault(key, []).append(round(r["frac_of_peak"], 2))
        out["sweep_n"] = sorted({r["n"] for r in sw})
        out["sweep_eff_tflops"] = eff
        out["sweep_frac_n4096_8192"] = frac
    if rows.get("semirings"):
        out["semiring_gops"] = {r["semiring"]: round(r["gops"]) for r in rows["semirings"]}
    if rows.get("outer"):
        out["outer_frac_hbm"] = {f"{r['op']}:{r['dtype']}": round(r["frac_hbm"], 2) for r in rows["outer"]}
    if rows.get("batched_10000"):
        b = rows["batched_10000"]
        out["batched"] = {"ms": b["ms"], "speedup_vs_one_call": b["speedup_vs_one_call_per_problem"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="moa", choices=["moa", "reference"])
    ap.add_argument("--rows", default="all",
                    help="comma list of extra rows to measure: sweep,semirings,outer,plain,batched,skinny,axes (all / none)")
    ap.add_argument("--skinny-n", type=int, default=None, help="n of the skinny row (default 2^26)")
    ap.add_argument("--no-rows", action="store_true", help="same as --rows none")
    ap.add_argument("--sweep-n", default="all", help="comma list of sweep sizes (default 256..8192)")
    ap.add_argument("--sweep-dist", default="uniform,loguniform", help="comma list of sweep value distributions")
    ap.add_argument("--sweep-forms", default="all",
                    help="comma list of form:dtype pairs for the sweep row (e.g. ozaki:f64,fp8_t128:f32)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--headline-n", type=int, default=N_HEAD,
                    help="matrix size of the headline product (smaller sizes for profiling captures only)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer (end-to-end) leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batched-count", type=int, default=10000, help="problems in the batched row")
    ap.add_argument("--batched-no-compare", action="store_true",
                    help="skip the one-call-per-problem comparison of the batched row")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, ws, local = _dist()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return

    import torch

    import paper_0907_0792_gb300 as moa
    import synth

    torch.cuda.set_device(local)
    all_cpus = os.sched_getaffinity(0)
    near_cpus = _bind_near_gpu(local)
    moa.lib()
    peaks = _peaks()
    stream = torch.cuda.current_stream()
    n = args.headline_n

    # ---- headline: FP64 8192^3 (+,*) in the Ozaki form through moa_inner, inputs resident in HBM.
    # With N ranks the problem is the (N n) x n . n x n product partitioned by rows of A and D
    # (rowpart): rank r holds its n rows of A (stream 100 + r of the seed for r > 0), rank 0 holds B and
    # broadcasts it once; no exchange inside a step.
    from paper_0907_0792_gb300 import rowpart
    A64, B64 = synth.square(n, "uniform")
    if rank > 0:
        A64 = synth.uniform(2, 100 + rank, (n, n), -1.0, 1.0)
    A = torch.from_numpy(A64).cuda()
    B = torch.from_numpy(B64).cuda() if rank == 0 else torch.empty((n, n), dtype=torch.float64, device="cuda")
    if ws > 1:
        rowpart.broadcast_operand(B, src=0)
        torch.cuda.synchronize()
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    step = lambda: moa.moa_inner("add", "mul", "f64", "ozaki", (n, n), A, (n, n), B, D, "f64", stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    _barrier(ws)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        torch.cuda.synchronize()
        _barrier(ws)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        moa.moa_kernel_timing(True)  # CUDA events around the slice-pair GEMM launch of every step
        t_start = time.time()
        s.record(stream)
        for _ in range(args.steps):
            step()
        e.record(stream)
        torch.cuda.synchronize()
        clk.window = (t_start, time.time())
        moa.moa_kernel_timing(False)
        _barrier(ws)
    gemm_launches, gemm_ms_total = moa.moa_kernel_timing_read()
    ms_local = s.elapsed_time(e) / args.steps
    ms = _max_over_ranks(ms_local, ws)
    flops = 2.0 * n ** 3
    value = whole_job_rate(flops, ms, ws) / 1e12
    st = moa.moa_device_status()
    if st != 0:
        raise RuntimeError("device status " + moa.moa_status_string(st))

    # ---- e2e: the same product through moa_inner_host, every step copying its
    # operands in from page-locked host memory and its result out (inside the
    # call, overlapped by row blocks), timed with CUDA events on the stream
    del A, B, D
    torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A64).pin_memory()
        hB = torch.from_numpy(B64).pin_memory()
        hD = torch.empty((n, n), dtype=torch.float64).pin_memory()
        e2e_call = lambda: moa.moa_inner_host("add", "mul", "f64", "ozaki", (n, n), hA, (n, n), hB, hD, "f64", stream)
        e2e_call()
        torch.cuda.synchronize()
        e2e_steps = max(3, min(args.steps, 10))
        ms_e2e = _max_over_ranks(_events_time(e2e_call, e2e_steps, stream), ws)
        e2e = {"value": round(ws * flops / (ms_e2e * 1e-3) / 1e12, 2), "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8), "d2h_bytes_per_step": int(hD.numel() * 8),
               "ms_per_step": round(ms_e2e, 3), "call": "moa_inner_host (pinned host buffers, row blocks overlapped)",
               "host_cpus": near_cpus}
        st = moa.moa_device_status()
        if st != 0:
            raise RuntimeError("device status " + moa.moa_status_string(st))
        del hA, hB, hD
    os.sched_setaffinity(0, all_cpus)  # the CPU baseline and the rows use every host core again
    moa.moa_release_workspace()
    torch.cuda.empty_cache()

    # roofline of the dominant kernel (the slice-pair GEMM): slice-product
    # flops per launch over its event-timed duration; a timed region of
    # continuous load past ~0.25 s runs at the power-capped clock, so the
    # sustained measured peak is the denominator there
    gemm_ms = gemm_ms_total / max(1, gemm_launches)
    S = ozaki_slices(n)
    slice_flops = S * (S + 1) // 2 * flops
    sustained = ms_local * args.steps > 250.0
    peak_tc = peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"]
    achieved = slice_flops / (gemm_ms * 1e-3) / 1e12
    kname = "tc_gemm_pair<3>"
    roofline = {"bound": "tensor", "achieved": round(achieved, 1), "peak": peak_tc, "unit": "TFLOP/s",
                "frac": round(achieved / peak_tc, 3), "traffic": _ncu_traffic(kname, n),
                "kernel": kname, "kernel_ms": round(gemm_ms, 4), "kernel_launches": gemm_launches,
                "work": f"{S * (S + 1) // 2} bf16 slice products of 2 n^3 flop (S = {S} slices per operand)",
                "algorithmic_bytes": 2 * S * n * n * 2 + n * n * 8,
                "peak_kind": f"bf16 dense {'sustained' if sustained else 'burst'}, {peaks['source']}",
                "timed_region_ms": round(ms_local * args.steps, 1), "peak_burst": peaks["bf16_tflops"],
                "share_of_step": round(gemm_ms / ms_local, 3)}

    rows = {}
    # the extra rows are single-GPU measurements: with N ranks only the headline runs
    want = set() if args.no_rows or args.rows == "none" or ws > 1 else (
        {"sweep", "semirings", "outer", "plain", "batched", "skinny", "axes"} if args.rows == "all"
        else set(args.rows.split(",")))
    if want:
        flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        flush = lambda: _flush_l2(flush_buf)
        if "sweep" in want:
            sizes = synth.SWEEP_N if args.sweep_n == "all" else tuple(int(v) for v in args.sweep_n.split(","))
            forms = SWEEP_FORMS
            if args.sweep_forms != "all":
                pick = set(args.sweep_forms.split(","))
                forms = tuple(f for f in forms if f"{f[0]}:{f[1]}" in pick)
            inputs = SweepInputs()
            sweep = []
            for dist in args.sweep_dist.split(","):
                for sn in sizes:
                    sweep += _row_sweep(moa, torch, inputs, sn, dist, stream, peaks, flush, forms)
            del inputs
            rows["square_sweep"] = sweep
        if "semirings" in want:
            rows["semirings"] = [
                _row_semiring(moa, torch, "tropical", "min", "add", 5, stream, flush),
                _row_semiring(moa, torch, "tropical", "max", "add", 5, stream, flush),
                _row_semiring(moa, torch, "maxmul", "max", "mul", 5, stream, flush),
                _row_semiring(moa, torch, "tropical", "max", "min", 5, stream, flush),
                _row_semiring(moa, torch, "int32", "add", "mul", 5, stream, flush),
                _row_semiring(moa, torch, "bool", "or", "and", 5, stream, flush)]
        if "outer" in want:
            rows["outer"] = [_row_outer(moa, torch, op, dt, 10, stream, peaks)
                             for op, dt in (("mul", "f32"), ("add", "f32"), ("sub", "f32"), ("div", "f32"),
                                            ("mul", "bf16"), ("div", "bf16"), ("mul", "i32"))]
        if "plain" in want:
            rows["plain_method_f64_rank4x3"] = _row_plain_method(moa, torch, 20, stream)
        if "axes" in want:
            rows["axes_transpose"] = _row_axes(moa, torch, 10, stream, peaks, flush)
        if "skinny" in want:
            rows["skinny_paper_m_x_128_x_n"] = _row_skinny(moa, torch, 10, stream, peaks, n=args.skinny_n,
                                                            cpu=not args.no_cpu)
        if "batched" in want:
            rows["batched_10000"] = _row_batched(moa, torch, 10, stream, compare=not args.batched_no_compare,
                                                 count=args.batched_count)
        del flush_buf
        st = moa.moa_device_status()
        if st != 0:
            raise RuntimeError("device status " + moa.moa_status_string(st))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:  # the CPU baseline belongs to the single-GPU line
        cpu = cpu_oracle_sample(args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": headline_config(ws, n),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * ozaki_kernels_per_call(n),
                "clocks": clk.summary(), "device_status": "ok", "rows": rows, "summary": _summary(rows)}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
