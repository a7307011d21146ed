"""Helpers for the GPU parity tests: move seeded inputs to the device, call
the library through its C ABI, and compare with the CPU oracle."""
import numpy as np

import oracle
import synth


def dev():
    import torch
    return torch.device("cuda:0")


def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def bf16_dev(bits):
    import torch
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).view(torch.bfloat16).to(dev())


def empty(shape, dtype):
    import torch
    return torch.empty(tuple(shape), dtype=dtype, device=dev())


def sample_idx(n_total, n, seed=99):
    if n_total <= n:
        return np.arange(n_total, dtype=np.int64)
    return synth.int_uniform(seed, 7, (n,), 0, int(min(n_total - 1, 2 ** 31 - 1))).astype(np.int64) if n_total < 2 ** 31 \
        else (synth.u64(seed, 7, n) % np.uint64(n_total)).astype(np.int64)


def check_status():
    import paper_0907_0792_gb300 as moa
    st = moa.moa_device_status()
    assert st == 0, moa.moa_status_string(st)


def assert_norm_err(D, A, B, tol, out_idx=None):
    """max |D - D_exact| / sum_p |A||B| <= tol, D_exact by Dot2 on the
    operands as given (exactly representable in float64)."""
    ref, S = oracle.inner_dot2(np.asarray(A, dtype=np.float64), np.asarray(B, dtype=np.float64), out_idx=out_idx)
    D = np.asarray(D, dtype=np.float64)
    if out_idx is not None:
        D = D.ravel()[out_idx] if D.size != len(out_idx) else D.ravel()
    err = oracle.normalised_error(D, ref, S)
    assert err <= tol, f"normalised error {err:.3e} > {tol:.1e}"
    return err
