"""The row partition of Eq. (2) over ranks (paper_0907_0792_gb300.rowpart)
on CPU with gloo, world sizes 2 and 3: every rank takes its block of A's
rows, B is broadcast from rank 0, each block is computed (here by the
oracle, there being no GPU), and the gathered D equals the oracle's result
for the whole problem, bit for bit for the exact semirings."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0907_0792_gb300 import rowpart  # noqa: E402


def test_row_blocks_cover_every_row_once():
    for M in (0, 1, 5, 7, 8192, 10007):
        for world in (1, 2, 3, 4, 8):
            blocks = [rowpart.row_block(M, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == M
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    assert rowpart.flat_extents((16, 12, 8, 64), (64, 24, 20)) == (1536, 64, 480)
    with pytest.raises(ValueError):
        rowpart.flat_extents((4, 5), (6, 7))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, kind, q):
    sys.path.insert(0, ROOT)
    import torch

    import oracle
    import synth
    from paper_0907_0792_gb300 import rowpart as rp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    shA, shB = (3, 41, 30), (30, 7, 9)
    M, K, N = rp.flat_extents(shA, shB)
    if kind == "minplus":
        A, B = synth.semiring_inputs("tropical", seed=81, shape_a=shA, shape_b=shB)
        fn = lambda a, b, o: o.copy_(torch.from_numpy(oracle.inner_f32("min", "add", a.numpy(), b.numpy())))
    elif kind == "int32":
        A, B = synth.int_uniform(81, 0, shA, -1000, 1000), synth.int_uniform(81, 1, shB, -1000, 1000)
        fn = lambda a, b, o: o.copy_(torch.from_numpy(oracle.inner_i32(a.numpy(), b.numpy())))
    else:
        A, B = synth.uniform(81, 0, shA, -1, 1), synth.uniform(81, 1, shB, -1, 1)
        fn = lambda a, b, o: o.copy_(torch.from_numpy(oracle.inner_dot2(a.numpy(), b.numpy())[0]))
    r0, r1 = rp.row_block(M, ws, rank)
    A_rows = torch.from_numpy(np.ascontiguousarray(A.reshape(M, K)[r0:r1]))  # each rank holds only its rows of A
    Bt = torch.from_numpy(np.ascontiguousarray(B.reshape(K, N))) if rank == 0 else \
        torch.zeros((K, N), dtype=torch.from_numpy(B).dtype)
    rp.broadcast_operand(Bt, src=0)
    out = torch.empty((r1 - r0, N), dtype=Bt.dtype)
    rp.sharded_inner(None, None, None, None, A_rows, Bt, out, None, compute=fn)
    D = rp.gather_rows(out, M).numpy()
    q.put((rank, D))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
@pytest.mark.parametrize("kind", ["minplus", "int32", "f64"])
def test_sharded_rows_reassemble_the_product(ws, kind):
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, kind, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shA, shB = (3, 41, 30), (30, 7, 9)
    if kind == "minplus":
        A, B = synth.semiring_inputs("tropical", seed=81, shape_a=shA, shape_b=shB)
        want = oracle.inner_f32("min", "add", A, B).reshape(123, 63)
    elif kind == "int32":
        A, B = synth.int_uniform(81, 0, shA, -1000, 1000), synth.int_uniform(81, 1, shB, -1000, 1000)
        want = oracle.inner_i32(A, B).reshape(123, 63)
    else:
        A, B = synth.uniform(81, 0, shA, -1, 1), synth.uniform(81, 1, shB, -1, 1)
        want = oracle.inner_dot2(A, B)[0].reshape(123, 63)
    for _, D in res:
        assert np.array_equal(D, want)
