"""Host logic of bench.py on CPU: the multi-rank (replica) mode with the gloo backend,
and the column layout of its per-mode error report.

Replicas share nothing on the data path; the only cross-rank step is the job total:
the slowest rank's time (max) and the work of all ranks (sum).
"""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, w = bench.job_totals(1.0 + rank, 1000 * (rank + 1), world, torch.device("cpu"))
    out.put((rank, t, w))
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_ranks():
    world = 2
    port = 29500 + os.getpid() % 2000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, t, w in res:
        assert t == 2.0          # slowest rank
        assert w == 3000.0       # all ranks' work


def test_job_totals_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(1.5, 7, 1, None) == (1.5, 7.0)


def test_h_mode_slices_follow_the_packed_mode_order():
    """The per-mode error columns of the bench line: each higher mode's block of the
    packed [N][h] layout, in the oracle's mode order and widths."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import tensors
    for trunc in (2, 3, 4):
        MB = tensors.ModeBasis(trunc)
        expect, off = [], 0
        for name, L, sig in MB.hmodes:
            k = 2 * (L - sig) + 1
            expect.append((name, off, k))
            off += k
        assert bench.h_mode_slices(trunc) == expect
        assert off == MB.h
