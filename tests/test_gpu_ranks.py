"""The benchmark's sharded multi-GPU path, run as two ranks on the one GPU a test has (gloo for
the single reduction; the ranks' solves are independent, no kernel waits on another rank): each
rank solves its own seeded batch (rank_batch) and the job time is the slowest rank's. Each rank's
supports and coefficients must be bit-identical to a single-process solve of the same seed, and
rank 1's results must match the FP64 oracle on sampled signals."""
import os
import socket

import numpy as np
import pytest

from oracle import omp as oracle
from tests import parity
from workloads import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WORKLOAD = dict(M=256, N=2048, B=512, S=24, s_min=8, s_max=24, sigma=1e-3, col_scale=1.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _solve(w, A, Y):
    from paper_2407_06434_gb300 import omp
    s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    X, sup, n, r, st = s.solve(Ad, torch.from_numpy(Y).cuda(), w.S, diagnostics=True)
    torch.cuda.synchronize()
    out = X.cpu().numpy(), sup.cpu().numpy(), n.cpu().numpy(), r.cpu().numpy()
    s.close()
    return out


def _worker(rank, world, port, out_dir):
    import time
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        w = gen.get_config("gaussian_64x256_s8_b16", **WORKLOAD)
        A = gen.dictionary(w)
        Y = bench.rank_batch(w, A, rank)
        t0 = time.perf_counter()
        X, sup, n, r = _solve(w, A, Y)
        t = bench.max_over_ranks(time.perf_counter() - t0, world)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), X=X, sup=sup, n=n, r=r, t=t)
    finally:
        dist.destroy_process_group()


def test_two_ranks_solve_their_shards():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import tempfile
    import torch.multiprocessing as mp
    from paper_2407_06434_gb300 import build
    build.build()
    out_dir = tempfile.mkdtemp()
    mp.spawn(_worker, args=(2, _free_port(), out_dir), nprocs=2, join=True)
    w = gen.get_config("gaussian_64x256_s8_b16", **WORKLOAD)
    A = gen.dictionary(w)
    ts = []
    for rank in (0, 1):
        d = np.load(os.path.join(out_dir, f"rank{rank}.npz"))
        Y, *_ = gen.signals(w, A, seed=rank)
        X, sup, n, r = _solve(w, A, Y)
        assert np.array_equal(d["sup"], sup)
        assert np.array_equal(d["X"].view(np.uint32), X.view(np.uint32))
        ts.append(float(d["t"]))
        if rank == 1:
            rows = np.arange(0, w.B, 8)
            ref = oracle.omp_batch(A, Y[rows], w.S)
            st = parity.compare(A, Y[rows], ref, sup[rows], X[rows], n[rows], r[rows], rows=rows)
            assert st["tie_diverged"] <= 2, st
    assert ts[0] == ts[1] > 0
