"""Host logic of a multi-GPU (weak-scaling) bench run, on CPU with world_size 2 over gloo: each
rank draws a distinct batch of the same workload (rank 0's is the single-GPU batch), and the
job time is the slowest rank's, agreed by both ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    from workloads import gen
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = gen.get_config("gaussian_64x256_s8_b16")
        A = gen.dictionary(w)
        Y = bench.rank_batch(w, A, rank)
        t = bench.max_over_ranks(1.5 + rank, world)
        np.save(os.path.join(out_dir, f"y{rank}.npy"), Y)
        np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_agree_on_time(tmp_path):
    import torch.multiprocessing as mp
    from workloads import gen
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    y0, y1 = np.load(tmp_path / "y0.npy"), np.load(tmp_path / "y1.npy")
    w = gen.get_config("gaussian_64x256_s8_b16")
    ref, *_ = gen.signals(w, gen.dictionary(w))
    assert np.array_equal(y0, ref)              # rank 0 = the single-GPU batch
    assert y0.shape == y1.shape and not np.allclose(y0, y1)
    t0, t1 = float(np.load(tmp_path / "t0.npy")[0]), float(np.load(tmp_path / "t1.npy")[0])
    assert t0 == t1 == 2.5                       # max over ranks, seen by both


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
