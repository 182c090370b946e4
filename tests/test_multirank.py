"""The N > 1 path of bench.py on CPU: two gloo ranks.  Each rank runs its own batch (weak
scaling, no collective on the data path); the job's throughput is the units every rank
processed over the slowest rank's time (an all-reduce MAX of the timing, the only exchange).
The reference arm runs on rank 0 alone."""

import io
import os
import shutil
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as D  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    D.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from gen import workloads as W
        # weak scaling: each rank its own batch of the same shape
        w = W.make_cfg2(seed=bench.rank_seed(2000, rank), n_steps=2)
        q0 = w["frames"][w["steps"][0]["q"]]
        sig = np.array([len(w["steps"]), float(q0["xy"][0, 0]), float(q0["n"])], np.float64)
        # the job's throughput: every rank's units over the slowest rank's time
        secs = 1.0 + rank  # rank 1 is the slower one
        value, t = bench.job_throughput(units_per_rank=64, seconds=secs, world=world, dist=True)
        # the reference arm: rank 0 alone prints its line
        class Args:
            seed, steps, warmup = 2000, 1, 0
        buf = io.StringIO()
        with redirect_stdout(buf):
            if rank != 0:
                bench.run_reference(Args, rank, world)
        np.save(os.path.join(out_dir, "r%d.npy" % rank),
                np.array([value, t, len(buf.getvalue())] + list(sig), np.float64))
        D.barrier()
    finally:
        D.destroy_process_group()


@pytest.fixture
def out_dir():
    # the ranks' results go to the tests' own (git-ignored) build folder
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "ranks_%d" % os.getpid())
    os.makedirs(d, exist_ok=True)
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_two_ranks_gloo(out_dir):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), out_dir), nprocs=world, join=True)
    r0 = np.load(os.path.join(out_dir, "r0.npy"))
    r1 = np.load(os.path.join(out_dir, "r1.npy"))
    # both ranks agree on the slowest time and the job throughput
    assert r0[1] == r1[1] == 2.0
    assert r0[0] == r1[0] == pytest.approx(64 * world / 2.0)
    # a non-zero rank of the reference arm does no work and prints nothing
    assert r1[2] == 0
    # each rank has its own batch of the same shape
    assert r0[3] == r1[3] == 2
    assert r0[4] != r1[4]


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    v, t = bench.job_throughput(units_per_rank=10, seconds=0.5, world=1, dist=False)
    assert (v, t) == (20.0, 0.5)
    assert bench.rank_seed(7, 0) == 7 and bench.rank_seed(7, 3) != 7
