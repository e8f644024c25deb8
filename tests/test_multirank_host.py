"""The multi-rank benchmark path on CPU: world_size-2 gloo ranks, no GPU.

Each rank solves its own spectrum slice (the units are sharded, so the data
path has no collective); after the timed region the ranks agree on the
whole-job figures, the max of the timed region and the sum of converged
eigenpairs, which is the only exchange."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    lo, hi = bench.rank_slice(rank)
    # rank-dependent timed region and eigenpair counts
    t_ms, pairs = bench.reduce_over_ranks(1000.0 + 250.0 * rank, 90 + 7 * rank, world, "cpu")
    out[rank] = (lo, hi, t_ms, pairs)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_slices_and_reduce():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    res = dict(out)
    assert sorted(res) == [0, 1]
    (lo0, hi0, t0, p0), (lo1, hi1, t1, p1) = res[0], res[1]
    # distinct, non-overlapping slices
    assert hi0 <= lo1 or hi1 <= lo0
    # every rank sees the same whole-job figures: max time, summed pairs
    assert t0 == t1 == 1250.0
    assert p0 == p1 == 90 + 97


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 3, 1, "cpu") == (12.5, 3)
    assert bench.rank_slice(0) == bench.SLICES_OMEGA[0]


def test_reference_arm_nonzero_rank_exits_without_work():
    """Under torchrun the reference arm runs on rank 0 alone; another rank
    returns at once with status 0 and prints nothing."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
