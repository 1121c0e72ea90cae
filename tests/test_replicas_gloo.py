"""The multi-GPU form is replicas (fields are independent; the path has no exchange step):
every rank transforms its own batch and the job's throughput is world x batch over the
slowest rank's time.  Checked here with two gloo ranks on the CPU: the max-over-ranks
reduction bench.py uses, and the reference arm's rank handling."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms = [3.0, 5.0][rank]                     # the two ranks' timed regions
    dist.barrier()
    worst = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (worst, bench.replica_throughput(32, world, worst * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (5.0, 2 * 32 / 5e-3)


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5, None, "cpu") == 4.5
    assert bench.replica_throughput(32, 1, 0.5) == 64.0


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun the reference arm (the CPU oracle) runs on rank 0 only; another
    rank exits 0 without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
