"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every
rank decodes its own batch with its own seed, the whole-job value is the
units of all ranks over the slowest rank's time, and under torchrun only
rank 0 of the reference arm runs and prints."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.0, 20.0][rank]
    units = [1000.0, 3000.0][rank]
    value, ms_max, total = bench.aggregate_ranks(ms, units)
    out.put((rank, value, ms_max, total))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max, total in res:
        assert ms_max == 20.0 and total == 4000.0
        assert value == pytest.approx(4000.0 / 0.020)


def test_ranks_decode_distinct_batches():
    import bench
    import workloads as W
    a = W.config2_lengths(seed=bench.rank_seed(0), n_seq=64)
    b = W.config2_lengths(seed=bench.rank_seed(1), n_seq=64)
    assert a.shape == b.shape and not np.array_equal(a, b)
    assert a.min() >= 500 and a.max() <= 4000 and b.min() >= 500 and b.max() <= 4000


def test_reference_arm_rank1_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
