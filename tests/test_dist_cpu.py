"""The multi-process path of bench.py on CPU (gloo, world size 2): the rank
helpers (barrier, maximum over ranks) and the reference arm launched the way a
multi-GPU run is, where rank 0 alone works and prints one JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init(world)
    bench.barrier(w)
    m = bench.max_over_ranks(1.5 + r, w)
    bench.barrier(w)
    q.put((r, w, m))
    dist.destroy_process_group()


def test_rank_helpers_over_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 2.5), (1, 2, 2.5)]


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def _partition_main(rank, world, port, q):
    """One rank of the request partition with a stub solver: request g's
    'weights' are (g, g + 0.5, ...), so the gathered rows show which request
    each came from."""
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import bench
    r, w = bench.dist_init(world)
    n_req, n = 64 * w, 5
    idx = bench.partition(n_req, r, w)
    W_local = np.asarray([[g + 0.5 * j for j in range(n)] for g in idx], dtype=np.float64)
    out = bench.gather_weights(W_local, idx, n_req, w)
    q.put((r, idx, None if out is None else out.tolist()))
    dist.destroy_process_group()


def test_request_partition_and_gather_over_gloo():
    """bench.py with N ranks: rank r solves requests r, r + N, ... of the global
    list (each request exactly once), and rank 0 receives every request's
    weights in global order."""
    import multiprocessing as mp

    import numpy as np
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seen = sorted(g for _, idx, _ in res for g in idx)
    assert seen == list(range(128))                      # every request once
    assert all(len(idx) == 64 for _, idx, _ in res)      # 64 per rank
    assert res[1][2] is None                             # only rank 0 gathers
    W = np.asarray(res[0][2])
    assert W.shape == (128, 5)
    assert np.array_equal(W, np.asarray([[g + 0.5 * j for j in range(5)] for g in range(128)]))


def test_sweep_requests_grow_with_ranks():
    """One rank: the 64 requests of the measured sweep; N ranks: 4 x 16 N
    distinct requests (finer target grid), the first rank's share distinct
    from the second's."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import panels
    R, lam1, tg1 = bench.sweep_requests(1)
    _, lam_ref, tg_ref = panels.workload("c4_batch_n5440_T12000")
    assert lam1.shape == (64, 4) and np.array_equal(np.unique(tg1), np.sort(tg_ref))
    _, lam2, tg2 = bench.sweep_requests(2)
    assert lam2.shape == (128, 4) and len(np.unique(tg2)) == 32
    a = set(zip(map(tuple, lam2[bench.partition(128, 0, 2)]), tg2[bench.partition(128, 0, 2)]))
    b = set(zip(map(tuple, lam2[bench.partition(128, 1, 2)]), tg2[bench.partition(128, 1, 2)]))
    assert not (a & b)
