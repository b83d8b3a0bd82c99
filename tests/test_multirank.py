"""The N > 1 host path of bench.py on CPU: two gloo ranks (torch.distributed,
world size 2, 127.0.0.1) run its process-group setup and the max / sum
reductions that turn per-rank times and pair counts into the whole-job
figure; each rank draws its own subject (weak scaling, no data-path
collective); the reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    os.environ.update({"WORLD_SIZE": "2", "RANK": str(rank), "LOCAL_RANK": str(rank), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup()
    t = 1.0 + rank          # per-rank time: the job time is the max
    pairs = 10.0 * (rank + 1)
    res = {"ws": ws, "rank": r, "max": bench.reduce_max(t, ws), "sum": bench.reduce_sum(pairs, ws)}
    case, _ = bench.workload("tiny", r)
    res["theta0"] = float(case["theta"][0])

    class A:
        workload = "tiny"
        steps = 1
        warmup = 0
    if r != 0:
        bench.run_reference(A, ws, r)  # returns at once on the other ranks
        res["reference_returned"] = True
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = res


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_and_shard():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0]["ws"] == res[1]["ws"] == 2
    assert res[0]["max"] == res[1]["max"] == 2.0
    assert res[0]["sum"] == res[1]["sum"] == 30.0
    assert res[0]["theta0"] != res[1]["theta0"]  # each rank its own subject
    assert res[1]["reference_returned"]


def test_bench_tile_spec():
    """Host only: the bench's launch-shape argument."""
    import bench
    assert bench.parse_tile("16x16") == (16, 16, 0)
    assert bench.parse_tile("32x8px4") == (32, 8, 4)
    assert bench.parse_tile("16x16px16") == (16, 16, 16)
    for bad in ("16", "16x", "x16", "16x16px", "16*16"):
        with pytest.raises(SystemExit):
            bench.parse_tile(bad)
