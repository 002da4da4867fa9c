"""The benchmark's multi-GPU path on the CPU: two gloo ranks (world size 2).

The hot path partitions into independent replicas (one workload copy per
rank, no data-path collective), so what N > 1 adds is the host logic: the
barrier around the timed region, the max over ranks of the measured time,
the whole-job value, and rank 0 alone running and printing the reference
arm.  Those pieces are exercised here with torch.distributed on gloo."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, outdir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    barrier, max_over_ranks = bench.dist_helpers(ws, torch.device("cpu"))
    barrier()
    slowest = max_over_ranks(10.0 + rank)            # rank r "took" 10 + r ms
    value = bench.replica_value(ws, 1000, 4, slowest)
    # the reference arm: rank 0 alone would run it; the others return at once
    ran = None
    if rank != 0:
        import argparse
        ran = bench.run_reference(argparse.Namespace(flux="lf", steps=1, warmup=0))
    barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "value": value, "ran": ran, "info": list(bench.dist_info())}, f)


def test_two_gloo_ranks(tmp_path):
    ws, port = 2, _free_port()
    torch.multiprocessing.spawn(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r, d in enumerate(res):
        assert d["slowest"] == 11.0                    # max over ranks, seen by every rank
        assert d["value"] == pytest.approx(2 * 1000 * 5 * 4 / 11e-3)
        assert d["info"] == [2, r, r]
    assert res[1]["ran"] is None


def test_replica_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    barrier, max_over_ranks = bench.dist_helpers(1, torch.device("cpu"))
    barrier()
    assert max_over_ranks(3.5) == 3.5
    assert bench.replica_value(1, 795780, 100, 536.0) == pytest.approx(795780 * 500 / 0.536)
