"""Host logic of the N > 1 benchmark path on CPU ranks (gloo, world size 2).

Replicas shard by independent images with no data-path collective; the only
cross-rank step is the max-over-ranks of the timed region, and rank 0 alone prints.
"""
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


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = 1.0 + 2.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, ws, "cpu")
    value = bench.whole_job_value(1000, ws, ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "value": value}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["ms"] == 3.0                         # the slowest rank's time
        assert r["value"] == pytest.approx(1000 * ws / 3e-3)


def test_reference_arm_prints_on_rank0_only(monkeypatch, capsys):
    """Under torchrun the reference arm runs on rank 0; the other ranks exit at once."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    ns = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    bench.run_reference(ns)
    assert capsys.readouterr().out == ""
