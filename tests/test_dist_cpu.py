"""The replica path of bench.py on CPU with the gloo backend, world size 2: barrier, the
max-over-ranks timing, and the reference arm running on rank 0 only."""
import json
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, outdir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import io
    import contextlib
    import bench
    from workloads import config_tiny
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(1.5 + rank, w)
    buf = io.StringIO()

    class Args:
        steps, warmup = 1, 0
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args, w, r, workload=config_tiny)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": m, "stdout": buf.getvalue()}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replicas_gloo_world2(tmp_path):
    pytest.importorskip("torch.distributed")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["max"] == r1["max"] == 2.5
    line = json.loads(r0["stdout"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert r1["stdout"] == ""
