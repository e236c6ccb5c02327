"""The multi-rank host logic of bench.py on CPU: two gloo ranks (no GPU).

* max_over_ranks gives every rank the slowest rank's time;
* job_throughput aggregates weak-scaled work (one independent trial per rank);
* the reference arm under two ranks: rank 0 alone times the oracle and prints one JSON line
  with impl "reference"; rank 1 exits without work or output.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist   # noqa: E402
import torch.multiprocessing as mp   # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = {"max": bench.max_over_ranks(1.0 + rank, dist, device="cpu"),
           "value": bench.job_throughput(100.0, world, bench.max_over_ranks(0.5 * (rank + 1), dist, "cpu"))}
    args = bench.parse_args_for_test(["--impl", "reference", "--gpus", str(world), "--n", "3000", "--T", "4",
                                      "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    out["stdout"] = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["max"] == 2.0
        assert res[r]["value"] == pytest.approx(100.0 * 2 / 1.0)
    assert res[1]["stdout"] == ""
    line = json.loads(res[0]["stdout"].strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
