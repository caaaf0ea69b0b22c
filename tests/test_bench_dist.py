"""bench.py's multi-rank aggregation (max time, summed units over ranks) with
two gloo ranks on CPU, as torchrun would launch them."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, l = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    elapsed = 1.0 + rank                 # rank 1 is the slow one
    units = 5 * (rank + 1)
    t_max = bench.reduce_scalar(elapsed, "max", w)
    total = bench.reduce_scalar(units, "sum", w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, l, t_max, total))


def test_two_rank_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, t_max, total) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert t_max == 2.0            # max over ranks
        assert total == 15.0           # 5 + 10 units
    # whole-job throughput as bench.py reports it
    assert total / t_max == 7.5


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_scalar(3.5, "max", 1) == 3.5
    assert bench.reduce_scalar(4, "sum", 1) == 4.0


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the CPU oracle arm) prints one JSON line
    with the contract's keys, on a host without a GPU."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "0",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Newton steps/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
