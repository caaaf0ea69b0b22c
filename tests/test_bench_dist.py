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


def _batch_rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import bench
    r, w, _ = bench.dist_env()
    bench.dist_init(w, "gloo")
    sizes = np.random.default_rng(7).integers(64, 1025, size=256)   # the batched workload's sizes
    parts = bench.partition_instances([float(nd) ** 3 for nd in sizes], w)
    mine = parts[r]
    # stand-in per-rank results: time proportional to the rank's load, one
    # failed solve on rank 1, a worst KKT error per rank
    local = {"t_seq": None, "t_bat": sum(float(sizes[i]) ** 3 for i in mine) / 1e9, "n": len(mine),
             "n_ok": len(mine) - (1 if r == 1 else 0), "iters": 15 * len(mine), "max_E0": 1e-9 * (r + 1)}
    agg = bench.batch_aggregate(local, w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, mine, local["t_bat"], agg))


def test_batch_partition_over_two_ranks():
    """The batched workload split over two gloo ranks: each instance solved on
    exactly one rank, the loads balanced, and the whole-job figures (max time,
    summed counts, max error) the same on both ranks."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mine0, t0, agg0), (r1, mine1, t1, agg1) = out
    assert sorted(mine0 + mine1) == list(range(256)) and not set(mine0) & set(mine1)
    assert agg0 == agg1
    assert agg0["t_bat"] == max(t0, t1) and agg0["n"] == 256 and agg0["n_ok"] == 255
    assert agg0["iters"] == 15 * 256 and agg0["max_E0"] == 2e-9 and agg0["t_seq"] is None


def test_partition_is_balanced_and_complete():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 4, 8):
        costs = [float(c) for c in rng.integers(1, 1000, size=97) ** 3]
        parts = bench.partition_instances(costs, world)
        assert len(parts) == world
        assert sorted(i for p in parts for i in p) == list(range(97))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)        # the greedy bound
        assert parts == bench.partition_instances(costs, world)   # deterministic
    assert bench.partition_instances([5.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3]]


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
