#!/usr/bin/env python
"""Throughput of the mixed dense-sparse interior-point Newton step on GB300.

A step is one IPM iteration (Section 2.1) on the benchmark family member
(default 1: n_d=2000, n_s=200000, m_E=100000, m_I=50, plain FP64): model
evaluation, residuals and norms, diagonal scaling, condensation (the FP64
A^T W^-1 A product), Bunch-Kaufman LDL^T with inertia (and inertia-correction
retries), solves, back-substitution, fraction-to-boundary, line-search trials
and the accept/barrier update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mdsip|reference]

W warm-up steps run from the default starting point; then exactly K steps run
from the W-th iterate (warm start), timed with CUDA events on the library's
stream between barriers: when the solve reaches E_0 <= 1e-8 before K steps,
it starts again from the W-th iterate, so the K steps are iterations W+1,
W+2, ... of the method's own trajectory, repeated.  One full solve to
E_0 <= 1e-8 is timed after that (solves/s).  `e2e` repeats the K steps
through the public API with the iterate copied from pinned host memory
before each step and back after it.  With N > 1 (torchrun) every rank solves
its own instance (independent problems, weak scaling); the value is the sum
of steps over the max time.  `--impl reference` times the CPU oracle on the
same workload and the same steps.

After the headline the default run also measures (rank 0, one GPU): the FP64
FMA rate (the roofline's FP64 peak, measured), mixed precision on member 2
(n_d=4000, m_E=200000) with the per-step gap to the FP64 direction and the
final objective against the oracle's, the batched workload (256 instances,
n_d in [64, 1024]) and the learned warm start (8192 training and 1024
held-out members), each against the plain FP64 GPU path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton steps/sec and solves/sec to 1e-8 KKT error, vs plain FP64 GPU path"
UNIT = "Newton steps/s"
# FP64 ALU peak of a GB300: 152 SMs x 2 DFMA/clk (4 flop) x 2.07 GHz.  A DFMA
# microbenchmark reached 1.20 TFLOP/s at ~1.97 GHz on this machine.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12   # 128 FP32 lanes per SM, 2 flop per FMA
# DRAM bytes per launch of the FP64 condensation kernel at n_d = 2000,
# m_E = 100000, scaled from an ncu capture of the current kernel at m = 20000
# (profiles/syrk_fp64_m20000_n2000.md): reads of A grow with m, the split
# partial writes do not.
SYRK_TRAFFIC_BYTES = 5 * 326.793216e6 + 183.695104e6


def measured_peak(key):
    """A peak from MEASURED_PEAKS.json (None if the file or key is absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdsip", choices=["mdsip", "reference"])
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--no-solve", action="store_true", help="skip the timed full solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=4,
                    help="oracle steps in the CPU baseline sample (all cores; the 1-thread sample takes 1)")
    ap.add_argument("--mixed-config", type=int, default=2,
                    help="member solved in FP64, BF16 and TF32 with per-step FP64 direction gaps (-1: skip)")
    ap.add_argument("--variants", default="bf16,tf32",
                    help="tensor-core precisions also timed on the same instance (comma list, '' for none)")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="instances of the batched measurement (0: skip); n_d ~ U{64..batch-max-nd}")
    ap.add_argument("--batch-max-nd", type=int, default=1024)
    ap.add_argument("--batch-seq-fp64", action="store_true",
                    help="batched measurement: also time the FP64 instances one after another")
    ap.add_argument("--batch-concurrency", type=int, default=32,
                    help="batched measurement: problems solved at once (host workers)")
    ap.add_argument("--batch-option", action="append", default=[],
                    help="NAME=VALUE integer solver option set on every batched instance (repeatable)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched measurement and print its own JSON line")
    ap.add_argument("--ws-train", type=int, default=8192,
                    help="learned warm start: training solves of the parametric family (0: skip)")
    ap.add_argument("--ws-eval", type=int, default=1024, help="learned warm start: held-out members")
    ap.add_argument("--ws-epochs", type=int, default=60)
    ap.add_argument("--ws-fp64-eval", type=int, default=128,
                    help="learned warm start: held-out members also solved cold with the plain FP64 path")
    ap.add_argument("--ws-workers", type=int, default=8, help="concurrent problems (contexts)")
    ap.add_argument("--ws-only", action="store_true",
                    help="run only the learned warm-start measurement and print its own JSON line")
    ap.add_argument("--kernel", choices=["syrk", "syrk_bf16", "syrk_tf32", "ldlt", "ldlt_solve", "ldlt_library",
                                         "gemm_bf16", "dfma", "gemv_pair_df"],
                    default=None,
                    help="time one kernel-level C-ABI call instead of the Newton step")
    ap.add_argument("--m", type=int, default=100000, help="--kernel syrk: rows of A")
    ap.add_argument("--n", type=int, default=2000, help="--kernel syrk: columns of A; ldlt: N; gemm: N")
    ap.add_argument("--k", type=int, default=512, help="--kernel gemm_bf16: K")
    ap.add_argument("--fp32-update", action="store_true",
                    help="--kernel ldlt: the mixed-precision factorization (FP32 update products)")
    ap.add_argument("--no-spec", action="store_true",
                    help="--kernel ldlt --fp32-update: every panel pivots (no verified no-interchange panels)")
    ap.add_argument("--persistent", action="store_true",
                    help="--kernel ldlt: the persistent no-interchange kernel at any order")
    ap.add_argument("--fused", action="store_true",
                    help="--kernel gemv_pair_df: the fused form (mdsip_gemv_pair_df_next, n <= 2048)")
    ap.add_argument("--refine-study", action="store_true",
                    help="refinement convergence of the mixed-precision direction on --config (one JSON line)")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--ldlt-matrix", choices=["kkt", "ipm"], default="kkt",
                    help="--kernel ldlt: kkt = [[H, J^T], [J, -I]] with J ~ N(0, 1) (pivots often); "
                         "ipm = the P1 Newton-step shape of a convex problem (H + Sigma dominant, J small)")
    return ap.parse_args()


# --------------------------------------------------------------------------
# ranks
# --------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_scalar(x: float, op: str, world: int, device=None) -> float:
    """max or sum of a float over ranks (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mdsip_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# --------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------
def blas_info():
    """BLAS library and thread count of this process's numpy."""
    try:
        import threadpoolctl
        info = [d for d in threadpoolctl.threadpool_info() if d.get("user_api") == "blas"]
        if info:
            return {"library": info[0].get("internal_api"), "threads": info[0].get("num_threads")}
    except ImportError:
        pass
    name = None
    try:
        import numpy as np
        name = np.show_config(mode="dicts")["Build Dependencies"]["blas"]["name"]
    except Exception:
        pass
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return {"library": name, "threads": int(os.environ[k])}
    return {"library": name, "threads": os.cpu_count()}


ONE_THREAD_ENV = {k: "1" for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS",
                                   "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")}


def oracle_warm(inst, warm: int):
    """The oracle's own W-th iterate (condensed P2 form) and its barrier parameter."""
    from oracle import ipm
    from oracle.model import SynthModel
    if warm <= 0:
        return None, None
    r = ipm.solve(SynthModel(inst), opt=ipm.Options(linsolve="p2", max_iter=warm))
    return r["point"], r["mu"]


def oracle_sample(inst, start, mu, steps: int):
    """Time `steps` oracle iterations from `start` (None: the default start);
    when the oracle reaches E_0 <= 1e-8 first it starts again from `start`, as
    the GPU's timed steps do.  Returns (iterations, seconds)."""
    from oracle import ipm
    from oracle.model import SynthModel
    model = SynthModel(inst)
    done, el = 0, 0.0
    while done < steps:
        t0 = time.perf_counter()
        r = ipm.solve(model, opt=ipm.Options(linsolve="p2", max_iter=steps - done), start=start, mu0=mu)
        el += time.perf_counter() - t0
        if r["iters"] == 0:
            break
        done += r["iters"]
    return done, el


def save_point(path, pt, mu):
    import numpy as np
    np.savez(path, mu=mu, **{k: getattr(pt, k) for k in ("x", "d", "yg", "yh", "zl", "zu", "vl", "vu")})


def load_point(path):
    import numpy as np
    from oracle import ipm
    z = np.load(path)
    return ipm.Point(*(z[k] for k in ("x", "d", "yg", "yh", "zl", "zu", "vl", "vu"))), float(z["mu"])


def oracle_sample_one_thread(cfg, point_path, steps):
    """The oracle sample in a child process whose BLAS runs one thread."""
    env = dict(os.environ, **ONE_THREAD_ENV)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", point_path, "--config", str(cfg),
           "--cpu-steps", str(steps)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else f"rc {r.returncode}"}
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_sample(args):
    """Child of oracle_sample_one_thread: prints {steps, seconds, blas}."""
    import synth
    start, mu = load_point(args.oracle_sample)
    n, el = oracle_sample(synth.make_config(args.config), start, mu, args.cpu_steps)
    print(json.dumps({"steps": n, "seconds": el, "blas": blas_info()}))


def cpu_baseline(inst, cfg, warm, steps):
    """The oracle on this host: `steps` iterations after its own `warm` warm-up
    iterations with the default (multithreaded) BLAS, and one iteration of the
    same sample with a one-thread BLAS."""
    start, mu = oracle_warm(inst, warm)
    n, el = oracle_sample(inst, start, mu, steps)
    out = {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "blas": blas_info(),
           "sample": f"iterations {warm + 1}..{warm + n} of the FP64 numpy/scipy oracle's own trajectory "
                     f"(condensed P2 form) from its iterate {warm}, restarted there if it converges first; "
                     f"the same steps the GPU times"}
    if start is not None:
        path = os.path.join(tempfile.gettempdir(), f"mdsip_oracle_point_{os.getpid()}.npz")
        try:
            save_point(path, start, mu)
            one = oracle_sample_one_thread(cfg, path, 1)
        finally:
            try:
                os.remove(path)
            except OSError:
                pass
        if "steps" in one:
            out["single_thread"] = {"value": one["steps"] / one["seconds"], "unit": UNIT, "cores": 1,
                                    "blas": one["blas"],
                                    "sample": f"iteration {warm + 1} of the same trajectory, BLAS limited to "
                                              f"one thread"}
        else:
            out["single_thread"] = one
    return out


def workload_name(cfg):
    import synth
    p = synth.CONFIGS[cfg]
    return (f"mds{cfg}: plain FP64 MDS NLP, n_d={p['n_d']}, n_s={2 * p['m_E']}, m_E={p['m_E']}, "
            f"m_I={p['m_I']}, a_i~N(0,{p['sigma_a']}^2), seed={cfg}")


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import synth
    inst = synth.make_config(args.config)
    start, mu = oracle_warm(inst, args.warmup)
    n, el = oracle_sample(inst, start, mu, args.steps)
    value = n / el
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(n, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.config), "path": "P2 (two-stage elimination)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "blas": blas_info(),
                             "sample": f"iterations {args.warmup + 1}.. of the FP64 numpy/scipy oracle's own "
                                       f"trajectory (condensed P2 form) from its iterate {args.warmup}, "
                                       f"restarted there if it converges first: {n} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def partition_instances(costs, world):
    """Instances (by index) over ranks: longest-processing-time first, each to
    the least-loaded rank (ties to the lower rank), so every rank gets a
    deterministic share whose summed cost is within the largest single cost
    of the mean.  Returns one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def batch_aggregate(local, world, device=None):
    """Whole-job figures of a partitioned batch from each rank's own: time =
    max over ranks (every rank starts after a barrier), counts summed, worst
    KKT error max'ed."""
    return {"t_seq": reduce_scalar(local["t_seq"], "max", world, device) if local["t_seq"] is not None else None,
            "t_bat": reduce_scalar(local["t_bat"], "max", world, device),
            "n": reduce_scalar(local["n"], "sum", world, device),
            "n_ok": reduce_scalar(local["n_ok"], "sum", world, device),
            "iters": reduce_scalar(local["iters"], "sum", world, device),
            "max_E0": reduce_scalar(local["max_E0"], "max", world, device)}


def run_batch(args, m, torch, local, rank=0, world=1):
    """Many independent instances (one IPM solve each): sequential on one stream
    vs mdsip_batch_solve with one context per instance.  The contexts' streams
    come from torch's stream pool (32 distinct streams per device), so at most
    32 instances run at once; instances sharing a stream run in turn.  With
    several ranks the instances are partitioned over them (partition_instances
    on n_d^3, the order of both the product and the factorization) and every
    rank solves its share on its own GPU; no data crosses ranks."""
    import numpy as np
    import synth
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(7)
    sizes = rng.integers(64, args.batch_max_nd + 1, size=args.batch_count)
    parts = partition_instances([float(nd) ** 3 for nd in sizes], world)
    mine = parts[rank]
    out = {"instances": len(sizes), "n_d_range": [int(sizes.min()), int(sizes.max())],
           "shape": "n_s = 100 n_d, m_E = 50 n_d, m_I = 50, a_i ~ N(0, 0.01^2), seeds 1000+i",
           "fp64_jacobian_gb": float(sum(50.0 * int(nd) * int(nd) * 8 for nd in sizes) / 1e9),
           "partition": {"ranks": world, "rule": "longest processing time first on n_d^3",
                         "instances_per_rank": [len(p) for p in parts],
                         "max_over_mean_load": (max(sum(float(sizes[i]) ** 3 for i in p) for p in parts) /
                                                (sum(float(nd) ** 3 for nd in sizes) / world))}}
    streams = [torch.cuda.Stream(device=local) for _ in mine]
    ctxs = [m.mdsip_ctx_create(local, st.cuda_stream) for st in streams]
    probs = []
    for c, i in zip(ctxs, mine):   # one host instance at a time
        nd = int(sizes[i])
        inst = synth.make_instance(nd, 50 * nd, 50, 0.01, seed=1000 + i)
        probs.append(m.mdsip_problem_create_synthetic(c, **m.synth_arrays(inst)))
        del inst
    try:
        for name, prec in (("fp64", m.MDSIP_PREC_FP64), ("bf16", m.MDSIP_PREC_BF16)):
            for p in probs:
                m.mdsip_set_option_int(p, "precision", prec)
                for kv in args.batch_option:
                    k, v = kv.split("=")
                    m.mdsip_set_option_int(p, k, int(v))
            # one untimed pass of two steps over every instance: workspaces, autotuned
            # shapes (first use per shape) and captured factorization graphs (second use)
            for p in probs:
                m.mdsip_set_option_int(p, "max_iter", 2)
            m.mdsip_batch_solve(probs, args.batch_concurrency)
            for p in probs:
                m.mdsip_set_option_int(p, "max_iter", 200)
            torch.cuda.synchronize()
            seq = []
            t_seq = None
            if name != "fp64" or args.batch_seq_fp64:
                barrier(world)
                t0 = time.perf_counter()
                seq = [m.mdsip_solve(p) for p in probs]
                t_seq = time.perf_counter() - t0
            barrier(world)
            t0 = time.perf_counter()
            bst = m.mdsip_batch_solve(probs, args.batch_concurrency)
            torch.cuda.synchronize()
            t_bat = time.perf_counter() - t0
            agg = batch_aggregate({"t_seq": t_seq, "t_bat": t_bat, "n": len(probs),
                                   "n_ok": sum(m.STATUS[x] == "OK" for x in bst) + sum(m.STATUS[x] == "OK" for x in seq),
                                   "iters": sum(m.mdsip_get_stats(p)["iters"] for p in probs),
                                   "max_E0": max([m.mdsip_get_stats(p)["E0"] for p in probs] or [0.0])}, world, dev)
            n_runs = agg["n"] * (2 if seq else 1)
            out[name] = {"sequential_solves_per_s": agg["n"] / agg["t_seq"] if agg["t_seq"] else None,
                         "batched_solves_per_s": agg["n"] / agg["t_bat"],
                         "batched_newton_steps_per_s": agg["iters"] / agg["t_bat"],
                         "speedup": agg["t_seq"] / agg["t_bat"] if agg["t_seq"] else None,
                         "all_ok": agg["n_ok"] == n_runs,
                         "solves_ok": f"{int(agg['n_ok'])} of {int(n_runs)}",
                         "statuses_sequential": {k: [m.STATUS[x] for x in seq].count(k) for k in set(m.STATUS[x] for x in seq)},
                         "statuses_batched": {k: [m.STATUS[x] for x in bst].count(k) for k in set(m.STATUS[x] for x in bst)},
                         "max_E0": agg["max_E0"]}
            if world > 1:
                out[name]["statuses_rank0_only"] = True
        out["bf16_vs_fp64_batched"] = out["bf16"]["batched_solves_per_s"] / out["fp64"]["batched_solves_per_s"]
    finally:
        for p in probs:
            m.mdsip_problem_destroy(p)
        for c in ctxs:
            m.mdsip_ctx_destroy(c)
    return out


def run_warmstart(args, m, torch, local):
    """Learned warm start on the parametric family (the benchmark structure at
    n_d = 512, n_s = 51 200, m_E = 25 600, m_I = 50, b = b0 (1 + 0.2 p),
    p in R^64): cold solves of training members -> network trained on the GPU
    -> warm-started solves of held-out members against their cold solves.
    Mixed-precision (BF16 condensation + FP64 refinement) solves throughout."""
    import numpy as np
    import synth
    from paper_2605_13736_gb300 import warmstart as ws
    fam = synth.FAMILY
    inst = synth.make_config(fam["config"])
    n_p, W = fam["n_p"], args.ws_workers
    streams = [torch.cuda.Stream(device=local) for _ in range(W)]
    ctxs = [m.mdsip_ctx_create(local, st.cuda_stream) for st in streams]
    probs = [m.mdsip_problem_create_synthetic(c, **m.synth_arrays(inst)) for c in ctxs]
    for p, c in zip(probs, ctxs):
        m.mdsip_set_option_int(p, "precision", m.MDSIP_PREC_BF16, c)

    def set_member(prob, p):
        m.mdsip_set_bounds(prob, inst.xl, inst.xu, inst.hl, inst.hu,
                           synth.family_rhs(inst, p, fam["amplitude"]), inst.x0)

    net = None
    try:
        P = m.mdsip_packed_size(probs[0])
        train_p = synth.draw_family_params(args.ws_train, n_p, seed=41)
        eval_p = synth.draw_family_params(args.ws_eval, n_p, seed=42)
        dev = torch.device("cuda", local)
        X = torch.from_numpy(train_p).to(dev)
        Y = torch.zeros((args.ws_train, P + 1), dtype=torch.float64, device=dev)
        gen = ws.solve_family(probs, set_member, train_p, Y, e0_level=1e-3)
        ok = gen["statuses"] == 0
        H = 512
        net = ws.WarmStartNet(ctxs[0], n_p, P, hidden=H, init=synth.mlp_init(n_p, H, P + 1, seed=3))
        batch = min(256, args.ws_train)
        losses, t_train = net.train(X, Y, args.ws_train, epochs=args.ws_epochs, batch=batch, lr=1e-3,
                                    lr_final=3e-5, seed=4)
        steps = args.ws_epochs * max(1, args.ws_train // batch)
        Xe = torch.from_numpy(eval_p).to(dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pred = net.predict(Xe, args.ws_eval)
        torch.cuda.synchronize(dev)
        t_pred = time.perf_counter() - t0
        cold = ws.solve_cold(probs, set_member, eval_p)
        warm = ws.solve_warm(probs, set_member, eval_p, pred, push=1e-4)
        # the plain FP64 GPU path on a sample of the same held-out members
        n64 = min(args.ws_fp64_eval, args.ws_eval)
        cold64 = None
        if n64 > 0:
            for p, c in zip(probs, ctxs):
                m.mdsip_set_option_int(p, "precision", m.MDSIP_PREC_FP64, c)
            cold64 = ws.solve_cold(probs, set_member, eval_p[:n64])
            for p, c in zip(probs, ctxs):
                m.mdsip_set_option_int(p, "precision", m.MDSIP_PREC_BF16, c)
        frel = np.abs(warm["f"] - cold["f"]) / np.maximum(1.0, np.abs(cold["f"]))
        hist = lambda st: {m.STATUS[k]: int(v) for k, v in zip(*np.unique(st, return_counts=True))}
        return {
            "family": f"n_d={inst.n_d}, n_s={inst.n_s}, m_E={inst.m_E}, m_I={inst.m_I}, b = b0 (1 + 0.2 p), "
                      f"p ~ U(-1,1)^{n_p} on blocks of {inst.m_E // n_p} rows; BF16 condensation + FP64 refinement",
            "network": f"MLP {n_p}->{H}->{H}->{P + 1} (packed primal-dual point + log mu0), BF16 tcgen05 GEMMs, "
                       f"FP32 Adam",
            "train_members": args.ws_train, "eval_members": args.ws_eval, "workers": W,
            "data_generation": {"solves_per_s": args.ws_train / gen["seconds"], "seconds": gen["seconds"],
                                "mean_iters": float(gen["iters"].mean()), "statuses": hist(gen["statuses"])},
            "training": {"epochs": args.ws_epochs, "batch": batch, "adam_steps": steps, "seconds": t_train,
                         "ms_per_step": 1e3 * t_train / max(1, steps), "loss_first_epoch": losses[0],
                         "loss_last_epoch": losses[-1], "usable_targets": int(ok.sum())},
            "inference_ms": 1e3 * t_pred,
            "cold": {"solves_per_s": args.ws_eval / cold["seconds"], "mean_iters": float(cold["iters"].mean()),
                     "statuses": hist(cold["statuses"]), "max_E0": float(cold["E0"].max())},
            "warm": {"solves_per_s": args.ws_eval / warm["seconds"], "mean_iters": float(warm["iters"].mean()),
                     "mean_iters_incl_fallback": float(warm["total_iters"].mean()),
                     "fallbacks": int(warm["fallbacks"]), "statuses": hist(warm["statuses"]),
                     "max_E0": float(warm["E0"].max()), "max_f_rel_diff_vs_cold": float(frel.max())},
            "speedup_solves_per_s": cold["seconds"] / warm["seconds"],
            "fp64_cold": ({"members": n64, "solves_per_s": n64 / cold64["seconds"],
                           "mean_iters": float(cold64["iters"].mean()), "statuses": hist(cold64["statuses"]),
                           "max_E0": float(cold64["E0"].max())} if cold64 else None),
            "warm_vs_fp64_cold_solves_per_s": ((args.ws_eval / warm["seconds"]) / (n64 / cold64["seconds"])
                                              if cold64 else None),
        }
    finally:
        if net is not None:
            net.close()
        for p in probs:
            m.mdsip_problem_destroy(p)
        for c in ctxs:
            m.mdsip_ctx_destroy(c)


def cond_ldlt_roofline(inst, syrk_ms, ldlt_ms, precision):
    """Roofline fraction of condensation + LDL^T together: (F_syrk / P_syrk +
    F_ldlt / P_ldlt) / (measured product + factorization time), F_syrk =
    n_d (n_d + 1) m_E flop, F_ldlt = N^3 / 3 flop (N = n_d + m_I); P_syrk the FP64
    ALU peak, the measured BF16 peak, or TF32 at half of it; P_ldlt the peak of
    the arithmetic the factorization's updates use: FP64 on the FP64 path, FP32
    (derived: 152 SMs x 128 lanes x 2 flop x 2.07 GHz) on the mixed-precision
    path.  `ldlt_time_vs_fp64_peak` compares the factorization with the time
    its flops take at the FP64 peak."""
    N = inst.n_d + inst.m_I
    f_syrk = inst.n_d * (inst.n_d + 1) * inst.m_E * 1.0
    f_ldlt = N ** 3 / 3.0
    p64 = FP64_PEAK_TFLOPS * 1e12
    bf16 = (measured_peak("bf16_tflops") or 1900.0) * 1e12
    p_syrk = {"fp64": p64, "bf16": bf16, "tf32": bf16 / 2.0}[precision]
    p_ldlt = p64 if precision == "fp64" else FP32_PEAK_TFLOPS * 1e12
    t_roof = f_syrk / p_syrk + f_ldlt / p_ldlt
    t_meas = (syrk_ms + ldlt_ms) / 1e3
    return {"t_roof_ms": 1e3 * t_roof, "t_measured_ms": 1e3 * t_meas, "frac": t_roof / t_meas if t_meas else None,
            "peaks": f"product at {p_syrk / 1e12:.1f} TFLOP/s ({precision}), LDL^T at {p_ldlt / 1e12:.1f} TFLOP/s "
                     f"({'FP64' if precision == 'fp64' else 'FP32, derived'})",
            "ldlt_time_vs_fp64_peak": (f_ldlt / p64) / (ldlt_ms / 1e3) if ldlt_ms else None}


def timed_steps(m, prob, ctx, packed, mu_w, K, mem):
    """Exactly K Newton steps from the W-th iterate `packed` (restarting there
    when the solve converges first).  Returns (steps, summed statistics)."""
    done, zero_calls = 0, 0
    acc = {k: 0.0 for k in ("t_syrk_ms", "n_syrk", "t_ldlt_ms", "n_ldlt", "t_condense_ms", "t_factor_ms",
                            "t_solve_ms", "t_refine_ms", "t_ls_ms", "n_refine", "n_fp64_fallback")}
    statuses = []
    while done < K and zero_calls < 2:
        m.mdsip_set_option_int(prob, "max_iter", K - done, ctx)
        m.mdsip_set_start(prob, packed, mu_w, mem, ctx)
        statuses.append(m.STATUS[m.mdsip_solve(prob, ctx)])
        st = m.mdsip_get_stats(prob)
        for k in acc:
            acc[k] += st[k]
        zero_calls = zero_calls + 1 if st["iters"] == 0 else 0
        done += st["iters"]
    acc["solve_calls"] = len(statuses)
    acc["statuses"] = sorted(set(statuses))
    return done, acc


def fp64_fma_probe(m, torch, ctx, local):
    """Measured FP64 FMA rate (TFLOP/s) of this GPU: mdsip_probe_fp64_fma over
    8 resident blocks per SM, median of 5 timed launches after 2 warm ones."""
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    blocks, iters = 8 * n_sm, 20000
    sink = torch.empty(blocks * 256, dtype=torch.float64, device=torch.device("cuda", local))
    times = []
    for it in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        m.mdsip_probe_fp64_fma(ctx, blocks, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        if it >= 2:
            times.append(e0.elapsed_time(e1) / 1e3)
    flops = blocks * 256.0 * iters * 8 * 2
    return {"tflops": flops / statistics.median(times) / 1e12, "blocks": blocks, "iters_per_thread": iters,
            "ms_median": 1e3 * statistics.median(times)}


def golden_objective(cfg):
    """Final objective of the oracle's own solve of member `cfg`
    (tests/golden/mds{cfg}_p2.json, written by tests/golden/make_golden.py)."""
    path = os.path.join(ROOT, "tests", "golden", f"mds{cfg}_p2.json")
    try:
        with open(path) as fh:
            g = json.load(fh)
        return {"f": g["f"], "iters": g["iters"], "E0": g["E0"], "source": os.path.relpath(path, ROOT)}
    except (OSError, KeyError, ValueError):
        return None


def run_mixed(args, m, torch, local):
    """Member `--mixed-config` (default 2: n_d=4000, n_s=400000, m_E=200000,
    m_I=50) solved to E_0 <= 1e-8 with the plain FP64 path and with the BF16 and
    TF32 tensor-core products (FP64 refinement); then the mixed solves once more
    with every step's direction compared with the FP64 direction from the same
    iterate (direction_check).  Objectives against the oracle's solve."""
    import synth
    cfg = args.mixed_config
    inst = synth.make_config(cfg)
    gold = golden_objective(cfg)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = m.mdsip_ctx_create(local, stream)
    prob = m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(inst))
    del inst
    out = {"workload": workload_name(cfg).replace("plain FP64 ", ""), "oracle": gold}
    try:
        for name, prec in (("fp64", m.MDSIP_PREC_FP64), ("bf16", m.MDSIP_PREC_BF16), ("tf32", m.MDSIP_PREC_TF32)):
            m.mdsip_set_option_int(prob, "precision", prec, ctx)
            m.mdsip_set_option_int(prob, "direction_check", 0, ctx)
            m.mdsip_set_start(prob, None)
            m.mdsip_set_option_int(prob, "max_iter", 2, ctx)     # workspaces, tile choices, graphs
            m.mdsip_solve(prob, ctx)
            m.mdsip_set_option_int(prob, "max_iter", 200, ctx)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = m.mdsip_solve(prob, ctx)
            e1.record()
            torch.cuda.synchronize()
            ss = m.mdsip_get_stats(prob)
            sec = e0.elapsed_time(e1) / 1e3
            rec = {"status": m.STATUS[st], "iters": ss["iters"], "seconds": sec, "solves_per_s": 1.0 / sec,
                   "newton_steps_per_s": ss["iters"] / sec, "E0": ss["E0"], "f": ss["f"],
                   "f_rel_err_vs_oracle": abs(ss["f"] - gold["f"]) / abs(gold["f"]) if gold else None,
                   "iters_oracle": gold["iters"] if gold else None,
                   "refine_sweeps_per_step": ss["n_refine"] / max(1, ss["iters"]),
                   "fp64_fallbacks": ss["n_fp64_fallback"],
                   "phase_ms_per_step": {k: ss[k] / max(1, ss["iters"]) for k in
                                         ("t_condense_ms", "t_factor_ms", "t_refine_ms", "t_ls_ms",
                                          "t_syrk_ms", "t_ldlt_ms")},
                   "condensation_plus_ldlt_roofline": cond_ldlt_roofline(
                       _dims(cfg),
                       ss["t_syrk_ms"] / max(1, ss["n_syrk"]), ss["t_ldlt_ms"] / max(1, ss["n_ldlt"]), name)}
            if name != "fp64":
                rec["speedup_vs_fp64_solves"] = out["fp64"]["seconds"] / sec
                # the same solve once more, each step's direction against the FP64 direction
                m.mdsip_set_option_int(prob, "direction_check", 1, ctx)
                m.mdsip_set_start(prob, None)
                cst = m.mdsip_solve(prob, ctx)
                log = m.mdsip_get_log(prob)
                cs = m.mdsip_get_stats(prob)
                errs = [r["dir_err_fp64"] for r in log if r["dir_err_fp64"] >= 0]
                rec["direction_check"] = {
                    "status": m.STATUS[cst], "iters": cs["iters"], "f": cs["f"],
                    "f_rel_err_vs_oracle": abs(cs["f"] - gold["f"]) / abs(gold["f"]) if gold else None,
                    "rel_err_per_step": errs, "max_rel_err": max(errs) if errs else None,
                    "fp64_fallbacks": cs["n_fp64_fallback"],
                    "what": "||D - D_64||_2 / ||D_64||_2 per Newton step: D the refined mixed-precision "
                            "direction, D_64 the FP64 GPU direction from the same iterate and shifts"}
                m.mdsip_set_option_int(prob, "direction_check", 0, ctx)
            out[name] = rec
    finally:
        m.mdsip_problem_destroy(prob)
        m.mdsip_ctx_destroy(ctx)
    return out


class _dims:
    """n_d, m_E, m_I of a benchmark member without drawing its arrays."""

    def __init__(self, cfg):
        import synth
        p = synth.CONFIGS[cfg]
        self.n_d, self.m_E, self.m_I = p["n_d"], p["m_E"], p["m_I"]


def run_gpu(args):
    rank, world, local = dist_env()
    import numpy as np
    import torch

    import paper_2605_13736_gb300 as m
    import synth

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    m.build()
    # every rank solves its own instance (independent problems)
    seed = args.config if rank == 0 else 1000 * args.config + rank
    inst = synth.make_config(args.config, seed=seed)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = m.mdsip_ctx_create(local, stream)
    prob = m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(inst))
    psize = m.mdsip_packed_size(prob)
    K = args.steps
    try:
        # warm-up: W steps from the default start
        m.mdsip_set_option_int(prob, "max_iter", args.warmup, ctx)
        m.mdsip_solve(prob, ctx)
        w_stats = m.mdsip_get_stats(prob)
        packed = torch.empty(psize, dtype=torch.float64, device=dev)
        m.mdsip_get_iterate(prob, packed, m.MDSIP_MEM_DEVICE, ctx)
        mu_w = w_stats["mu"]
        # timed: exactly K steps from the W-th iterate
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = m.mdsip_launch_count()
        with ClockSampler(local) as clk:
            barrier(world)
            torch.cuda.synchronize()
            e0.record()
            steps_done, acc = timed_steps(m, prob, ctx, packed, mu_w, K, m.MDSIP_MEM_DEVICE)
            e1.record()
            torch.cuda.synchronize()
            barrier(world)
        launches = m.mdsip_launch_count() - launches0
        elapsed = e0.elapsed_time(e1) / 1e3
        t_max = reduce_scalar(elapsed, "max", world, dev)
        units = reduce_scalar(steps_done, "sum", world, dev)
        value = units / t_max

        # full solve to 1e-8 from the default start
        solve = None
        if not args.no_solve:
            m.mdsip_set_start(prob, None)
            m.mdsip_set_option_int(prob, "max_iter", 200, ctx)
            barrier(world)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            sst = m.mdsip_solve(prob, ctx)
            s1.record()
            torch.cuda.synchronize()
            ss = m.mdsip_get_stats(prob)
            sec = s0.elapsed_time(s1) / 1e3
            sec_max = reduce_scalar(sec, "max", world, dev)
            gold = golden_objective(args.config) if rank == 0 else None
            solve = {"status": m.STATUS[sst], "iters": ss["iters"], "E0": ss["E0"], "f": ss["f"],
                     "seconds": sec, "solves_per_s": reduce_scalar(1.0, "sum", world, dev) / sec_max,
                     "newton_steps_per_s": reduce_scalar(ss["iters"], "sum", world, dev) / sec_max,
                     "factorizations": ss["n_factorizations"],
                     "f_rel_err_vs_oracle": abs(ss["f"] - gold["f"]) / abs(gold["f"]) if gold else None,
                     "iters_oracle": gold["iters"] if gold else None}

        # end to end through the public API with host buffers: one step per call,
        # the iterate copied in from pinned memory before and out after it
        host = torch.empty(psize, dtype=torch.float64, pin_memory=True)
        hview = host.numpy()
        w_host = packed.cpu().numpy()
        hview[:] = w_host
        m.mdsip_set_option_int(prob, "max_iter", 1, ctx)
        mu_e = mu_w
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e, idle = 0, 0
        while n_e2e < K and idle < 2:
            m.mdsip_set_start(prob, hview, mu_e, m.MDSIP_MEM_HOST, ctx)   # H2D from pinned memory
            m.mdsip_solve(prob, ctx)
            m.mdsip_get_iterate(prob, hview, m.MDSIP_MEM_HOST, ctx)       # D2H into pinned memory
            es = m.mdsip_get_stats(prob)
            if es["iters"] == 0:         # converged: start again from the W-th iterate
                hview[:] = w_host
                mu_e = mu_w
                idle += 1
                continue
            idle = 0
            mu_e = es["mu"]
            n_e2e += es["iters"]
        torch.cuda.synchronize()
        e2e_t = time.perf_counter() - t0
        e2e_max = reduce_scalar(e2e_t, "max", world, dev)
        e2e_units = reduce_scalar(n_e2e, "sum", world, dev)

        # the same K steps and full solve with the tensor-core condensation product
        variants = {}
        for name in [v for v in args.variants.split(",") if v]:
            prec = {"bf16": m.MDSIP_PREC_BF16, "tf32": m.MDSIP_PREC_TF32}[name]
            m.mdsip_set_option_int(prob, "precision", prec, ctx)
            timed_steps(m, prob, ctx, packed, mu_w, min(K, 4), m.MDSIP_MEM_DEVICE)   # warm the workspace
            barrier(world)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record()
            vdone, vs = timed_steps(m, prob, ctx, packed, mu_w, K, m.MDSIP_MEM_DEVICE)
            v1.record()
            torch.cuda.synchronize()
            vt = reduce_scalar(v0.elapsed_time(v1) / 1e3, "max", world, dev)
            vunits = reduce_scalar(vdone, "sum", world, dev)
            rec = {"value": vunits / vt, "unit": UNIT, "steps": vdone, "ms_per_step": 1e3 * vt / max(1, vdone),
                   "refine_sweeps_per_step": vs["n_refine"] / max(1, vdone),
                   "fp64_fallbacks": vs["n_fp64_fallback"],
                   "syrk_ms_per_launch": vs["t_syrk_ms"] / max(1, vs["n_syrk"]),
                   "phase_ms_per_step": {k: vs[k] / max(1, vdone) for k in
                                         ("t_condense_ms", "t_factor_ms", "t_refine_ms", "t_ls_ms",
                                          "t_syrk_ms", "t_ldlt_ms")}}
            if not args.no_solve:
                m.mdsip_set_start(prob, None)
                m.mdsip_set_option_int(prob, "max_iter", 200, ctx)
                torch.cuda.synchronize()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record()
                sst = m.mdsip_solve(prob, ctx)
                s1.record()
                torch.cuda.synchronize()
                ss = m.mdsip_get_stats(prob)
                sec = reduce_scalar(s0.elapsed_time(s1) / 1e3, "max", world, dev)
                rec["solve"] = {"status": m.STATUS[sst], "iters": ss["iters"], "E0": ss["E0"], "f": ss["f"],
                                "seconds": sec,
                                "solves_per_s": reduce_scalar(1.0, "sum", world, dev) / sec,
                                "refine_sweeps": ss["n_refine"], "fp64_fallbacks": ss["n_fp64_fallback"],
                                "f_rel_diff_vs_fp64": (abs(ss["f"] - solve["f"]) / abs(solve["f"])
                                                        if solve else None)}
                rec["speedup_vs_fp64_solves"] = (rec["solve"]["solves_per_s"] / solve["solves_per_s"]
                                                 if solve else None)
            rec["speedup_vs_fp64_steps"] = rec["value"] / value
            rec["condensation_plus_ldlt_roofline"] = cond_ldlt_roofline(
                inst, vs["t_syrk_ms"] / max(1, vs["n_syrk"]), vs["t_ldlt_ms"] / max(1, vs["n_ldlt"]), name)
            variants[name] = rec
            m.mdsip_set_option_int(prob, "precision", m.MDSIP_PREC_FP64, ctx)
        probe = fp64_fma_probe(m, torch, ctx, local) if rank == 0 else None
    finally:
        m.mdsip_problem_destroy(prob)
        m.mdsip_ctx_destroy(ctx)

    # the batched workload on every rank (its instances partitioned over them)
    batch = run_batch(args, m, torch, local, rank, world) if args.batch_count > 0 else None
    if rank != 0:
        return
    D = dict(n_d=inst.n_d, n_s=inst.n_s, m_E=inst.m_E, m_I=inst.m_I)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(inst, args.config, args.warmup, args.cpu_steps)
    del inst
    mixed = run_mixed(args, m, torch, local) if (args.mixed_config >= 0 and world == 1) else None
    wstart = run_warmstart(args, m, torch, local) if (args.ws_train > 0 and world == 1) else None
    flops = D["n_d"] * (D["n_d"] + 1) / 2 * D["m_E"] * 2.0
    syrk_ms = acc["t_syrk_ms"] / max(1, acc["n_syrk"])
    achieved = flops / (syrk_ms / 1e3) / 1e12 if acc["n_syrk"] else None
    roofline = {"kernel": "k_syrk_fp64 (A^T W^-1 A, FP64 DFMA)", "bound": "alu",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": SYRK_TRAFFIC_BYTES if (D["n_d"], D["m_E"]) == (2000, 100000) else None,
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz (FP64 is not in MEASURED_PEAKS.json)",
                "peak_probe": probe,
                "frac_of_probe": achieved / probe["tflops"] if (achieved and probe) else None,
                "flops_per_launch": flops, "avg_launch_ms": syrk_ms, "launches": int(acc["n_syrk"]),
                "share_of_step": acc["t_syrk_ms"] / (1e3 * elapsed) if elapsed else None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps_done,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / max(1, steps_done),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.config), "path": "P2 (two-stage elimination)",
                   "reduced_N": D["n_d"] + D["m_I"], "steps_requested": K,
                   "steps_timed": steps_done, "solve_calls": acc["solve_calls"],
                   "timed_steps": f"iterations {args.warmup + 1}.. of the solve from its iterate {args.warmup}, "
                                  f"restarted there when it converges",
                   "statuses": acc["statuses"],
                   "l2": "no flush: every step streams A (m_E x n_d FP64 = "
                         f"{D['m_E'] * D['n_d'] * 8 / 1e9:.2f} GB) > 135 MB L2",
                   "parallelism": f"replicas x{world} (independent instances)"},
        "roofline": roofline,
        "condensation_plus_ldlt_roofline": cond_ldlt_roofline(
            _dims(args.config), syrk_ms, acc["t_ldlt_ms"] / max(1, acc["n_ldlt"]), "fp64"),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_units / e2e_max, "unit": UNIT, "h2d_bytes_per_step": psize * 8,
                "d2h_bytes_per_step": psize * 8, "steps": n_e2e},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "solve": solve,
        "variants": variants,
        "mixed_precision": mixed,
        "batched": batch,
        "warm_start": wstart,
        "phase_ms_per_step": {k: acc[k] / max(1, steps_done) for k in
                              ("t_condense_ms", "t_factor_ms", "t_solve_ms", "t_ls_ms", "t_syrk_ms",
                               "t_ldlt_ms")},
    }
    print(json.dumps(line))


def run_ws_only(args):
    """The learned warm-start measurement alone, as its own JSON line (rank 0;
    other ranks exit)."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_2605_13736_gb300 as m
    m.build()
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        ws = run_warmstart(args, m, torch, local)
    print(json.dumps({"metric": "solves/s to 1e-8 KKT error, learned warm start vs cold start (same solver)",
                      "value": ws["warm"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
                      "higher_is_better": True, "dtype": "bf16+f64", "data": "synthetic",
                      "config": {"workload": "parametric family " + ws["family"]},
                      "clocks": clk.summary(), "warm_start": ws}))


def run_batch_only(args):
    """The batched measurement alone, as its own JSON line (rank 0)."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_2605_13736_gb300 as m
    m.build()
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        b = run_batch(args, m, torch, local)
    print(json.dumps({"metric": "solves/s to 1e-8 KKT error, many independent instances (batched vs sequential)",
                      "value": b["bf16"]["batched_solves_per_s"], "unit": "solves/s", "n_gpus": 1,
                      "higher_is_better": True, "dtype": "bf16+f64", "data": "synthetic",
                      "config": {"workload": f"{b['instances']} instances, n_d in {b['n_d_range']}, " + b["shape"]},
                      "clocks": clk.summary(), "batched": b}))


def run_refine_study(args):
    """How the mixed-precision direction converges under refinement, on member
    `--config`: at iterates 3, 9 and 14 of the FP64 trajectory, the relative
    gap between the direction after k = 1 .. 4 sweeps (BF16 and TF32 factors,
    stopping test off, no FP64 fallback) and the FP64 direction from the same
    iterate; then BF16 solves with refine_tol 1e-14 (the default) and 1e-12:
    sweeps, solve time, final residuals and the per-step gap to FP64."""
    import numpy as np
    import torch
    import paper_2605_13736_gb300 as m
    import synth
    m.build()
    torch.cuda.set_device(0)
    inst = synth.make_config(args.config)
    ctx = m.mdsip_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    prob = m.mdsip_problem_create_synthetic(ctx, **m.synth_arrays(inst))
    del inst
    psize = m.mdsip_packed_size(prob)
    precs = (("bf16", m.MDSIP_PREC_BF16), ("tf32", m.MDSIP_PREC_TF32))
    points, solves = [], []
    try:
        for it in (3, 9, 14):
            m.mdsip_set_option_int(prob, "precision", m.MDSIP_PREC_FP64, ctx)
            m.mdsip_set_start(prob, None)
            m.mdsip_set_option_int(prob, "max_iter", it, ctx)
            m.mdsip_solve(prob, ctx)
            mu = m.mdsip_get_stats(prob)["mu"]
            pk, d64 = np.zeros(psize), np.zeros(psize)
            m.mdsip_get_iterate(prob, pk, m.MDSIP_MEM_HOST, ctx)
            m.mdsip_debug_direction(prob, pk, mu, 0.0, 0.0, d64, ctx=ctx)
            rec = {"iterate": it, "mu": mu}
            for name, prec in precs:
                m.mdsip_set_option_int(prob, "precision", prec, ctx)
                m.mdsip_set_option_double(prob, "refine_tol", 0.0, ctx)
                m.mdsip_set_option_double(prob, "refine_fallback_tol", 1.0, ctx)
                gaps = []
                for k in (1, 2, 3, 4):
                    d = np.zeros(psize)
                    m.mdsip_debug_direction(prob, pk, mu, 0.0, 0.0, d, refine=k, ctx=ctx)
                    gaps.append(float(np.linalg.norm(d - d64) / np.linalg.norm(d64)))
                rec[name + "_gap_after_k_sweeps"] = gaps
            m.mdsip_set_option_double(prob, "refine_tol", 1e-14, ctx)
            m.mdsip_set_option_double(prob, "refine_fallback_tol", 1e-10, ctx)
            points.append(rec)
        m.mdsip_set_option_int(prob, "precision", m.MDSIP_PREC_BF16, ctx)
        for tol in (1e-14, 1e-12):
            m.mdsip_set_option_double(prob, "refine_tol", tol, ctx)
            m.mdsip_set_option_int(prob, "direction_check", 0, ctx)
            m.mdsip_set_option_int(prob, "max_iter", 200, ctx)
            m.mdsip_set_start(prob, None)
            m.mdsip_solve(prob, ctx)   # warm: workspaces, tiles
            m.mdsip_set_start(prob, None)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = m.mdsip_solve(prob, ctx)
            e1.record()
            torch.cuda.synchronize()
            ss = m.mdsip_get_stats(prob)
            log = m.mdsip_get_log(prob)
            rec = {"refine_tol": tol, "status": m.STATUS[st], "iters": ss["iters"], "f": ss["f"],
                   "solve_ms": e0.elapsed_time(e1), "sweeps_per_step": ss["n_refine"] / max(1, ss["iters"]),
                   "refine_ms_per_step": ss["t_refine_ms"] / max(1, ss["iters"]),
                   "final_residual_per_step": [r["refine_res"] for r in log[:-1]]}
            m.mdsip_set_option_int(prob, "direction_check", 1, ctx)
            m.mdsip_set_start(prob, None)
            m.mdsip_solve(prob, ctx)
            rec["gap_to_fp64_per_step"] = [r["dir_err_fp64"] for r in m.mdsip_get_log(prob)[:-1]]
            solves.append(rec)
        m.mdsip_set_option_double(prob, "refine_tol", 1e-14, ctx)
        m.mdsip_set_option_int(prob, "direction_check", 0, ctx)
    finally:
        m.mdsip_problem_destroy(prob)
        m.mdsip_ctx_destroy(ctx)
    print(json.dumps({"study": "refinement sweeps", "workload": workload_name(args.config),
                      "points": points, "solves": solves}))


def run_kernel(args):
    """Kernel-level timing: `--kernel syrk` (A^T diag(1/w) A, FP64, m x n) or
    `--kernel ldlt` (Bunch-Kaufman LDL^T of an N x N KKT-like matrix)."""
    import numpy as np
    import torch

    import paper_2605_13736_gb300 as m
    m.build()
    ctx = m.mdsip_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(0)
    times = []
    panels = None
    try:
        if args.kernel == "syrk":
            mm, n = args.m, args.n
            lda = n + (n & 1)
            A = torch.zeros((mm, lda), dtype=torch.float64, device="cuda")
            A[:, :n] = torch.randn((mm, n), dtype=torch.float64, device="cuda") * 0.01
            w = torch.rand(mm, dtype=torch.float64, device="cuda") + 0.5
            Cm = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            flops = n * (n + 1) / 2 * mm * 2.0
            call = lambda: m.mdsip_syrk_scaled(ctx, mm, n, A, lda, w, 0.0, Cm, n)
        elif args.kernel in ("syrk_bf16", "syrk_tf32"):
            mm, n = args.m, args.n
            A = torch.randn((mm, n), dtype=torch.float64, device="cuda") * 0.01
            w = torch.rand(mm, dtype=torch.float64, device="cuda") + 0.5
            Cm = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            flops = n * (n + 1) / 2 * mm * 2.0
            prec = m.MDSIP_PREC_BF16 if args.kernel == "syrk_bf16" else m.MDSIP_PREC_TF32
            call = lambda: m.mdsip_syrk_scaled_tc(ctx, mm, n, A, n, w, 0.0, Cm, n, prec)
        elif args.kernel == "dfma":
            p = fp64_fma_probe(m, torch, ctx, 0)
            print(json.dumps({"kernel": "dfma", "tflops": p["tflops"], "ms_median": p["ms_median"],
                              "blocks": p["blocks"], "iters_per_thread": p["iters_per_thread"],
                              "derived_peak_tflops": FP64_PEAK_TFLOPS,
                              "frac_of_derived": p["tflops"] / FP64_PEAK_TFLOPS}))
            return
        elif args.kernel == "gemv_pair_df":
            # the refinement residual's two products with A (m_E x n_d) in double-float,
            # one call = split of A into FP32 halves + the fused pass
            mm, n = args.m, args.n
            lda = (n + 3) // 4 * 4
            A = torch.zeros((mm, lda), dtype=torch.float64, device="cuda")
            A[:, :n] = torch.randn((mm, n), dtype=torch.float64, device="cuda") * 0.01
            x = torch.randn(n, dtype=torch.float64, device="cuda")
            v = torch.randn(mm, dtype=torch.float64, device="cuda")
            Ax = torch.empty(mm, dtype=torch.float64, device="cuda")
            ATv = torch.empty(n, dtype=torch.float64, device="cuda")
            flops = 4.0 * mm * n
            call = lambda: m.mdsip_gemv_pair_df(ctx, mm, n, A, lda, x, v, Ax, ATv)
            if args.fused:   # the form that also takes the next approximate solve's A^T product
                cpre = torch.randn(mm, dtype=torch.float64, device="cuda")
                winv = torch.rand(mm, dtype=torch.float64, device="cuda") + 0.5
                ATw = torch.empty(n, dtype=torch.float64, device="cuda")
                flops = 6.0 * mm * n
                call = lambda: m.mdsip_gemv_pair_df_next(ctx, mm, n, A, lda, x, v, cpre, winv, Ax, ATv, ATw)
        elif args.kernel == "gemm_bf16":
            # the warm-start network's output layer: (batch m) x (outputs n) x (hidden k)
            M, N, K = args.m, args.n, args.k
            ld = (K + 7) // 8 * 8
            A = torch.randn((M, ld), device="cuda").to(torch.bfloat16)
            B = torch.randn((N, ld), device="cuda").to(torch.bfloat16)
            Cm = torch.empty((M, N), dtype=torch.float32, device="cuda")
            flops = 2.0 * M * N * K
            call = lambda: m.mdsip_gemm_bf16(ctx, M, N, K, A, ld, B, ld, Cm, N)
        else:
            N = args.n
            k = N * 40 // 41
            if N <= 4096:
                G = rng.standard_normal((k, k))
                H = G @ G.T / k + 0.1 * np.eye(k)
                J = rng.standard_normal((N - k, k))
                if args.ldlt_matrix == "ipm":
                    H = H + np.diag(rng.uniform(1.0, 3.0, k))
                    J *= 0.1
                K = np.zeros((N, N))
                K[:k, :k] = H
                K[k:, :k] = J
                K[:k, k:] = J.T
                K[k:, k:] = (-np.eye(N - k) if args.ldlt_matrix == "kkt"
                             else -np.diag(rng.uniform(0.5, 2.0, N - k)))
                S0 = torch.as_tensor(np.tril(K).T.copy()).cuda()
            else:
                # large orders, drawn on the device (seeded): H = 3 I + a symmetric random block
                # of spectral radius ~1.4, J ~ N(0, 1) (kkt) or 0.1 N(0, 1) plus a diagonal lift (ipm)
                gen = torch.Generator(device="cuda").manual_seed(N)
                S0 = torch.zeros((N, N), dtype=torch.float64, device="cuda")
                B = torch.randn((k, k), dtype=torch.float64, device="cuda", generator=gen) / np.sqrt(k)
                S0[:k, :k] = 0.5 * (B + B.T)
                del B
                S0[:k, :k] += torch.diag(torch.full((k,), 3.0, dtype=torch.float64, device="cuda"))
                J = torch.randn((N - k, k), dtype=torch.float64, device="cuda", generator=gen)
                if args.ldlt_matrix == "ipm":
                    S0[:k, :k] += torch.diag(1.0 + 2.0 * torch.rand(k, dtype=torch.float64, device="cuda",
                                                                    generator=gen))
                    J *= 0.1
                S0[k:, :k] = J
                S0[:k, k:] = J.T
                del J
                S0[k:, k:] = (-torch.eye(N - k, dtype=torch.float64, device="cuda") if args.ldlt_matrix == "kkt"
                              else -torch.diag(0.5 + 1.5 * torch.rand(N - k, dtype=torch.float64, device="cuda",
                                                                      generator=gen)))
                K = None            # symmetric: S0's row-major storage is its column-major lower triangle
            S = torch.empty_like(S0)
            L = torch.empty((N, N), dtype=torch.float64, device="cuda")
            Dd = torch.empty(N, dtype=torch.float64, device="cuda")
            Doff = torch.empty_like(Dd)
            perm = torch.empty(N, dtype=torch.int32, device="cuda")
            kind = torch.empty_like(perm)
            inr = torch.empty(3, dtype=torch.int32, device="cuda")
            flops = N ** 3 / 3.0

            flags = m.MDSIP_LDLT_FP32_UPDATES if args.fp32_update else 0
            if args.no_spec:
                flags |= m.MDSIP_LDLT_NO_SPECULATION
            if args.persistent:
                flags |= m.MDSIP_LDLT_PERSISTENT

            def call():
                S.copy_(S0)
                m.mdsip_ldlt_factor_ex(ctx, N, S, N, 1e-14, flags, L, Dd, Doff, perm, kind, inr)
            if args.kernel == "ldlt_library":
                # context only: the vendor library's Bunch-Kaufman (cuSOLVER sytrf behind
                # torch.linalg.ldl_factor_ex) on the same matrix, full symmetric storage
                Kf = torch.as_tensor(K).cuda() if K is not None else S0.clone()
                Kw = torch.empty_like(Kf)

                def call():
                    Kw.copy_(Kf)
                    torch.linalg.ldl_factor_ex(Kw, hermitian=False, check_errors=False)
            if args.kernel == "ldlt_solve":
                call()
                rhs = torch.randn((4, N), dtype=torch.float64, device="cuda")
                flops = 2.0 * N * N * 4

                def call():
                    m.mdsip_ldlt_solve(ctx, N, L, Dd, Doff, perm, 4, rhs, N)
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            call()
            e1.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
        if args.kernel == "ldlt":
            panels = m.mdsip_ldlt_panel_counts(ctx)
    finally:
        m.mdsip_ctx_destroy(ctx)
    ms = statistics.median(times)
    tf = flops / (ms / 1e3) / 1e12
    out = {"kernel": args.kernel, "m": args.m, "n": args.n, "ms_median": ms, "ms_all": times, "tflops": tf}
    if panels is not None:
        out["panels_no_interchange_kept_handed_back"] = panels
    if args.kernel == "gemv_pair_df":
        out["bytes_per_call"] = {"split_read_write": 16.0 * args.m * args.n, "pass_read": 8.0 * args.m * args.n}
    elif args.kernel in ("syrk", "ldlt", "ldlt_solve", "ldlt_library"):
        out["frac_fp64_peak"] = tf / FP64_PEAK_TFLOPS
    else:
        peak = measured_peak("bf16_tflops")
        if args.kernel == "syrk_tf32" and peak:
            peak = peak / 2.0      # nominal TF32 : BF16 dense ratio 1.1 : 2.25
        out["k"] = args.k if args.kernel == "gemm_bf16" else None
        out["peak_tflops"] = peak
        out["frac_of_measured_peak"] = tf / peak if peak else None
    print(json.dumps(out))


def main():
    args = parse()
    if args.oracle_sample:
        run_oracle_sample(args)
        return
    if args.kernel:
        run_kernel(args)
        return
    if args.refine_study:
        run_refine_study(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.ws_only:
        run_ws_only(args)
    elif args.batch_only:
        run_batch_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
