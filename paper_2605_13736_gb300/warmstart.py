"""Learned warm start for a parametric family of problems.

Workflow (argument marshalling around the C ABI; every numeric step runs in
libmdsip's kernels):

1. ``solve_family``: solve members of the family with the plain method
   (cold start), many problems concurrently (``mdsip_batch_solve``), and write
   each member's training target (``mdsip_warmstart_target``: the solution's
   packed primal-dual point and log of a barrier parameter) into a device
   matrix.
2. ``train``: fit the warm-start network (``mdsip_mlp_*``: BF16 tensor-core
   forward and backward passes, Adam) to (parameters -> targets).
3. ``solve_warm``: predict starting points for new members in one batched
   forward pass, start each solve from its prediction pushed into the
   interior (``mdsip_set_start_predicted``), and fall back to a cold start for
   any member whose warm-started solve does not end with status OK.  The
   plain method's own termination test (E_0 <= tol) decides every result.

The family is described by a callable ``set_member(problem, p)`` that loads
member p's data into a problem (for the synthetic family: the equality
right-hand side through ``mdsip_set_bounds``).
"""
from __future__ import annotations

import time

import numpy as np

from . import (MDSIP_MEM_DEVICE, mdsip_batch_solve, mdsip_get_stats, mdsip_mlp_create,
               mdsip_mlp_destroy, mdsip_mlp_fit_scaling, mdsip_mlp_forward, mdsip_mlp_num_params,
               mdsip_mlp_param_offsets, mdsip_mlp_set_params, mdsip_mlp_train_step, mdsip_packed_size,
               mdsip_set_start, mdsip_set_start_predicted, mdsip_warmstart_target)


def _torch():
    import torch
    return torch


def pack_params(mlp, blocks: dict) -> np.ndarray:
    """Parameter vector of the network from blocks W1, b1, W2, b2, W3, b3."""
    off = mdsip_mlp_param_offsets(mlp)
    flat = np.zeros(mdsip_mlp_num_params(mlp), dtype=np.float32)
    for o, k in zip(off, ("W1", "b1", "W2", "b2", "W3", "b3")):
        v = np.ascontiguousarray(blocks[k], dtype=np.float32).reshape(-1)
        flat[o:o + v.size] = v
    return flat


def unpack_params(mlp, flat, n_in, n_hidden, n_out) -> dict:
    """Blocks W1, b1, W2, b2, W3, b3 of a parameter vector."""
    off = mdsip_mlp_param_offsets(mlp)
    shapes = ((n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden), (n_out,))
    out = {}
    for o, k, sh in zip(off, ("W1", "b1", "W2", "b2", "W3", "b3"), shapes):
        out[k] = np.asarray(flat[o:o + int(np.prod(sh))]).reshape(sh)
    return out


def _run_batches(problems, members, prepare, after=None):
    """Solve members in groups of len(problems); prepare(problem, i) loads
    member i, after(problem, i, status) runs once it is solved.  Returns
    dict(statuses, iters, f, E0, seconds)."""
    n = len(members)
    out = dict(statuses=np.zeros(n, dtype=np.int32), iters=np.zeros(n, dtype=np.int32),
               f=np.zeros(n), E0=np.zeros(n))
    t0 = time.perf_counter()
    W = len(problems)
    for s in range(0, n, W):
        group = list(range(s, min(n, s + W)))
        for j, i in enumerate(group):
            prepare(problems[j], i)
        st = mdsip_batch_solve(problems[:len(group)])
        for j, i in enumerate(group):
            stats = mdsip_get_stats(problems[j])
            out["statuses"][i] = st[j]
            out["iters"][i] = stats["iters"]
            out["f"][i] = stats["f"]
            out["E0"][i] = stats["E0"]
            if after is not None:
                after(problems[j], i, st[j])
    out["seconds"] = time.perf_counter() - t0
    return out


def solve_family(problems, set_member, params, targets=None, e0_level=1e-3):
    """Cold-start solves of members params[i]; if ``targets`` (device float64
    tensor, rows >= len(params), row length packed_size + 1) is given, row i
    receives member i's training target (members that do not reach status OK
    leave their row unchanged).  Returns dict(statuses, iters, f, E0, seconds)."""
    def prepare(prob, i):
        set_member(prob, params[i])
        mdsip_set_start(prob, None)

    def after(prob, i, status):
        if targets is not None and status == 0:
            mdsip_warmstart_target(prob, e0_level, targets[i], MDSIP_MEM_DEVICE)

    return _run_batches(problems, params, prepare, after)


class WarmStartNet:
    """The warm-start network of one family: n_p inputs, packed_size + 1 outputs."""

    def __init__(self, ctx, n_p, packed_size, hidden=512, init=None):
        self.ctx = ctx
        self.n_in, self.n_hidden, self.n_out = int(n_p), int(hidden), int(packed_size) + 1
        self.mlp = mdsip_mlp_create(ctx, self.n_in, self.n_hidden, self.n_out)
        if init is not None:
            mdsip_mlp_set_params(self.mlp, pack_params(self.mlp, init), ctx=ctx)

    def close(self):
        if self.mlp:
            mdsip_mlp_destroy(self.mlp)
            self.mlp = None

    def __del__(self):
        self.close()

    def train(self, X, Y, count, epochs, batch, lr, seed=0, lr_final=None, log=None):
        """Fit to rows 0..count-1 of X (device float64, count x n_p) and Y
        (device float64, count x n_out): standardisation from the data, then
        `epochs` passes of shuffled batches of Adam steps; the learning rate
        decays geometrically from lr to lr_final.  Returns the per-epoch loss
        of the last batch and the seconds spent."""
        torch = _torch()
        dev = X.device
        mdsip_mlp_fit_scaling(self.mlp, X, X.shape[1], Y, Y.shape[1], count, ctx=self.ctx)
        rng = np.random.Generator(np.random.PCG64(seed))
        nb = max(1, count // batch)
        total = epochs * nb
        lr_final = lr if lr_final is None else lr_final
        losses = []
        step = 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for e in range(epochs):
            perm = rng.permutation(count).astype(np.int32)
            idx = torch.from_numpy(perm[:nb * batch].copy()).to(dev)
            loss = None
            for b in range(nb):
                rate = lr * (lr_final / lr) ** (step / max(1, total - 1))
                last = b == nb - 1
                loss = mdsip_mlp_train_step(self.mlp, X, X.shape[1], Y, Y.shape[1], idx[b * batch:],
                                            batch, rate, want_loss=last, ctx=self.ctx)
                step += 1
            losses.append(loss)
            if log is not None:
                log(e, loss)
        torch.cuda.synchronize(dev)
        return losses, time.perf_counter() - t0

    def predict(self, X, count):
        """Predictions for rows 0..count-1 of X (device float64): device float32
        tensor count x n_out (packed point, then log mu0)."""
        torch = _torch()
        out = torch.empty((count, self.n_out), dtype=torch.float32, device=X.device)
        mdsip_mlp_forward(self.mlp, X, X.shape[1], count, out, self.n_out, ctx=self.ctx)
        return out


def solve_warm(problems, set_member, params, pred, push=1e-4, fallback=True):
    """Solve members params[i] started from pred[i] (device float32 rows of
    packed_size + 1); members whose status is not OK are solved again from the
    cold start when ``fallback``.  Returns dict(statuses, iters (warm attempt),
    total_iters (incl. fallback), f, E0, fallbacks, seconds)."""
    def prepare(prob, i):
        set_member(prob, params[i])
        mdsip_set_start_predicted(prob, pred[i], push, MDSIP_MEM_DEVICE)

    r = _run_batches(problems, params, prepare)
    r["total_iters"] = r["iters"].copy()
    bad = [i for i in range(len(params)) if r["statuses"][i] != 0]
    r["fallbacks"] = len(bad)
    if fallback and bad:
        def prepare_cold(prob, k):
            set_member(prob, params[bad[k]])
            mdsip_set_start(prob, None)
        r2 = _run_batches(problems, bad, prepare_cold)
        for k, i in enumerate(bad):
            r["statuses"][i] = r2["statuses"][k]
            r["total_iters"][i] += r2["iters"][k]
            r["f"][i] = r2["f"][k]
            r["E0"][i] = r2["E0"][k]
        r["seconds"] += r2["seconds"]
    return r


def solve_cold(problems, set_member, params):
    """Plain cold-start solves (the reference the warm start is measured
    against).  Returns dict(statuses, iters, f, E0, seconds)."""
    def prepare(prob, i):
        set_member(prob, params[i])
        mdsip_set_start(prob, None)

    return _run_batches(problems, params, prepare)


def output_size(problem) -> int:
    return mdsip_packed_size(problem) + 1
