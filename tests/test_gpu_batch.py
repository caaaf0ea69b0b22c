"""Batched solves (mdsip_batch_solve): independent instances of uneven sizes,
each on its own context/stream, solved concurrently, give exactly the results
of solving each one alone (the kernels are deterministic), and each batched
result is the CPU oracle's own solve of that instance: the same iteration
count and inertia-correction sequence, the objective to 1e-8 relative."""
import numpy as np
import pytest

import paper_2605_13736_gb300 as m
import synth
from oracle import ipm
from oracle.model import SynthModel
from gpu_util import make_problem, torch_cuda


@pytest.fixture(scope="module")
def oracle_runs():
    """The oracle's solve of every instance of _instances() (two-stage condensed
    directions, pinned against the full 4x4 solve by the oracle's own tests)."""
    return [ipm.solve(SynthModel(inst), opt=ipm.Options(linsolve="p2")) for inst in _instances()]

pytestmark = pytest.mark.gpu


def _instances():
    rng = np.random.default_rng(3)
    sizes = rng.integers(8, 40, size=6)
    return [synth.make_instance(int(nd), int(20 * nd), 5, 0.05, seed=1000 + i) for i, nd in enumerate(sizes)]


@pytest.mark.parametrize("prec", [m.MDSIP_PREC_FP64, m.MDSIP_PREC_BF16])
def test_batch_equals_individual_solves(prec, oracle_runs):
    torch = torch_cuda()
    m.build()
    insts = _instances()
    streams = [torch.cuda.Stream() for _ in insts]
    ctxs = [m.mdsip_ctx_create(0, s.cuda_stream) for s in streams]
    probs = []
    try:
        for c, inst in zip(ctxs, insts):
            p = make_problem(c, inst)
            m.mdsip_set_option_int(p, "precision", prec, c)
            probs.append(p)
        statuses = m.mdsip_batch_solve(probs, max_concurrent=4)
        assert [m.STATUS[s] for s in statuses] == ["OK"] * len(insts)
        batched = [m.mdsip_get_stats(p) for p in probs]
        for p, st, r in zip(probs, batched, oracle_runs):
            assert r["status_str"] == "OK"
            assert st["iters"] == r["iters"]
            assert abs(st["f"] - r["f"]) <= 1e-8 * abs(r["f"])
            log = m.mdsip_get_log(p)
            for rec, orec in zip(log, r["log"]):
                assert [tuple(c[2]) for c in rec["ic"]] == [tuple(c[2]) for c in orec.get("ic", [])]
        xb = []
        for p in probs:
            buf = np.zeros(m.mdsip_packed_size(p))
            m.mdsip_get_iterate(p, buf)
            xb.append(buf)
        # the same problems one at a time
        for i, p in enumerate(probs):
            assert m.STATUS[m.mdsip_solve(p)] == "OK"
            st = m.mdsip_get_stats(p)
            assert st["iters"] == batched[i]["iters"]
            assert st["f"] == batched[i]["f"]
            buf = np.zeros(m.mdsip_packed_size(p))
            m.mdsip_get_iterate(p, buf)
            np.testing.assert_array_equal(buf, xb[i])
            assert st["E0"] <= 1e-8
    finally:
        for p in probs:
            m.mdsip_problem_destroy(p)
        for c in ctxs:
            m.mdsip_ctx_destroy(c)


def test_batch_contexts_sharing_a_stream():
    """Several contexts on one CUDA stream (for instance streams handed out by
    a framework's pool): their problems are solved in turn by one worker, with
    the results of solving them alone, while other streams run concurrently;
    graphs are captured on the shared stream (second and later solves)."""
    torch = torch_cuda()
    m.build()
    insts = _instances()
    shared = torch.cuda.Stream()
    other = torch.cuda.Stream()
    ctxs = [m.mdsip_ctx_create(0, (shared if i % 3 else other).cuda_stream) for i in range(len(insts))]
    probs = []
    try:
        for c, inst in zip(ctxs, insts):
            p = make_problem(c, inst)
            m.mdsip_set_option_int(p, "precision", m.MDSIP_PREC_BF16, c)
            probs.append(p)
        for rep in range(3):
            statuses = m.mdsip_batch_solve(probs, max_concurrent=8)
            assert [m.STATUS[s] for s in statuses] == ["OK"] * len(insts)
        batched = [m.mdsip_get_stats(p) for p in probs]
        for i, p in enumerate(probs):
            assert m.STATUS[m.mdsip_solve(p)] == "OK"
            st = m.mdsip_get_stats(p)
            assert st["iters"] == batched[i]["iters"] and st["f"] == batched[i]["f"]
    finally:
        for p in probs:
            m.mdsip_problem_destroy(p)
        for c in ctxs:
            m.mdsip_ctx_destroy(c)


def test_batch_shared_context_runs_sequentially():
    torch = torch_cuda()
    m.build()
    ctx = m.mdsip_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    insts = _instances()[:3]
    probs = [make_problem(ctx, inst) for inst in insts]
    try:
        statuses = m.mdsip_batch_solve(probs)
        assert [m.STATUS[s] for s in statuses] == ["OK"] * 3
    finally:
        for p in probs:
            m.mdsip_problem_destroy(p)
        m.mdsip_ctx_destroy(ctx)


def test_batch_many_sizes_all_concurrent():
    """Many concurrent problems of different sizes (different launch shapes and
    shared-memory sizes at the same time): every solve succeeds."""
    torch = torch_cuda()
    m.build()
    rng = np.random.default_rng(11)
    sizes = rng.integers(8, 120, size=16)
    insts = [synth.make_instance(int(nd), int(10 * nd), 3, 0.05, seed=2000 + i) for i, nd in enumerate(sizes)]
    streams = [torch.cuda.Stream() for _ in insts]
    ctxs = [m.mdsip_ctx_create(0, s.cuda_stream) for s in streams]
    probs = []
    try:
        for c, inst in zip(ctxs, insts):
            probs.append(make_problem(c, inst))
        for prec in (m.MDSIP_PREC_FP64, m.MDSIP_PREC_BF16):
            for p, c in zip(probs, ctxs):
                m.mdsip_set_option_int(p, "precision", prec, c)
            statuses = m.mdsip_batch_solve(probs)
            errs = [m.mdsip_ctx_last_error(c) for c, st in zip(ctxs, statuses) if st != 0]
            assert [m.STATUS[s] for s in statuses] == ["OK"] * len(insts), errs
    finally:
        for p in probs:
            m.mdsip_problem_destroy(p)
        for c in ctxs:
            m.mdsip_ctx_destroy(c)


@pytest.mark.parametrize("prec", [m.MDSIP_PREC_FP64, m.MDSIP_PREC_BF16])
def test_graph_replay_equals_separate_launches(prec):
    """The factorization phase replayed as a CUDA graph gives bit for bit the
    iterates of separate launches (same kernels, same arguments)."""
    torch = torch_cuda()
    m.build()
    inst = synth.make_instance(48, 960, 5, 0.05, seed=31)
    out = []
    stream = torch.cuda.Stream()   # stream capture needs a stream other than the legacy default
    before = m.mdsip_launch_count()
    for graphs in (0, 1):
        ctx = m.mdsip_ctx_create(0, stream.cuda_stream)
        p = make_problem(ctx, inst)
        try:
            m.mdsip_set_option_int(p, "precision", prec, ctx)
            m.mdsip_set_option_int(p, "graphs", graphs, ctx)
            assert m.mdsip_solve(p, ctx) == 0
            buf = np.zeros(m.mdsip_packed_size(p))
            m.mdsip_get_iterate(p, buf)
            out.append((buf, m.mdsip_get_stats(p)["iters"], [r["E0"] for r in m.mdsip_get_log(p)]))
        finally:
            m.mdsip_problem_destroy(p)
            m.mdsip_ctx_destroy(ctx)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]


def test_autotuned_shapes_solve_to_the_same_optimum():
    """Tile shapes chosen by the autotuner (panel width, product tile edge) give
    the optimum of the analytic choices (a different rounding order only)."""
    torch = torch_cuda()
    m.build()
    inst = synth.make_instance(150, 7500, 10, 0.02, seed=77)
    res = []
    stream = torch.cuda.Stream()
    for tune in (0, 1):
        ctx = m.mdsip_ctx_create(0, stream.cuda_stream)
        p = make_problem(ctx, inst)
        try:
            m.mdsip_set_option_int(p, "autotune", tune, ctx)
            assert m.mdsip_solve(p, ctx) == 0
            res.append(m.mdsip_get_stats(p))
        finally:
            m.mdsip_problem_destroy(p)
            m.mdsip_ctx_destroy(ctx)
    assert all(r["E0"] <= 1e-8 for r in res)
    assert abs(res[0]["f"] - res[1]["f"]) <= 1e-10 * max(1.0, abs(res[0]["f"]))
