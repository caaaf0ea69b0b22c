"""Newton-step and whole-solve parity of the GPU path against the oracle.

* direction parity: from the same iterate and shifts, the GPU direction (P1
  and P2 paths, through mdsip_debug_direction) equals the oracle's solve of
  the full 4x4 system of Eq. (linsys4x4) to a relative 1e-10, and the GPU's
  Haynsworth inertia equals the oracle's LDL^T inertia exactly;
* the benchmark family member 0 (n_d=32, n_s=2000, m_E=1000, m_I=1) and its
  nonconvex variant: the GPU run has the oracle's iteration count and
  inertia-correction sequence, and the final objective within 1e-8 relative.
"""
import json
import os

import numpy as np
import pytest

import paper_2605_13736_gb300 as m
import synth
from oracle import ipm
from oracle.model import SynthModel
from gpu_util import make_ctx, make_problem, pack_dir

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    m.mdsip_ctx_destroy(c)


def _point(it):
    return ipm.Point(it["x"], it["d"], it["yg"], it["yh"], it["zl"], it["zu"], it["vl"], it["vu"])


CASES = [
    # (n_d, m_E, m_I, sigma_a, seed, q_shift)
    (4, 6, 2, 0.3, 1, 0.1),
    (5, 40, 1, 0.3, 2, 0.1),
    (33, 70, 3, 0.1, 3, 0.1),
    (6, 9, 1, 0.3, 4, -3.0),      # indefinite Q: wrong inertia at dw = 0
    (70, 130, 7, 0.05, 5, 0.1),   # reduced size 77 (P2) / 207 (P1), several BK tiles
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("path", [m.MDSIP_PATH_P1, m.MDSIP_PATH_P2])
@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (1e-4, 0.0), (3.0, 1e-7)])
def test_direction_parity(ctx, case, path, dw, dc):
    n_d, m_E, m_I, sa, seed, qs = case
    inst = synth.make_instance(n_d, m_E, m_I, sa, seed=seed, q_shift=qs)
    model = SynthModel(inst)
    it = synth.random_iterate(inst, seed + 100)
    pt = _point(it)
    mu = 0.05
    want = ipm.direction_at(model, pt, mu, dw, dc, "full")
    prob = make_problem(ctx, inst, path)
    try:
        out = np.zeros(m.mdsip_packed_size(prob))
        inertia = m.mdsip_debug_direction(prob, pt.packed(), mu, dw, dc, out, ctx=ctx)
    finally:
        m.mdsip_problem_destroy(prob)
    assert inertia == tuple(want["inertia"])
    ref = pack_dir(want)
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel <= 1e-10, rel


def _golden(name):
    with open(os.path.join(HERE, "golden", name + ".json")) as fh:
        return json.load(fh)


def _inst_for(case):
    if case["kind"] == "config":
        return synth.make_config(case["k"])
    return synth.make_instance(case["n_d"], case["m_E"], case["m_I"], case["sigma_a"],
                               seed=case["seed"], q_shift=case["q_shift"])


@pytest.mark.parametrize("name", ["mds0_full", "mds0_nonconvex_full"])
@pytest.mark.parametrize("path", [m.MDSIP_PATH_P1, m.MDSIP_PATH_P2])
def test_solve_matches_oracle_trajectory(ctx, name, path):
    g = _golden(name)
    inst = _inst_for(g["case"])
    prob = make_problem(ctx, inst, path)
    try:
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == g["status"] == "OK"
    assert stats["iters"] == g["iters"]
    assert stats["E0"] <= 1e-8
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    # inertia-correction sequence: every attempt's shift and inertia
    for rec, grec in zip(log, g["log"]):
        want = grec.get("ic", [])
        got = rec["ic"]
        assert len(got) == len(want), (rec["iter"], got, want)
        for (dw, dc, inr), (gdw, gdc, ginr) in zip(got, want):
            assert tuple(inr) == tuple(ginr)
            assert dw == pytest.approx(gdw, rel=1e-12, abs=0)
            assert dc == pytest.approx(gdc, rel=1e-12, abs=0)
    compare_iterations(log, g["log"])


# Per-iteration quantities of the trajectory against the oracle's log.  Both
# sides run the same decisions in FP64 on iterates that differ only by
# rounding order (the directions agree to ~1e-13 relative, bounded by 1e-10 in
# the direction tests), so:
#  * discrete decisions -- backtracking count n_ls, the f-type flag -- match exactly;
#  * mu is the same sequence of products and powers: 1e-12 relative;
#  * step lengths alpha_max, alpha_z (minima of ratios of the iterate to the
#    direction) and alpha = alpha_max / 2^n_ls: 1e-8 relative, the direction
#    bound amplified by the ratio's conditioning;
#  * the objective f: 1e-10 relative;
#  * norms that fall toward zero (E_0, theta, the primal/dual infeasibility,
#    gphi) lose relative accuracy as they shrink: 1e-6 relative plus an
#    absolute floor of 1e-12 times their value at the first iteration.
def compare_iterations(log, glog):
    assert len(log) == len(glog)
    first = glog[0]
    for rec, grec in zip(log, glog):
        it = rec["iter"]
        assert it == grec["iter"]
        assert rec["mu"] == pytest.approx(grec["mu"], rel=1e-12), it
        assert rec["f"] == pytest.approx(grec["f"], rel=1e-10, abs=1e-12), it
        for key in ("E0", "theta", "inf_pr", "inf_du"):
            assert rec[key] == pytest.approx(grec[key], rel=1e-6, abs=1e-12 * abs(first[key])), (it, key)
        if "alpha" not in grec:          # the last record: the stopping test only
            continue
        assert rec["n_ls"] == grec["n_ls"], it
        assert bool(rec["ftype"]) == bool(grec["ftype"]), it
        for key in ("alpha_max", "alpha_z", "alpha"):
            assert rec[key] == pytest.approx(grec[key], rel=1e-8), (it, key)
        assert rec["gphi"] == pytest.approx(grec["gphi"], rel=1e-6, abs=1e-12 * abs(first["gphi"])), it


def test_directions_along_oracle_trajectory(ctx):
    """Directions from the oracle's own iterates of the small instance (n_d = 32;
    P2 condensed oracle for the iterates, full 4x4 solve for the reference
    direction)."""
    inst = synth.make_config(0)
    model = SynthModel(inst)
    opt = ipm.Options(linsolve="p2", max_iter=6)
    r = ipm.solve(model, opt=opt)
    pt = r["point"]
    mu = r["mu"]
    want = ipm.direction_at(model, pt, mu, 0.0, 0.0, "full")
    for path in (m.MDSIP_PATH_P1, m.MDSIP_PATH_P2):
        prob = make_problem(ctx, inst, path)
        try:
            out = np.zeros(m.mdsip_packed_size(prob))
            inertia = m.mdsip_debug_direction(prob, pt.packed(), mu, 0.0, 0.0, out, ctx=ctx)
        finally:
            m.mdsip_problem_destroy(prob)
        assert inertia == tuple(want["inertia"])
        ref = pack_dir(want)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-10


@pytest.fixture(scope="module")
def mds1():
    return synth.make_config(1)


def test_direction_parity_full_size(ctx, mds1):
    """At the benchmark size (n_d=2000, n_s=200000, m_E=100000, m_I=50; P2 as in
    bench.py): the GPU direction from a random interior iterate equals the
    oracle's two-stage direction (itself pinned to the full 4x4 solve on small
    inputs) to 1e-10, with the same inertia, and satisfies Eq. (linsys4x4)."""
    inst = mds1
    model = SynthModel(inst)
    it = synth.random_iterate(inst, 77)
    pt = _point(it)
    mu, dw, dc = 0.01, 0.0, 0.0
    want = ipm.direction_at(model, pt, mu, dw, dc, "p2")
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        out = np.zeros(m.mdsip_packed_size(prob))
        inertia = m.mdsip_debug_direction(prob, pt.packed(), mu, dw, dc, out, ctx=ctx)
    finally:
        m.mdsip_problem_destroy(prob)
    assert inertia == tuple(want["inertia"]) == (inst.n, inst.m, 0)
    ref = pack_dir(want)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-10
    # the GPU direction satisfies the 4x4 system (operator applied block by block)
    P = ipm.Problem(model)
    ev = ipm.Evals(P, pt.x, pt.d)
    sy = ipm.newton_system(P, pt, ev, mu)
    n_s, n_d, m_E, m_I = sy.dims
    o = np.cumsum([0, inst.n, m_I, m_E, m_I])
    dx, dd, dyg, dyh = (out[o[i]:o[i + 1]] for i in range(4))
    dxs, dxd = dx[:n_s], dx[n_s:]
    Dh = sy.sig_d + dw
    res = np.concatenate([
        (sy.Hss + sy.sig_xs + dw) * dxs + sy.Jsg.T @ dyg + sy.r_xs,
        sy.Hdd @ dxd + (sy.sig_xd + dw) * dxd + sy.A.T @ dyg + sy.Jdh.T @ dyh + sy.r_xd,
        sy.Jsg @ dxs + sy.A @ dxd - dc * dyg + sy.r_g,
        sy.Jdh @ dxd - (1.0 / Dh + dc) * dyh + sy.r_h + sy.r_d / Dh])
    rhs = np.concatenate([sy.r_xs, sy.r_xd, sy.r_g, sy.r_h + sy.r_d / Dh])
    assert np.abs(res).max() <= 1e-9 * (1.0 + np.abs(rhs).max())


def test_full_size_solve_reaches_tolerance(ctx, mds1):
    """The benchmark-size solve ends with E_0 <= 1e-8, recomputed by the oracle
    from the GPU's final iterate (a property that holds at any size), with the
    oracle's iteration count, inertia-correction sequence and objective to 1e-8
    relative (tests/golden/mds1_p2.json, the condensed oracle's solve)."""
    inst = mds1
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        packed = np.zeros(m.mdsip_packed_size(prob))
        m.mdsip_get_iterate(prob, packed, ctx=ctx)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK"
    model = SynthModel(inst)
    P = ipm.Problem(model)
    n, m_I, m_E = inst.n, inst.m_I, inst.m_E
    o = np.cumsum([0, n, m_I, m_E, m_I, n, n, m_I, m_I])
    pt = ipm.Point(*(packed[o[i]:o[i + 1]] for i in range(8)))
    ev = ipm.Evals(P, pt.x, pt.d)
    E0 = ipm.kkt_error(P, pt, ev, 0.0, ipm.Options())[0]
    assert E0 <= 1e-8
    assert abs(E0 - stats["E0"]) <= 1e-10
    assert abs(ev.f - stats["f"]) <= 1e-12 * abs(ev.f)
    for rec in log[:-1]:
        assert rec["ic"][-1][2] == (inst.n, inst.m, 0)
    g = _golden("mds1_p2")
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    for rec, grec in zip(log, g["log"]):
        assert [tuple(c[2]) for c in rec["ic"]] == [tuple(c[2]) for c in grec.get("ic", [])]
    compare_iterations(log, g["log"])


TC_PRECS = [m.MDSIP_PREC_BF16, m.MDSIP_PREC_TF32]


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("case", CASES[:3] + CASES[4:])
def test_direction_parity_tensor_core_refined(ctx, case, prec):
    """Condensation product on the tensor cores (BF16 / TF32, FP32 accumulation),
    direction refined in FP64 on the unreduced system: equal to the oracle's
    full 4x4 solve to 1e-10 with the same inertia."""
    n_d, m_E, m_I, sa, seed, qs = case
    inst = synth.make_instance(n_d, m_E, m_I, sa, seed=seed, q_shift=qs)
    model = SynthModel(inst)
    pt = _point(synth.random_iterate(inst, seed + 100))
    mu = 0.05
    want = ipm.direction_at(model, pt, mu, 0.0, 0.0, "full")
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        m.mdsip_set_option_int(prob, "precision", prec, ctx)
        out = np.zeros(m.mdsip_packed_size(prob))
        inertia = m.mdsip_debug_direction(prob, pt.packed(), mu, 0.0, 0.0, out, refine=40, ctx=ctx)
    finally:
        m.mdsip_problem_destroy(prob)
    assert inertia == tuple(want["inertia"])
    ref = pack_dir(want)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-10


@pytest.mark.parametrize("spec", [1, 0])
@pytest.mark.parametrize("prec", TC_PRECS)
def test_tensor_core_solve_matches_oracle_trajectory(ctx, prec, spec):
    """The refined tensor-core solve, with (spec = 1, the default) and without
    the verified no-interchange panels of the FP32-update factorization: the
    oracle's iteration count, objective and inertia-correction sequence."""
    g = _golden("mds0_full")
    inst = _inst_for(g["case"])
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        m.mdsip_set_option_int(prob, "precision", prec, ctx)
        m.mdsip_set_option_int(prob, "ldlt_spec", spec, ctx)
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK" and stats["E0"] <= 1e-8
    assert stats["precision"] == prec
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    for rec, grec in zip(log, g["log"]):
        assert [tuple(c[2]) for c in rec["ic"]] == [tuple(c[2]) for c in grec.get("ic", [])]
    assert sum(r["n_refine"] for r in log) > 0
    compare_iterations(log, g["log"])


@pytest.mark.parametrize("prec", TC_PRECS)
def test_tensor_core_full_size(ctx, mds1, prec):
    """Benchmark size with the tensor-core product: refined direction equal to
    the oracle's to 1e-10, and the solve ends at E_0 <= 1e-8 (recomputed by the
    oracle) with the FP64 path's objective."""
    inst = mds1
    model = SynthModel(inst)
    pt = _point(synth.random_iterate(inst, 77))
    want = ipm.direction_at(model, pt, 0.01, 0.0, 0.0, "p2")
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        m.mdsip_set_option_int(prob, "precision", prec, ctx)
        out = np.zeros(m.mdsip_packed_size(prob))
        inertia = m.mdsip_debug_direction(prob, pt.packed(), 0.01, 0.0, 0.0, out, refine=40, ctx=ctx)
        assert inertia == tuple(want["inertia"])
        ref = pack_dir(want)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-10
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        packed = np.zeros(m.mdsip_packed_size(prob))
        m.mdsip_get_iterate(prob, packed, ctx=ctx)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK"
    P = ipm.Problem(model)
    n, m_I, m_E = inst.n, inst.m_I, inst.m_E
    o = np.cumsum([0, n, m_I, m_E, m_I, n, n, m_I, m_I])
    fin = ipm.Point(*(packed[o[i]:o[i + 1]] for i in range(8)))
    ev = ipm.Evals(P, fin.x, fin.d)
    assert ipm.kkt_error(P, fin, ev, 0.0, ipm.Options())[0] <= 1e-8
    g = _golden("mds1_p2")          # the oracle's own solve of this instance
    assert abs(ev.f - g["f"]) <= 1e-8 * abs(g["f"])
    assert stats["iters"] == g["iters"]


@pytest.mark.parametrize("prec", TC_PRECS)
def test_fp64_fallback_records_the_factor_used(ctx, prec):
    """A refinement target below any reachable residual sends every step of the
    mixed-precision solve to the FP64 re-factorization.  Each step then records
    the inertia of the FP64 factor its direction came from, which must be the
    target (n, m, 0), and the solve follows the oracle's trajectory (the
    nonconvex member, whose steps need inertia correction)."""
    g = _golden("mds0_nonconvex_full")
    inst = _inst_for(g["case"])
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        m.mdsip_set_option_int(prob, "precision", prec, ctx)
        m.mdsip_set_option_double(prob, "refine_fallback_tol", 1e-300, ctx)
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK" and stats["E0"] <= 1e-8
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    assert stats["n_fp64_fallback"] >= stats["iters"]
    for rec in log[:-1]:
        assert rec["fp64_fallback"] == 1
        assert rec["factor_inertia"] == (inst.n, inst.m, 0)
        assert rec["ic"][-1][2] == (inst.n, inst.m, 0)


def test_option_strings(ctx):
    """mdsip_set_option_str sets the same options as the integer setter, by
    word, and rejects unknown names and values with INVALID_ARG."""
    g = _golden("mds0_full")
    inst = _inst_for(g["case"])
    prob = make_problem(ctx, inst)
    try:
        m.mdsip_set_option_str(prob, "path", "p2", ctx)
        m.mdsip_set_option_str(prob, "precision", "bf16", ctx)
        m.mdsip_set_option_str(prob, "ldlt_spec", "no", ctx)
        for name, value in (("path", "p3"), ("precision", "fp16"), ("colour", "blue")):
            with pytest.raises(m.MdsipError) as ei:
                m.mdsip_set_option_str(prob, name, value, ctx)
            assert ei.value.status == 1
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK"
    assert stats["path"] == m.MDSIP_PATH_P2 and stats["precision"] == m.MDSIP_PREC_BF16
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])


@pytest.mark.parametrize("prec", TC_PRECS)
def test_direction_check_logs_the_gap_to_fp64(ctx, prec):
    """With direction_check on, every step of a mixed-precision solve logs the
    relative gap between its refined direction and the FP64 direction from the
    same iterate; the refined directions meet the FP64 bound of 1e-10 there,
    and the check leaves the trajectory as it was (same count, objective and
    per-iteration record as the oracle's)."""
    g = _golden("mds0_full")
    inst = _inst_for(g["case"])
    prob = make_problem(ctx, inst, m.MDSIP_PATH_P2)
    try:
        m.mdsip_set_option_int(prob, "precision", prec, ctx)
        m.mdsip_set_option_int(prob, "direction_check", 1, ctx)
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == "OK" and stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    errs = [r["dir_err_fp64"] for r in log[:-1]]
    assert len(errs) == g["iters"] and all(0.0 <= e <= 1e-10 for e in errs), errs
    assert log[-1]["dir_err_fp64"] == -1.0
    compare_iterations(log, g["log"])


# ---------------------------------------------------------------- J_sh != 0

JSH_CASES = [
    # (n_d, m_E, m_I, sigma_a, seed, q_shift, jsh_per_row)
    (4, 6, 2, 0.3, 1, 0.1, 2),
    (33, 70, 5, 0.1, 3, 0.1, 4),
    (6, 9, 3, 0.3, 4, -3.0, 3),     # indefinite Q
    (70, 130, 7, 0.05, 5, 0.1, 6),
]


@pytest.mark.parametrize("case", JSH_CASES)
@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (1e-4, 0.0), (3.0, 1e-7)])
def test_direction_parity_sparse_inequality_block(ctx, case, dw, dc):
    """Inequalities with a sparse x_s part (J_sh != 0): path AUTO takes P1, whose
    compressed matrix carries the J_sh blocks of J_s Q_s^-1 J_s^T; the direction
    equals the oracle's full 4x4 solve to 1e-10 with the same inertia."""
    n_d, m_E, m_I, sa, seed, qs, jsh = case
    inst = synth.make_instance(n_d, m_E, m_I, sa, seed=seed, q_shift=qs, jsh_per_row=jsh)
    model = SynthModel(inst)
    pt = _point(synth.random_iterate(inst, seed + 100))
    mu = 0.05
    want = ipm.direction_at(model, pt, mu, dw, dc, "full")
    prob = make_problem(ctx, inst)
    try:
        out = np.zeros(m.mdsip_packed_size(prob))
        inertia = m.mdsip_debug_direction(prob, pt.packed(), mu, dw, dc, out, ctx=ctx)
        assert m.mdsip_get_stats(prob)["path"] in (0, m.MDSIP_PATH_P1)
        m.mdsip_set_option_int(prob, "path", m.MDSIP_PATH_P2, ctx)
        with pytest.raises(m.MdsipError) as ei:      # P2's precondition: J_sh = 0
            m.mdsip_debug_direction(prob, pt.packed(), mu, dw, dc, out, ctx=ctx)
        assert ei.value.status == 10 and "J_sh" in str(ei.value)
    finally:
        m.mdsip_problem_destroy(prob)
    assert inertia == tuple(want["inertia"])
    ref = pack_dir(want)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-10


def test_sparse_inequality_block_trajectory(ctx):
    """The member-0 shape with four active inequalities carrying a sparse x_s
    part (nonconvex, so inertia correction runs): the oracle's iteration
    count, inertia-correction sequence, per-iteration record and objective."""
    g = _golden("mds0_jsh_full")
    c = g["case"]
    inst = synth.make_instance(c["n_d"], c["m_E"], c["m_I"], c["sigma_a"], seed=c["seed"],
                               q_shift=c["q_shift"], jsh_per_row=c["jsh_per_row"])
    prob = make_problem(ctx, inst)
    try:
        st = m.mdsip_solve(prob, ctx)
        stats = m.mdsip_get_stats(prob)
        log = m.mdsip_get_log(prob)
    finally:
        m.mdsip_problem_destroy(prob)
    assert m.STATUS[st] == g["status"] == "OK"
    assert stats["path"] == m.MDSIP_PATH_P1
    assert stats["iters"] == g["iters"]
    assert abs(stats["f"] - g["f"]) <= 1e-8 * abs(g["f"])
    for rec, grec in zip(log, g["log"]):
        want = grec.get("ic", [])
        assert len(rec["ic"]) == len(want), (rec["iter"], rec["ic"], want)
        for (dw, dc, inr), (gdw, gdc, ginr) in zip(rec["ic"], want):
            assert tuple(inr) == tuple(ginr)
            assert dw == pytest.approx(gdw, rel=1e-12, abs=0)
            assert dc == pytest.approx(gdc, rel=1e-12, abs=0)
    compare_iterations(log, g["log"])
