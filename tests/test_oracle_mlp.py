"""Pins of the warm-start oracle (oracle/mlp.py) against facts that do not
depend on it: finite differences, a direct matrix product, torch's bfloat16
conversion, Adam's closed form for a constant gradient, numpy's moments and
the defining inequalities of the interior projection."""
import math

import numpy as np
import pytest

from oracle import mlp as om
import synth


def _net(I=5, H=7, O=4, seed=0):
    p = synth.mlp_init(I, H, O, seed, out_scale=1.0)
    p = {k: v.astype(np.float64) for k, v in p.items()}
    rng = np.random.default_rng(seed + 1)
    p["b1"] = rng.uniform(-0.3, 0.3, H)
    p["b2"] = rng.uniform(-0.3, 0.3, H)
    p["b3"] = rng.uniform(-0.3, 0.3, O)
    return p


def _scaling(I, O, seed=3):
    rng = np.random.default_rng(seed)
    return dict(in_mean=rng.uniform(-0.2, 0.2, I), in_std=rng.uniform(0.5, 2.0, I),
                out_mean=rng.uniform(-1, 1, O), out_std=rng.uniform(0.5, 2.0, O))


def test_gradient_matches_central_differences():
    I, H, O, B = 5, 7, 4, 6
    p = _net(I, H, O)
    sc = _scaling(I, O)
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, (B, I))
    Y = rng.normal(size=(B, O))
    L, g = om.loss_and_grad(p, X, Y, sc)
    h = 1e-6
    for k in om.BLOCKS:
        flat = p[k].reshape(-1)
        for j in range(flat.size):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k].reshape(-1)[j] += h
            Lp, _ = om.loss_and_grad(q, X, Y, sc)
            q[k].reshape(-1)[j] -= 2 * h
            Lm, _ = om.loss_and_grad(q, X, Y, sc)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[j]) <= 1e-7 + 1e-6 * abs(fd), (k, j, fd, g[k].reshape(-1)[j])


def test_linear_regime_equals_matrix_product():
    # biases large enough that no unit is cut by the ReLU: the net is affine
    I, H, O, B = 4, 6, 3, 5
    p = _net(I, H, O, seed=5)
    p["b1"] = np.full(H, 50.0)
    p["b2"] = np.full(H, 500.0)
    p["W2"] = np.abs(p["W2"])
    sc = dict(in_mean=np.zeros(I), in_std=np.ones(I), out_mean=np.zeros(O), out_std=np.ones(O))
    X = np.random.default_rng(2).uniform(-1, 1, (B, I))
    got = om.predict(p, X, sc)
    Wc = np.linalg.multi_dot([p["W3"], p["W2"], p["W1"]])
    bc = p["W3"] @ (p["W2"] @ p["b1"] + p["b2"]) + p["b3"]
    np.testing.assert_allclose(got, X @ Wc.T + bc, rtol=1e-12, atol=1e-10)


def test_scaling_is_applied_on_both_ends():
    I, H, O = 3, 4, 2
    p = _net(I, H, O, seed=9)
    sc = _scaling(I, O)
    X = np.random.default_rng(4).uniform(-1, 1, (3, I))
    c = om.forward(p, X, sc["in_mean"], sc["in_std"])
    np.testing.assert_allclose(c["xn"], (X - sc["in_mean"]) / sc["in_std"], rtol=1e-15)
    np.testing.assert_allclose(om.predict(p, X, sc), c["yn"] * sc["out_std"] + sc["out_mean"], rtol=1e-15)


def test_bf16_round_hand_worked_and_torch():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert om.bf16_round(one) == 1.0
    assert om.bf16_round(1.0 + 2.0 ** -8) == 1.0                 # tie -> even (down)
    assert om.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert om.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert om.bf16_round(-2.5) == -2.5
    v = np.random.default_rng(0).normal(size=4096) * np.exp(np.random.default_rng(1).uniform(-20, 20, 4096))
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(om.bf16_round(v), ref)


def test_bf16_mode_differs_only_by_rounding():
    I, H, O, B = 8, 16, 5, 7
    p = _net(I, H, O, seed=2)
    sc = _scaling(I, O)
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (B, I))
    Y = rng.normal(size=(B, O))
    L0, g0 = om.loss_and_grad(p, X, Y, sc, bf16=False)
    L1, g1 = om.loss_and_grad(p, X, Y, sc, bf16=True)
    assert abs(L1 - L0) <= 0.05 * L0
    for k in om.BLOCKS:
        assert np.linalg.norm(g1[k] - g0[k]) <= 0.05 * np.linalg.norm(g0[k]) + 1e-12, k


def test_adam_two_steps_constant_gradient_closed_form():
    # with a constant gradient g, m_t / (1 - b1^t) = g and v_t / (1 - b2^t) = g^2
    # for every t, so each step moves w by -lr g / (|g| + eps)
    g = {"w": np.array([1e-3, -2.0, 0.5, 0.0, -1e-9])}
    w0 = {"w": np.array([0.1, 0.2, -0.3, 0.4, 0.5])}
    m = {"w": np.zeros(5)}
    v = {"w": np.zeros(5)}
    lr, eps = 0.01, 1e-8
    w1, m, v = om.adam_step(w0, g, m, v, 1, lr, eps=eps)
    w2, m, v = om.adam_step(w1, g, m, v, 2, lr, eps=eps)
    step = lr * g["w"] / (np.abs(g["w"]) + eps)
    np.testing.assert_allclose(w1["w"], w0["w"] - step, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(w2["w"], w0["w"] - 2 * step, rtol=1e-12, atol=1e-15)


def test_col_stats_matches_numpy_and_floor():
    Y = np.random.default_rng(7).normal(size=(50, 6)) * [1, 2, 3, 0, 1e-9, 5] + [0, 1, -2, 7, 3, 0]
    mu, sd = om.col_stats(Y)
    np.testing.assert_allclose(mu, Y.mean(axis=0), rtol=1e-14, atol=1e-14)
    ref = Y.std(axis=0)
    np.testing.assert_allclose(sd[[0, 1, 2, 5]], ref[[0, 1, 2, 5]], rtol=1e-13)
    assert sd[3] == pytest.approx(7e-6) and sd[4] == pytest.approx(3e-6)


def test_push_inside_rule():
    lo = np.array([-1.0, -np.inf, 0.0, -3.0, 5.0])
    hi = np.array([1.0, 2.0, np.inf, 3.0, 5.0 + 1e-3])
    v = np.array([-1.0, 2.5, -4.0, 0.0, 7.0])
    out = om.push_inside(v, lo, hi, 1e-2, 1e-2)
    assert out[0] == -1.0 + 1e-2              # at the lower bound: pushed by k1 max(1, |lo|)
    assert out[1] == 2.0 - 2e-2               # above the upper bound: clamped, push 1e-2 * 2
    assert out[2] == 0.0 + 1e-2
    assert out[3] == 0.0                      # interior, unchanged
    assert out[4] == pytest.approx(5.0 + 1e-3 - 1e-5, abs=1e-15)  # narrow box: upper push k2 (hi - lo)
    assert np.all((out > lo) | ~np.isfinite(lo)) and np.all((out < hi) | ~np.isfinite(hi))


def test_project_start_interior_and_centred():
    n, m_E, m_I = 6, 2, 2
    xl = np.array([-1, -1, -1, -np.inf, -np.inf, 0.0])
    xu = np.array([1, 1, np.inf, np.inf, 1.0, np.inf])
    hl = np.array([-np.inf, 0.0])
    hu = np.array([1.0, 2.0])
    rng = np.random.default_rng(0)
    pred = rng.normal(size=3 * n + 4 * m_I + m_E) * 2
    mu0 = 1e-3
    out = om.project_start(pred, n, m_E, m_I, xl, xu, hl, hu, 1e-4, mu0)
    off = np.cumsum([0, n, m_I, m_E, m_I, n, n, m_I, m_I])
    x, d, yg, yh, zl, zu, vl, vu = (out[off[i]:off[i + 1]] for i in range(8))
    assert np.all(x[np.isfinite(xl)] > xl[np.isfinite(xl)]) and np.all(x[np.isfinite(xu)] < xu[np.isfinite(xu)])
    assert np.all(d[np.isfinite(hl)] > hl[np.isfinite(hl)]) and np.all(d[np.isfinite(hu)] < hu[np.isfinite(hu)])
    for z, s, fin in ((zl, x - xl, np.isfinite(xl)), (zu, xu - x, np.isfinite(xu)),
                      (vl, d - hl, np.isfinite(hl)), (vu, hu - d, np.isfinite(hu))):
        assert np.all(z[~fin] == 0.0)
        assert np.all(z[fin] * s[fin] >= mu0 * (1 - 1e-15))
    np.testing.assert_array_equal(yg, pred[off[2]:off[3]])
    np.testing.assert_array_equal(yh, pred[off[3]:off[4]])
    # an interior, well-centred prediction is returned unchanged
    x0 = np.array([0.2, -0.3, 0.1, 5.0, 0.5, 2.0])
    d0 = np.array([0.5, 1.0])
    zl0 = np.where(np.isfinite(xl), 1.0, 0.0)
    zu0 = np.where(np.isfinite(xu), 1.0, 0.0)
    vl0 = np.where(np.isfinite(hl), 1.0, 0.0)
    vu0 = np.where(np.isfinite(hu), 1.0, 0.0)
    p0 = np.concatenate([x0, d0, [0.3, -0.1], [0.2, 0.4], zl0, zu0, vl0, vu0])
    np.testing.assert_array_equal(om.project_start(p0, n, m_E, m_I, xl, xu, hl, hu, 1e-4, 1e-3), p0)


def test_clamp_and_target_rules():
    assert om.clamp_mu0(math.log(1e-4), 1e-8, 0.1) == pytest.approx(1e-4)
    assert om.clamp_mu0(math.log(1e-20), 1e-8, 0.1) == pytest.approx(1e-9)
    assert om.clamp_mu0(5.0, 1e-8, 0.1) == pytest.approx(0.1)
    assert om.clamp_mu0(float("nan"), 1e-8, 0.1) == pytest.approx(0.1)
    rec = [(10.0, 0.1), (0.5, 0.02), (1e-3, 2.8e-3), (1e-6, 1e-5), (1e-9, 1e-9)]
    assert om.warmstart_log_mu(rec, 1e-2) == pytest.approx(math.log(2.8e-3))
    assert om.warmstart_log_mu(rec, 1e-12) == pytest.approx(math.log(1e-9))


def test_family_rhs_blocks():
    inst = synth.make_instance(4, 10, 1, 0.1, seed=0)
    p = np.array([1.0, -1.0, 0.5])
    b = synth.family_rhs(inst, p, 0.2)
    f = np.array([1.2] * 3 + [0.8] * 3 + [1.1] * 4)
    np.testing.assert_allclose(b, inst.b * f, rtol=1e-15)
