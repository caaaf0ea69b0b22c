"""Pins of oracle.kkt and of the Newton system built by oracle.ipm.

* the full (Eq. (linsys4x4)), compressed (Eq. (compressed)) and two-stage
  directions agree with each other and with the unreduced system that keeps
  the slack d as an unknown;
* with no shifts, the direction (including the bound-multiplier steps) is the
  Newton step on the perturbed KKT conditions, whose Jacobian is taken here by
  finite differences -- a formula independent of the Sigma-form elimination;
* inertias from LDL^T, Haynsworth sums and dense eigenvalues coincide.
"""
import numpy as np
import pytest

import synth
from oracle import kkt, ipm
from oracle.model import SynthModel


def _setup(n_d=4, m_E=6, m_I=2, seed=5, q_shift=0.1, spread=1.0, jsh=0):
    inst = synth.make_instance(n_d, m_E, m_I, 0.3, seed=seed, q_shift=q_shift, jsh_per_row=jsh)
    model = SynthModel(inst)
    it = synth.random_iterate(inst, seed + 1, spread=spread)
    pt = ipm.Point(it["x"], it["d"], it["yg"], it["yh"], it["zl"], it["zu"], it["vl"], it["vu"])
    P = ipm.Problem(model)
    ev = ipm.Evals(P, pt.x, pt.d)
    return inst, model, P, pt, ev


def _unreduced(sy, dw, dc):
    """5x5 system with d kept: [[W+Sx+dw,0,Jg^T,Jh^T],[0,Sd+dw,0,-I],[Jg,0,-dc,0],[Jh,-I,0,-dc]]."""
    n_s, n_d, m_E, m_I = sy.dims
    n = n_s + n_d
    N = n + m_I + m_E + m_I
    K = np.zeros((N, N))
    W = np.zeros((n, n))
    W[:n_s, :n_s] = np.diag(sy.Hss)
    W[n_s:, n_s:] = sy.Hdd
    K[:n, :n] = W + np.diag(np.concatenate([sy.sig_xs, sy.sig_xd])) + dw * np.eye(n)
    o_d, o_g, o_h = n, n + m_I, n + m_I + m_E
    K[o_d:o_g, o_d:o_g] = np.diag(sy.sig_d + dw)
    Jg = np.hstack([sy.Jsg.toarray(), sy.A])
    Jh = np.hstack([sy.Jsh.toarray(), sy.Jdh])
    K[o_g:o_h, :n] = Jg
    K[:n, o_g:o_h] = Jg.T
    K[o_h:, :n] = Jh
    K[:n, o_h:] = Jh.T
    K[o_h:, o_d:o_g] = -np.eye(m_I)
    K[o_d:o_g, o_h:] = -np.eye(m_I)
    K[o_g:o_h, o_g:o_h] = -dc * np.eye(m_E)
    K[o_h:, o_h:] = -dc * np.eye(m_I)
    rhs = -np.concatenate([sy.r_xs, sy.r_xd, sy.r_d, sy.r_g, sy.r_h])
    sol = np.linalg.solve(K, rhs)
    return dict(dx=sol[:n], dd=sol[o_d:o_g], dyg=sol[o_g:o_h], dyh=sol[o_h:])


@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (1e-3, 0.0), (0.5, 1e-6)])
def test_three_directions_agree_with_unreduced(dw, dc):
    inst, model, P, pt, ev = _setup()
    sy = ipm.newton_system(P, pt, ev, mu=0.05)
    ref = _unreduced(sy, dw, dc)
    scale = np.linalg.norm(np.concatenate([ref["dx"], ref["dd"], ref["dyg"], ref["dyh"]]))
    for name, fn in kkt.DIRECTIONS.items():
        r = fn(sy, dw, dc)
        got = np.concatenate([r["dxs"], r["dxd"], r["dd"], r["dyg"], r["dyh"]])
        want = np.concatenate([ref["dx"], ref["dd"], ref["dyg"], ref["dyh"]])
        assert np.linalg.norm(got - want) <= 1e-11 * scale, name


def _kkt_F(P, model, v, mu, sizes):
    n, m_I, m_E = sizes
    o = np.cumsum([0, n, m_I, m_E, m_I, n, n, m_I, m_I])
    x, d, yg, yh, zl, zu, vl, vu = (v[o[i]:o[i + 1]] for i in range(8))
    Jsg, Jsh, A, Jdh = model.jac(x)
    Jg = np.hstack([Jsg.toarray(), A])
    Jh = np.hstack([Jsh.toarray(), Jdh])
    sl, su, tl, tu = P.slacks(x, d)
    F1 = model.grad_f(x) + Jg.T @ yg + Jh.T @ yh - zl + zu
    F2 = -yh - vl + vu
    F3 = model.g(x) - model.gE
    F4 = model.h(x) - d
    hxl, hxu, hdl, hdu = P.masks()
    F5 = np.where(hxl, sl * zl - mu, zl)        # multipliers of absent bounds pinned at 0
    F6 = np.where(hxu, su * zu - mu, zu)
    F7 = np.where(hdl, tl * vl - mu, vl)
    F8 = np.where(hdu, tu * vu - mu, vu)
    return np.concatenate([F1, F2, F3, F4, F5, F6, F7, F8])


def test_direction_is_newton_step_on_perturbed_kkt():
    inst, model, P, pt, ev = _setup(n_d=3, m_E=4, m_I=1, seed=9)
    mu = 0.03
    n, m_I, m_E = P.n, P.m_I, P.m_E
    v0 = pt.packed()
    F0 = _kkt_F(P, model, v0, mu, (n, m_I, m_E))
    J = np.zeros((F0.size, v0.size))
    eps = 1e-6
    for i in range(v0.size):
        e = np.zeros_like(v0)
        e[i] = eps
        J[:, i] = (_kkt_F(P, model, v0 + e, mu, (n, m_I, m_E)) - _kkt_F(P, model, v0 - e, mu, (n, m_I, m_E))) / (2 * eps)
    newton = np.linalg.solve(J, -F0)
    r = ipm.direction_at(model, pt, mu, 0.0, 0.0, "full")
    ours = np.concatenate([r["dx"], r["dd"], r["dyg"], r["dyh"], r["dzl"], r["dzu"], r["dvl"], r["dvu"]])
    np.testing.assert_allclose(ours, newton, rtol=1e-6, atol=1e-7 * np.abs(newton).max())


def _eig_inertia(K):
    ev = np.linalg.eigvalsh(K)
    tol = 1e-12 * np.abs(ev).max()
    return int(np.sum(ev > tol)), int(np.sum(ev < -tol)), int(np.sum(np.abs(ev) <= tol))


@pytest.mark.parametrize("q_shift", [0.1, -3.0])
@pytest.mark.parametrize("dw", [0.0, 1e-4, 10.0])
def test_inertia_haynsworth(q_shift, dw):
    inst, model, P, pt, ev = _setup(n_d=6, m_E=5, m_I=1, seed=21, q_shift=q_shift)
    sy = ipm.newton_system(P, pt, ev, mu=0.1)
    K, _ = kkt.assemble_k4(sy, dw, 0.0)
    want = _eig_inertia(K)
    assert kkt.direction_full(sy, dw, 0.0)["inertia"] == want
    assert kkt.direction_p1(sy, dw, 0.0)["inertia"] == want
    assert kkt.direction_p2(sy, dw, 0.0)["inertia"] == want
    if q_shift > 0:
        assert want == (P.n, P.m_E + P.m_I, 0)      # convex: correct without correction
    if dw >= 10.0:
        assert want == (P.n, P.m_E + P.m_I, 0)      # large shift restores the target


def test_nonconvex_needs_correction():
    inst, model, P, pt, ev = _setup(n_d=6, m_E=5, m_I=1, seed=21, q_shift=-3.0)
    sy = ipm.newton_system(P, pt, ev, mu=0.1)
    assert kkt.direction_p2(sy, 0.0, 0.0)["inertia"] != (P.n, P.m_E + P.m_I, 0)
    state = dict(dw_last=0.0)
    res, attempts = ipm.compute_direction(P, pt, ev, 0.1, ipm.Options(linsolve="p2"), state)
    assert res is not None and len(attempts) >= 2
    assert attempts[-1][2] == (P.n, P.m_E + P.m_I, 0)
    assert attempts[1][0] == 1e-4                    # first shift dw0
    for (a, _, _), (b, _, _) in zip(attempts[1:], attempts[2:]):
        assert b == pytest.approx(100.0 * a)         # first-time growth factor
    assert state["dw_last"] == attempts[-1][0]


# ---------------------------------------------------------------- J_sh != 0

@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (1e-3, 0.0), (0.5, 1e-6)])
def test_sparse_inequality_block_directions_agree(dw, dc):
    """Inequalities with a sparse x_s part (J_sh != 0): the full and compressed
    solves agree with the unreduced system, the two-stage form does not apply
    (J_s Q_s^-1 J_s^T couples g and h rows), and both inertias are the
    eigenvalue inertia of the 4x4 matrix."""
    inst, model, P, pt, ev = _setup(n_d=5, m_E=7, m_I=3, seed=31, jsh=3)
    sy = ipm.newton_system(P, pt, ev, mu=0.05)
    assert sy.Jsh.nnz == 9
    assert not kkt.p2_applicable(sy.Jsg, sy.Jsh)
    ref = _unreduced(sy, dw, dc)
    want = np.concatenate([ref["dx"], ref["dd"], ref["dyg"], ref["dyh"]])
    K, _ = kkt.assemble_k4(sy, dw, dc)
    for name in ("full", "p1"):
        r = kkt.DIRECTIONS[name](sy, dw, dc)
        got = np.concatenate([r["dxs"], r["dxd"], r["dd"], r["dyg"], r["dyh"]])
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want), name
        assert r["inertia"] == _eig_inertia(K), name


def test_sparse_inequality_block_newton_step():
    """With J_sh != 0 the direction is still the Newton step on the perturbed
    KKT conditions (Jacobian by finite differences)."""
    inst, model, P, pt, ev = _setup(n_d=3, m_E=4, m_I=2, seed=13, jsh=2)
    assert model.Jsh.nnz == 4
    mu = 0.03
    n, m_I, m_E = P.n, P.m_I, P.m_E
    v0 = pt.packed()
    F0 = _kkt_F(P, model, v0, mu, (n, m_I, m_E))
    J = np.zeros((F0.size, v0.size))
    eps = 1e-6
    for i in range(v0.size):
        e = np.zeros_like(v0)
        e[i] = eps
        J[:, i] = (_kkt_F(P, model, v0 + e, mu, (n, m_I, m_E)) - _kkt_F(P, model, v0 - e, mu, (n, m_I, m_E))) / (2 * eps)
    newton = np.linalg.solve(J, -F0)
    r = ipm.direction_at(model, pt, mu, 0.0, 0.0, "p1")
    ours = np.concatenate([r["dx"], r["dd"], r["dyg"], r["dyh"], r["dzl"], r["dzu"], r["dvl"], r["dvu"]])
    np.testing.assert_allclose(ours, newton, rtol=1e-6, atol=1e-7 * np.abs(newton).max())
