"""Pins of oracle.ipm (filter line-search IPM of Section 2.1).

Closed-form optima:
 (i)   equality QP  min 1/2 x_d^T Q x_d + c_d^T x_d + 1/2 ||x_s||^2  s.t. identity-pair
       rows:  x_d* = (Q + A^T A / 2)^-1 (A^T b / 2 - c_d),  x_s,i = -x_s,i+m = (b_i - a_i^T x_d*) / 2
 (ii)  ball         min 1/2 ||x_d - t||^2  s.t. ||x_d||^2 <= 4,  ||t|| = 3:
       x* = 2 t / 3, multiplier 1/4
 (iii) box          min sum 1/2 (x_i - t_i)^2  s.t. -1 <= x <= 1:  x* = clip(t)
and an independent library optimizer (scipy trust-constr) on a tiny synthetic
instance; every accepted factorization has the target inertia.
"""
import numpy as np
import pytest
import warnings
import scipy.optimize as so
import scipy.sparse as sp

import synth
from oracle import ipm
from oracle.model import SynthModel


class _Model:
    """Generic small MDS model: f = 1/2 x_d^T Q x_d + c_d^T x_d + sum 1/2 p_i x_s,i^2 + c_s^T x_s,
    g = Jsg x_s + A x_d, h_j = ||x_d[S_j]||^2 (x_d free unless bounds given)."""

    def __init__(self, n_s, n_d, Q, c_d, p, c_s, Jsg, A, gE, h_set, hu, xl, xu):
        self.n_s, self.n_d = n_s, n_d
        self.m_E = A.shape[0]
        self.m_I = hu.size
        self.n = n_s + n_d
        self.Q, self.c_d, self.p, self.c_s = Q, c_d, p, c_s
        self.Jsg = sp.csr_matrix(Jsg)
        self.Jsh = sp.csr_matrix((self.m_I, n_s))
        self.A, self.gE = A, gE
        k = np.nonzero(h_set >= 0)[0]
        self.E = sp.csr_matrix((np.ones(k.size), (h_set[k], k)), shape=(self.m_I, n_d))
        self.hu = hu
        self.hl = np.full(self.m_I, -np.inf)
        self.xl, self.xu = xl, xu

    def f(self, x):
        xs, xd = x[:self.n_s], x[self.n_s:]
        return 0.5 * xd @ self.Q @ xd + self.c_d @ xd + 0.5 * np.sum(self.p * xs ** 2) + self.c_s @ xs

    def grad_f(self, x):
        xs, xd = x[:self.n_s], x[self.n_s:]
        return np.concatenate([self.p * xs + self.c_s, self.Q @ xd + self.c_d])

    def g(self, x):
        return self.Jsg @ x[:self.n_s] + self.A @ x[self.n_s:]

    def h(self, x):
        xd = x[self.n_s:]
        return self.E @ (xd * xd)

    def jac(self, x):
        xd = x[self.n_s:]
        return self.Jsg, self.Jsh, self.A, self.E.toarray() * (2 * xd)[None, :]

    def hess(self, x, yg, yh):
        return self.p.copy(), self.Q + np.diag(2.0 * (self.E.T @ yh))


def test_equality_qp_closed_form():
    rng = np.random.default_rng(1)
    n_d, m = 5, 7
    G = rng.standard_normal((n_d, n_d))
    Q = G.T @ G / n_d + 0.1 * np.eye(n_d)
    c_d = rng.uniform(-1, 1, n_d)
    A = 0.3 * rng.standard_normal((m, n_d))
    b = rng.uniform(-0.5, 0.5, m)
    Jsg = np.hstack([np.eye(m), -np.eye(m)])
    mod = _Model(2 * m, n_d, Q, c_d, np.ones(2 * m), np.zeros(2 * m), Jsg, A, b,
                 -np.ones(n_d, dtype=np.int32), np.zeros(0),
                 np.full(2 * m + n_d, -np.inf), np.full(2 * m + n_d, np.inf))
    for ls in ("full", "p1", "p2"):
        r = ipm.solve(mod, x0=np.zeros(mod.n), opt=ipm.Options(linsolve=ls))
        assert r["status"] == 0 and r["E0"] <= 1e-8
        xd = np.linalg.solve(Q + 0.5 * A.T @ A, 0.5 * A.T @ b - c_d)
        xs = (b - A @ xd) / 2
        np.testing.assert_allclose(r["point"].x[2 * m:], xd, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(r["point"].x[:m], xs, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(r["point"].x[m:2 * m], -xs, rtol=1e-9, atol=1e-10)


def test_ball_closed_form_with_multiplier():
    rng = np.random.default_rng(2)
    n_d = 6
    t = rng.standard_normal(n_d)
    t *= 3.0 / np.linalg.norm(t)
    mod = _Model(0, n_d, np.eye(n_d), -t, np.zeros(0), np.zeros(0), np.zeros((0, 0)),
                 np.zeros((0, n_d)), np.zeros(0), np.zeros(n_d, dtype=np.int32), np.array([4.0]),
                 np.full(n_d, -np.inf), np.full(n_d, np.inf))
    r = ipm.solve(mod, x0=np.zeros(n_d))
    assert r["status"] == 0
    np.testing.assert_allclose(r["point"].x, 2 * t / 3, atol=1e-7)
    assert r["point"].yh[0] == pytest.approx(0.25, abs=1e-7)
    assert r["point"].vu[0] == pytest.approx(0.25, abs=1e-7)


def test_box_closed_form():
    t = np.array([-2.5, -1.0, -0.3, 0.0, 0.7, 1.2, 3.0])
    n = t.size
    mod = _Model(n, 0, np.zeros((0, 0)), np.zeros(0), np.ones(n), -t, np.zeros((0, n)),
                 np.zeros((0, 0)), np.zeros(0), np.zeros(0, dtype=np.int32), np.zeros(0),
                 -np.ones(n), np.ones(n))
    r = ipm.solve(mod, x0=np.zeros(n))
    assert r["status"] == 0
    # t = -1 sits on its bound with a zero multiplier (no strict complementarity):
    # there the barrier bias decays like sqrt(mu) instead of mu.
    strict = t != -1.0
    np.testing.assert_allclose(r["point"].x[strict], np.clip(t, -1, 1)[strict], atol=1e-7)
    assert abs(r["point"].x[~strict][0] + 1.0) <= 1e-3
    np.testing.assert_allclose(r["point"].zu, np.maximum(t - 1, 0), atol=1e-6)
    np.testing.assert_allclose(r["point"].zl[strict], np.maximum(-1 - t, 0)[strict], atol=1e-6)
    assert r["point"].zl[~strict][0] <= 1e-3


def _scipy_opt(inst):
    m = SynthModel(inst)
    cons = [so.NonlinearConstraint(m.g, inst.b, inst.b, jac=lambda x: np.hstack([m.jac(x)[0].toarray(), m.jac(x)[2]])),
            so.NonlinearConstraint(m.h, inst.hl, inst.hu, jac=lambda x: np.hstack([m.jac(x)[1].toarray(), m.jac(x)[3]]))]
    bounds = so.Bounds(inst.xl, inst.xu)
    warnings.filterwarnings("ignore", category=UserWarning)
    res = so.minimize(m.f, np.zeros(m.n), jac=m.grad_f, method="trust-constr", constraints=cons,
                      bounds=bounds, options=dict(gtol=1e-12, xtol=1e-14, maxiter=5000))
    return res


@pytest.mark.parametrize("ls", ["full", "p1", "p2"])
def test_synthetic_matches_library_optimizer(ls):
    inst = synth.make_instance(4, 6, 2, 0.3, seed=3)
    r = ipm.solve(SynthModel(inst), opt=ipm.Options(linsolve=ls))
    assert r["status"] == 0 and r["E0"] <= 1e-8
    ref = _scipy_opt(inst)
    assert abs(r["f"] - ref.fun) <= 1e-6 * max(1.0, abs(ref.fun))
    np.testing.assert_allclose(r["point"].x, ref.x, atol=1e-4)
    target = (inst.n, inst.m, 0)
    for rec in r["log"][:-1]:
        assert rec["ic"][-1][2] == target


def test_nonconvex_synthetic_uses_inertia_correction():
    inst = synth.make_instance(6, 8, 1, 0.3, seed=4, q_shift=-1.0)
    r = ipm.solve(SynthModel(inst), opt=ipm.Options(linsolve="full"))
    assert r["status"] == 0 and r["E0"] <= 1e-8
    tries = [len(rec["ic"]) for rec in r["log"][:-1]]
    assert max(tries) >= 2
    target = (inst.n, inst.m, 0)
    for rec in r["log"][:-1]:
        assert rec["ic"][-1][2] == target
    # second-order condition at the solution: the reduced Hessian is PSD on the
    # null space of the active constraints -> a local minimum; compare with the
    # library optimizer started from the same solution
    ref = _scipy_opt(inst)
    assert r["f"] <= ref.fun + 1e-6 * max(1.0, abs(ref.fun))


def test_sparse_inequality_block_matches_library_optimizer():
    """Inequalities with a sparse x_s part (J_sh != 0, path P1 and the full
    solve): the oracle's optimum equals scipy's trust-constr optimum, and every
    accepted factorization has the target inertia."""
    inst = synth.make_instance(4, 6, 2, 0.3, seed=3, jsh_per_row=2)
    ref = _scipy_opt(inst)
    for ls in ("full", "p1"):
        r = ipm.solve(SynthModel(inst), opt=ipm.Options(linsolve=ls))
        assert r["status"] == 0 and r["E0"] <= 1e-8
        assert abs(r["f"] - ref.fun) <= 1e-6 * max(1.0, abs(ref.fun))
        np.testing.assert_allclose(r["point"].x, ref.x, atol=1e-4)
        for rec in r["log"][:-1]:
            assert rec["ic"][-1][2] == (inst.n, inst.m, 0)
