"""Hand-worked pins of the step rules inside oracle.ipm (W&B filter line search,
which Section 2.1 delegates to).

Each expected value below is worked out by hand in the comment beside it from
the rule as W&B state it, not recomputed with the oracle's own expression, so
that a dropped term, a wrong side of tau, a swapped scaling or a wrong branch
fails here on the CPU:

* fraction-to-boundary (W&B eq. (15)) and which slacks/steps enter it;
* the scaled KKT error's s_d / s_c (W&B eq. (5));
* the barrier-parameter update (W&B eq. (7));
* alpha_min (eq. (23)), the switching condition, Armijo, sufficient decrease,
  the theta_min branch, theta_max and the filter (eqs. (18)-(22));
* Algorithm IC's shift schedule (W&B Section 3.1), through a stand-in linear
  solve whose inertia is scripted;
* the starting-point push (W&B Section 3.6) and the kappa_Sigma safeguard
  (eq. (16)).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ipm, kkt


OPT = ipm.Options()


class _Box:
    """min sum 1/2 x_i^2 - t_i x_i over n_s sparse variables with -1 <= x <= 1,
    equality rows J x = gE (J given), no dense part, no inequalities."""

    def __init__(self, t, J, gE):
        self.n_s, self.n_d = t.size, 0
        self.m_E, self.m_I = J.shape[0], 0
        self.n = self.n_s
        self.t = t
        self.J = sp.csr_matrix(J)
        self.gE = np.asarray(gE, dtype=np.float64)
        self.xl, self.xu = -np.ones(self.n), np.ones(self.n)
        self.hl = self.hu = np.zeros(0)

    def f(self, x):
        return 0.5 * x @ x - self.t @ x

    def grad_f(self, x):
        return x - self.t

    def g(self, x):
        return self.J @ x

    def h(self, x):
        return np.zeros(0)

    def jac(self, x):
        return self.J, sp.csr_matrix((0, self.n)), np.zeros((self.m_E, 0)), np.zeros((0, 0))

    def hess(self, x, yg, yh):
        return np.ones(self.n), np.zeros((0, 0))


def _pt(x, yg, zl, zu):
    e = np.zeros(0)
    return ipm.Point(np.array(x, float), e, np.array(yg, float), e, np.array(zl, float),
                     np.array(zu, float), e, e)


# ---------------------------------------------------------------- fraction to boundary

def test_fraction_to_boundary_hand_worked():
    tau = 0.99
    # only the first pair decreases: alpha = tau * 1 / 2 = 0.495
    assert ipm.fraction_to_boundary(tau, [np.array([1.0, 2.0])], [np.array([-2.0, 1.0])]) == 0.495
    # both decrease: min(0.99 * 1 / 4, 0.99 * 4 / 1) = 0.2475
    assert ipm.fraction_to_boundary(tau, [np.array([1.0, 4.0])], [np.array([-4.0, -1.0])]) == 0.2475
    # nothing decreases, or the bound lies beyond a full step: alpha = 1
    assert ipm.fraction_to_boundary(tau, [np.array([1.0])], [np.array([3.0])]) == 1.0
    assert ipm.fraction_to_boundary(tau, [np.array([1.0])], [np.array([-0.5])]) == 1.0
    # the minimum runs over every array: 0.99 * 3 / 10 = 0.297
    a = ipm.fraction_to_boundary(tau, [np.array([0.5]), np.array([3.0])],
                                 [np.array([1.0]), np.array([-10.0])])
    assert a == pytest.approx(0.297, rel=1e-15)
    # at the returned alpha the binding entry sits exactly at (1 - tau) of its value
    v, dv = np.array([1.0, 4.0]), np.array([-4.0, -1.0])
    a = ipm.fraction_to_boundary(0.9, [v], [dv])
    assert v[0] + a * dv[0] == pytest.approx(0.1 * v[0], rel=1e-14)


def test_step_to_boundary_uses_the_right_slacks_and_signs():
    # x in [-1, 1]^2 at x = (0.5, 0.0): slacks x - xl = (1.5, 1.0), xu - x = (0.5, 1.0)
    # dx = (1.0, -4.0): x_1 approaches its upper bound (slack 0.5, rate 1) -> 0.99*0.5 = 0.495
    #                   x_2 approaches its lower bound (slack 1.0, rate 4) -> 0.99*1/4 = 0.2475
    # so alpha_max = 0.2475.  Multipliers zl = (1, 2), zu = (3, 4) with steps
    # dzl = (-0.5, 0), dzu = (0, -8): 0.99*1/0.5 = 1.98 (> 1), 0.99*4/8 = 0.495 -> alpha_z = 0.495
    P = ipm.Problem(_Box(np.zeros(2), np.zeros((0, 2)), []))
    pt = _pt([0.5, 0.0], [], [1.0, 2.0], [3.0, 4.0])
    e = np.zeros(0)
    amax, az = ipm.step_to_boundary(P, pt, np.array([1.0, -4.0]), e,
                                    (np.array([-0.5, 0.0]), np.array([0.0, -8.0]), e, e), 0.99)
    assert amax == 0.2475
    assert az == 0.495
    # an unbounded variable takes no part: free x_2 (no bounds) leaves only x_1's 0.495
    b = _Box(np.zeros(2), np.zeros((0, 2)), [])
    b.xl = np.array([-1.0, -np.inf])
    b.xu = np.array([1.0, np.inf])
    P = ipm.Problem(b)
    amax, _ = ipm.step_to_boundary(P, pt, np.array([1.0, -4.0]), e,
                                   (np.zeros(2), np.zeros(2), e, e), 0.99)
    assert amax == 0.495


# ---------------------------------------------------------------- scaled KKT error

def test_kkt_error_scalings_hand_worked():
    # two bounded variables, one equality x_1 + x_2 = 0.2, f = 1/2 |x|^2 (t = 0)
    # at x = (0.5, -0.5): grad f = (0.5, -0.5), g - gE = 0 - 0.2 -> primal = 0.2
    mod = _Box(np.zeros(2), np.array([[1.0, 1.0]]), [0.2])
    P = ipm.Problem(mod)
    assert P.n_bounds == 4
    # case 1 (dual error dominates): yg = 1197, zl = (300, 2), zu = (1, 500)
    #   r_x = grad + J^T y - zl + zu = (0.5+1197-300+1, -0.5+1197-2+500) = (898.5, 1694.5)
    #   ||y||_1 + ||z||_1 = 1197 + 803 = 2000 over m + n_bounds = 5 -> 400: s_d = 4
    #   ||z||_1 / n_bounds = 200.75 -> s_c = 2.0075
    #   complementarity: (x - xl) zl = (1.5*300, 0.5*2) = (450, 1), (xu - x) zu = (0.5, 750)
    #   E_0 = max(1694.5 / 4, 0.2, 750 / 2.0075) = 423.625
    pt = _pt([0.5, -0.5], [1197.0], [300.0, 2.0], [1.0, 500.0])
    ev = ipm.Evals(P, pt.x, pt.d)
    E, dual, primal, comp = ipm.kkt_error(P, pt, ev, 0.0, OPT)
    assert (dual, primal, comp) == (1694.5, pytest.approx(0.2, abs=1e-16), 750.0)
    assert E == 423.625
    # case 2 (complementarity dominates): yg = 1000, zl = (1200.5, 1000), zu = (200, 0.5)
    #   r_x = (0.5+1000-1200.5+200, -0.5+1000-1000+0.5) = (0, 0)
    #   ||z||_1 = 2401 -> s_c = max(100, 600.25)/100 = 6.0025; s_d = max(100, 3401/5)/100 = 6.802
    #   complementarity: (1.5*1200.5, 0.5*1000, 0.5*200, 1.5*0.5) = (1800.75, 500, 100, 0.75)
    #   E_0 = 1800.75 / 6.0025 = 300;  E_mu at mu = 0.75: (1800.75 - 0.75) / 6.0025 = 299.875...
    pt = _pt([0.5, -0.5], [1000.0], [1200.5, 1000.0], [200.0, 0.5])
    ev = ipm.Evals(P, pt.x, pt.d)
    E, dual, primal, comp = ipm.kkt_error(P, pt, ev, 0.0, OPT)
    assert dual == 0.0 and comp == 1800.75
    assert E == pytest.approx(300.0, rel=1e-15)
    E_mu, _, _, comp_mu = ipm.kkt_error(P, pt, ev, 0.75, OPT)
    assert comp_mu == 1800.0
    assert E_mu == pytest.approx(1800.0 / 6.0025, rel=1e-15)
    # case 3 (small multipliers): both scalings floor at 1 -> E_0 = max(dual, primal, comp)
    #   yg = 1, zl = (2, 1), zu = (1, 3): r_x = (0.5+1-2+1, -0.5+1-1+3) = (0.5, 2.5)
    #   complementarity (3, 0.5, 0.5, 4.5) -> E_0 = 4.5
    pt = _pt([0.5, -0.5], [1.0], [2.0, 1.0], [1.0, 3.0])
    ev = ipm.Evals(P, pt.x, pt.d)
    assert ipm.kkt_error(P, pt, ev, 0.0, OPT)[0] == 4.5


# ---------------------------------------------------------------- barrier update

def test_barrier_update_hand_worked():
    # mu = 0.1: min(0.2 * 0.1, 0.1^1.5 = 0.0316) = 0.02 (linear decrease)
    assert ipm.next_mu(0.1, OPT) == pytest.approx(0.02, rel=1e-15)
    # mu = 1e-3: min(2e-4, 1e-4.5 = 3.1623e-5) = 3.16227766e-5 (superlinear decrease)
    assert ipm.next_mu(1e-3, OPT) == pytest.approx(3.1622776601683795e-05, rel=1e-14)
    # floor tol / 10 = 1e-9
    assert ipm.next_mu(2e-9, OPT) == 1e-9
    assert ipm.next_mu(1e-9, OPT) == 1e-9


# ---------------------------------------------------------------- line-search acceptance

def test_alpha_min_hand_worked():
    # theta_k > theta_min, descent: 0.05 * min(1e-5, 1e-8 * 1 / 2) = 2.5e-10
    assert ipm.alpha_min(1.0, -2.0, 1e-4, OPT) == pytest.approx(2.5e-10, rel=1e-15)
    # no descent: 0.05 * 1e-5 = 5e-7
    assert ipm.alpha_min(1.0, 0.0, 1e-4, OPT) == pytest.approx(5e-7, rel=1e-15)
    assert ipm.alpha_min(1.0, 3.0, 1e-4, OPT) == pytest.approx(5e-7, rel=1e-15)
    # theta_k = 1e-6 <= theta_min with a steep descent gphi = -1e7:
    #   gamma_phi theta / (-gphi) = 1e-21;  delta theta^1.1 / (-gphi)^2.3 = 10^(-6.6 - 16.1) = 10^-22.7
    #   -> 0.05 * 10^-22.7  (the exponents swapped would give 10^(-13.8 - 7.7) = 10^-21.5)
    assert ipm.alpha_min(1e-6, -1e7, 1e-4, OPT) == pytest.approx(0.05 * 10 ** -22.7, rel=1e-12)


def _acc(th_t, phi_t, th_k=1.0, phi_k=0.0, gphi=-1.0, alpha=1.0, theta_min=1e-4, theta_max=1e4,
         filt=(), inside=True):
    return ipm.trial_acceptable(th_t, phi_t, inside, th_k, phi_k, gphi, alpha, theta_min, theta_max,
                                list(filt), OPT)


def test_switching_condition_hand_worked():
    # switching: alpha (-gphi)^2.3 > theta_k^1.1.  theta_k = 1, gphi = -1: alpha = 1 gives 1 > 1
    # false; gphi = -2: 2^2.3 = 4.92 > 1 true; alpha = 0.1: 0.492 > 1 false
    assert _acc(0.5, 0.0, gphi=-1.0)[1] is False
    assert _acc(0.5, 0.0, gphi=-2.0)[1] is True
    assert _acc(0.5, 0.0, gphi=-2.0, alpha=0.1)[1] is False
    assert _acc(0.5, 0.0, gphi=0.5)[1] is False
    # theta_k = 0.5, gphi = -0.5, alpha = 1: 0.5^2.3 = 0.203 > 0.5^1.1 = 0.467 is false
    # (with the exponents swapped it would hold)
    assert _acc(0.1, 0.0, th_k=0.5, gphi=-0.5)[1] is False
    # theta_k = 0.5, gphi = -1.5, alpha = 0.7: 0.7 * 1.5^2.3 = 1.78 > 0.467 holds
    assert _acc(0.1, 0.0, th_k=0.5, gphi=-1.5, alpha=0.7)[1] is True


def test_armijo_branch_when_theta_is_small():
    # theta_k = 1e-6 <= theta_min = 1e-4 and switching holds (1 > 1e-6.6): the trial must
    # satisfy Armijo phi_t <= phi_k + 1e-8 * alpha * gphi = -1e-8 (gphi = -1, alpha = 1)
    ok, sw, arm = _acc(0.0, -0.5e-8, th_k=1e-6, phi_k=0.0)
    assert sw and not arm and not ok          # theta fell to 0, but Armijo fails: rejected
    ok, sw, arm = _acc(0.0, -2e-8, th_k=1e-6, phi_k=0.0)
    assert sw and arm and ok
    # the same numbers with theta_k above theta_min: sufficient decrease in theta suffices
    ok, sw, arm = _acc(0.0, -0.5e-8, th_k=1e-6, phi_k=0.0, theta_min=1e-7)
    assert ok and not arm


def test_sufficient_decrease_hand_worked():
    # theta_k = 1 > theta_min, phi_k = 0, gphi = -1 (no switching at alpha = 1):
    # accept iff theta_t <= 1 - 1e-5 or phi_t <= -1e-8
    assert _acc(1.0 - 2e-5, 10.0)[0]          # theta reduced enough, phi may grow
    assert not _acc(1.0 - 5e-6, -5e-9)[0]     # neither reduced enough
    assert _acc(1.0 - 5e-6, -2e-8)[0]         # phi reduced enough
    assert _acc(1.5, -2e-8)[0]                # theta may grow if phi falls enough ...
    assert not _acc(1.5, -2e-8, theta_max=1.5)[0]   # ... but never to theta_max
    # a trial outside the bounds or with a non-finite value is rejected
    assert not _acc(0.0, -1.0, inside=False)[0]
    assert not _acc(np.nan, -1.0)[0]


def test_filter_rejects_dominated_trials():
    # one entry (0.5, 0.0) excludes theta_t >= 0.5 together with phi_t >= 0.0
    filt = [(0.5, 0.0)]
    assert not _acc(0.6, 0.1, filt=filt)[0]     # sufficient decrease holds, but in the filter
    assert _acc(0.4, 0.1, filt=filt)[0]         # below the entry's theta
    assert _acc(0.6, -0.1, filt=filt)[0]        # below the entry's phi
    assert not _acc(0.5, 0.0, filt=filt)[0]     # the corner itself is excluded


def test_filter_entry_hand_worked():
    # ((1 - 1e-5) * 2, 5 - 1e-8 * 2)
    a, b = ipm.filter_entry(2.0, 5.0, OPT)
    assert a == pytest.approx(1.99998, rel=1e-15)
    assert b == pytest.approx(4.99999998, rel=1e-15)


# ---------------------------------------------------------------- inertia correction

def _scripted_ic(monkeypatch, rule, dw_last, mu):
    """Run compute_direction with a stand-in solve whose inertia is rule(dw, dc)."""
    mod = _Box(np.zeros(2), np.array([[1.0, 1.0]]), [0.2])
    P = ipm.Problem(mod)
    pt = _pt([0.5, -0.5], [0.0], [1.0, 1.0], [1.0, 1.0])
    ev = ipm.Evals(P, pt.x, pt.d)

    def fake(sy, dw, dc):
        return dict(inertia=rule(dw, dc))

    monkeypatch.setitem(kkt.DIRECTIONS, "scripted", fake)
    state = dict(dw_last=dw_last)
    res, attempts = ipm.compute_direction(P, pt, ev, mu, ipm.Options(linsolve="scripted"), state)
    return res, attempts, state


def test_ic_first_time_with_zero_eigenvalue(monkeypatch):
    # target (2, 1, 0).  dw = 0 gives a zero eigenvalue: dc = 1e-8 * mu^0.25 = 1e-8 * 0.1 = 1e-9.
    # No earlier shift: dw = 1e-4, then x100 until the inertia is right at dw >= 0.5:
    # 1e-4, 1e-2, 1 -> accepted at 1, remembered as the last shift.
    rule = lambda dw, dc: (2, 1, 0) if dw >= 0.5 else ((1, 1, 1) if dw == 0 else (1, 2, 0))
    res, att, st = _scripted_ic(monkeypatch, rule, 0.0, 1e-4)
    assert res is not None
    assert [a[0] for a in att] == [0.0, 1e-4, pytest.approx(1e-2, rel=1e-15), pytest.approx(1.0, rel=1e-15)]
    assert att[0][1] == 0.0
    assert all(a[1] == pytest.approx(1e-9, rel=1e-15) for a in att[1:])
    assert st["dw_last"] == att[-1][0]


def test_ic_after_an_earlier_shift(monkeypatch):
    # last shift 0.3: start at 0.3 / 3 = 0.1, then x8: 0.8 -> accepted; no zero eigenvalue -> dc = 0
    rule = lambda dw, dc: (2, 1, 0) if dw >= 0.5 else (1, 2, 0)
    res, att, st = _scripted_ic(monkeypatch, rule, 0.3, 1e-4)
    assert [a[0] for a in att] == [0.0, pytest.approx(0.1, rel=1e-15), pytest.approx(0.8, rel=1e-15)]
    assert all(a[1] == 0.0 for a in att)
    assert st["dw_last"] == att[-1][0]
    # a tiny last shift is floored at dw_min = 1e-20 (1.5e-20 / 3 = 5e-21 -> 1e-20)
    rule = lambda dw, dc: (2, 1, 0) if dw > 0 else (1, 2, 0)
    _, att, _ = _scripted_ic(monkeypatch, rule, 1.5e-20, 1e-4)
    assert [a[0] for a in att] == [0.0, 1e-20]


def test_ic_no_retry_when_inertia_is_right(monkeypatch):
    res, att, st = _scripted_ic(monkeypatch, lambda dw, dc: (2, 1, 0), 0.7, 1e-4)
    assert res is not None and att == [(0.0, 0.0, (2, 1, 0))]
    assert st["dw_last"] == 0.7               # unchanged


def test_ic_gives_up_above_dw_max(monkeypatch):
    res, att, st = _scripted_ic(monkeypatch, lambda dw, dc: (1, 2, 0), 1.0, 1e-4)
    assert res is None
    # 1/3, then x8 while the shift stays <= 1e40: the last one tried is the largest such shift
    shifts = [a[0] for a in att[1:]]
    assert shifts[0] == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert all(b == pytest.approx(8.0 * a, rel=1e-15) for a, b in zip(shifts, shifts[1:]))
    assert shifts[-1] <= 1e40 < 8.0 * shifts[-1]
    assert st["dw_last"] == 1.0


# ---------------------------------------------------------------- start and safeguard

def test_initial_push_hand_worked():
    # bounds [-1, 1]: push p = min(0.01 * max(1, 1), 0.01 * 2) = 0.01
    #   0 stays, -1 -> -0.99, 3 -> 0.99
    lo, hi = -np.ones(3), np.ones(3)
    has = np.ones(3, bool)
    v = ipm._push(np.array([0.0, -1.0, 3.0]), lo, hi, has, has, 0.01, 0.01)
    assert v.tolist() == [0.0, -0.99, 0.99]
    # bounds [0, 0.5]: p = min(0.01, 0.01 * 0.5) = 0.005 -> 5 goes to 0.495, -2 to 0.005
    v = ipm._push(np.array([5.0, -2.0]), np.zeros(2), np.full(2, 0.5), np.ones(2, bool),
                  np.ones(2, bool), 0.01, 0.01)
    assert v.tolist() == [0.495, 0.005]
    # one-sided upper bound 4: p = 0.01 * max(1, 4) = 0.04 -> 4 goes to 3.96; no lower bound
    v = ipm._push(np.array([4.0, -100.0]), np.full(2, -np.inf), np.full(2, 4.0),
                  np.zeros(2, bool), np.ones(2, bool), 0.01, 0.01)
    assert v.tolist() == [3.96, -100.0]


def test_kappa_sigma_safeguard_hand_worked():
    # mu = 1e-2, kappa = 1e10, slack 1: z kept in [1e-12, 1e8]; slack 4: [2.5e-13, 2.5e7]
    z = np.array([1e-13, 1.0, 1e12, 1e8])
    s = np.array([1.0, 1.0, 1.0, 4.0])
    out = ipm.kappa_sigma_safeguard(z, s, 1e-2, 1e10)
    np.testing.assert_allclose(out, [1e-12, 1.0, 1e8, 2.5e7], rtol=1e-15)
