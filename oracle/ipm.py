"""Filter line-search interior-point method (Section 2.1).

Oracle (test infrastructure only).  Section 2.1 delegates the method to
Waechter & Biegler (filter line search, inertia correction); this module
implements it step by step in FP64, computing every Newton direction from the
4x4 system of Eq. (linsys4x4) (`kkt.direction_full`; the condensed forms are
selectable for sizes where the dense 4x4 matrix does not fit).

Formulation (Section 2, Eqs. (obj)-(bounds), with the slack reformulation of
Section 2.1): variables x = [x_s; x_d] and slacks d for h,

    min f(x)  s.t.  g(x) - g_E = 0,  h(x) - d = 0,  x^l <= x <= x^u,  h^l <= d <= h^u,

multipliers y_g, y_h for the equalities and z_l, z_u (for x), v_l, v_u (for d)
for the finite bounds.  Optimality: grad f + J_g^T y_g + J_h^T y_h - z_l + z_u = 0,
-y_h - v_l + v_u = 0, and the complementarity products equal mu.

One iteration (W&B Algorithm A, no second-order correction, no restoration):
  A.2  stop if E_0 <= tol                      (scaled KKT error, s_max = 100)
  A.3  if E_mu <= kappa_eps mu: mu <- max(tol/10, min(kappa_mu mu, mu^theta_mu)),
       tau <- max(tau_min, 1 - mu), reset the filter (repeated only at k = 0)
  A.4  Newton direction with inertia correction (Algorithm IC): target
       inertia (n, m, 0) in (positive, negative, zero) order, shifts dw on the
       Hessian blocks and -dc on blocks (3,3)/(4,4) (Section 2.1)
  A.5  fraction-to-boundary alpha_max and alpha_z (Section 2.1: the search
       starts at the farthest bound-feasible point), then backtracking by
       halving with the filter / switching-condition / Armijo tests
  A.6  accept; y <- y + alpha dy, z <- z + alpha_z dz, kappa_Sigma safeguard
  A.7  augment the filter unless the step was of f-type with Armijo

Readings where the paper is silent are collected in `Options`.
Pinned by tests/test_oracle_ipm.py: closed-form optima of convex instances
(equality QP, ball constraint with known multiplier, box projection), a
library optimizer's optimum, the KKT error at exit and the target inertia of
every accepted factorization.  The step rules are pinned one by one on
hand-worked values by tests/test_oracle_ipm_rules.py: `fraction_to_boundary`
and `step_to_boundary`, `kkt_error`'s s_d/s_c scalings, `next_mu`,
`alpha_min`, `trial_acceptable` (switching condition, Armijo, sufficient
decrease, the theta_min branch, theta_max, the filter), `filter_entry`, the
Algorithm IC shift schedule of `compute_direction`, `_push` and
`kappa_sigma_safeguard`.  How `solve` strings these together (the order of
A.3-A.7) is pinned only through the closed-form optima above.
"""
from __future__ import annotations

import dataclasses
import math
import numpy as np

from . import kkt


@dataclasses.dataclass
class Options:
    tol: float = 1e-8
    max_iter: int = 200
    mu0: float = 0.1
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    s_max: float = 100.0
    kappa_1: float = 1e-2
    kappa_2: float = 1e-2
    kappa_sigma: float = 1e10
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-8
    delta: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-8
    gamma_alpha: float = 0.05
    theta_max_fact: float = 1e4
    theta_min_fact: float = 1e-4
    max_ls: int = 60
    dw0: float = 1e-4
    dw_min: float = 1e-20
    dw_max: float = 1e40
    kw_minus: float = 1.0 / 3.0
    kw_plus: float = 8.0
    kw_plus_bar: float = 100.0
    dc_bar: float = 1e-8
    kappa_c: float = 0.25
    linsolve: str = "full"          # full | p1 | p2


STATUS = {0: "OK", 8: "MAX_ITER", 6: "INERTIA", 7: "RESTORATION_NEEDED", 5: "NONFINITE"}


class Point:
    """Primal-dual iterate."""

    def __init__(self, x, d, yg, yh, zl, zu, vl, vu):
        self.x, self.d, self.yg, self.yh = x, d, yg, yh
        self.zl, self.zu, self.vl, self.vu = zl, zu, vl, vu

    def copy(self):
        return Point(*(np.array(v, copy=True) for v in
                       (self.x, self.d, self.yg, self.yh, self.zl, self.zu, self.vl, self.vu)))

    def packed(self):
        return np.concatenate([self.x, self.d, self.yg, self.yh, self.zl, self.zu, self.vl, self.vu])


class Problem:
    """Bounds, masks and evaluations around a model (oracle.model.SynthModel)."""

    def __init__(self, model):
        self.mod = model
        self.n_s, self.n_d, self.m_E, self.m_I = model.n_s, model.n_d, model.m_E, model.m_I
        self.n = self.n_s + self.n_d
        self.xl, self.xu, self.hl, self.hu = model.xl, model.xu, model.hl, model.hu
        self.gE = model.gE
        self.hxl, self.hxu = np.isfinite(self.xl), np.isfinite(self.xu)
        self.hdl, self.hdu = np.isfinite(self.hl), np.isfinite(self.hu)
        self.n_bounds = int(self.hxl.sum() + self.hxu.sum() + self.hdl.sum() + self.hdu.sum())

    # slacks to the finite bounds (zero where the bound is infinite)
    def slacks(self, x, d):
        sl = np.where(self.hxl, x - np.where(self.hxl, self.xl, 0.0), 0.0)
        su = np.where(self.hxu, np.where(self.hxu, self.xu, 0.0) - x, 0.0)
        tl = np.where(self.hdl, d - np.where(self.hdl, self.hl, 0.0), 0.0)
        tu = np.where(self.hdu, np.where(self.hdu, self.hu, 0.0) - d, 0.0)
        return sl, su, tl, tu

    def masks(self):
        return self.hxl, self.hxu, self.hdl, self.hdu


def _push(v, lo, hi, has_lo, has_hi, k1, k2):
    """W&B Section 3.6: move a starting value strictly inside its bounds."""
    v = v.copy()
    both = has_lo & has_hi
    width = np.where(both, np.where(both, hi, 0.0) - np.where(both, lo, 0.0), np.inf)
    lo0 = np.where(has_lo, lo, 0.0)
    hi0 = np.where(has_hi, hi, 0.0)
    pl = np.minimum(k1 * np.maximum(1.0, np.abs(lo0)), k2 * width)
    pu = np.minimum(k1 * np.maximum(1.0, np.abs(hi0)), k2 * width)
    v = np.where(has_lo, np.maximum(v, lo0 + pl), v)
    v = np.where(has_hi, np.minimum(v, hi0 - pu), v)
    return v


def initial_point(P: Problem, x0, opt: Options) -> Point:
    x = _push(np.asarray(x0, dtype=np.float64), P.xl, P.xu, P.hxl, P.hxu, opt.kappa_1, opt.kappa_2)
    d = _push(P.mod.h(x), P.hl, P.hu, P.hdl, P.hdu, opt.kappa_1, opt.kappa_2)
    yg = np.zeros(P.m_E)
    yh = np.zeros(P.m_I)
    zl = P.hxl.astype(np.float64)
    zu = P.hxu.astype(np.float64)
    vl = P.hdl.astype(np.float64)
    vu = P.hdu.astype(np.float64)
    return Point(x, d, yg, yh, zl, zu, vl, vu)


class Evals:
    """Model values at a primal point (x, d)."""

    def __init__(self, P: Problem, x, d):
        m = P.mod
        self.f = m.f(x)
        self.grad = m.grad_f(x)
        self.g = m.g(x)
        self.h = m.h(x)
        self.cg = self.g - P.gE
        self.ch = self.h - d


def barrier_phi(P: Problem, f, x, d, mu):
    sl, su, tl, tu = P.slacks(x, d)
    hxl, hxu, hdl, hdu = P.masks()
    return f - mu * (np.sum(np.log(sl[hxl])) + np.sum(np.log(su[hxu]))
                     + np.sum(np.log(tl[hdl])) + np.sum(np.log(tu[hdu])))


def theta(ev: Evals):
    return float(np.sum(np.abs(ev.cg)) + np.sum(np.abs(ev.ch)))


def dual_residual(P: Problem, pt: Point, ev: Evals):
    Jsg, Jsh, A, Jdh = P.mod.jac(pt.x)
    r_s = ev.grad[:P.n_s] + Jsg.T @ pt.yg + Jsh.T @ pt.yh
    r_d = ev.grad[P.n_s:] + A.T @ pt.yg + Jdh.T @ pt.yh
    rx = np.concatenate([r_s, r_d]) - pt.zl + pt.zu
    rdd = -pt.yh - pt.vl + pt.vu
    return rx, rdd


def kkt_error(P: Problem, pt: Point, ev: Evals, mu, opt: Options):
    """Scaled optimality error E_mu (W&B eq. (5)); E_0 with mu = 0."""
    rx, rdd = dual_residual(P, pt, ev)
    sl, su, tl, tu = P.slacks(pt.x, pt.d)
    hxl, hxu, hdl, hdu = P.masks()
    z1 = np.sum(np.abs(pt.zl)) + np.sum(np.abs(pt.zu)) + np.sum(np.abs(pt.vl)) + np.sum(np.abs(pt.vu))
    y1 = np.sum(np.abs(pt.yg)) + np.sum(np.abs(pt.yh))
    nm = P.m_E + P.m_I + P.n_bounds
    s_d = max(opt.s_max, (y1 + z1) / nm) / opt.s_max if nm > 0 else 1.0
    s_c = max(opt.s_max, z1 / P.n_bounds) / opt.s_max if P.n_bounds > 0 else 1.0
    dual = max(_inf(rx), _inf(rdd))
    primal = max(_inf(ev.cg), _inf(ev.ch))
    comp = max(_inf((sl * pt.zl - mu)[hxl]), _inf((su * pt.zu - mu)[hxu]),
               _inf((tl * pt.vl - mu)[hdl]), _inf((tu * pt.vu - mu)[hdu]))
    return max(dual / s_d, primal, comp / s_c), dual, primal, comp


def _inf(v):
    return float(np.max(np.abs(v))) if v.size else 0.0


def newton_system(P: Problem, pt: Point, ev: Evals, mu) -> kkt.NewtonSystem:
    """Barrier diagonals and residuals of the primal-dual system."""
    mod = P.mod
    Hss, Hdd = mod.hess(pt.x, pt.yg, pt.yh)
    Jsg, Jsh, A, Jdh = mod.jac(pt.x)
    sl, su, tl, tu = P.slacks(pt.x, pt.d)
    hxl, hxu, hdl, hdu = P.masks()
    sig_x = np.where(hxl, pt.zl / np.where(hxl, sl, 1.0), 0.0) + np.where(hxu, pt.zu / np.where(hxu, su, 1.0), 0.0)
    sig_d = np.where(hdl, pt.vl / np.where(hdl, tl, 1.0), 0.0) + np.where(hdu, pt.vu / np.where(hdu, tu, 1.0), 0.0)
    # gradient of the barrier objective
    gphi_x = ev.grad - np.where(hxl, mu / np.where(hxl, sl, 1.0), 0.0) + np.where(hxu, mu / np.where(hxu, su, 1.0), 0.0)
    gphi_d = -np.where(hdl, mu / np.where(hdl, tl, 1.0), 0.0) + np.where(hdu, mu / np.where(hdu, tu, 1.0), 0.0)
    n_s = P.n_s
    r_xs = gphi_x[:n_s] + Jsg.T @ pt.yg + Jsh.T @ pt.yh
    r_xd = gphi_x[n_s:] + A.T @ pt.yg + Jdh.T @ pt.yh
    r_d = gphi_d - pt.yh
    return kkt.NewtonSystem(Hss=Hss, Hdd=Hdd, Jsg=Jsg, Jsh=Jsh, A=A, Jdh=Jdh,
                            sig_xs=sig_x[:n_s], sig_xd=sig_x[n_s:], sig_d=sig_d,
                            r_xs=r_xs, r_xd=r_xd, r_g=ev.cg, r_h=ev.ch, r_d=r_d)


def bound_multiplier_steps(P: Problem, pt: Point, dx, dd, mu):
    """dz = mu S^-1 e - z - S^-1 Z ds for every finite bound (W&B eq. (11))."""
    sl, su, tl, tu = P.slacks(pt.x, pt.d)
    hxl, hxu, hdl, hdu = P.masks()
    one = lambda s, m: np.where(m, s, 1.0)
    dzl = np.where(hxl, mu / one(sl, hxl) - pt.zl - pt.zl / one(sl, hxl) * dx, 0.0)
    dzu = np.where(hxu, mu / one(su, hxu) - pt.zu + pt.zu / one(su, hxu) * dx, 0.0)
    dvl = np.where(hdl, mu / one(tl, hdl) - pt.vl - pt.vl / one(tl, hdl) * dd, 0.0)
    dvu = np.where(hdu, mu / one(tu, hdu) - pt.vu + pt.vu / one(tu, hdu) * dd, 0.0)
    return dzl, dzu, dvl, dvu


def fraction_to_boundary(tau, vals, steps):
    """Largest alpha in (0, 1] with v + alpha dv >= (1 - tau) v for all pairs."""
    a = 1.0
    for v, dv in zip(vals, steps):
        neg = dv < 0
        if np.any(neg):
            a = min(a, float(np.min(-tau * v[neg] / dv[neg])))
    return a


def step_to_boundary(P: Problem, pt: Point, dx, dd, dz, tau):
    """alpha_max and alpha_z of one direction (W&B eqs. (15) and (14b)).

    alpha_max keeps every slack to a finite bound at least (1 - tau) of its
    current value: x - x^l moves by +dx, x^u - x by -dx, d - h^l by +dd and
    h^u - d by -dd.  alpha_z does the same for the bound multipliers
    (z_l, z_u, v_l, v_u) and their steps dz = (dzl, dzu, dvl, dvu).  Entries
    without a finite bound take no part."""
    sl, su, tl, tu = P.slacks(pt.x, pt.d)
    hxl, hxu, hdl, hdu = P.masks()
    dzl, dzu, dvl, dvu = dz
    alpha_max = fraction_to_boundary(tau, [sl[hxl], su[hxu], tl[hdl], tu[hdu]],
                                     [dx[hxl], -dx[hxu], dd[hdl], -dd[hdu]])
    alpha_z = fraction_to_boundary(tau, [pt.zl[hxl], pt.zu[hxu], pt.vl[hdl], pt.vu[hdu]],
                                   [dzl[hxl], dzu[hxu], dvl[hdl], dvu[hdu]])
    return alpha_max, alpha_z


def kappa_sigma_safeguard(z, s, mu, kappa_sigma):
    """Keep each bound multiplier within [mu / (kappa_sigma s), kappa_sigma mu / s]
    of its slack s (W&B eq. (16)), so that the primal-dual Sigma stays within a
    factor kappa_sigma of the primal barrier Hessian mu / s^2."""
    return np.maximum(np.minimum(z, kappa_sigma * mu / s), mu / (kappa_sigma * s))


def next_mu(mu, opt: Options):
    """Barrier parameter after the subproblem for mu is solved (W&B eq. (7)):
    the smaller of a linear (kappa_mu mu) and a superlinear (mu^theta_mu)
    decrease, never below tol/10."""
    return max(opt.tol / 10.0, min(opt.kappa_mu * mu, mu ** opt.theta_mu))


def alpha_min(th_k, gphi, theta_min, opt: Options):
    """Smallest step before the backtracking gives up (W&B eq. (23)).

    With a descent direction (gphi < 0) the bound is gamma_alpha times the
    smallest of gamma_theta, gamma_phi theta_k / (-gphi) and, when theta_k is
    already small (<= theta_min), delta theta_k^s_theta / (-gphi)^s_phi;
    otherwise gamma_alpha gamma_theta."""
    if gphi < 0 and th_k <= theta_min:
        return opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * th_k / (-gphi),
                                     opt.delta * th_k ** opt.s_theta / (-gphi) ** opt.s_phi)
    if gphi < 0:
        return opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * th_k / (-gphi))
    return opt.gamma_alpha * opt.gamma_theta


def trial_acceptable(th_t, phi_t, inside, th_k, phi_k, gphi, alpha, theta_min, theta_max, filt,
                     opt: Options):
    """Acceptance test of one trial point (W&B Section 2.3, A-5.2 to A-5.4).

    switching condition (eq. (19)): gphi < 0 and alpha (-gphi)^s_phi > delta theta_k^s_theta;
    Armijo (eq. (20)): phi_t <= phi_k + eta_phi alpha gphi.
    If theta_k <= theta_min and the switching condition holds, the trial must
    satisfy Armijo; otherwise it must reduce theta or phi sufficiently
    (eq. (18): theta_t <= (1 - gamma_theta) theta_k or phi_t <= phi_k - gamma_phi theta_k).
    In both cases it must lie below theta_max and outside every filter entry
    (a pair (a, b) excludes theta_t >= a together with phi_t >= b).  A trial
    outside the bounds (inside = False) or with a non-finite value is rejected.
    Returns (accepted, switching, armijo)."""
    ftype = gphi < 0 and alpha * (-gphi) ** opt.s_phi > opt.delta * th_k ** opt.s_theta
    armijo = phi_t <= phi_k + opt.eta_phi * alpha * gphi
    ok = False
    if inside and np.isfinite(phi_t) and np.isfinite(th_t):
        if th_k <= theta_min and ftype:
            ok = armijo
        else:
            ok = th_t <= (1 - opt.gamma_theta) * th_k or phi_t <= phi_k - opt.gamma_phi * th_k
        if ok:
            ok = th_t < theta_max and not any(th_t >= a and phi_t >= b for a, b in filt)
    return ok, ftype, armijo


def filter_entry(th_k, phi_k, opt: Options):
    """Corner point added to the filter after a step that was not of f-type with
    Armijo (W&B eq. (22))."""
    return ((1 - opt.gamma_theta) * th_k, phi_k - opt.gamma_phi * th_k)


def compute_direction(P: Problem, pt: Point, ev: Evals, mu, opt: Options, state):
    """W&B Algorithm IC around the chosen linear solve; returns (dir, attempts)."""
    sy = newton_system(P, pt, ev, mu)
    target = (P.n, P.m_E + P.m_I, 0)
    solve = kkt.DIRECTIONS[opt.linsolve]
    attempts = []
    dw, dc = 0.0, 0.0
    res = solve(sy, dw, dc)
    attempts.append((dw, dc, res["inertia"]))
    if res["inertia"] != target:
        if res["inertia"][2] > 0:
            dc = opt.dc_bar * mu ** opt.kappa_c
        dw = opt.dw0 if state["dw_last"] == 0.0 else max(opt.dw_min, opt.kw_minus * state["dw_last"])
        while True:
            res = solve(sy, dw, dc)
            attempts.append((dw, dc, res["inertia"]))
            if res["inertia"] == target:
                state["dw_last"] = dw
                break
            dw = opt.kw_plus_bar * dw if state["dw_last"] == 0.0 else opt.kw_plus * dw
            if dw > opt.dw_max:
                return None, attempts
    return res, attempts


def solve(model, x0=None, opt: Options | None = None, start: Point | None = None, mu0=None):
    """Run the interior-point method.  Returns dict(point, status, iters, log, ...)."""
    opt = opt or Options()
    P = Problem(model)
    pt = start.copy() if start is not None else initial_point(P, model.inst.x0 if x0 is None else x0, opt)
    mu = opt.mu0 if mu0 is None else mu0
    tau = max(opt.tau_min, 1.0 - mu)
    ev = Evals(P, pt.x, pt.d)
    th0 = theta(ev)
    theta_max = opt.theta_max_fact * max(1.0, th0)
    theta_min = opt.theta_min_fact * max(1.0, th0)
    filt = []
    state = dict(dw_last=0.0)
    log = []
    k = 0
    status = 8
    while True:
        E0, inf_du, inf_pr, inf_co = kkt_error(P, pt, ev, 0.0, opt)
        rec = dict(iter=k, mu=mu, f=float(ev.f), theta=theta(ev), inf_pr=inf_pr, inf_du=inf_du, E0=E0)
        if not np.isfinite(E0):
            status = 5
            log.append(rec)
            break
        if E0 <= opt.tol:
            status = 0
            log.append(rec)
            break
        if k >= opt.max_iter:
            status = 8
            log.append(rec)
            break
        # A.3 barrier update
        while True:
            Emu = kkt_error(P, pt, ev, mu, opt)[0]
            if Emu <= opt.kappa_eps * mu:
                mu_new = next_mu(mu, opt)
                if mu_new == mu:
                    break
                mu = mu_new
                tau = max(opt.tau_min, 1.0 - mu)
                filt = []
                if k == 0:
                    continue
            break
        rec["mu"] = mu
        # A.4 direction
        res, attempts = compute_direction(P, pt, ev, mu, opt, state)
        rec["ic"] = [(float(a), float(b), tuple(int(t) for t in c)) for a, b, c in attempts]
        if res is None:
            status = 6
            log.append(rec)
            break
        dx = np.concatenate([res["dxs"], res["dxd"]])
        dd = res["dd"]
        dyg, dyh = res["dyg"], res["dyh"]
        dzl, dzu, dvl, dvu = bound_multiplier_steps(P, pt, dx, dd, mu)
        # A.5 line search
        sl, su, tl, tu = P.slacks(pt.x, pt.d)
        hxl, hxu, hdl, hdu = P.masks()
        alpha_max, alpha_z = step_to_boundary(P, pt, dx, dd, (dzl, dzu, dvl, dvu), tau)
        phi_k = barrier_phi(P, ev.f, pt.x, pt.d, mu)
        th_k = theta(ev)
        # directional derivative of the barrier objective
        gphi_x = ev.grad - np.where(hxl, mu / np.where(hxl, sl, 1.0), 0.0) + np.where(hxu, mu / np.where(hxu, su, 1.0), 0.0)
        gphi_d = -np.where(hdl, mu / np.where(hdl, tl, 1.0), 0.0) + np.where(hdu, mu / np.where(hdu, tu, 1.0), 0.0)
        gphi = float(gphi_x @ dx + gphi_d @ dd)
        a_min = alpha_min(th_k, gphi, theta_min, opt)
        alpha = alpha_max
        n_ls = 0
        accepted = False
        while True:
            xt = pt.x + alpha * dx
            dt = pt.d + alpha * dd
            evt = Evals(P, xt, dt)
            sl_t, su_t, tl_t, tu_t = P.slacks(xt, dt)
            inside = (np.all(sl_t[hxl] > 0) and np.all(su_t[hxu] > 0)
                      and np.all(tl_t[hdl] > 0) and np.all(tu_t[hdu] > 0))
            th_t = theta(evt)
            phi_t = barrier_phi(P, evt.f, xt, dt, mu) if inside else np.inf
            ok, ftype, armijo = trial_acceptable(th_t, phi_t, inside, th_k, phi_k, gphi, alpha,
                                                 theta_min, theta_max, filt, opt)
            if ok:
                accepted = True
                break
            n_ls += 1
            alpha *= 0.5
            if alpha < a_min or n_ls >= opt.max_ls:
                break
        rec.update(alpha_max=alpha_max, alpha_z=alpha_z, n_ls=n_ls, gphi=gphi)
        if not accepted:
            status = 7
            log.append(rec)
            break
        rec.update(alpha=alpha, ftype=bool(ftype and armijo))
        # A.7 filter augmentation (before moving the reference point)
        if not (ftype and armijo):
            filt.append(filter_entry(th_k, phi_k, opt))
        # A.6 accept
        pt.x, pt.d = xt, dt
        pt.yg = pt.yg + alpha * dyg
        pt.yh = pt.yh + alpha * dyh
        pt.zl = pt.zl + alpha_z * dzl
        pt.zu = pt.zu + alpha_z * dzu
        pt.vl = pt.vl + alpha_z * dvl
        pt.vu = pt.vu + alpha_z * dvu
        # kappa_Sigma safeguard (W&B eq. (16))
        sl, su, tl, tu = P.slacks(pt.x, pt.d)
        for z, s, msk in ((pt.zl, sl, hxl), (pt.zu, su, hxu), (pt.vl, tl, hdl), (pt.vu, tu, hdu)):
            z[msk] = kappa_sigma_safeguard(z[msk], s[msk], mu, opt.kappa_sigma)
        ev = evt
        log.append(rec)
        k += 1
    E0 = kkt_error(P, pt, ev, 0.0, opt)[0]
    return dict(point=pt, status=status, status_str=STATUS[status], iters=k, log=log,
                f=float(ev.f), E0=E0, mu=mu)


def direction_at(model, pt: Point, mu, dw, dc, linsolve="full"):
    """Direction and inertia of one Newton system at a given iterate (no IC).

    Returns dict with dx (n), dd, dyg, dyh, dzl, dzu, dvl, dvu and inertia.
    """
    P = Problem(model)
    ev = Evals(P, pt.x, pt.d)
    sy = newton_system(P, pt, ev, mu)
    res = kkt.DIRECTIONS[linsolve](sy, dw, dc)
    dx = np.concatenate([res["dxs"], res["dxd"]])
    dzl, dzu, dvl, dvu = bound_multiplier_steps(P, pt, dx, res["dd"], mu)
    return dict(dx=dx, dd=res["dd"], dyg=res["dyg"], dyh=res["dyh"], dzl=dzl, dzu=dzu,
                dvl=dvl, dvu=dvu, inertia=res["inertia"])
