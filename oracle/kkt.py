"""KKT systems of one Newton step (Sections 2.1-2.3).

Oracle (test infrastructure only).  Unknowns are ordered
[dx_s; dx_d; dy_g; dy_h] as in Eq. (linsys4x4):

    [ Q_s    0     Jsg^T  Jsh^T        ] [dx_s]   [b_s]
    [ 0      Q_d   A^T    Jdh^T        ] [dx_d] = [b_d]
    [ Jsg    A     -dc I  0            ] [dy_g]   [b_g]
    [ Jsh    Jdh   0      -Dh^-1 - dc I] [dy_h]   [b_h]

Q_s = diag(H_ss + Sigma_xs + dw),  Q_d = H_dd + Sigma_xd + dw I,
Dh = Sigma_d + dw.  The inertia-correction shifts follow Section 2.1: +dw on
the Hessian blocks (and on the eliminated slack block, hence Dh), -dc on
blocks (3,3) and (4,4).  The right-hand side is b = -[r_x; r_g; r_h + Dh^-1 r_d]
and the eliminated slack step is dd = Dh^-1 (dy_h - r_d).

Three ways to the same direction:

* `direction_full`   forms the dense 4x4 matrix and solves it (the definition).
* `direction_p1`     the compressed 3x3 matrix of Eq. (compressed): dx_s
                     eliminated by Gauss elimination, In(K) = In(Q_s) + In(M)
                     (Haynsworth, Section 2.3).
* `direction_p2`     one further exact block elimination of dy_g, valid when
                     J_sh = 0 and the rows of J_sg have disjoint supports, so that
                     W = J_sg Q_s^-1 J_sg^T + dc I is diagonal:
                     S = [[Q_d + A^T W^-1 A, Jdh^T], [Jdh, -Dh^-1 - dc I]],
                     In(K) = In(Q_s) + In(-W) + In(S).

Pinned by tests/test_oracle_kkt.py: the three directions agree with each other
and satisfy the unreduced 5x5 system (slack row included) to rounding on tiny
inputs; inertias agree with numpy.linalg.eigvalsh of the dense 4x4 matrix.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

ZERO_TOL = 1e-14


@dataclasses.dataclass
class NewtonSystem:
    Hss: np.ndarray       # (n_s,) diagonal of the x_s Hessian block
    Hdd: np.ndarray       # (n_d, n_d)
    Jsg: sp.spmatrix      # (m_E, n_s)
    Jsh: sp.spmatrix      # (m_I, n_s)
    A: np.ndarray         # (m_E, n_d)  J_{x_d} g
    Jdh: np.ndarray       # (m_I, n_d)  J_{x_d} h
    sig_xs: np.ndarray    # (n_s,) primal-dual barrier diagonal of x_s
    sig_xd: np.ndarray    # (n_d,)
    sig_d: np.ndarray     # (m_I,) barrier diagonal of the slack d
    r_xs: np.ndarray      # residuals (gradient of the barrier Lagrangian etc.)
    r_xd: np.ndarray
    r_g: np.ndarray
    r_h: np.ndarray
    r_d: np.ndarray

    @property
    def dims(self):
        return self.Hss.size, self.Hdd.shape[0], self.A.shape[0], self.Jdh.shape[0]


def inertia_from_ldl_D(D, scale, zero_tol=ZERO_TOL):
    """Inertia (pos, neg, zero) from the block-diagonal D of an LDL^T."""
    N = D.shape[0]
    pos = neg = zero = 0
    i = 0
    while i < N:
        if i + 1 < N and D[i + 1, i] != 0.0:
            ev = np.linalg.eigvalsh(D[i:i + 2, i:i + 2])
            for v in ev:
                if abs(v) <= zero_tol * scale:
                    zero += 1
                elif v > 0:
                    pos += 1
                else:
                    neg += 1
            i += 2
        else:
            v = D[i, i]
            if v == 0.0 or abs(v) <= zero_tol * scale:
                zero += 1
            elif v > 0:
                pos += 1
            else:
                neg += 1
            i += 1
    return pos, neg, zero


def inertia_ldl(K, zero_tol=ZERO_TOL):
    """Inertia of a dense symmetric K through the library Bunch-Kaufman LDL^T."""
    if K.shape[0] == 0:
        return (0, 0, 0)
    _, D, _ = sla.ldl(K, lower=True, hermitian=True)
    return inertia_from_ldl_D(D, float(np.max(np.abs(K))), zero_tol)


def inertia_diag(v):
    """Inertia of a diagonal matrix: counts of positive, negative and zero entries."""
    v = np.asarray(v)
    return int(np.sum(v > 0)), int(np.sum(v < 0)), int(np.sum(v == 0))


def _add(a, b):
    return tuple(int(x) + int(y) for x, y in zip(a, b))


def assemble_k4(sy: NewtonSystem, dw: float, dc: float):
    """Dense matrix and right-hand side of Eq. (linsys4x4) with shifts."""
    n_s, n_d, m_E, m_I = sy.dims
    n, m = n_s + n_d, m_E + m_I
    Dh = sy.sig_d + dw
    K = np.zeros((n + m, n + m))
    K[np.arange(n_s), np.arange(n_s)] = sy.Hss + sy.sig_xs + dw
    K[n_s:n, n_s:n] = sy.Hdd + np.diag(sy.sig_xd + dw)
    J = np.block([[sy.Jsg.toarray(), sy.A], [sy.Jsh.toarray(), sy.Jdh]])
    K[n:, :n] = J
    K[:n, n:] = J.T
    K[n + np.arange(m_E), n + np.arange(m_E)] = -dc
    K[n + m_E + np.arange(m_I), n + m_E + np.arange(m_I)] = -1.0 / Dh - dc
    rhs = -np.concatenate([sy.r_xs, sy.r_xd, sy.r_g, sy.r_h + sy.r_d / Dh])
    return K, rhs


def _finish(sy, dw, dxs, dxd, dyg, dyh, inertia):
    dd = (dyh - sy.r_d) / (sy.sig_d + dw)
    return dict(dxs=dxs, dxd=dxd, dyg=dyg, dyh=dyh, dd=dd, inertia=inertia)


def direction_full(sy: NewtonSystem, dw: float, dc: float, want_solve=True):
    """Solve the dense 4x4 system; inertia from its Bunch-Kaufman LDL^T."""
    n_s, n_d, m_E, m_I = sy.dims
    K, rhs = assemble_k4(sy, dw, dc)
    inertia = inertia_ldl(K)
    if not want_solve:
        return dict(inertia=inertia)
    sol = np.linalg.solve(K, rhs)
    n = n_s + n_d
    return _finish(sy, dw, sol[:n_s], sol[n_s:n], sol[n:n + m_E], sol[n + m_E:], inertia)


def compressed_p1(sy: NewtonSystem, dw: float, dc: float):
    """Matrix M of Eq. (compressed) (with shifts), Q_s diagonal and In(Q_s)."""
    n_s, n_d, m_E, m_I = sy.dims
    q = sy.Hss + sy.sig_xs + dw
    Js = sp.vstack([sy.Jsg, sy.Jsh]).tocsr()
    Jd = np.vstack([sy.A, sy.Jdh])
    M = np.zeros((n_d + m_E + m_I,) * 2)
    M[:n_d, :n_d] = sy.Hdd + np.diag(sy.sig_xd + dw)
    M[n_d:, :n_d] = Jd
    M[:n_d, n_d:] = Jd.T
    JQ = Js.multiply(1.0 / q[None, :]).tocsr()         # Js Q_s^-1
    M[n_d:, n_d:] = -(JQ @ Js.T).toarray()
    idx = n_d + np.arange(m_E + m_I)
    M[idx, idx] -= dc
    ih = n_d + m_E + np.arange(m_I)
    M[ih, ih] -= 1.0 / (sy.sig_d + dw)
    return M, q


def direction_p1(sy: NewtonSystem, dw: float, dc: float):
    n_s, n_d, m_E, m_I = sy.dims
    M, q = compressed_p1(sy, dw, dc)
    inertia = _add(inertia_diag(q), inertia_ldl(M))
    Js = sp.vstack([sy.Jsg, sy.Jsh]).tocsr()
    b_s = -sy.r_xs
    b_d = -sy.r_xd
    b_y = -np.concatenate([sy.r_g, sy.r_h + sy.r_d / (sy.sig_d + dw)])
    rhs = np.concatenate([b_d, b_y - Js @ (b_s / q)])
    sol = np.linalg.solve(M, rhs)
    dxd, dy = sol[:n_d], sol[n_d:]
    dxs = (b_s - Js.T @ dy) / q
    return _finish(sy, dw, dxs, dxd, dy[:m_E], dy[m_E:], inertia)


def p2_applicable(Jsg, Jsh) -> bool:
    """J_sh = 0 and every column of J_sg has at most one nonzero."""
    if Jsh.nnz:
        return False
    col_counts = np.bincount(sp.coo_matrix(Jsg).col, minlength=Jsg.shape[1])
    return bool(np.all(col_counts <= 1))


def reduced_p2(sy: NewtonSystem, dw: float, dc: float):
    """S of the two-stage elimination, with q = diag(Q_s) and diagonal W."""
    n_s, n_d, m_E, m_I = sy.dims
    q = sy.Hss + sy.sig_xs + dw
    J2 = sy.Jsg.multiply(sy.Jsg).tocsr()
    w = J2 @ (1.0 / q) + dc
    S = np.zeros((n_d + m_I,) * 2)
    S[:n_d, :n_d] = sy.Hdd + np.diag(sy.sig_xd + dw) + sy.A.T @ (sy.A / w[:, None])
    S[n_d:, :n_d] = sy.Jdh
    S[:n_d, n_d:] = sy.Jdh.T
    ih = n_d + np.arange(m_I)
    S[ih, ih] = -1.0 / (sy.sig_d + dw) - dc
    return S, q, w


def direction_p2(sy: NewtonSystem, dw: float, dc: float):
    assert p2_applicable(sy.Jsg, sy.Jsh)
    n_s, n_d, m_E, m_I = sy.dims
    S, q, w = reduced_p2(sy, dw, dc)
    inertia = _add(_add(inertia_diag(q), inertia_diag(-w)), inertia_ldl(S))
    b_s, b_d, b_g = -sy.r_xs, -sy.r_xd, -sy.r_g
    b_h = -(sy.r_h + sy.r_d / (sy.sig_d + dw))
    bt_g = b_g - sy.Jsg @ (b_s / q)
    rhs = np.concatenate([b_d + sy.A.T @ (bt_g / w), b_h])
    sol = np.linalg.solve(S, rhs)
    dxd, dyh = sol[:n_d], sol[n_d:]
    dyg = (sy.A @ dxd - bt_g) / w
    dxs = (b_s - sy.Jsg.T @ dyg) / q
    return _finish(sy, dw, dxs, dxd, dyg, dyh, inertia)


DIRECTIONS = dict(full=direction_full, p1=direction_p1, p2=direction_p2)
