"""Evaluation of the synthetic MDS problem (Section 2, Eqs. (obj)-(bounds)).

Oracle (test infrastructure only).  The Hessian is that of the Lagrangian
L = f + y_g^T g + y_h^T h (Section 2, display after assumption A2), so
grad_x L = grad f + J_g^T y_g + J_h^T y_h.  Assumption A1 (zero cross
Hessians) holds by construction, so the Hessian is returned as the diagonal
x_s block and the dense x_d block.

Pinned by tests/test_oracle_model.py: every derivative is checked against
central finite differences of the value it differentiates.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class SynthModel:
    """f, g, h and their derivatives for a `synth.Instance`."""

    def __init__(self, inst):
        self.inst = inst
        self.n_s, self.n_d, self.m_E, self.m_I = inst.n_s, inst.n_d, inst.m_E, inst.m_I
        self.n = inst.n_s + inst.n_d
        self.Jsg = sp.csr_matrix((inst.Jsg_vals, (inst.Jsg_rows, inst.Jsg_cols)),
                                 shape=(inst.m_E, inst.n_s))
        # sparse block of the inequalities (zero in the benchmark family); h is
        # linear in x_s, so it adds nothing to the Hessian
        self.Jsh = sp.csr_matrix((inst.Jsh_vals, (inst.Jsh_rows, inst.Jsh_cols)),
                                 shape=(inst.m_I, inst.n_s))
        self.A = inst.A
        self.Q = inst.Q
        self.c = inst.c
        self.gE = inst.b
        self.h_set = inst.h_set
        # membership matrix E (m_I x n_d): E[j, k] = 1 iff x_d[k] is in subset S_j
        k = np.nonzero(inst.h_set >= 0)[0]
        self.E = sp.csr_matrix((np.ones(k.size), (inst.h_set[k], k)), shape=(inst.m_I, inst.n_d))
        self.xl, self.xu, self.hl, self.hu = inst.xl, inst.xu, inst.hl, inst.hu

    def split(self, x):
        return x[:self.n_s], x[self.n_s:]

    def f(self, x):
        xs, xd = self.split(x)
        return 0.5 * xd @ (self.Q @ xd) + 0.25 * np.sum(xs ** 4) + self.c @ x

    def grad_f(self, x):
        xs, xd = self.split(x)
        return np.concatenate([xs ** 3, self.Q @ xd]) + self.c

    def g(self, x):
        xs, xd = self.split(x)
        return self.Jsg @ xs + self.A @ xd

    def h(self, x):
        xs, xd = self.split(x)
        return self.E @ (xd * xd) + self.Jsh @ xs

    def jac(self, x):
        """Blocks of the constraint Jacobian: (J_sg, J_sh, J_dg = A, J_dh)."""
        xs, xd = self.split(x)
        Jdh = self.E.toarray() * (2.0 * xd)[None, :]
        return self.Jsg, self.Jsh, self.A, Jdh

    def hess(self, x, yg, yh):
        """Hessian of the Lagrangian: (diagonal of the x_s block, dense x_d block)."""
        xs, xd = self.split(x)
        Hss = 3.0 * xs ** 2
        Hdd = self.Q + np.diag(2.0 * (self.E.T @ yh))
        return Hss, Hdd
