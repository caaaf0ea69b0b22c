"""Pins of oracle.model: derivatives against central finite differences."""
import numpy as np

import synth
from oracle.model import SynthModel


def _fd(fun, x, eps=1e-6):
    cols = []
    for i in range(x.size):
        e = np.zeros_like(x)
        e[i] = eps
        cols.append((np.atleast_1d(fun(x + e)) - np.atleast_1d(fun(x - e))) / (2 * eps))
    return np.stack(cols, axis=-1)


import pytest


@pytest.mark.parametrize("jsh", [0, 3])
def test_derivatives_match_finite_differences(jsh):
    inst = synth.make_instance(5, 6, 2, 0.3, seed=11, jsh_per_row=jsh)
    m = SynthModel(inst)
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.8, 0.8, size=m.n)
    # gradient of f
    np.testing.assert_allclose(m.grad_f(x), _fd(m.f, x)[0], rtol=1e-7, atol=1e-8)
    # Jacobians of g and h, block by block
    Jsg, Jsh, A, Jdh = m.jac(x)
    Jg = np.hstack([Jsg.toarray(), A])
    Jh = np.hstack([Jsh.toarray(), Jdh])
    np.testing.assert_allclose(Jg, _fd(m.g, x), rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(Jh, _fd(m.h, x), rtol=1e-7, atol=1e-8)
    # Hessian of the Lagrangian f + y_g^T g + y_h^T h
    yg = rng.standard_normal(m.m_E)
    yh = rng.uniform(0, 1, size=m.m_I)
    gradL = lambda v: m.grad_f(v) + Jg.T @ yg + np.hstack([Jsh.toarray(), m.jac(v)[3]]).T @ yh
    H = _fd(gradL, x)
    Hss, Hdd = m.hess(x, yg, yh)
    full = np.zeros((m.n, m.n))
    full[np.arange(m.n_s), np.arange(m.n_s)] = Hss
    full[m.n_s:, m.n_s:] = Hdd
    np.testing.assert_allclose(full, H, rtol=1e-6, atol=1e-7)
    # assumption A1: no cross-term Hessians, and the x_s block is diagonal (A2)
    assert np.allclose(H[:m.n_s, m.n_s:], 0, atol=1e-7)
    off = H[:m.n_s, :m.n_s] - np.diag(np.diag(H[:m.n_s, :m.n_s]))
    assert np.allclose(off, 0, atol=1e-7)


def test_instance_structure():
    inst = synth.make_config(0)
    assert (inst.n_d, inst.n_s, inst.m_E, inst.m_I) == (32, 2000, 1000, 1)
    m = SynthModel(inst)
    # row i: x_s,i - x_s,i+m_E
    J = m.Jsg.toarray()
    assert np.all(J[np.arange(1000), np.arange(1000)] == 1)
    assert np.all(J[np.arange(1000), np.arange(1000) + 1000] == -1)
    assert np.count_nonzero(J) == 2000
    # Q symmetric positive definite
    assert np.allclose(inst.Q, inst.Q.T)
    assert np.linalg.eigvalsh(inst.Q).min() > 0.09
    # the c1-shaped family splits x_d into m_I disjoint chunks
    small = synth.make_instance(100, 10, 5, 0.01, seed=1)
    counts = np.bincount(small.h_set[small.h_set >= 0], minlength=5)
    assert np.all(counts == 20)


def test_sparse_inequality_part():
    """jsh_per_row adds h_j += sum e_ja x_s,a with that many distinct indices per
    row, and leaves every other array of the instance as it was."""
    a = synth.make_instance(8, 20, 3, 0.1, seed=5)
    b = synth.make_instance(8, 20, 3, 0.1, seed=5, jsh_per_row=4)
    for k in ("Q", "c", "A", "b", "h_set", "hu", "xl", "xu"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert a.Jsh_rows.size == 0 and b.Jsh_rows.size == 12
    for j in range(3):
        cols = b.Jsh_cols[b.Jsh_rows == j]
        assert cols.size == 4 and np.unique(cols).size == 4
    m = SynthModel(b)
    x = np.random.default_rng(1).uniform(-0.5, 0.5, m.n)
    xs, xd = x[:m.n_s], x[m.n_s:]
    h = np.array([np.sum(xd[b.h_set == j] ** 2) for j in range(3)])
    for r, c, v in zip(b.Jsh_rows, b.Jsh_cols, b.Jsh_vals):
        h[r] += v * xs[c]
    np.testing.assert_allclose(m.h(x), h, rtol=1e-15, atol=1e-15)
