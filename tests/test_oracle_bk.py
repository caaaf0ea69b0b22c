"""Pins of oracle.bk (Bunch-Kaufman LDL^T with inertia, Section 2.3)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.bk import bk_ldlt, bk_solve, ALPHA


def _sym(rng, n, kind):
    if kind == "rand":
        a = rng.standard_normal((n, n))
        return a + a.T
    if kind == "zero_diag":           # forces 2x2 pivots
        a = rng.standard_normal((n, n))
        a = a + a.T
        np.fill_diagonal(a, 0.0)
        return a
    if kind == "saddle":              # KKT-like [[H, J^T], [J, -c]]
        k = n // 2
        h = rng.standard_normal((k, k))
        h = h @ h.T / k + 0.1 * np.eye(k)
        j = rng.standard_normal((n - k, k))
        out = np.zeros((n, n))
        out[:k, :k] = h
        out[k:, :k] = j
        out[:k, k:] = j.T
        out[k:, k:] = -1e-3 * np.eye(n - k)
        return out
    raise ValueError(kind)


def _eig_inertia(K):
    ev = np.linalg.eigvalsh(K)
    tol = 1e-10 * max(1.0, np.abs(ev).max())
    return int(np.sum(ev > tol)), int(np.sum(ev < -tol)), int(np.sum(np.abs(ev) <= tol))


def _scipy_pattern(D):
    pat = []
    i = 0
    while i < D.shape[0]:
        if i + 1 < D.shape[0] and D[i + 1, i] != 0:
            pat += [2, 0]
            i += 2
        else:
            pat.append(1)
            i += 1
    return pat


@pytest.mark.parametrize("n", [1, 2, 3, 7, 17, 40])
@pytest.mark.parametrize("kind", ["rand", "zero_diag", "saddle"])
def test_bk_reconstructs_and_inertia(n, kind):
    rng = np.random.default_rng(100 * n + len(kind))
    K = _sym(rng, n, kind)
    fac = bk_ldlt(K)
    p, L, D = fac["perm"], fac["L"], fac["D"]
    R = K[np.ix_(p, p)] - L @ D @ L.T
    assert np.abs(R).max() <= 1e-12 * max(1.0, np.abs(K).max())
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
    # Sylvester: the inertia of D is that of K
    assert fac["inertia"] == _eig_inertia(K)
    # |L| bounded by the Bunch-Kaufman growth guarantee (1/(1-alpha) for 1x1 columns)
    if fac["inertia"][2] == 0:
        x = rng.standard_normal(n)
        np.testing.assert_allclose(bk_solve(fac, K @ x), x, rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("n", [5, 16, 33, 60])
def test_bk_matches_lapack_sytrf_pivots(n):
    """Same pivoting rule as LAPACK ?sytrf: same block pattern and same D."""
    rng = np.random.default_rng(n)
    for kind in ("rand", "zero_diag", "saddle"):
        K = _sym(rng, n, kind)
        fac = bk_ldlt(K)
        _, Dl, _ = sla.ldl(K, lower=True, hermitian=True)
        ours = [int(v) for v in fac["kind"]]
        assert ours == _scipy_pattern(Dl)
        np.testing.assert_allclose(np.diag(fac["D"]), np.diag(Dl), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(np.diag(fac["D"], -1), np.diag(Dl, -1), rtol=1e-9, atol=1e-12)


def test_bk_singular_and_special_cases():
    # zero matrix: every pivot is a zero 1x1
    fac = bk_ldlt(np.zeros((4, 4)))
    assert fac["inertia"] == (0, 0, 4)
    # [[0,1],[1,0]]: one 2x2 pivot with eigenvalues +1, -1
    fac = bk_ldlt(np.array([[0.0, 1.0], [1.0, 0.0]]))
    assert list(fac["kind"]) == [2, 0] and fac["inertia"] == (1, 1, 0)
    # diagonal: no interchanges, D = K
    d = np.array([3.0, -2.0, 1.0, -5.0])
    fac = bk_ldlt(np.diag(d))
    assert fac["inertia"] == (2, 2, 0) and np.allclose(np.diag(fac["D"]), d)
    assert list(fac["perm"]) == [0, 1, 2, 3]
    # rank-deficient PSD: one zero eigenvalue
    v = np.array([1.0, 2.0, 3.0])
    fac = bk_ldlt(np.outer(v, v) + np.outer([1.0, 0, -1.0], [1.0, 0, -1.0]))
    assert fac["inertia"] == (2, 0, 1)
    assert 0.6 < ALPHA < 0.65


def _ldlt_no_pivoting(K):
    """Textbook LDL^T without interchanges (right-looking, 1x1 pivots)."""
    a = np.array(K, dtype=float)
    n = a.shape[0]
    L = np.eye(n)
    d = np.zeros(n)
    for j in range(n):
        d[j] = a[j, j]
        L[j + 1:, j] = a[j + 1:, j] / d[j]
        a[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], a[j + 1:, j])
    return L, d


@pytest.mark.parametrize("case", ["dominant", "row_test_keeps"])
def test_bk_without_interchanges_is_the_unpivoted_factor(case):
    """The reading behind the mixed-precision factorization's no-interchange
    panels: when the Bunch-Kaufman rule keeps every diagonal pivot (1x1, no
    interchange, including columns that pass only the row test), its factor is
    the LDL^T factor without pivoting."""
    rng = np.random.default_rng(17)
    n = 60
    if case == "dominant":
        g = rng.standard_normal((n, n))
        K = 0.1 * (g + g.T) + np.diag(rng.uniform(2.0, 4.0, n))
    else:
        # column j: |a_jj| = 1 < alpha * 2 fails the column test; row r = 59 - j
        # holds 2 at (r, j) and 3 at (r, j + 1), so rowmax 3 passes the row test
        K = 10.0 * np.eye(n)
        for j, r in ((0, 59), (7, 58), (14, 57)):
            K[j, j] = 1.0
            K[r, j] = K[j, r] = 2.0
            K[r, j + 1] = K[j + 1, r] = 3.0
            K[r, r] = 100.0
    f = bk_ldlt(K)
    np.testing.assert_array_equal(f["perm"], np.arange(n))
    assert list(f["kind"]) == [1] * n
    if case == "row_test_keeps":   # the column test really fails at these columns
        for j in (0, 7, 14):
            assert abs(K[j, j]) < ALPHA * 2.0
    L, d = _ldlt_no_pivoting(K)
    np.testing.assert_allclose(f["L"], L, rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.diag(f["D"]), d, rtol=1e-12)
