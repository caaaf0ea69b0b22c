"""Kernel-level parity on the GPU, through the C ABI:

* the FP64 condensation product A^T diag(1/w) A against the oracle's
  definition (numpy product), element by element, at sizes that span several
  64x64 tiles, split-K and ragged edges;
* the Bunch-Kaufman LDL^T against the oracle's plain Bunch-Kaufman
  (oracle.bk): inertia bit-exact, the same 1x1/2x2 pattern and permutation,
  D to 1e-10, the factorization reconstructs the input, and the solve.
"""
import numpy as np
import pytest

import paper_2605_13736_gb300 as m
from oracle.bk import bk_ldlt
from gpu_util import dev, make_ctx, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    m.mdsip_ctx_destroy(c)


@pytest.mark.parametrize("mrows,n", [(1, 1), (37, 5), (1000, 64), (1037, 130), (5000, 257), (20011, 64)])
def test_syrk_matches_definition(ctx, mrows, n):
    torch = torch_cuda()
    rng = np.random.default_rng(mrows + n)
    A = rng.standard_normal((mrows, n)) * 0.1
    w = rng.uniform(0.5, 4.0, mrows)
    lda = n + (n & 1)
    Ap = np.zeros((mrows, lda))
    Ap[:, :n] = A
    C0 = rng.standard_normal((n, n))
    for beta in (0.0, 1.0):
        Cd = dev(C0.T.copy())             # column-major storage of C0
        m.mdsip_syrk_scaled(ctx, mrows, n, dev(Ap), lda, dev(w), beta, Cd, n)
        torch.cuda.synchronize()
        got = Cd.cpu().numpy().T           # back to row-major view: got[p, q] = C[p][q]
        want = A.T @ (A / w[:, None]) + beta * C0
        scale = np.abs(A).T @ (np.abs(A) / w[:, None]) + abs(beta) * np.abs(C0)
        low = np.tril_indices(n)
        err = np.abs(got[low] - want[low]) / np.maximum(scale[low], 1e-300)
        assert err.max() <= 1e-13, err.max()
        up = np.triu_indices(n, 1)
        np.testing.assert_array_equal(got[up], C0[up])    # upper triangle untouched


def _sym(rng, n, kind):
    if kind == "rand":
        a = rng.standard_normal((n, n))
        return a + a.T
    if kind == "zero_diag":
        a = rng.standard_normal((n, n))
        a = a + a.T
        np.fill_diagonal(a, 0.0)
        return a
    k = n // 2
    h = rng.standard_normal((k, k))
    h = h @ h.T / max(k, 1) + 0.1 * np.eye(k)
    j = rng.standard_normal((n - k, k))
    out = np.zeros((n, n))
    out[:k, :k] = h
    out[k:, :k] = j
    out[:k, k:] = j.T
    out[k:, k:] = -1e-3 * np.eye(n - k)
    return out


def _gpu_ldlt(ctx, K):
    torch = torch_cuda()
    N = K.shape[0]
    S = dev(np.asfortranarray(np.tril(K)).T.copy())   # column-major lower triangle
    L = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    Dd = torch.zeros(N, dtype=torch.float64, device="cuda")
    Doff = torch.zeros(N, dtype=torch.float64, device="cuda")
    perm = torch.zeros(N, dtype=torch.int32, device="cuda")
    kind = torch.zeros(N, dtype=torch.int32, device="cuda")
    inertia = torch.zeros(3, dtype=torch.int32, device="cuda")
    m.mdsip_ldlt_factor(ctx, N, S, N, 1e-14, L, Dd, Doff, perm, kind, inertia)
    torch.cuda.synchronize()
    Lh = np.tril(L.cpu().numpy().T)            # L stored column-major
    return dict(L=Lh, Dd=Dd.cpu().numpy(), Doff=Doff.cpu().numpy(), perm=perm.cpu().numpy(),
                kind=kind.cpu().numpy(), inertia=tuple(int(v) for v in inertia.cpu().numpy()),
                dev=(L, Dd, Doff, perm))


@pytest.mark.parametrize("N", [1, 2, 3, 17, 33, 100, 257, 600, 1033])
@pytest.mark.parametrize("kind", ["rand", "zero_diag", "saddle"])
def test_ldlt_matches_oracle_bunch_kaufman(ctx, N, kind):
    torch = torch_cuda()
    rng = np.random.default_rng(N * 7 + len(kind))
    K = _sym(rng, N, kind)
    g = _gpu_ldlt(ctx, K)
    o = bk_ldlt(K)
    assert g["inertia"] == o["inertia"]
    np.testing.assert_array_equal(g["kind"], o["kind"])
    np.testing.assert_array_equal(g["perm"], o["perm"])
    # entries of D carry a forward error of order N u max|K| (u = 2^-53) from
    # the N rank-1/rank-2 updates each side performs in its own order
    tol_d = 1e-13 * N * max(1.0, np.abs(K).max())
    np.testing.assert_allclose(g["Dd"], np.diag(o["D"]), rtol=1e-10, atol=tol_d)
    np.testing.assert_allclose(g["Doff"], np.concatenate([np.diag(o["D"], -1), [0.0]]), rtol=1e-10, atol=tol_d)
    D = np.diag(g["Dd"]) + np.diag(g["Doff"][:-1], -1) + np.diag(g["Doff"][:-1], 1)
    p = g["perm"]
    R = K[np.ix_(p, p)] - g["L"] @ D @ g["L"].T
    assert np.abs(R).max() <= 1e-11 * max(1.0, np.abs(K).max()) * max(1, N) ** 0.5
    if g["inertia"][2] == 0:
        B = rng.standard_normal((2, N))
        Bd = dev(B.copy())
        L, Dd, Doff, perm = g["dev"]
        m.mdsip_ldlt_solve(ctx, N, L, Dd, Doff, perm, 2, Bd, N)
        torch.cuda.synchronize()
        X = Bd.cpu().numpy()
        for r in range(2):
            res = K @ X[r] - B[r]
            assert np.abs(res).max() <= 1e-9 * (np.abs(K).max() * np.abs(X[r]).max() + np.abs(B[r]).max())


@pytest.mark.parametrize("N,kind", [(2600, "saddle"), (4200, "zero_diag")])
def test_ldlt_large_orders(ctx, N, kind):
    """Orders that take many panels and (at 4200) the narrower panel width:
    reconstruction and the inertia of numpy.linalg.eigvalsh."""
    rng = np.random.default_rng(N)
    K = _sym(rng, N, kind)
    g = _gpu_ldlt(ctx, K)
    ev = np.linalg.eigvalsh(K)
    tol = 1e-9 * np.abs(ev).max()
    assert np.min(np.abs(ev)) > tol
    assert g["inertia"] == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    D = np.diag(g["Dd"]) + np.diag(g["Doff"][:-1], -1) + np.diag(g["Doff"][:-1], 1)
    p = g["perm"]
    R = K[np.ix_(p, p)] - g["L"] @ D @ g["L"].T
    assert np.abs(R).max() <= 1e-11 * max(1.0, np.abs(K).max()) * N ** 0.5


@pytest.mark.parametrize("N,kind", [(600, "saddle"), (2100, "saddle"), (300, "zero_diag")])
def test_ldlt_fp32_updates(ctx, N, kind):
    """The mixed-precision factorization (FP32 update products, FP64 pivots):
    inertia of numpy.linalg.eigvalsh and a reconstruction at FP32 accuracy."""
    torch = torch_cuda()
    rng = np.random.default_rng(N + 5)
    K = _sym(rng, N, kind)
    S = dev(np.asfortranarray(np.tril(K)).T.copy())
    L = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    Dd = torch.zeros(N, dtype=torch.float64, device="cuda")
    Doff = torch.zeros(N, dtype=torch.float64, device="cuda")
    perm = torch.zeros(N, dtype=torch.int32, device="cuda")
    kd = torch.zeros(N, dtype=torch.int32, device="cuda")
    inr = torch.zeros(3, dtype=torch.int32, device="cuda")
    m.mdsip_ldlt_factor_ex(ctx, N, S, N, 1e-14, m.MDSIP_LDLT_FP32_UPDATES, L, Dd, Doff, perm, kd, inr)
    torch.cuda.synchronize()
    ev = np.linalg.eigvalsh(K)
    assert tuple(int(v) for v in inr.cpu().numpy()) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    Lh = np.tril(L.cpu().numpy().T)
    dd, do, p = Dd.cpu().numpy(), Doff.cpu().numpy(), perm.cpu().numpy()
    D = np.diag(dd) + np.diag(do[:-1], -1) + np.diag(do[:-1], 1)
    R = K[np.ix_(p, p)] - Lh @ D @ Lh.T
    assert np.abs(R).max() <= 1e-4 * np.abs(K).max()
    with pytest.raises(m.MdsipError):
        m.mdsip_ldlt_factor_ex(ctx, N, S, N, 1e-14, 8, L, Dd, Doff, perm, kd, inr)
    with pytest.raises(m.MdsipError):     # pivot every panel and run the persistent kernel: contradictory
        m.mdsip_ldlt_factor_ex(ctx, N, S, N, 1e-14, m.MDSIP_LDLT_NO_SPECULATION | m.MDSIP_LDLT_PERSISTENT,
                               L, Dd, Doff, perm, kd, inr)


def _ipm_like(rng, nd, mi):
    """A Newton-step matrix of the P1 form [[H + Sigma, J^T], [J, -D]]: H + Sigma
    positive definite and diagonally dominant, J small, D > 0 (the shape of
    the condensed systems of a convex problem at a usual iterate)."""
    g = rng.standard_normal((nd, nd)) / np.sqrt(nd)
    h = g @ g.T + np.diag(rng.uniform(1.0, 3.0, nd))
    j = 0.1 * rng.standard_normal((mi, nd))
    out = np.zeros((nd + mi, nd + mi))
    out[:nd, :nd] = h
    out[nd:, :nd] = j
    out[:nd, nd:] = j.T
    out[nd:, nd:] = -np.diag(rng.uniform(0.5, 2.0, mi))
    return out


def _row_test_matrix(n, second):
    """Diagonal 10 with, for every 7th column j < n - 60, a_jj = 1, a_rj = 2 in
    a late row r, and a_rc = `second` in column c = j + 1, a_rr = 100.  At
    column j the Bunch-Kaufman column test fails (1 < alpha 2); the row test
    keeps the 1x1 pivot without interchange when second = 3 (rowmax 3) and
    interchanges j and r when second = 2.1 (rowmax 2.1)."""
    K = 10.0 * np.eye(n)
    r = n - 1
    for j in range(0, n - 60, 7):
        K[j, j] = 1.0
        K[r, j] = K[j, r] = 2.0
        K[r, j + 1] = K[j + 1, r] = second
        K[r, r] = 100.0
        r -= 1
    return K


def _fp32_ldlt(ctx, K, flags):
    torch = torch_cuda()
    N = K.shape[0]
    S = dev(np.asfortranarray(np.tril(K)).T.copy())
    L = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    Dd = torch.zeros(N, dtype=torch.float64, device="cuda")
    Doff = torch.zeros(N, dtype=torch.float64, device="cuda")
    perm = torch.zeros(N, dtype=torch.int32, device="cuda")
    kd = torch.zeros(N, dtype=torch.int32, device="cuda")
    inr = torch.zeros(3, dtype=torch.int32, device="cuda")
    m.mdsip_ldlt_factor_ex(ctx, N, S, N, 1e-14, flags, L, Dd, Doff, perm, kd, inr)
    torch.cuda.synchronize()
    out = dict(L=np.tril(L.cpu().numpy().T), Dd=Dd.cpu().numpy(), Doff=Doff.cpu().numpy(),
               perm=perm.cpu().numpy(), kind=kd.cpu().numpy(),
               inertia=tuple(int(v) for v in inr.cpu().numpy()), panels=m.mdsip_ldlt_panel_counts(ctx))
    D = np.diag(out["Dd"]) + np.diag(out["Doff"][:-1], -1) + np.diag(out["Doff"][:-1], 1)
    p = out["perm"]
    out["resid"] = np.abs(K[np.ix_(p, p)] - out["L"] @ D @ out["L"].T).max() / np.abs(K).max()
    return out


@pytest.mark.parametrize("N,kind", [(2050, "ipm"), (700, "row_keep"), (700, "row_swap"), (2100, "saddle"),
                                    (1500, "mixed"), (64, "ipm"), (65, "ipm"), (1, "ipm")])
def test_ldlt_fp32_speculation(ctx, N, kind):
    """The mixed-precision factorization with the verified no-interchange
    panels against the same factorization with every panel pivoting and
    against the oracle's Bunch-Kaufman: the same inertia, 1x1/2x2 pattern and
    permutation (the matrices keep every pivot decision far from its
    threshold), D within FP32 accuracy, the reconstruction at FP32 accuracy,
    and the panel counts show which path took the panels."""
    rng = np.random.default_rng(N * 7 + len(kind))
    if kind == "ipm":
        K = _ipm_like(rng, N - min(50, N // 3), min(50, N // 3))
    elif kind == "row_keep":
        K = _row_test_matrix(N, 3.0)
    elif kind == "row_swap":
        K = _row_test_matrix(N, 2.1)
    elif kind == "mixed":     # a convex block, then a block that pivots
        K = np.zeros((N, N))
        K[:900, :900] = _ipm_like(rng, 860, 40)
        K[900:, 900:] = _sym(rng, N - 900, "saddle")
    else:
        K = _sym(rng, N, kind)
    spec = _fp32_ldlt(ctx, K, m.MDSIP_LDLT_FP32_UPDATES)
    piv = _fp32_ldlt(ctx, K, m.MDSIP_LDLT_FP32_UPDATES | m.MDSIP_LDLT_NO_SPECULATION)
    assert piv["panels"] == (0, 0)
    o = bk_ldlt(K)
    # FP32 products: a reconstruction error of a few 2^-24 times the growth of
    # the factors, which interchanges on the saddle matrices make larger
    tol = 1e-4 if kind in ("saddle", "mixed") else 1e-5
    for g in (spec, piv):
        assert g["inertia"] == o["inertia"]
        if kind != "saddle":   # a random saddle matrix has near-ties in its pivot tests
            np.testing.assert_array_equal(g["kind"], o["kind"])
            np.testing.assert_array_equal(g["perm"], o["perm"])
        assert g["resid"] <= tol, (spec["resid"], piv["resid"])
    if kind != "saddle":   # (the saddle block's late pivots carry the growth of its interchanges)
        nd = 900 if kind == "mixed" else N
        np.testing.assert_allclose(spec["Dd"][:nd], np.diag(o["D"])[:nd], rtol=1e-4, atol=1e-5 * np.abs(K).max())
    acc, rej = spec["panels"]
    if kind in ("ipm", "row_keep"):
        assert acc >= 1 and rej == 0
        np.testing.assert_array_equal(spec["perm"], np.arange(N))
    elif kind == "row_swap":
        assert rej >= 1
    elif kind == "mixed":
        assert acc >= 1 and rej >= 1


@pytest.mark.parametrize("N", [2600, 4200])
def test_ldlt_fp32_speculation_large(ctx, N):
    """Orders with many panels and (at 4200) the 32-column panels: every panel
    of a convex Newton-step matrix is kept without interchanges, the inertia is
    that of numpy.linalg.eigvalsh, and the reconstruction has FP32 accuracy."""
    rng = np.random.default_rng(N + 11)
    K = _ipm_like(rng, N - 50, 50)
    g = _fp32_ldlt(ctx, K, m.MDSIP_LDLT_FP32_UPDATES)
    ev = np.linalg.eigvalsh(K)
    assert g["inertia"] == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    acc, rej = g["panels"]
    assert acc >= N // 64 and rej == 0
    np.testing.assert_array_equal(g["perm"], np.arange(N))
    assert g["resid"] <= 1e-5


@pytest.mark.parametrize("mrows,n", [(1, 1), (5, 3), (1000, 2000), (3001, 2500), (700, 4100), (20011, 64)])
def test_gemv_pair_df_within_bound(ctx, mrows, n):
    """A x and A^T v from the double-float pass against the exact products
    (FP64 products summed exactly by math.fsum: their own error is below
    2^-53 of the sum of |terms|), element by element, with entries spread over
    2^-20 .. 2^20 so that the low halves of A and x matter."""
    import math
    torch = torch_cuda()
    rng = np.random.default_rng(mrows * 7 + n)
    A = rng.standard_normal((mrows, n)) * np.exp2(rng.integers(-20, 21, (mrows, n)))
    x = rng.standard_normal(n) * np.exp2(rng.integers(-20, 21, n))
    v = rng.standard_normal(mrows) * np.exp2(rng.integers(-20, 21, mrows))
    lda = (n + 3) // 4 * 4
    Ap = np.zeros((mrows, lda))
    Ap[:, :n] = A
    Ax, ATv = dev(np.full(mrows, np.nan)), dev(np.full(n, np.nan))
    m.mdsip_gemv_pair_df(ctx, mrows, n, dev(Ap), lda, dev(x), dev(v), Ax, ATv)
    torch.cuda.synchronize()
    Ax, ATv = Ax.cpu().numpy(), ATv.cpu().numpy()
    P, Q = A * x[None, :], A * v[:, None]
    ex_r = np.array([math.fsum(P[i]) for i in range(mrows)])
    ex_c = np.array([math.fsum(Q[:, p]) for p in range(n)])
    S_r, S_c = np.abs(P).sum(axis=1), np.abs(Q).sum(axis=0)
    err_r, err_c = np.abs(Ax - ex_r) / S_r, np.abs(ATv - ex_c) / S_c
    assert err_r.max() <= 2.0 ** -36 and err_c.max() <= 2.0 ** -36
    # typical errors: the split and cross-term roundings, about 2^-49 of each
    # term (an FP64 product of these sizes errs by up to 2^-53 per term plus
    # n 2^-53 in its sum); a dropped low half or cross term would leave
    # errors near 2^-24
    assert np.median(err_r) <= 2.0 ** -46 and np.median(err_c) <= 2.0 ** -46


@pytest.mark.parametrize("mrows,n", [(1, 1), (5, 3), (150, 7), (1000, 2000), (3001, 2048), (20011, 64)])
def test_gemv_pair_df_next_folds_the_solve_half(ctx, mrows, n):
    """The fused form of the pass: A x and A^T v bit for bit as the plain pass,
    and A_hi^T w, w_i = fl32(d_i fl32(winv_i)) with d_i the double-float
    difference cpre_i - (A x)_i rounded to FP32, within its stated bound of
    sum_i A_hi[i][p] (cpre_i - (A x)_i) winv_i: the FP32 block sums, the
    roundings of d_i, winv_i and w_i (2^-22 of |w|), and 2^-46 |cpre_i| winv_i.
    A_hi times a float64 is summed exactly by math.fsum.  cpre is A x plus a
    small offset on half of the rows, so that the difference cancels; the
    magnitudes are of order one, so that a row paired with another row's w
    (the pass learns w one batch late) misses the bound by orders of
    magnitude."""
    import math
    torch = torch_cuda()
    rng = np.random.default_rng(mrows * 11 + n)
    A = rng.standard_normal((mrows, n)) * np.exp2(rng.integers(-3, 4, (mrows, n)))
    x, v = rng.standard_normal(n), rng.standard_normal(mrows)
    winv = rng.uniform(0.5, 2.0, mrows)
    lda = (n + 3) // 4 * 4
    Ap = np.zeros((mrows, lda))
    Ap[:, :n] = A
    dA, dx, dv = dev(Ap), dev(x), dev(v)
    Ax0, ATv0 = dev(np.full(mrows, np.nan)), dev(np.full(n, np.nan))
    m.mdsip_gemv_pair_df(ctx, mrows, n, dA, lda, dx, dv, Ax0, ATv0)
    torch.cuda.synchronize()
    Ax0 = Ax0.cpu().numpy()
    cpre = np.where(rng.random(mrows) < 0.5, Ax0 * (1.0 + 1e-6 * rng.standard_normal(mrows)),
                    4.0 * rng.standard_normal(mrows))
    Ax, ATv, ATw = dev(np.full(mrows, np.nan)), dev(np.full(n, np.nan)), dev(np.full(n, np.nan))
    m.mdsip_gemv_pair_df_next(ctx, mrows, n, dA, lda, dx, dv, dev(cpre), dev(winv), Ax, ATv, ATw)
    torch.cuda.synchronize()
    Ax, ATv, ATw = (t.cpu().numpy() for t in (Ax, ATv, ATw))
    np.testing.assert_array_equal(Ax, Ax0)
    np.testing.assert_array_equal(ATv, ATv0.cpu().numpy())
    Ah = np.abs(A.astype(np.float32).astype(np.float64))
    w_ref = (cpre - Ax) * winv
    Q = A.astype(np.float32).astype(np.float64) * w_ref[:, None]
    ex = np.array([math.fsum(Q[:, p]) for p in range(n)])
    S = Ah.T @ np.abs(w_ref)
    S3 = Ah.T @ (np.abs(cpre) * winv)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows = -(-mrows // min(sms, 152))
    err = np.abs(ATw - ex)
    bound = (rows + 7) * 2.0 ** -24 * S + 2.0 ** -45 * S3
    assert np.all(err <= bound), float((err / bound).max())


def test_gemv_pair_df_next_rejects_a_row_wider_than_a_slice(ctx):
    torch = torch_cuda()
    A = dev(np.zeros((4, 2052)))
    out = dev(np.zeros(2052))
    with pytest.raises(m.MdsipError):   # n > 2048
        m.mdsip_gemv_pair_df_next(ctx, 4, 2049, A, 2052, out, out, out, out, out, out, out)
    with pytest.raises(m.MdsipError):   # n = 0
        m.mdsip_gemv_pair_df_next(ctx, 4, 0, A, 4, out, out, out, out, out, out, out)
    torch.cuda.synchronize()


def test_gemv_pair_df_rejects_bad_arguments(ctx):
    torch = torch_cuda()
    A = dev(np.zeros((4, 8)))
    out = dev(np.zeros(8))
    with pytest.raises(m.MdsipError):   # lda not a multiple of 4
        m.mdsip_gemv_pair_df(ctx, 4, 6, A, 6, out, out, out, out)
    with pytest.raises(m.MdsipError):   # lda < n
        m.mdsip_gemv_pair_df(ctx, 4, 8, A, 4, out, out, out, out)
    m.mdsip_gemv_pair_df(ctx, 0, 0, None, 4, None, None, None, None)
    torch.cuda.synchronize()


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("N", [1, 20, 63, 64, 65, 200, 1033, 2600])
def test_ldlt_persistent_keeps_every_panel(ctx, N, fp32):
    """Convex Newton-step matrices (every Bunch-Kaufman decision keeps the
    diagonal): the persistent no-interchange factorization (forced below the
    order where it runs by itself) keeps every panel of
    64 columns, so no pivoting panel runs; the oracle's permutation (identity),
    1x1 pivots and inertia, D to rounding (FP64) or FP32 accuracy, and the
    reconstruction."""
    rng = np.random.default_rng(N * 13 + fp32)
    K = _ipm_like(rng, N - min(50, N // 3), min(50, N // 3))
    g = _fp32_ldlt(ctx, K, (m.MDSIP_LDLT_FP32_UPDATES if fp32 else 0) | m.MDSIP_LDLT_PERSISTENT)
    o = bk_ldlt(K)
    assert g["inertia"] == o["inertia"]
    np.testing.assert_array_equal(g["kind"], o["kind"])
    np.testing.assert_array_equal(g["perm"], np.arange(N))
    np.testing.assert_array_equal(o["perm"], np.arange(N))
    assert g["panels"] == ((N + 63) // 64, 0)
    if fp32:
        np.testing.assert_allclose(g["Dd"], np.diag(o["D"]), rtol=1e-4, atol=1e-5 * np.abs(K).max())
        assert g["resid"] <= 1e-5
    else:
        tol_d = 1e-13 * N * max(1.0, np.abs(K).max())
        np.testing.assert_allclose(g["Dd"], np.diag(o["D"]), rtol=1e-10, atol=tol_d)
        assert g["resid"] <= 1e-12 * max(1, N) ** 0.5


@pytest.mark.parametrize("fp32", [False, True])
def test_ldlt_persistent_hands_over_midway(ctx, fp32):
    """A convex block, then a block whose pivots need interchanges: the
    persistent kernel keeps the leading panels and stops at the first panel
    the column test rejects; the pivoting panels finish from there with the
    oracle's permutation, pivot kinds and inertia.  (The FP32-update form
    takes a saddle block, whose pivot tests are far from their thresholds; on
    a random block with a zero diagonal its FP32 products may tip near-ties.)"""
    rng = np.random.default_rng(91 + fp32)
    N = 1500
    K = np.zeros((N, N))
    K[:900, :900] = _ipm_like(rng, 860, 40)
    K[900:, 900:] = _sym(rng, N - 900, "saddle" if fp32 else "zero_diag")
    g = _fp32_ldlt(ctx, K, (m.MDSIP_LDLT_FP32_UPDATES if fp32 else 0) | m.MDSIP_LDLT_PERSISTENT)
    o = bk_ldlt(K)
    assert g["inertia"] == o["inertia"]
    np.testing.assert_array_equal(g["kind"], o["kind"])
    np.testing.assert_array_equal(g["perm"], o["perm"])
    acc, _ = g["panels"]
    assert 900 // 64 <= acc < (N + 63) // 64
    assert g["resid"] <= (1e-4 if fp32 else 1e-11)


@pytest.mark.parametrize("fp32", [False, True])
def test_ldlt_order_beyond_the_pivoting_panel(ctx, fp32):
    """N = 20003, beyond the order whose pivoting panel fits shared memory: a
    convex Newton-step matrix [[H, J^T], [J, -D]] (H, D positive definite, so
    its inertia is (n_d, m_I, 0) by Sylvester's law) factors through the
    persistent kernel alone, with that inertia, the identity permutation, and
    a solve whose residual is at the factor's precision."""
    torch = torch_cuda()
    nd, mi = 19953, 50
    N = nd + mi
    gen = torch.Generator(device="cuda").manual_seed(5)
    K = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    B = torch.randn((nd, nd), dtype=torch.float64, device="cuda", generator=gen) * (0.5 / np.sqrt(2.0 * nd))
    K[:nd, :nd] = B + B.T      # spectrum within about [-1, 1]
    del B
    K[:nd, :nd] += torch.diag(2.0 + torch.rand(nd, dtype=torch.float64, device="cuda", generator=gen))
    J = 0.1 * torch.randn((mi, nd), dtype=torch.float64, device="cuda", generator=gen)
    K[nd:, :nd] = J
    K[:nd, nd:] = J.T
    K[nd:, nd:] = -torch.diag(0.5 + 1.5 * torch.rand(mi, dtype=torch.float64, device="cuda", generator=gen))
    S = K.clone()           # symmetric: its row-major storage is the column-major lower triangle
    L = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    Dd = torch.zeros(N, dtype=torch.float64, device="cuda")
    Doff = torch.zeros(N, dtype=torch.float64, device="cuda")
    perm = torch.zeros(N, dtype=torch.int32, device="cuda")
    kd = torch.zeros(N, dtype=torch.int32, device="cuda")
    inr = torch.zeros(3, dtype=torch.int32, device="cuda")
    flags = m.MDSIP_LDLT_FP32_UPDATES if fp32 else 0
    m.mdsip_ldlt_factor_ex(ctx, N, S, N, 1e-14, flags, L, Dd, Doff, perm, kd, inr)
    torch.cuda.synchronize()
    del S
    assert tuple(int(v) for v in inr.cpu().numpy()) == (nd, mi, 0)
    assert torch.equal(perm.cpu(), torch.arange(N, dtype=torch.int32))
    assert bool((kd == 1).all())
    assert m.mdsip_ldlt_panel_counts(ctx) == ((N + 63) // 64, 0)
    b = torch.randn((1, N), dtype=torch.float64, device="cuda", generator=gen)
    x = b.clone()
    m.mdsip_ldlt_solve(ctx, N, L, Dd, Doff, perm, 1, x, N)
    torch.cuda.synchronize()
    r = (K @ x[0] - b[0]).abs().max().item()
    scale = K.abs().max().item() * x.abs().max().item() + b.abs().max().item()
    assert r <= (1e-4 if fp32 else 1e-11) * scale, r / scale


def test_ldlt_singular_and_edge_cases(ctx):
    g = _gpu_ldlt(ctx, np.zeros((5, 5)))
    assert g["inertia"] == (0, 0, 5)
    g = _gpu_ldlt(ctx, np.array([[0.0, 1.0], [1.0, 0.0]]))
    assert g["inertia"] == (1, 1, 0) and list(g["kind"]) == [2, 0]
    d = np.array([3.0, -2.0, 1.0, -5.0, 0.5])
    g = _gpu_ldlt(ctx, np.diag(d))
    assert g["inertia"] == (3, 2, 0)
    np.testing.assert_array_equal(g["perm"], np.arange(5))
    np.testing.assert_array_equal(g["Dd"], d)


@pytest.mark.parametrize("prec", [m.MDSIP_PREC_BF16, m.MDSIP_PREC_TF32])
@pytest.mark.parametrize("mrows,n", [(64, 8), (1000, 64), (5000, 130), (20011, 300)])
def test_syrk_tensor_core_matches_definition(ctx, prec, mrows, n):
    """tcgen05 product vs the FP64 definition: error per entry within the
    operand type's rounding (BF16 2^-8, TF32 2^-10 per product, both operands
    rounded) plus FP32 accumulation, relative to sum_i |A_ip A_iq| / w_i."""
    torch = torch_cuda()
    rng = np.random.default_rng(mrows * 3 + n + prec)
    A = rng.standard_normal((mrows, n)) * 0.1
    w = rng.uniform(0.05, 4.0, mrows)
    C0 = rng.standard_normal((n, n))
    want = A.T @ (A / w[:, None]) + C0
    scale = np.abs(A).T @ (np.abs(A) / w[:, None])
    Cd = dev(C0.T.copy())
    m.mdsip_syrk_scaled_tc(ctx, mrows, n, dev(A), n, dev(w), 1.0, Cd, n, prec)
    torch.cuda.synchronize()
    got = Cd.cpu().numpy().T
    low = np.tril_indices(n)
    rel = np.abs(got[low] - want[low]) / scale[low]
    bound = 2.0 ** -7 if prec == m.MDSIP_PREC_BF16 else 2.0 ** -9
    assert rel.max() <= bound, rel.max()
    # and it is a real low-precision product, not an FP64 one in disguise
    assert rel.max() > 1e-9
    up = np.triu_indices(n, 1)
    np.testing.assert_array_equal(got[up], C0.T.T[up])
