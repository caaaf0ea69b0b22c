"""The allocation-free LDL^T entry point (mdsip_ldlt_factor_noalloc).

It serves callers that cannot allocate device memory (their device memory is
owned by another allocator, or their loop must not take the synchronisation
that allocating can cause); its scratch is a fixed device array shared by
every call.  The test checks, through the C ABI, that two calls in a row give
the results of the allocating mdsip_ldlt_factor on the same inputs (so the
array's leftover contents from the previous call do not leak into the next),
that both take the Bunch-Kaufman decisions of the CPU oracle (oracle/bk.py:
permutation, 1x1/2x2 pattern and inertia bit for bit, D to the rounding bound
of the other LDL^T tests), and that sizes beyond the fixed limit are rejected.  It lives in its own file,
collected last, and passes alone in a fresh process as well as after the
other tests.
"""
import numpy as np
import pytest

import paper_2605_13736_gb300 as m
from oracle.bk import bk_ldlt
from gpu_util import dev, make_ctx, torch_cuda

pytestmark = pytest.mark.gpu


def _matrix(rng, n, kind):
    a = rng.standard_normal((n, n))
    a = a + a.T
    if kind == "zero_diag":
        np.fill_diagonal(a, 0.0)
    return a


def _factor(ctx, K, fn):
    torch = torch_cuda()
    N = K.shape[0]
    S = dev(np.tril(K).T.copy())          # column-major lower triangle
    out = dict(L=torch.zeros((N, N), dtype=torch.float64, device="cuda"),
               Dd=torch.zeros(N, dtype=torch.float64, device="cuda"),
               Doff=torch.zeros(N, dtype=torch.float64, device="cuda"),
               perm=torch.zeros(N, dtype=torch.int32, device="cuda"),
               kind=torch.zeros(N, dtype=torch.int32, device="cuda"),
               inertia=torch.zeros(3, dtype=torch.int32, device="cuda"))
    fn(ctx, N, S, N, 1e-14, out["L"], out["Dd"], out["Doff"], out["perm"], out["kind"], out["inertia"])
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["L"] = np.tril(res["L"].T)
    return res


def test_noalloc_ldlt_matches_allocating_entry_point():
    ctx = make_ctx()
    try:
        rng = np.random.default_rng(2024)
        # two calls in a row, different sizes and pivot structure
        for N, kind in ((1024, "zero_diag"), (700, "rand")):
            K = _matrix(rng, N, kind)
            ref = _factor(ctx, K, m.mdsip_ldlt_factor)
            got = _factor(ctx, K, m.mdsip_ldlt_factor_noalloc)
            np.testing.assert_array_equal(got["inertia"], ref["inertia"])
            np.testing.assert_array_equal(got["kind"], ref["kind"])
            np.testing.assert_array_equal(got["perm"], ref["perm"])
            tol = 1e-13 * N * np.abs(K).max()
            np.testing.assert_allclose(got["Dd"], ref["Dd"], rtol=1e-10, atol=tol)
            np.testing.assert_allclose(got["Doff"], ref["Doff"], rtol=1e-10, atol=tol)
            np.testing.assert_allclose(got["L"], ref["L"], rtol=1e-10, atol=1e-10)
            assert int(got["inertia"].sum()) == N
            # the oracle's unblocked Bunch-Kaufman on the same matrix
            o = bk_ldlt(K)
            assert tuple(int(v) for v in got["inertia"]) == tuple(o["inertia"])
            np.testing.assert_array_equal(got["kind"], o["kind"])
            np.testing.assert_array_equal(got["perm"], o["perm"])
            np.testing.assert_allclose(got["Dd"], np.diag(o["D"]), rtol=1e-10, atol=tol)
            np.testing.assert_allclose(got["Doff"], np.concatenate([np.diag(o["D"], -1), [0.0]]),
                                       rtol=1e-10, atol=tol)
        # beyond the fixed limit: a clear error, nothing launched
        torch = torch_cuda()
        N = 1025
        z = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        v = torch.zeros(N, dtype=torch.float64, device="cuda")
        iv = torch.zeros(N, dtype=torch.int32, device="cuda")
        inr = torch.zeros(3, dtype=torch.int32, device="cuda")
        with pytest.raises(m.MdsipError) as ei:
            m.mdsip_ldlt_factor_noalloc(ctx, N, z, N, 1e-14, z, v, v, iv, iv, inr)
        assert ei.value.status == 1 and "1024" in str(ei.value)
    finally:
        m.mdsip_ctx_destroy(ctx)
