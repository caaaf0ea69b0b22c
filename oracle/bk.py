"""Bunch-Kaufman symmetric indefinite LDL^T with inertia (Section 2.3).

Oracle (test infrastructure only).  The dense solver of Section 2.3 factors
P K P^T = L D L^T with D block diagonal (1x1 and 2x2 blocks), choosing pivots
by the partial-pivoting rule of Bunch and Kaufman (1977) with
alpha = (1 + sqrt(17)) / 8, and reads the inertia of K from D.  This is that
rule, written out unblocked on the lower triangle: at column k

    colmax  = max_{i>k} |a_ik|           (first index on ties)
    if |a_kk| >= alpha colmax                          -> 1x1 pivot, no swap
    else rowmax = max_{j != r} |a_rj| over the trailing block, r = argmax
         if |a_kk| >= alpha colmax (colmax / rowmax)  -> 1x1, no swap
         elif |a_rr| >= alpha rowmax                  -> 1x1, swap k <-> r
         else                                         -> 2x2, swap k+1 <-> r

followed by the rank-1 or rank-2 update of the trailing block.

Inertia: a 1x1 block counts by its sign, with |d| <= zero_tol * max|K| counted
as zero; a 2x2 block chosen by the rule above has a negative determinant
(|a_kk a_rr| < alpha^2 colmax^2 < a_rk^2) and counts (1 positive, 1 negative).

Pinned by tests/test_oracle_bk.py: P K P^T = L D L^T to rounding, the inertia
equals that of numpy.linalg.eigvalsh, the 1x1/2x2 block pattern and the
permutation equal those of scipy.linalg.ldl (LAPACK sytrf) on random inputs.
"""
from __future__ import annotations

import math
import numpy as np

ALPHA = (1.0 + math.sqrt(17.0)) / 8.0


def bk_ldlt(K, zero_tol=1e-14):
    """Factor symmetric K.  Returns dict(perm, L, D, kind, inertia).

    perm: row order with P K P^T = L D L^T, i.e. K[perm][:, perm] = L D L^T.
    kind: per column, 1 (1x1 pivot) or 2 (first column of a 2x2 pivot) or
          0 (second column of a 2x2 pivot).
    swaps: per pivot step, (k, kp, kstep) in the order they happened.
    inertia: (npos, nneg, nzero).
    """
    a = np.array(K, dtype=np.float64, copy=True)
    N = a.shape[0]
    scale = np.max(np.abs(a)) if N else 0.0
    perm = np.arange(N)
    L = np.eye(N)
    D = np.zeros((N, N))
    kind = np.zeros(N, dtype=np.int64)
    swaps = []
    npos = nneg = nzero = 0

    def swap(i, j):
        # symmetric interchange of rows/columns i and j of the working matrix,
        # and of the rows of the already computed columns of L
        if i == j:
            return
        a[[i, j], :] = a[[j, i], :]
        a[:, [i, j]] = a[:, [j, i]]
        L[[i, j], :k] = L[[j, i], :k]
        perm[[i, j]] = perm[[j, i]]

    k = 0
    while k < N:
        absakk = abs(a[k, k])
        if k + 1 < N:
            col = np.abs(a[k + 1:, k])
            r = k + 1 + int(np.argmax(col))
            colmax = float(col[r - k - 1])
        else:
            r, colmax = k, 0.0
        kstep = 1
        kp = k
        if max(absakk, colmax) == 0.0:
            kp = k
        elif absakk >= ALPHA * colmax:
            kp = k
        else:
            # largest off-diagonal magnitude in row/column r of the trailing block
            rowvals = np.concatenate([np.abs(a[r, k:r]), np.abs(a[r + 1:, r])])
            rowmax = float(np.max(rowvals))
            if absakk >= ALPHA * colmax * (colmax / rowmax):
                kp = k
            elif abs(a[r, r]) >= ALPHA * rowmax:
                kp = r
            else:
                kp = r
                kstep = 2
        kk = k + kstep - 1
        swaps.append((k, kp, kstep))
        swap(kk, kp)
        if kstep == 1:
            d = a[k, k]
            D[k, k] = d
            kind[k] = 1
            if abs(d) <= zero_tol * scale or d == 0.0:
                nzero += 1
            elif d > 0:
                npos += 1
            else:
                nneg += 1
            if d != 0.0 and k + 1 < N:
                l = a[k + 1:, k] / d
                L[k + 1:, k] = l
                a[k + 1:, k + 1:] -= np.outer(l, a[k + 1:, k])
        else:
            Dk = a[k:k + 2, k:k + 2].copy()
            Dk[0, 1] = Dk[1, 0]
            D[k:k + 2, k:k + 2] = Dk
            kind[k], kind[k + 1] = 2, 0
            npos += 1
            nneg += 1
            if k + 2 < N:
                C = a[k + 2:, k:k + 2]
                l = np.linalg.solve(Dk, C.T).T        # C D^{-1}
                L[k + 2:, k:k + 2] = l
                a[k + 2:, k + 2:] -= l @ C.T
        k += kstep
    return dict(perm=perm, L=L, D=D, kind=kind, swaps=swaps, inertia=(npos, nneg, nzero))


def bk_solve(fac, b):
    """Solve K x = b with the factors of `bk_ldlt`."""
    perm, L, D = fac["perm"], fac["L"], fac["D"]
    y = np.linalg.solve(L, np.asarray(b, dtype=np.float64)[perm])
    z = np.linalg.solve(D, y)
    w = np.linalg.solve(L.T, z)
    x = np.empty_like(w)
    x[perm] = w
    return x
