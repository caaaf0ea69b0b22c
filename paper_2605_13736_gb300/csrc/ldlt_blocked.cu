// Blocked Bunch-Kaufman LDL^T with inertia (Section 2.3): the same pivot rule
// as the unblocked kernel in ldlt.cu (alpha = (1 + sqrt 17) / 8, LAPACK
// ?sytf2 comparisons, first-index ties), organised as panels of NB columns
// whose updates of the trailing matrix are delayed and applied once per panel.
//
// Panel (one thread-block cluster, the column pivot chain):
//   the panel's NB + 1 columns (rows k..N-1) are distributed by contiguous row
//   ranges over the cluster's CTAs and live in shared memory together with W,
//   the panel's updated columns.  For each column j the cluster
//     - updates it with the panel's earlier columns, W(:, j) = A(:, j) - L W(j, :)^T,
//     - finds the column maximum (integer compares of |.| bit patterns, a
//       cluster barrier, every CTA combining all CTAs' candidates through
//       distributed shared memory, so all take the same decision),
//     - if the rule needs it, updates column r = argmax the same way and takes
//       its maximum,
//     - interchanges rows/columns kk <-> kp (copying the raw column kk into
//       position kp: column kk becomes L anyway; swapping rows kk, kp of the
//       panel's L and W columns, of the earlier L columns, and of perm),
//     - forms the L column(s) from W and D (1x1 or 2x2).
//   Pivot values, the pivot test, D and the inertia count stay in FP64.
// Trailing update (all SMs): A22 -= L21 W21^T on the lower triangle, W = L D;
//   FP64 for the FP64 path, FP32 products subtracted from the FP64 matrix for
//   the refined mixed-precision path (the update has K = NB, so it is bound by
//   the L2 traffic of A22, not by arithmetic).  On that path the panel's own
//   column updates also take FP32 products (from FP32 shadows of L and of the
//   broadcast W row): at 1/64 of the FP32 rate, FP64 products were the largest
//   part of each column's time.
// Mixed-precision path: each panel is first factored without interchanges and
// kept when the pivot rule's tests confirm every pivot (k_bk_spec,
// k_bk_spec_rows, below); k_bk_panel then returns at once.
// Panel state (next column, inertia counts) lives in device memory, so the
// host enqueues all panels without reading anything back; the panel loop's
// kernels use programmatic dependent launch.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace mdsip {

namespace {

constexpr int kPanelThreads = 512;
constexpr int kUpdThreads = 256;
constexpr int kUT = 64;   // trailing-update tile edge

// Programmatic dependent launch: the kernels of the panel loop are launched
// with programmatic stream serialization, so a kernel's launch overlaps the
// tail of the one before it.  Each waits for its predecessor's completion (and
// memory) before touching data, then lets its own successor launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

struct PanelState {
    int k;       // first column of the next panel
    int kb;      // columns factored by the last panel
    int npos, nneg, nzero;
    int spec;    // 1: the last panel was taken by the verified no-interchange path
    int nacc, nrej;   // panels that path accepted / handed to the pivoting panel
    unsigned done;    // k_bk_spec CTAs done with the current panel (reset by the last)
    int nfail;        // columns of the pending panel whose row test k_bk_spec_rows evaluates
    unsigned done2;   // k_bk_spec_rows CTAs done (reset by the last)
};

struct Cand {                  // one CTA's candidate of a cluster-wide arg-max
    unsigned long long bits;   // |v| bit pattern
    int idx;                   // global row (first index on ties)
    int pad;
    double val;                // diagonal value, when this CTA owns it
    unsigned long long abits;  // bit pattern of alpha |v| (rounded), for the pivot test
};

struct PanelArgs {
    int N, NB, C, R;           // order, panel width, cluster size, row capacity per CTA
    double *A;                 // lower triangle, column-major, ld N (updated in place)
    double *L, *Dd, *Doff;
    int32_t *perm, *kind;
    double *Wg;                // W of the last panel: N x (NB + 1), column-major, ld N
    float *Lf, *Wf;            // F32: FP32 L and W columns of the last panel (N x (NB + 1), ld N)
    PanelState *st;
    const double *maxabs;
    double zero_tol;
};

__device__ __forceinline__ unsigned long long absbits64(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

__device__ __forceinline__ void cand_combine(unsigned long long &b, int &i, unsigned long long b2, int i2) {
    if (b2 > b || (b2 == b && i2 < i)) {
        b = b2;
        i = i2;
    }
}

// warp arg-max (first index on ties), result in every lane: three warp
// reductions (maximum of the high words, maximum of the low words among the
// lanes holding that high word, minimum index among the lanes holding both)
__device__ __forceinline__ void warp_cand(unsigned long long &b, int &idx) {
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    const bool top = hi == mhi && lo == mlo;
    idx = __reduce_min_sync(0xffffffffu, top ? idx : 0x7fffffff);
    b = ((unsigned long long)mhi << 32) | mlo;
}

// block arg-max into *out (bits, idx, and alpha |max| as abits); val = *diag
// (a shared-memory value written before the call, read after the barrier; 0
// if diag is null).  One __syncthreads; *out is complete when warp 0 returns.
// Since rounding is monotone, the cluster-wide maximum of the CTAs' abits is
// the bit pattern of fl(alpha colmax): the common pivot test then needs no
// FP64 instruction on the column's critical path.
__device__ void block_cand_to(unsigned long long b, int idx, const double *diag, unsigned long long *sb,
                              int *si, Cand *out, double alpha) {
    warp_cand(b, idx);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sb[wid] = b;
        si[wid] = idx;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (int)(blockDim.x >> 5);
        b = lane < nw ? sb[lane] : 0ULL;
        idx = lane < nw ? si[lane] : 0x7fffffff;
        warp_cand(b, idx);
        if (lane == 0) {
            out->bits = b;
            out->idx = idx;
            out->val = diag ? *diag : 0.0;
            out->abits = absbits64(alpha * __longlong_as_double((long long)b));
        }
    }
}

// 1/d by Newton-Raphson iteration x <- x (2 - d x) (two steps, as fused
// multiply-adds) from the single-precision reciprocal of d: each step squares
// the relative error, 2^-23 -> 2^-46 -> below the double rounding.  Takes six
// FP64 instructions; d outside the normal float range goes through the
// division operator.
__device__ __forceinline__ double rcp_newton(double d) {
    if (d == 0.0) return 0.0;
    const float df = (float)d;
    if (!(fabsf(df) >= 1.17549435e-38f && fabsf(df) <= 3.0e38f)) return 1.0 / d;
    double x = (double)__frcp_rn(df);
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}

// Cluster-wide arg-max of the candidates cand[slot] of all C CTAs (C <= 32),
// computed by warp 0: lane c reads CTA c's candidate, a shuffle reduction
// combines them (first index on ties); lane 0 returns true with the result
// and the diagonal value held by CTA `vrank`.
__device__ bool cluster_cand(cg::cluster_group &cl, Cand *cand, int slot, int C, int vrank, Cand &res) {
    if (threadIdx.x >= 32) return false;
    const int c = threadIdx.x;
    unsigned long long b = 0, ab = 0;
    int idx = 0x7fffffff;
    double v = 0.0;
    if (c < C) {
        const Cand *o = cl.map_shared_rank(cand, c) + slot;
        b = o->bits;
        idx = o->idx;
        v = o->val;
        ab = o->abits;
    }
    const double vsel = __shfl_sync(0xffffffffu, v, vrank);
    warp_cand(b, idx);
    const unsigned ahi = __reduce_max_sync(0xffffffffu, (unsigned)(ab >> 32));
    const unsigned alo = __reduce_max_sync(0xffffffffu, (unsigned)(ab >> 32) == ahi ? (unsigned)ab : 0u);
    res.bits = b;
    res.idx = idx;
    res.val = vsel;
    res.abits = ((unsigned long long)ahi << 32) | alo;
    return c == 0;
}

// F32: the panel's column updates (the products with earlier L columns) in
// FP32 from single-precision shadows of L and of the broadcast W row (the
// refined mixed-precision path); pivot tests, D and inertia stay FP64.
template <bool F32>
__global__ void __launch_bounds__(kPanelThreads, 1) k_bk_panel(PanelArgs a) {
    pdl_wait();
    pdl_release();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = a.C, N = a.N, NB = a.NB, S = NB + 1;
    const int tid = threadIdx.x;
    extern __shared__ double smem[];
    double *Ap = smem;                       // R x S: raw A columns, then L columns
    double *Wp = Ap + (size_t)a.R * S;       // R x S: updated columns
    double *wrow = Wp + (size_t)a.R * S;     // S: row j (or r) of W
    // candidates [parity of the column step][column / row maximum]: double
    // buffered, so a CTA that starts the next column before a slower one has
    // read this column's candidates writes the other pair
    Cand *cand = reinterpret_cast<Cand *>(wrow + S);
    float *Apf = reinterpret_cast<float *>(cand + 4);   // F32 only: R x S shadow of the L columns
    float *wrowf = Apf + (size_t)a.R * S;                // F32 only: S
    __shared__ unsigned long long s_b[32];
    __shared__ Cand s_cand;
    __shared__ double s_rcp;
    __shared__ int s_i[32];
    __shared__ double s_d[6];
    __shared__ double s_sc[2];
    __shared__ int s_dec[3];

    if (a.st->spec) return;                  // the panel was taken without interchanges
    const int k = a.st->k;
    if (k >= N) return;                      // uniform over the cluster
    const int rows = N - k;
    const int R = (rows + C - 1) / C;
    const int r0 = min(N, k + rank * R), r1 = min(N, r0 + R);
    const int ncols = min(S, N - k);
    const double alpha = 0.6403882032022076;   // (1 + sqrt 17) / 8
    const double ztol = a.zero_tol * __ldg(a.maxabs);
    auto owner = [&](int i) { return (i - k) / R; };
    auto rAp = [&](int i) -> double * { return cl.map_shared_rank(Ap, owner(i)) + (size_t)(i - (k + owner(i) * R)) * S; };
    auto rWp = [&](int i) -> double * { return cl.map_shared_rank(Wp, owner(i)) + (size_t)(i - (k + owner(i) * R)) * S; };

    // load the panel's columns (lower part) for the owned rows
    const int nrows = max(0, r1 - r0);
    for (int e = tid; e < nrows * ncols; e += kPanelThreads) {   // rows fastest: coalesced columns
        const int t = e / nrows, lr = e % nrows, i = r0 + lr;
        Ap[(size_t)lr * S + t] = i >= k + t ? a.A[i + (int64_t)(k + t) * N] : 0.0;
    }
    int npos = 0, nneg = 0, nzero = 0;
    cl.sync();

    // tpr threads per row for the row-times-W-row products (a power of two,
    // as many as fit one pass over the owned rows)
    int tpr = 1;
    while (tpr < 32 && 2 * tpr * R <= kPanelThreads) tpr *= 2;
    const int q4 = tid & (tpr - 1), rsub = tid / tpr, rpp = kPanelThreads / tpr;
    int jj = 0, it = 0;
    while (jj < NB && k + jj < N) {
        const int j = k + jj;
        Cand *cpair = cand + 2 * (it & 1);
        // ---- W(:, jj) = A(:, j) - L(:, 0:jj) W(j, 0:jj)^T over the owned rows >= j
        if (tid < jj) {
            const double v = rWp(j)[tid];
            if constexpr (F32) wrowf[tid] = (float)v;
            else wrow[tid] = v;
        }
        __syncthreads();
        unsigned long long b = 0;
        int bi = 0x7fffffff;
        for (int lr0 = 0; lr0 < r1 - r0; lr0 += rpp) {
            const int lr = lr0 + rsub, i = r0 + lr;
            double s;
            if constexpr (F32) {
                float sf = 0.0f;
                if (lr < r1 - r0 && i >= j)
                    for (int t = q4; t < jj; t += tpr) sf = fmaf(Apf[(size_t)lr * S + t], wrowf[t], sf);
                for (int o = 1; o < tpr; o <<= 1) sf += __shfl_xor_sync(0xffffffffu, sf, o);
                s = (double)sf;
            } else {
                s = 0.0;
                if (lr < r1 - r0 && i >= j)
                    for (int t = q4; t < jj; t += tpr) s = fma(Ap[(size_t)lr * S + t], wrow[t], s);
                for (int o = 1; o < tpr; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            }
            if (lr < r1 - r0 && i >= j && q4 == 0) {
                const double v = Ap[(size_t)lr * S + jj] - s;
                Wp[(size_t)lr * S + jj] = v;
                if (i > j) cand_combine(b, bi, absbits64(v), i);
            }
        }
        block_cand_to(b, bi, (j >= r0 && j < r1) ? Wp + (size_t)(j - r0) * S + jj : nullptr, s_b, s_i, &cpair[0], alpha);
        cl.sync();   // #1
        {
            Cand res;
            if (cluster_cand(cl, cpair, 0, C, owner(j), res)) s_cand = res;
        }
        __syncthreads();
        // scalar FP64 work by single threads of two warps in parallel (GB300
        // issues FP64 at 1/64 rate: 512 threads repeating it would cost
        // microseconds): the pivot test in warp 0, the reciprocal of the
        // diagonal (used when the test keeps it) in warp 1
        if (tid == 0) {
            // |a_kk| >= alpha colmax, or both zero, as integer compares of the
            // non-negative FP64 bit patterns
            const unsigned long long akb = absbits64(s_cand.val);
            s_dec[0] = s_cand.idx == 0x7fffffff ? j : s_cand.idx;
            const bool plain = (akb == 0ULL && s_cand.bits == 0ULL) || akb >= s_cand.abits;
            s_dec[1] = plain ? 0 : 1;
            s_sc[0] = __longlong_as_double((long long)akb);
            s_sc[1] = __longlong_as_double((long long)s_cand.bits);
        } else if (tid == 32) {
            s_rcp = rcp_newton(s_cand.val);
        }
        __syncthreads();
        const int imax = s_dec[0];
        int kstep = 1, kp = j;
        bool copy_r = false;
        if (s_dec[1]) {
            const int r = imax;
            // ---- V = column r updated: V(i) = A_sym(i, r) - L(i, 0:jj) W(r, 0:jj)^T into W(:, jj+1)
            if (tid < jj) {
                const double v = rWp(r)[tid];
                if constexpr (F32) wrowf[tid] = (float)v;
                else wrow[tid] = v;
            }
            __syncthreads();
            unsigned long long b2 = 0;
            int bi2 = 0x7fffffff;
            const bool r_in_panel = r - k < S;
            for (int lr0 = 0; lr0 < r1 - r0; lr0 += rpp) {
                const int lr = lr0 + rsub, i = r0 + lr;
                const bool act = lr < r1 - r0 && i >= j;
                double s;
                if constexpr (F32) {
                    float sf = 0.0f;
                    if (act)
                        for (int t = q4; t < jj; t += tpr) sf = fmaf(Apf[(size_t)lr * S + t], wrowf[t], sf);
                    for (int o = 1; o < tpr; o <<= 1) sf += __shfl_xor_sync(0xffffffffu, sf, o);
                    s = (double)sf;
                } else {
                    s = 0.0;
                    if (act)
                        for (int t = q4; t < jj; t += tpr) s = fma(Ap[(size_t)lr * S + t], wrow[t], s);
                    for (int o = 1; o < tpr; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                }
                if (act && q4 == 0) {
                    double air;
                    if (i < r)
                        air = (i - k < S) ? rAp(r)[i - k] : a.A[r + (int64_t)i * N];
                    else
                        air = r_in_panel ? Ap[(size_t)lr * S + (r - k)] : a.A[i + (int64_t)r * N];
                    const double v = air - s;
                    Wp[(size_t)lr * S + jj + 1] = v;
                    if (i != r) cand_combine(b2, bi2, absbits64(v), i);
                }
            }
            block_cand_to(b2, bi2, (r >= r0 && r < r1) ? Wp + (size_t)(r - r0) * S + jj + 1 : nullptr, s_b, s_i,
                          &cpair[1], alpha);
            cl.sync();   // #2
            {
                Cand res;
                if (cluster_cand(cl, cpair, 1, C, owner(r), res)) {
                    const double absakk = s_sc[0], colmax = s_sc[1];
                    const double rowmax = __longlong_as_double((long long)res.bits);
                    if (absakk >= alpha * colmax * (colmax / rowmax)) s_dec[2] = 0;   // 1x1, no interchange
                    else if (fabs(res.val) >= alpha * rowmax) s_dec[2] = 1;         // 1x1 on V, interchange
                    else s_dec[2] = 2;                                              // 2x2, interchange
                }
            }
            __syncthreads();
            if (s_dec[2] == 1) {
                kp = r;
                copy_r = true;   // the pivot column is V
            } else if (s_dec[2] == 2) {
                kp = r;
                kstep = 2;
            }
        }
        const int kk = j + kstep - 1;
        if (copy_r) {
            for (int lr = tid; lr < r1 - r0; lr += kPanelThreads)
                if (r0 + lr >= j) Wp[(size_t)lr * S + jj] = Wp[(size_t)lr * S + jj + 1];
        }
        if (kp != kk) {
            cl.sync();   // every CTA is done with this column's reads of rows kk and kp
            const bool kp_in_panel = kp - k < S;
            // raw column kk moves to position kp (kk's own column becomes L)
            if (kk >= r0 && kk < r1 && tid == 0) {
                const double v = Ap[(size_t)(kk - r0) * S + (kk - k)];
                if (kp_in_panel) rAp(kp)[kp - k] = v;
                else a.A[kp + (int64_t)kp * N] = v;
            }
            for (int lr = tid; lr < r1 - r0; lr += kPanelThreads) {
                const int i = r0 + lr;
                if (i > kk && i < kp) {          // A(kp, i) = A(i, kk)
                    const double v = Ap[(size_t)lr * S + (kk - k)];
                    if (i - k < S) rAp(kp)[i - k] = v;
                    else a.A[kp + (int64_t)i * N] = v;
                } else if (i > kp) {             // A(i, kp) = A(i, kk)
                    const double v = Ap[(size_t)lr * S + (kk - k)];
                    if (kp_in_panel) Ap[(size_t)lr * S + (kp - k)] = v;
                    else a.A[i + (int64_t)kp * N] = v;
                }
            }
            // rows kk <-> kp of the panel's L columns (t < jj) and W columns (t <= kk - k)
            if (kk >= r0 && kk < r1) {
                double *ak = Ap + (size_t)(kk - r0) * S, *wk = Wp + (size_t)(kk - r0) * S;
                double *ap = rAp(kp), *wp = rWp(kp);
                for (int t = tid; t < jj; t += kPanelThreads) {
                    const double x = ak[t];
                    ak[t] = ap[t];
                    ap[t] = x;
                }
                if constexpr (F32) {
                    float *fk = Apf + (size_t)(kk - r0) * S;
                    float *fp = cl.map_shared_rank(Apf, owner(kp)) + (size_t)(kp - (k + owner(kp) * R)) * S;
                    for (int t = tid; t < jj; t += kPanelThreads) {
                        const float x = fk[t];
                        fk[t] = fp[t];
                        fp[t] = x;
                    }
                }
                for (int t = tid; t <= kk - k; t += kPanelThreads) {
                    const double x = wk[t];
                    wk[t] = wp[t];
                    wp[t] = x;
                }
            }
            // rows kk <-> kp of the earlier panels' L columns
            for (int t = rank * kPanelThreads + tid; t < k; t += C * kPanelThreads) {
                double *Lt = a.L + (int64_t)t * N;
                const double x = Lt[kk];
                Lt[kk] = Lt[kp];
                Lt[kp] = x;
            }
            if (rank == 0 && tid == 0) {
                const int x = a.perm[kk];
                a.perm[kk] = a.perm[kp];
                a.perm[kp] = x;
            }
            cl.sync();
        }
        // ---- D block and L column(s)
        const bool d_ready = s_dec[1] == 0;   // plain 1x1: d = the diagonal, 1/d = s_rcp
        if (tid == 0 && !d_ready) {
            const double d11 = rWp(j)[jj];
            const double d21 = kstep == 2 ? rWp(j + 1)[jj] : 0.0;
            const double d22 = kstep == 2 ? rWp(j + 1)[jj + 1] : 0.0;
            s_d[0] = d11;
            s_d[1] = d21;
            s_d[2] = d22;
            if (kstep == 1) {
                s_d[3] = rcp_newton(d11);
                s_d[4] = s_d[5] = 0.0;
            } else {
                const double inv = rcp_newton(d11 * d22 - d21 * d21);
                s_d[3] = d22 * inv;
                s_d[4] = -d21 * inv;
                s_d[5] = d11 * inv;
            }
        }
        if (!d_ready) __syncthreads();
        const double d11 = d_ready ? s_cand.val : s_d[0];
        const double d21 = d_ready ? 0.0 : s_d[1], d22 = d_ready ? 0.0 : s_d[2];
        const double e11 = d_ready ? s_rcp : s_d[3], e21 = d_ready ? 0.0 : s_d[4], e22 = d_ready ? 0.0 : s_d[5];
        for (int lr = tid; lr < r1 - r0; lr += kPanelThreads) {
            const int i = r0 + lr;
            double *arow = Ap + (size_t)lr * S;
            const double *wr = Wp + (size_t)lr * S;
            float *frow = Apf + (size_t)lr * S;
            if (kstep == 1) {
                if (i > j) {
                    arow[jj] = wr[jj] * e11;
                    if constexpr (F32) frow[jj] = (float)arow[jj];
                }
            } else {
                if (i >= j + 2) {
                    const double x = wr[jj], y = wr[jj + 1];
                    arow[jj] = x * e11 + y * e21;
                    arow[jj + 1] = x * e21 + y * e22;
                    if constexpr (F32) {
                        frow[jj] = (float)arow[jj];
                        frow[jj + 1] = (float)arow[jj + 1];
                    }
                } else if (i == j + 1) {
                    arow[jj] = 0.0;
                    if constexpr (F32) frow[jj] = 0.0f;
                }
            }
        }
        if (rank == 0 && tid == kPanelThreads - 32) {   // a warp without L rows at these sizes
            if (kstep == 1) {
                a.Dd[j] = d11;
                a.Doff[j] = 0.0;
                a.kind[j] = 1;
                if (d11 == 0.0 || fabs(d11) <= ztol) ++nzero;
                else if (d11 > 0.0) ++npos;
                else ++nneg;
            } else {
                a.Dd[j] = d11;
                a.Doff[j] = d21;
                a.Dd[j + 1] = d22;
                a.Doff[j + 1] = 0.0;
                a.kind[j] = 2;
                a.kind[j + 1] = 0;
                ++npos;
                ++nneg;
            }
        }
        jj += kstep;
        ++it;
        // No cluster barrier here: the next column reads only W rows finished
        // before this column's last barrier, writes W columns no CTA still
        // reads, and its candidates go to the other buffer pair.
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
    const int kb = jj;
    // ---- write back: L columns (strict lower, unit diagonal), W rows below the
    // panel for the trailing update, and the panel's raw columns not factored
    for (int e = tid; e < nrows * ncols; e += kPanelThreads) {
        const int t = e / nrows, lr = e % nrows, i = r0 + lr;
        const double v = Ap[(size_t)lr * S + t];
        if (t < kb) {
            if (i > k + t) a.L[i + (int64_t)(k + t) * N] = v;
            else if (i == k + t) a.L[i + (int64_t)i * N] = 1.0;
            if constexpr (F32) {   // the FP32 trailing update reads FP32 copies
                if (i > k + t) a.Lf[i + (int64_t)t * N] = Apf[(size_t)lr * S + t];
                if (i >= k + kb) a.Wf[i + (int64_t)t * N] = (float)Wp[(size_t)lr * S + t];
            } else {
                if (i >= k + kb) a.Wg[i + (int64_t)t * N] = Wp[(size_t)lr * S + t];
            }
        } else if (i >= k + t) {
            a.A[i + (int64_t)(k + t) * N] = v;
        }
    }
    if (rank == 0 && tid == kPanelThreads - 32) {   // the thread that counted the inertia
        a.st->k = k + kb;
        a.st->kb = kb;
        a.st->npos += npos;
        a.st->nneg += nneg;
        a.st->nzero += nzero;
    }
}

// A(i, c) -= sum_{t < kb} L(i, k + t) W(c, t)  for k + kb <= c <= i < N.
// Block = one 64 x 64 tile of the trailing lower triangle (tiles beyond the
// actual trailing size return).  256 threads, 4 x 4 outputs each.
// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}
__device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
    const double2 x = reinterpret_cast<const double2 *>(p)[0], y = reinterpret_cast<const double2 *>(p)[1];
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
}

// One 64 x 64 tile (number `tile` in row-major order over the lower
// triangle of tiles) of the trailing update after a panel of kb columns
// starting at k0: A(i, c) -= sum_t L(i, k0 + t) W(c, t) for i >= c >= base =
// k0 + kb.  kUpdThreads threads; smem holds 2 S 64 values of T, S >= kb the
// pitch the launch sized it for (panel width + 1: a pivoting panel may end
// with a 2x2 pivot and take one column more).
template <typename T>
__device__ void trailing_tile(int tile, int N, int kb, int k0, int S, double *__restrict__ A,
                              const double *__restrict__ L, const double *__restrict__ Wg,
                              const float *__restrict__ Lf, const float *__restrict__ Wf, unsigned char *usmem) {
    T *Lt = reinterpret_cast<T *>(usmem);          // [S][64]: Lt[t][r]
    T *Wt = Lt + (size_t)S * kUT;                   // [S][64]: Wt[t][c]
    const int base = k0 + kb;
    if (base >= N || kb <= 0) return;
    int tr = (int)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
    while ((tr + 1) * (tr + 2) / 2 <= tile) ++tr;
    while (tr * (tr + 1) / 2 > tile) --tr;
    const int tc = tile - tr * (tr + 1) / 2;
    const int i0 = base + tr * kUT, c0 = base + tc * kUT;
    if (i0 >= N) return;
    const int tid = threadIdx.x;
    {   // stage the panel's L rows and W rows of this tile: all loads in flight
        // before the first shared-memory store (thread: row r, columns t0 + 4 j)
        constexpr int kJ = (65 + 3) / 4;   // panel width <= 65
        const int r = tid & (kUT - 1), t0 = tid >> 6;
        const int i = i0 + r, c = c0 + r;
        T lv[kJ], wv[kJ];
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int t = t0 + 4 * j;
            lv[j] = wv[j] = (T)0;
            if (t < kb) {
                if constexpr (sizeof(T) == sizeof(float)) {   // the panel's FP32 copies
                    if (i < N) lv[j] = Lf[i + (int64_t)t * N];
                    if (c < N) wv[j] = Wf[c + (int64_t)t * N];
                } else {
                    if (i < N) lv[j] = (T)L[i + (int64_t)(k0 + t) * N];
                    if (c < N) wv[j] = (T)Wg[c + (int64_t)t * N];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int t = t0 + 4 * j;
            if (t < kb) {
                Lt[t * kUT + r] = lv[j];
                Wt[t * kUT + r] = wv[j];
            }
        }
    }
    __syncthreads();
    // rows 4 tx .. 4 tx + 3, columns 4 ty .. 4 ty + 3: each step reads its
    // four L and four W values as 16-byte shared-memory loads
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
    for (int t = 0; t < kb; ++t) {
        T lv[4], wv[4];
        load4(Lt + t * kUT + 4 * tx, lv);
        load4(Wt + t * kUT + 4 * ty, wv);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(lv[u], wv[v], acc[u][v]);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int c = c0 + 4 * ty + v;
        if (c >= N) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + 4 * tx + u;
            if (i < N && i >= c) A[i + (int64_t)c * N] -= (double)acc[u][v];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kUpdThreads) k_bk_trailing(int N, int NB, double *__restrict__ A,
                                                             const double *__restrict__ L,
                                                             const double *__restrict__ Wg,
                                                             const float *__restrict__ Lf,
                                                             const float *__restrict__ Wf,
                                                             const PanelState *__restrict__ st) {
    pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) unsigned char usmem[];
    const int kb = st->kb;
    trailing_tile<T>((int)blockIdx.x, N, kb, st->k - kb, NB + 1, A, L, Wg, Lf, Wf, usmem);
}

// ---------------------------------------------------------------------------
// Verified no-interchange panel (refined mixed-precision path).
//
// On the Newton-step matrices of a convex problem the Bunch-Kaufman rule
// almost always keeps the diagonal: the rule's choice at column j is a 1x1
// pivot without interchange exactly when
//     max(|a_jj|, colmax_j) = 0,  or  |a_jj| >= alpha colmax_j,  or
//     |a_jj| >= alpha colmax_j (colmax_j / rowmax_r),
// where colmax_j, r are the maximum and its row below the diagonal of the
// column after j eliminations and rowmax_r the maximum off-diagonal entry of
// row r of that active matrix.  If those decisions hold for every column of
// a panel, the panel's Bunch-Kaufman factor is the factor without pivoting,
// and that factor needs no cluster-wide arg-max per column: k_bk_spec
// factors the panel without interchanges (all CTAs, each for a slice of the
// rows, repeating the short pivot chain of the diagonal block), then its last
// CTA applies the column test to every column (the column maxima gathered by
// atomicMax; the arg-max row is the first among the entries whose |w| agree
// to 28 mantissa bits).  Columns that fail it go to k_bk_spec_rows, which recomputes
// row r of the active matrix from the stored matrix and the panel's earlier
// columns on all SMs and applies the row test.  A panel that passes is kept;
// otherwise k_bk_panel factors it with interchanges from the unchanged
// matrix.  Decisions, D and the inertia stay FP64; the chain and the products
// are FP32 as in the FP32-update panel.  A pivot with |d| <= zero_tol maxabs
// also hands the panel over, so zero pivots keep the pivoting panel's rules.
constexpr int kSpecThreads = 256;   // k_bk_spec_rows
constexpr int kSpecChainThreads = 512;                 // k_bk_spec
constexpr int kSpecTC = kSpecChainThreads / 16;         // column groups of the register tile
constexpr int kSpecY = 64 / kSpecTC;                    // columns per thread
constexpr int kSpecRB = 32;   // rows below the diagonal block per CTA
constexpr int kSpecP = 65;    // shared-memory row pitch (floats)

struct RowTest {               // a column that needs the rule's row test
    int jj, r;                 // column (in the panel) and the row of its column maximum
    double colmax, absakk;
};

struct SpecArgs {
    int N, NB;
    const double *A;          // lower triangle, column-major, ld N (not written)
    double *L, *Dd, *Doff;
    int32_t *kind;
    float *Lf, *Wf;           // FP32 L and W columns of the panel, ld N
    unsigned long long *cmax; // [2][64]: per column the maximum |w| (bits) and the arg-max key
    RowTest *fail;            // [NB]: the columns whose row test is pending
    unsigned long long *rowpart;   // [CTAs of k_bk_spec_rows][NB]: partial row maxima (bit patterns)
    PanelState *st;
    const double *maxabs;
    double zero_tol;
};

size_t spec_smem(int NB) {
    return 2 * (size_t)NB * sizeof(double) + (size_t)(NB + kSpecRB) * kSpecP * sizeof(double) +
           (size_t)3 * (NB + kSpecRB) * kSpecP * sizeof(float);
}

// Keep the panel (all threads of the block): 1x1 pivots without interchange,
// inertia from the signs of D, the next panel starts after it.
__device__ void spec_accept(const SpecArgs &a, int k, int nb) {
    int pos = 0;
    if ((int)threadIdx.x < nb) {
        a.kind[k + threadIdx.x] = 1;
        a.Doff[k + threadIdx.x] = 0.0;
        pos = __ldcg(&a.Dd[k + threadIdx.x]) > 0.0 ? 1 : 0;
    }
    const int np = __syncthreads_count(pos);
    if (threadIdx.x == 0) {
        a.st->npos += np;
        a.st->nneg += nb - np;
        a.st->k = k + nb;
        a.st->kb = nb;
        a.st->spec = 1;
        a.st->nacc += 1;
    }
}

__global__ void __launch_bounds__(kSpecChainThreads, 1) k_bk_spec(SpecArgs a) {
    pdl_wait();
    pdl_release();
    extern __shared__ double spsm[];
    const int N = a.N, NB = a.NB, G = (int)gridDim.x, g = (int)blockIdx.x;
    const int tid = threadIdx.x;
    constexpr int P = kSpecP;
    double *dd = spsm;                                      // NB: FP64 pivots
    double *rr = dd + NB;                                   // NB: their reciprocals
    double *Ad = rr + NB;                                   // rows x P: the raw values (FP64)
    float *Wsh = reinterpret_cast<float *>(Ad + (size_t)(NB + kSpecRB) * P);   // rows x P: W columns (FP32)
    float *U = Wsh + (size_t)(NB + kSpecRB) * P;            // rows x P: sums of the panel's products
    float *Ls = U + (size_t)(NB + kSpecRB) * P;             // rows x P: FP32 L columns
    __shared__ float s_rf[64];                              // FP32 reciprocals of the chain's pivots
    __shared__ int s_last;
    const int k = a.st->k;
    const int nb = min(NB, N - k);
    const int rb0 = k + nb + g * kSpecRB;
    const int nown = k < N ? max(0, min(N, rb0 + kSpecRB) - rb0) : 0;
    const int nloc = nb + nown;
    if (k < N && (g == 0 || nown > 0)) {        // CTAs beyond the last row have no work
        // Local rows 0..nb-1: the diagonal block; nb..nloc-1: this CTA's rows
        // below it.  Thread (tr, tc) keeps the entries (tr + 16 x, tc + kSpecTC y),
        // x < 6, y < kSpecY, in registers: their raw value and the running sum of
        // the panel's products (right-looking, one barrier per column).
        const int tr = tid & 15, tc = tid >> 4;
        float ar[6][kSpecY], u[6][kSpecY];
#pragma unroll
        for (int x = 0; x < 6; ++x) {
            const int i = tr + 16 * x;
            const int gi = i < nb ? k + i : rb0 + (i - nb);
#pragma unroll
            for (int y = 0; y < kSpecY; ++y) {
                const int c = tc + kSpecTC * y;
                const bool valid = i < nloc && c < nb && (i >= nb || c <= i);
                const double v = valid ? a.A[gi + (int64_t)(k + c) * N] : 0.0;
                ar[x][y] = (float)v;
                u[x][y] = 0.0f;
                if (valid) {
                    Ad[i * P + c] = v;
                    if (c == 0) Wsh[i * P] = (float)v;   // column 0's working values
                    if (i == 0 && c == 0) s_rf[0] = __frcp_rn((float)v);
                }
            }
        }
        __syncthreads();
        for (int jj = 0; jj < nb; ++jj) {
            const float rf = s_rf[jj];
            float lf[6], wc[kSpecY];
#pragma unroll
            for (int x = 0; x < 6; ++x) {
                const int i = tr + 16 * x;
                lf[x] = (i > jj && i < nloc) ? Wsh[i * P + jj] * rf : 0.0f;
            }
#pragma unroll
            for (int y = 0; y < kSpecY; ++y) {
                const int c = tc + kSpecTC * y;
                wc[y] = (c > jj && c < nb) ? Wsh[c * P + jj] : 0.0f;
            }
            if (tc == 0) {
#pragma unroll
                for (int x = 0; x < 6; ++x) {
                    const int i = tr + 16 * x;
                    if (i > jj && i < nloc) Ls[i * P + jj] = lf[x];
                }
            }
#pragma unroll
            for (int x = 0; x < 6; ++x)
#pragma unroll
                for (int y = 0; y < kSpecY; ++y) u[x][y] = fmaf(lf[x], wc[y], u[x][y]);
            // the owners of column jj + 1 publish its working values
#pragma unroll
            for (int y = 0; y < kSpecY; ++y) {
                if (tc + kSpecTC * y == jj + 1) {
#pragma unroll
                    for (int x = 0; x < 6; ++x) {
                        const int i = tr + 16 * x;
                        if (i > jj && i < nloc) {
                            const float v = ar[x][y] - u[x][y];
                            Wsh[i * P + jj + 1] = v;
                            if (i == jj + 1) s_rf[jj + 1] = __frcp_rn(v);   // the next pivot's reciprocal
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int x = 0; x < 6; ++x)
#pragma unroll
            for (int y = 0; y < kSpecY; ++y) {
                const int i = tr + 16 * x, c = tc + kSpecTC * y;
                if (i < nloc && c < nb && (i >= nb || c <= i)) U[i * P + c] = u[x][y];
            }
        __syncthreads();
        // ---- FP64: pivots, reciprocals, W and L; column candidates
        if (tid < nb) {
            const double d = Ad[tid * P + tid] - (double)U[tid * P + tid];
            dd[tid] = d;
            rr[tid] = rcp_newton(d);
        }
        __syncthreads();
        const int lane = tid & 31, wid = tid >> 5;
        const int below = max(0, N - k - nb);
        const int Gw = max(1, (below + kSpecRB - 1) / kSpecRB);   // CTAs with rows (CTA 0 always)
        // the column maxima of this CTA's rows, and of the diagonal block's
        // rows for the columns jj = g, g + Gw, ..., go to the per-column
        // maxima by atomicMax: the exact |w| bits, and a key whose high bits
        // are |w| truncated to 28 mantissa bits and whose low 24 bits are the
        // complemented row (the arg-max, first row among maxima equal to 2^-28)
        auto put_max = [&](int jj, unsigned long long b, int bi) {
            if (b == 0ULL) return;
            atomicMax(&a.cmax[jj], b);
            atomicMax(&a.cmax[64 + jj], ((b >> 24) << 24) | (unsigned long long)(0xFFFFFFu - (unsigned)bi));
        };
        for (int jj = wid; jj < nb; jj += kSpecChainThreads / 32) {
            unsigned long long b = 0;
            int bi = 0x7fffffff;
            if (lane < nown) {
                const int li = nb + lane, i = rb0 + lane;
                const double w = Ad[li * P + jj] - (double)U[li * P + jj];
                a.L[i + (int64_t)(k + jj) * N] = w * rr[jj];
                a.Lf[i + (int64_t)jj * N] = Ls[li * P + jj];
                a.Wf[i + (int64_t)jj * N] = Wsh[li * P + jj];
                b = absbits64(w);
                bi = i;
            }
            warp_cand(b, bi);
            if (lane == 0) put_max(jj, b, bi);
        }
        for (int q = wid;; q += kSpecChainThreads / 32) {   // the diagonal block's columns
            const int jj = g + q * Gw;
            if (jj >= nb) break;
            unsigned long long b2 = 0;
            int bi2 = 0x7fffffff;
            for (int li = jj + lane; li < nb; li += 32) {
                const int i = k + li;
                if (li == jj) {
                    a.L[i + (int64_t)i * N] = 1.0;
                    a.Dd[i] = dd[jj];
                    a.Wf[i + (int64_t)jj * N] = Wsh[li * P + jj];
                    continue;
                }
                const double w = Ad[li * P + jj] - (double)U[li * P + jj];
                a.L[i + (int64_t)(k + jj) * N] = w * rr[jj];
                a.Lf[i + (int64_t)jj * N] = Ls[li * P + jj];
                a.Wf[i + (int64_t)jj * N] = Wsh[li * P + jj];
                cand_combine(b2, bi2, absbits64(w), i);
            }
            warp_cand(b2, bi2);
            if (lane == 0) put_max(jj, b2, bi2);
        }
    }
    // ---- arrival; the last CTA decides
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&a.st->done, 1u) == (unsigned)(G - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (k >= N) {
        if (tid == 0) a.st->done = 0u;
        return;
    }
    __shared__ int s_reject, s_nf, s_cnt0;
    const int lane = tid & 31;
    const double alpha = 0.6403882032022076;   // (1 + sqrt 17) / 8
    if (tid == 0) {
        s_reject = 0;
        s_nf = 0;
    }
    __syncthreads();
    const double ztol = a.zero_tol * __ldg(a.maxabs);
    bool fail = false;
    RowTest rt{};
    if (tid < 64) {
        const unsigned long long cb = __ldcg(&a.cmax[tid]), key = __ldcg(&a.cmax[64 + tid]);
        a.cmax[tid] = 0ULL;                  // cleared for the next panel
        a.cmax[64 + tid] = 0ULL;
        if (tid < nb) {
            const double d = __ldcg(&a.Dd[k + tid]);
            const unsigned long long akb = absbits64(d);
            const double colmax = __longlong_as_double((long long)cb);
            const bool plain = (akb == 0ULL && cb == 0ULL) || akb >= absbits64(alpha * colmax);
            // zero pivots, and values that are not finite, go to the pivoting panel
            if (d == 0.0 || fabs(d) <= ztol || !isfinite(d) || !isfinite(colmax)) atomicOr(&s_reject, 1);
            if (!plain) {
                const int r = (int)(0xFFFFFFu - (unsigned)(key & 0xFFFFFFULL));
                if (r <= k + tid || r >= N) atomicOr(&s_reject, 1);   // no valid row
                fail = true;
                rt = RowTest{tid, r, colmax, fabs(d)};
            }
        }
    }
    // columns that need the row test: listed (in column order) for k_bk_spec_rows
    const unsigned bal = __ballot_sync(0xffffffffu, fail);
    if (tid == 0) s_cnt0 = __popc(bal);
    __syncthreads();
    if (fail) {
        const int pos = __popc(bal & ((1u << lane) - 1u)) + (tid >= 32 ? s_cnt0 : 0);
        a.fail[pos] = rt;
        atomicAdd(&s_nf, 1);
    }
    __syncthreads();
    const int nf = s_nf;
    if (tid == 0) a.st->nfail = s_reject ? 0 : nf;
    if (s_reject) {
        if (tid == 0) {
            a.st->spec = 0;
            a.st->nrej += 1;
            a.st->nfail = 0;
        }
    } else if (nf == 0) {
        spec_accept(a, k, nb);
    } else if (tid == 0) {
        a.st->spec = 0;   // decided by k_bk_spec_rows
    }
    if (tid == 0) a.st->done = 0u;
}

// The row tests of the listed columns: rowmax_r = max over c >= j, c != r of
// |S(c, r) - sum_{t < jj} L(c, k + t) W(r, t)| (the active matrix's row r
// after j eliminations, FP32 products as in the panel), partial maxima per CTA
// over 32 rows c (one per lane; warp w takes the listed columns w, w + 8, ...),
// then the last CTA applies the rule and keeps or hands over the panel.
__global__ void __launch_bounds__(kSpecThreads) k_bk_spec_rows(SpecArgs a) {
    pdl_wait();
    pdl_release();
    __shared__ float s_w[64 * 64];
    __shared__ RowTest s_t[64];
    __shared__ int s_last, s_reject;
    const int nf = a.st->nfail;
    if (nf == 0) return;                       // uniform: nothing pending
    const int N = a.N, NB = a.NB, k = a.st->k, nb = min(NB, N - k);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = (int)gridDim.x, g = (int)blockIdx.x;
    for (int f = tid; f < nf; f += kSpecThreads) s_t[f] = a.fail[f];
    __syncthreads();
    for (int e = tid; e < nf * 64; e += kSpecThreads) {
        const int f = e >> 6, t = e & 63;
        s_w[e] = t < s_t[f].jj ? __ldcg(&a.Wf[s_t[f].r + (int64_t)t * N]) : 0.0f;
    }
    const int c = k + g * 32 + lane;
    float lf[64];
#pragma unroll
    for (int t = 0; t < 64; ++t) lf[t] = (c < N && t < nb) ? __ldcg(&a.Lf[c + (int64_t)t * N]) : 0.0f;
    __syncthreads();
    for (int f = wid; f < nf; f += kSpecThreads / 32) {
        const RowTest rt = s_t[f];
        const float *wr = s_w + f * 64;
        unsigned long long b = 0;
        if (c < N && c >= k + rt.jj && c != rt.r) {
            float sf = 0.0f;
#pragma unroll
            for (int t = 0; t < 64; ++t)
                if (t < rt.jj) sf = fmaf(lf[t], wr[t], sf);
            const double asym = c < rt.r ? a.A[rt.r + (int64_t)c * N] : a.A[c + (int64_t)rt.r * N];
            b = absbits64(asym - (double)sf);
        }
        const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(b >> 32));
        const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(b >> 32) == hi ? (unsigned)b : 0u);
        if (lane == 0) a.rowpart[(size_t)g * NB + f] = ((unsigned long long)hi << 32) | lo;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&a.st->done2, 1u) == (unsigned)(G - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid == 0) s_reject = 0;
    __syncthreads();
    const double alpha = 0.6403882032022076;   // (1 + sqrt 17) / 8
    for (int f = wid; f < nf; f += kSpecThreads / 32) {
        unsigned long long b = 0;
        for (int q = lane; q < G; q += 32) {
            const unsigned long long v = __ldcg(&a.rowpart[(size_t)q * NB + f]);
            b = v > b ? v : b;
        }
        const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(b >> 32));
        const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(b >> 32) == hi ? (unsigned)b : 0u);
        if (lane == 0) {
            const double rowmax = __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
            const RowTest rt = s_t[f];
            if (!(rt.absakk >= alpha * rt.colmax * (rt.colmax / rowmax))) atomicOr(&s_reject, 1);
        }
    }
    __syncthreads();
    if (!s_reject) {
        spec_accept(a, k, nb);
    } else if (tid == 0) {
        a.st->spec = 0;
        a.st->nrej += 1;
    }
    if (tid == 0) {
        a.st->nfail = 0;
        a.st->done2 = 0u;
    }
}

// ---------------------------------------------------------------------------
// Persistent speculative factorization (one cooperative launch for all panels),
// FP64 form (the FP32-update form is k_bk_persist32 below).
//
// The same no-interchange speculation as k_bk_spec, organised so that a kept
// panel costs no launch: one grid of co-resident CTAs walks the panels of 64
// columns, with a grid barrier after the panel (all column maxima known) and
// one after its trailing update.  Per panel:
//   A1 every CTA factors the 64 x 64 diagonal block in shared memory without
//      interchanges, in four sub-panels of 16 columns: warp 0 factors the
//      16 x 16 diagonal sub-block with register shuffles, one thread per row
//      solves the rows below it, and a rank-16 update brings the rest of the
//      block up to date (three block barriers per sub-panel instead of one
//      per column);
//   A2 each CTA takes a slice of the rows below the block, one thread per
//      row: 64-row chunks in shared memory, solved against the block's
//      factor in the same 16-column steps; the FP64 values w = A - sum L W,
//      L = w / d and the column maxima of |w| (exact FP64 bit patterns,
//      atomicMax) follow;
//   B  after the grid barrier every CTA applies the rule's column test to the
//      64 columns with the same data: the panel is kept when every column
//      keeps its diagonal pivot (|a_jj| >= alpha colmax_j, or a zero column)
//      and no pivot is within zero_tol max|S| of zero;
//   C  the trailing update of a kept panel, tiles of the lower triangle over
//      all CTAs; grid barrier.
// The first panel that fails the column test (the rule would look at a row
// or interchange) ends the kernel with st->k at its first column; the host
// then runs the pivoting panels from there.  All arithmetic is FP64.
// ---------------------------------------------------------------------------
constexpr int kPThreads = 256;
constexpr int kPP = 65;      // shared-memory row pitch of the diagonal block

struct PanelBar {
    unsigned count;   // grid-barrier arrivals of the current launch
    unsigned pad0;
    int err, pad;
};

struct PersistArgs {
    int N;
    double *A;                      // lower triangle, column-major, ld N (trailing part updated in place)
    double *L, *Dd, *Doff;
    int32_t *kind;
    double *Wg;                     // FP64 W of the current panel (T = double), ld N
    float *Lf, *Wf;                 // FP32 L and W of the current panel (T = float), ld N
    unsigned long long *cmax;       // [2][64]: per-column maxima of |w| (bit patterns), by panel parity
    PanelState *st;
    PanelBar *bar;
    const double *maxabs;
    double zero_tol;
    long long wait_ns;              // bound of each grid-barrier wait
    float *Af;                      // FP32 copy of the lower triangle, ld N (FP32-update kernel)
    float *Lf2, *Wf2;               // FP32-update kernel: the odd panels' L and W columns (ld N)
    unsigned *colcnt;               // FP32-update kernel: per 64-column block, trailing tiles updated
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident).  The
// arrival counter only grows within a launch (k_bk_init clears it): the
// barrier numbered `epoch` (counted by each CTA's thread 0) completes when
// the counter reaches epoch x gridDim.x, so arriving is one release-add with
// no reply to wait for and nobody resets anything.  Every wait is bounded: a
// CTA that waits longer than wait_ns sets the error word and returns false,
// and so does every CTA that sees the word set.
__device__ bool panel_barrier(PanelBar *b, unsigned &epoch, long long wait_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = ++epoch * gridDim.x;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&b->count) : "memory");
        const long long t0 = global_ns();
        for (unsigned it = 0;; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&b->count) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((it & 63) == 63) {
                if (*(volatile int *)&b->err) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > wait_ns) {
                    atomicExch(&b->err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile int *)&b->err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Wait (thread 0, then the whole CTA) until *cnt reaches target; bounded like
// panel_barrier and sharing its error word.
__device__ bool wait_count(const unsigned *cnt, unsigned target, PanelBar *b, long long wait_ns) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = global_ns();
        for (unsigned it = 0;; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
            if ((int)(v - target) >= 0) break;
            if ((it & 63) == 63) {
                if (*(volatile int *)&b->err) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > wait_ns) {
                    atomicExch(&b->err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T chain_rcp(T d) {
    if constexpr (sizeof(T) == sizeof(float)) return d != 0.0f ? __frcp_rn(d) : 0.0f;
    else return d != 0.0 ? 1.0 / d : 0.0;
}

// w in FP64 from a chain value v: for FP32 chains the part of A that the FP32
// copy dropped is added back (v started as float(A))
template <typename T>
__device__ __forceinline__ double chain_w64(T v, double a) {
    if constexpr (sizeof(T) == sizeof(float)) return (double)v + (a - (double)(float)a);
    else return v;
}

// The rule's column test for the panel at k (all threads of every CTA take
// the same decision from the FP64 pivots s_d and the maxima gathered in
// cmax[buf]); CTA 0 records a kept panel (kind, inertia, next column) and
// clears cmax[clear] for a later panel.  Returns whether the panel is kept.
__device__ bool persist_keep(const PersistArgs &a, int k, int nb, int buf, int clear, double ztol, const double *s_d) {
    const double alpha = 0.6403882032022076;   // (1 + sqrt 17) / 8
    const int tid = threadIdx.x;
    int keep = 1;
    if (tid < nb) {
        const double d = s_d[tid];
        const unsigned long long cb = __ldcg(&a.cmax[buf * 64 + tid]);
        const double colmax = __longlong_as_double((long long)cb);
        const bool diag_ok = absbits64(d) >= absbits64(alpha * colmax);
        if (!diag_ok || d == 0.0 || fabs(d) <= ztol || !isfinite(d) || !isfinite(colmax)) keep = 0;
    }
    keep = __syncthreads_and(keep);
    if (!keep) return false;
    if (blockIdx.x == 0) {
        int pos = 0;
        if (tid < nb) {
            a.kind[k + tid] = 1;
            a.Doff[k + tid] = 0.0;
            pos = s_d[tid] > 0.0 ? 1 : 0;
        }
        if (tid < 64) a.cmax[clear * 64 + tid] = 0ULL;   // a later panel's maxima start at zero
        const int np = __syncthreads_count(pos);
        if (tid == 0) {
            a.st->npos += np;
            a.st->nneg += nb - np;
            a.st->k = k + nb;
            a.st->kb = nb;
            a.st->nacc += 1;
        }
    }
    return true;
}

__global__ void __launch_bounds__(kPThreads, 1) k_bk_persist(PersistArgs a) {
    using T = double;
    extern __shared__ __align__(16) unsigned char psm[];
    T *V = reinterpret_cast<T *>(psm);      // [64][kPP]: the diagonal block; W values once factored
                                            // (then [64][kPP]: a chunk of the rows below it)
    __shared__ double s_d[64], s_rd[64];    // FP64 pivots and their reciprocals
    __shared__ T s_rc[64];                  // the chain's reciprocals
    __shared__ unsigned long long s_cmax[64];
    const int N = a.N, G = (int)gridDim.x, g = (int)blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31;
    const double ztol = a.zero_tol * __ldg(a.maxabs);
    unsigned epoch = 0;   // grid barriers passed (thread 0)
    int p = 0;
    for (int k = a.st->k; k < N; k += 64, ++p) {
        const int nb = min(64, N - k);
        const int buf = p & 1;
        // ---------------- A1: the diagonal block
        for (int e = tid; e < 64 * 64; e += kPThreads) {
            const int c = e >> 6, r = e & 63;
            T v = (T)0;
            if (r < nb && c <= r) v = (T)a.A[(int64_t)(k + r) + (int64_t)(k + c) * N];
            V[r * kPP + c] = v;
        }
        if (tid < 64) {
            s_cmax[tid] = 0ULL;
            s_rc[tid] = (T)0;      // columns beyond a narrow last panel stay zero
        }
        __syncthreads();
        for (int c0 = 0; c0 < nb; c0 += 16) {
            const int cw = min(16, nb - c0);
            if (tid < 32) {   // warp 0: the 16 x 16 sub-block, lane = row c0 + lane
                T v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = (lane < cw && j <= lane) ? V[(c0 + lane) * kPP + c0 + j] : (T)0;
                // (lanes that take no part get a zero multiplier: a conditional
                // update kept v in local memory; the entries above a lane's
                // diagonal that the zero-free form touches are never read)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const T dj = __shfl_sync(0xffffffffu, v[j], j);
                    const T rj = j < cw ? chain_rcp(dj) : (T)0;
                    const T l = (lane > j && lane < cw) ? v[j] * rj : (T)0;
#pragma unroll
                    for (int t = 0; t < 16; ++t)
                        if (t > j) v[t] = fma(-l, __shfl_sync(0xffffffffu, v[j], t), v[t]);
                    if (lane == j && j < cw) s_rc[c0 + j] = rj;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (lane < cw && j <= lane) V[(c0 + lane) * kPP + c0 + j] = v[j];
            }
            __syncthreads();
            // rows of the block below the sub-block
            for (int r = c0 + 16 + tid; r < nb; r += kPThreads) {
                T v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = j < cw ? V[r * kPP + c0 + j] : (T)0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const T l = j < cw ? v[j] * s_rc[c0 + j] : (T)0;
#pragma unroll
                    for (int t = j + 1; t < 16; ++t)
                        if (t < cw) v[t] = fma(-l, V[(c0 + t) * kPP + c0 + j], v[t]);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < cw) V[r * kPP + c0 + j] = v[j];
            }
            __syncthreads();
            // rank-16 update of the rest of the block (lower triangle)
            const int m0 = c0 + 16, mw = nb - m0;
            if (mw > 0) {
                const int npairs = mw * (mw + 1) / 2;
                for (int e = tid; e < npairs; e += kPThreads) {
                    int rr = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                    while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
                    while (rr * (rr + 1) / 2 > e) --rr;
                    const int r = m0 + rr, c = m0 + (e - rr * (rr + 1) / 2);
                    T acc = V[r * kPP + c];
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j < cw) acc = fma(-(V[r * kPP + c0 + j] * s_rc[c0 + j]), V[c * kPP + c0 + j], acc);
                    V[r * kPP + c] = acc;
                }
            }
            __syncthreads();
        }
        // FP64 pivots
        if (tid < 64) {
            double d = 0.0, rd = 0.0;
            if (tid < nb) {
                d = chain_w64<T>(V[tid * kPP + tid], a.A[(int64_t)(k + tid) * (N + 1)]);
                rd = rcp_newton(d);
            }
            s_d[tid] = d;
            s_rd[tid] = rd;
        }
        __syncthreads();
        const int wid = tid >> 5;
        constexpr int kWarps = kPThreads / 32;
        // the block's L and D and the column maxima of its rows: column c by
        // CTA c mod G, one warp per column, lanes over rows (warp maxima)
        for (int c = g + G * wid; c < nb; c += G * kWarps) {
            unsigned long long bm = 0ULL;
            for (int r = c + lane; r < nb; r += 32) {
                const int64_t o = (int64_t)(k + r) + (int64_t)(k + c) * N;
                if (r == c) {
                    a.L[o] = 1.0;
                    a.Dd[k + c] = s_d[c];
                } else {
                    const T w = V[r * kPP + c];
                    a.L[o] = w * s_rd[c];
                    const unsigned long long bw = absbits64((double)w);
                    bm = bw > bm ? bw : bm;
                }
            }
            const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(bm >> 32));
            const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(bm >> 32) == hi ? (unsigned)bm : 0u);
            if (lane == 0 && (hi | lo)) atomicMax(&s_cmax[c], ((unsigned long long)hi << 32) | lo);
        }
        // ---------------- A2: this CTA's rows below the block, 64 at a time
        // in shared memory, solved against the block's factor in the same
        // 16-column steps (row solves, then a rank-16 update of the rest)
        T *U = V + 64 * kPP;                  // [64][kPP]: a chunk of rows
        const int brow = N - k - nb;
        const int R = (brow + G - 1) / G;
        const int r_begin = k + nb + g * R, r_end = min(N, r_begin + R);
        for (int cb = r_begin; cb < r_end; cb += 64) {
            const int nr = min(64, r_end - cb);
            __syncthreads();                   // the previous chunk is written out
            for (int e = tid; e < 64 * 64; e += kPThreads) {
                const int c = e >> 6, r = e & 63;
                U[r * kPP + c] = (r < nr && c < nb) ? (T)a.A[(int64_t)(cb + r) + (int64_t)(k + c) * N] : (T)0;
            }
            __syncthreads();
            for (int c0 = 0; c0 < nb; c0 += 16) {
                const int cw = min(16, nb - c0);
                for (int r = tid; r < nr; r += kPThreads) {
                    T v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = j < cw ? U[r * kPP + c0 + j] : (T)0;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const T l = j < cw ? v[j] * s_rc[c0 + j] : (T)0;
#pragma unroll
                        for (int t = j + 1; t < 16; ++t)
                            if (t < cw) v[t] = fma(-l, V[(c0 + t) * kPP + c0 + j], v[t]);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j < cw) U[r * kPP + c0 + j] = v[j];
                }
                __syncthreads();
                const int m0 = c0 + 16, mw = nb - m0;
                if (mw > 0) {
                    for (int e = tid; e < nr * mw; e += kPThreads) {
                        const int r = e / mw, c = m0 + (e - (e / mw) * mw);
                        T acc = U[r * kPP + c];
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j < cw) acc = fma(-(U[r * kPP + c0 + j] * s_rc[c0 + j]), V[c * kPP + c0 + j], acc);
                        U[r * kPP + c] = acc;
                    }
                }
                __syncthreads();
            }
            // outputs and column maxima: one warp per column, lanes over rows
            for (int c = wid; c < nb; c += kWarps) {
                unsigned long long bm = 0ULL;
                for (int r = lane; r < nr; r += 32) {
                    const int i = cb + r;
                    const int64_t o = (int64_t)i + (int64_t)(k + c) * N;
                    const double w = U[r * kPP + c];
                    a.L[o] = w * s_rd[c];
                    a.Wg[(int64_t)i + (int64_t)c * N] = w;
                    const unsigned long long bw = absbits64(w);
                    bm = bw > bm ? bw : bm;
                }
                const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(bm >> 32));
                const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(bm >> 32) == hi ? (unsigned)bm : 0u);
                if (lane == 0 && (hi | lo)) atomicMax(&s_cmax[c], ((unsigned long long)hi << 32) | lo);
            }
        }
        __syncthreads();
        if (tid < 64 && s_cmax[tid]) atomicMax(&a.cmax[buf * 64 + tid], s_cmax[tid]);
        if (!panel_barrier(a.bar, epoch, a.wait_ns)) return;
        // ---------------- B: the rule's column test, the same in every CTA
        if (!persist_keep(a, k, nb, buf, buf ^ 1, ztol, s_d)) {
            if (g == 0 && tid == 0) {   // the panel loop takes over at column k
                a.st->k = k;
                a.st->kb = 0;
                a.st->spec = 0;
            }
            return;
        }
        if (k + nb >= N) break;
        // ---------------- C: trailing update
        {
            const int base = k + nb;
            const int nt = (N - base + kUT - 1) / kUT;
            const int tiles = nt * (nt + 1) / 2;
            for (int t = g; t < tiles; t += G) {
                trailing_tile<T>(t, N, nb, k, 65, a.A, a.L, a.Wg, a.Lf, a.Wf, psm);
                __syncthreads();
            }
        }
        __threadfence();
        if (!panel_barrier(a.bar, epoch, a.wait_ns)) return;
    }
}

// ---------------------------------------------------------------------------
// Persistent no-interchange factorization, FP32-update form (the refined
// mixed-precision path).  The same panel sequence, column test and hand-over
// as k_bk_persist, with the arithmetic of the loop in FP32 only:
//   - the prologue copies the lower triangle of S into Af (FP32, ld N); the
//     trailing updates run on Af in place, and the FP64 matrix keeps S;
//   - each 64-column panel is factored in Q-column sub-panels (Q = 16).  A
//     warp holds the sub-panel's Q diagonal-block rows (lane = row) and 32
//     rows below them (lane = row) in registers and runs the Q-step pivot
//     chain, each step's column broadcast through shared memory; every warp
//     repeats the short diagonal chain for its own rows, so no block barrier
//     is needed per column.  A rank-Q update (2 x 4 outputs per thread, from
//     shared memory) brings the later columns up to date;
//   - the FP64 pivot is the chain's FP32 value plus the part of S's diagonal
//     that the FP32 copy dropped; L (FP64 copy), W and the column maxima come
//     from the FP32 chain values.
// One grid barrier per panel (after its rows, for the column test); the
// trailing update has none: its 64 x 64 blocks are spread over the CTAs with
// the blocks of the next panel's columns first, those count themselves done,
// and the next panel starts on that count while the remaining blocks are
// still being updated (L and W of successive panels alternate between two
// buffers, the column maxima rotate over three).  On a rejected panel every
// CTA writes the FP32 updates of the trailing matrix back into the FP64
// matrix (A += Af - fl32(A)) before the pivoting panels take over.
// ---------------------------------------------------------------------------
// Sub-panel width Q (16 or 32; 16 measured faster: 32-step chains are twice
// as long per column and the rank updates do not shrink in proportion): a
// warp holds the Q diagonal-block rows of a sub-panel and 32 rows below
// them.  Own rows staged per pass: what the warps left after the block's
// target groups take (at most 8 groups in all).
constexpr int kPersistQ = 16;   // sub-panel width of the FP32-update kernel
template <int Q> constexpr int own_rows() { return (8 - (64 - Q + 31) / 32) * 32; }
constexpr int kRowsBuf = 64 + own_rows<32>();   // the larger of the two (224 own rows)

// Pivot chain of one Q-column sub-panel in one warp.  vA: the sub-block's row
// `lane` (lanes >= Q hold zeros), vB: one row below it (zeros where a lane
// has no row).  Before step j the sub-block's lanes put column j (their
// vA[j]) into the warp's slot `col` (Q floats, 16-byte aligned) and every
// lane reads it back as 16-byte broadcasts: the loads issue back to back,
// where Q - j - 1 shuffles per step had their latencies exposed one after
// another.  The reciprocal pivot is the hardware approximation (about one
// unit in the last place; the factor is refined against the FP64 operator).
// With `factored`, vA holds the factored sub-block (its W values) and rcl the
// reciprocal pivot of column `lane`: vA is only read.  On return vB holds the
// row's W values (L = W / d); the result is the reciprocal pivot of column
// `lane`.
__device__ __forceinline__ float rcp_approx(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}

template <int Q>
__device__ __forceinline__ float chain_q(float (&vA)[Q], float (&vB)[Q], bool factored, float rcl, int cw,
                                         int lane, float *col) {
    float rc = 0.0f;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        if (lane < Q) col[lane] = vA[j];
        __syncwarp();
        float w[Q];
#pragma unroll
        for (int t = 0; t < Q; t += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(col + t);
            w[t] = x.x;
            w[t + 1] = x.y;
            w[t + 2] = x.z;
            w[t + 3] = x.w;
        }
        __syncwarp();   // every lane has read the column before the next one is written
        float rj;
        if (factored) rj = __shfl_sync(0xffffffffu, rcl, j);
        else rj = (j < cw && w[j] != 0.0f) ? rcp_approx(w[j]) : 0.0f;
        // zero multipliers, not conditional updates: v stays in registers
        const float lA = (!factored && lane > j) ? vA[j] * rj : 0.0f;
        const float lB = vB[j] * rj;
#pragma unroll
        for (int t = j + 1; t < Q; ++t) {
            vA[t] = fmaf(-lA, w[t], vA[t]);
            vB[t] = fmaf(-lB, w[t], vB[t]);
        }
        rc = lane == j ? rj : rc;
    }
    return rc;
}

// One sub-panel (columns c0 .. c0 + cw - 1 of the staged rows Rb, pitch kPP):
// the targets are the block rows c0 + Q .. nb - 1 (when `blk`) and the nr
// staged own rows (Rb rows 64 ..).  Each warp takes one group of 32 targets;
// warp 0 also keeps the factored sub-block and writes it back, with its
// reciprocal pivots, after every warp has read it.
template <int Q>
__device__ void persist_subpanel(float *Rb, float *s_rc, float *s_col, int c0, int cw, int nb, bool blk, int nr,
                                 bool factored) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gb = blk ? max(0, nb - c0 - Q + 31) / 32 : 0;   // groups of block rows
    const int ng = gb + (nr + 31) / 32;                       // <= 8 by the staging size
    float vA[Q], vB[Q];
    float rc = 0.0f;
    if (wid < ng || wid == 0) {
        int row = -1;
        if (wid < gb) {
            const int r = c0 + Q + 32 * wid + lane;
            if (r < nb) row = r;
        } else if (wid < ng) {
            const int r = 32 * (wid - gb) + lane;
            if (r < nr) row = 64 + r;
        }
#pragma unroll
        for (int t = 0; t < Q; ++t) {
            vA[t] = (lane < cw && t <= lane) ? Rb[(c0 + lane) * kPP + c0 + t] : 0.0f;
            vB[t] = (row >= 0 && t < cw) ? Rb[row * kPP + c0 + t] : 0.0f;
        }
        const float rcl = (factored && lane < Q) ? s_rc[c0 + lane] : 0.0f;
        rc = chain_q<Q>(vA, vB, factored, rcl, cw, lane, s_col + wid * Q);
        if (row >= 0) {
#pragma unroll
            for (int t = 0; t < Q; ++t)
                if (t < cw) Rb[row * kPP + c0 + t] = vB[t];
        }
    }
    __syncthreads();   // every warp has read the sub-block
    if (wid == 0 && !factored) {
#pragma unroll
        for (int t = 0; t < Q; ++t)
            if (lane < cw && t <= lane) Rb[(c0 + lane) * kPP + c0 + t] = vA[t];
        if (lane < cw) s_rc[c0 + lane] = rc;
    }
    __syncthreads();
}

// Rank-Q update of columns c0 + Q .. nb - 1 with the sub-panel at c0: block
// rows c0 + Q .. nb - 1 (lower triangle, when `blk`) and the nr staged own
// rows.  2 rows x 4 columns per thread.
template <int Q>
__device__ void persist_rank_q(float *Rb, const float *s_rc, int c0, int nb, bool blk, int nr) {
    const int m0 = c0 + Q;                    // first row / column updated
    const int ncq = (64 - m0) / 4;            // column quads
    const int nbp = blk ? (64 - m0) / 2 : 0;  // row pairs of the block
    const int items = (nbp + (nr + 1) / 2) * ncq;
    for (int it = threadIdx.x; it < items; it += kPThreads) {
        const int rp = it / ncq, cq = it - rp * ncq;
        const int r0 = rp < nbp ? m0 + 2 * rp : 64 + 2 * (rp - nbp);
        const int col0 = m0 + 4 * cq;
        if (col0 >= nb || (rp < nbp && (r0 + 1 < col0 || r0 >= nb))) continue;   // nothing of it is kept
        float acc[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float rcj = s_rc[c0 + j];
            const float l0 = Rb[r0 * kPP + c0 + j] * rcj, l1 = Rb[(r0 + 1) * kPP + c0 + j] * rcj;
            float w[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) w[v] = Rb[(col0 + v) * kPP + c0 + j];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                acc[0][v] = fmaf(l0, w[v], acc[0][v]);
                acc[1][v] = fmaf(l1, w[v], acc[1][v]);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int r = r0 + u;
            const bool live = rp < nbp ? r < nb : r - 64 < nr;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int c = col0 + v;
                if (live && c < nb && (rp >= nbp || c <= r)) Rb[r * kPP + c] -= acc[u][v];
            }
        }
    }
    __syncthreads();
}

// The TE x TE block (TE = 64 or 32) of the lower triangle at rows i0..,
// columns c0.. of the FP32 copy: Af(i, c) -= sum_{t < kb} Lf(i, t) Wf(c, t)
// for i >= c.  256 threads, (TE / 16)^2 outputs each; smem: 2 x 64 x TE floats.
template <int P>
__device__ __forceinline__ void load_p(const float *p, float (&v)[P]) {
    if constexpr (P == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    } else {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
}

template <int TE>
__device__ void block_update_f32(int i0, int c0, int N, int kb, float *__restrict__ Af,
                                 const float *__restrict__ Lf, const float *__restrict__ Wf,
                                 unsigned char *usmem) {
    constexpr int P = TE / 16;      // outputs per thread along rows and along columns
    constexpr int RS = 256 / TE;    // panel columns staged per pass of the threads
    float *Lt = reinterpret_cast<float *>(usmem);   // [64][TE]: Lt[t][r]
    float *Wt = Lt + 64 * TE;                       // [64][TE]: Wt[t][c]
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // this thread's entries of the block, loaded ahead of the products
    float cur[P][P];
#pragma unroll
    for (int v = 0; v < P; ++v) {
        const int c = c0 + P * ty + v;
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int i = i0 + P * tx + u;
            cur[u][v] = (i < N && c < N && i >= c) ? Af[i + (int64_t)c * N] : 0.0f;
        }
    }
    {
        const int r = tid % TE, t0 = tid / TE;
        const int i = i0 + r, c = c0 + r;
        float lv[64 / RS], wv[64 / RS];
#pragma unroll
        for (int j = 0; j < 64 / RS; ++j) {
            const int t = t0 + RS * j;
            lv[j] = (t < kb && i < N) ? Lf[i + (int64_t)t * N] : 0.0f;
            wv[j] = (t < kb && c < N) ? Wf[c + (int64_t)t * N] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 64 / RS; ++j) {
            const int t = t0 + RS * j;
            Lt[t * TE + r] = lv[j];
            Wt[t * TE + r] = wv[j];
        }
    }
    __syncthreads();
    float acc[P][P];
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
        for (int v = 0; v < P; ++v) acc[u][v] = 0.0f;
    for (int t = 0; t < kb; ++t) {
        float lv[P], wv[P];
        load_p<P>(Lt + t * TE + P * tx, lv);
        load_p<P>(Wt + t * TE + P * ty, wv);
#pragma unroll
        for (int u = 0; u < P; ++u)
#pragma unroll
            for (int v = 0; v < P; ++v) acc[u][v] = fmaf(lv[u], wv[v], acc[u][v]);
    }
#pragma unroll
    for (int v = 0; v < P; ++v) {
        const int c = c0 + P * ty + v;
        if (c >= N) continue;
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int i = i0 + P * tx + u;
            if (i < N && i >= c) Af[i + (int64_t)c * N] = cur[u][v] - acc[u][v];
        }
    }
}

// Two vertically adjacent 64 x 64 blocks of the trailing update on the tensor
// cores: rows i0 .. i0 + 127, columns c0 .. c0 + 63 of the FP32 copy,
// Af(i, c) -= sum_{t < 64} Lf(i, t) Wf(c, t) for i >= c.  One tcgen05.mma of
// shape 128 x 64 per 8-wide K step (kind::tf32), in three products
// (hi hi + hi lo + lo hi, x = hi + lo with hi = x cut to the TF32 mantissa):
// about 2^-21 relative per product, the FP32 accuracy of the CUDA-core form,
// instead of TF32's 2^-11.  All 256 threads stage L and W in shared memory in
// the 128-byte-swizzled K-major layout; one thread issues the 24 MMAs into a
// 64-column FP32 accumulator in TMEM and commits them to an mbarrier; the
// eight warps read the accumulator back (warp w: TMEM lanes 32 (w mod 4) ..,
// columns 32 (w / 4) ..) and write Af.  Returns false when the bounded wait
// for the MMAs expires.
constexpr int kTcA = 128 * 128;   // bytes per K slab of the 128 L rows (32 floats per row)
constexpr int kTcB = 64 * 128;    // bytes per K slab of the 64 W rows
constexpr size_t kTcSmem = 2 * 2 * (size_t)kTcA + 2 * 2 * (size_t)kTcB + 1024;   // hi and lo, two slabs each, alignment

__device__ __forceinline__ uint32_t sw128_off(int r, int chunk) {
    return (uint32_t)(r * 128 + (((chunk ^ r) & 7) << 4));
}

__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

__device__ bool pair_update_tc(int i0, int c0, int N, float *__restrict__ Af, const float *__restrict__ Lf,
                               const float *__restrict__ Wf, unsigned char *usmem, uint32_t tmem, uint64_t *bar,
                               uint32_t &phase) {
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(usmem) + 1023) & ~uintptr_t(1023));
    unsigned char *Ahi = base, *Alo = Ahi + 2 * kTcA, *Bhi = Alo + 2 * kTcA, *Blo = Bhi + 2 * kTcB;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // stage: L rows (128 x 16 chunks of 4 K values), W rows (64 x 16 chunks)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int r = tid & 127, ch = (tid >> 7) + 2 * j;
        const int i = i0 + r;
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) tf32_split(i < N ? Lf[i + (int64_t)(4 * ch + u) * N] : 0.0f, h[u], l[u]);
        const uint32_t off = (uint32_t)(ch >> 3) * kTcA + sw128_off(r, ch & 7);
        *reinterpret_cast<float4 *>(Ahi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(Alo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = tid & 63, ch = (tid >> 6) + 4 * j;
        const int c = c0 + r;
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) tf32_split(c < N ? Wf[c + (int64_t)(4 * ch + u) * N] : 0.0f, h[u], l[u]);
        const uint32_t off = (uint32_t)(ch >> 3) * kTcB + sw128_off(r, ch & 7);
        *reinterpret_cast<float4 *>(Bhi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(Blo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the tensor core reads what the threads wrote
    __syncthreads();
    if (tid == 0) {
        tc::fence_after();
        constexpr uint32_t kIdesc = tc::instr_desc(true, 128, 64);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int k = 0; k < 4; ++k) {   // four K steps of 8 TF32 values (32 bytes) per slab
                const uint32_t ao = (uint32_t)s * kTcA + 32 * k, bo = (uint32_t)s * kTcB + 32 * k;
                const uint64_t ah = tc::sw128_kmajor_desc(tc::smem_u32(Ahi + ao));
                const uint64_t al = tc::sw128_kmajor_desc(tc::smem_u32(Alo + ao));
                const uint64_t bh = tc::sw128_kmajor_desc(tc::smem_u32(Bhi + bo));
                const uint64_t bl = tc::sw128_kmajor_desc(tc::smem_u32(Blo + bo));
                tc::mma<true, kIdesc>(tmem, ah, bh, (s > 0 || k > 0) ? 1u : 0u);
                tc::mma<true, kIdesc>(tmem, ah, bl, 1u);
                tc::mma<true, kIdesc>(tmem, al, bh, 1u);
            }
        tc::commit(bar);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    tc::fence_after();
    if (ok) {
        const int q = wid & 3, h = wid >> 2;
        uint32_t v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h), v);
        const int i = i0 + 32 * q + lane;
        if (i < N) {
            float cur[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = c0 + 32 * h + j;
                cur[j] = (c < N && i >= c) ? Af[i + (int64_t)c * N] : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = c0 + 32 * h + j;
                if (c < N && i >= c) Af[i + (int64_t)c * N] = cur[j] - __uint_as_float(v[j]);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    return ok;
}

template <int Q>
__global__ void __launch_bounds__(kPThreads, 1) k_bk_persist32(PersistArgs a) {
    constexpr int kOwn = own_rows<Q>();
    extern __shared__ __align__(16) unsigned char psm[];
    float *Rb = reinterpret_cast<float *>(psm);   // [kRowsBuf][kPP]: block rows 0..63, then own rows
    __shared__ double s_d[64];
    __shared__ float s_rc[64];
    __shared__ __align__(16) float s_col[kPThreads / 32 * Q];   // each warp's pivot-chain column
    // column maxima of |w| as FP32 bit patterns: the diagonal block's rows
    // (written by the one warp that outputs the column) and this CTA's rows
    // (one warp per column): plain stores, no shared atomics
    __shared__ unsigned s_cmax_blk[64], s_cmax_own[64];
    __shared__ __align__(8) uint64_t s_mma_bar;   // completion of a trailing block pair's MMAs
    __shared__ uint32_t s_tmem;
    const int N = a.N, G = (int)gridDim.x, g = (int)blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    constexpr int kWarps = kPThreads / 32;
    const double ztol = a.zero_tol * __ldg(a.maxabs);
    const int kstart = a.st->k;
    unsigned epoch = 0;   // grid barriers passed (thread 0)
    // 64 TMEM columns for the trailing block pairs' accumulator (one CTA per SM),
    // released on every way out
    if (tid == 0) {
        tc::mbar_init(&s_mma_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wid == 0) tc::tmem_alloc(&s_tmem, 64);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t mma_phase = 0;
    auto release = [&]() {
        tc::fence_before();
        __syncthreads();
        if (wid == 0) tc::tmem_dealloc(tmem, 64);
    };
    // prologue: the FP32 copy of columns kstart .. N - 1 (whole columns: the
    // entries above the diagonal are copied too and never read), eight
    // 16-byte loads in flight per thread
    {
        const int64_t e0 = (int64_t)kstart * N, total = (int64_t)N * N;
        const int64_t stride = (int64_t)G * kPThreads;
        const int64_t first = (int64_t)g * kPThreads + tid;
        if (((reinterpret_cast<uintptr_t>(a.A) | reinterpret_cast<uintptr_t>(a.Af)) & 15) == 0 && (e0 & 1) == 0) {
            const double2 *src = reinterpret_cast<const double2 *>(a.A + e0);
            float2 *dst = reinterpret_cast<float2 *>(a.Af + e0);
            const int64_t n2 = (total - e0) / 2;
            for (int64_t e = first; e < n2; e += 8 * stride) {
                double2 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e + u * stride < n2) x[u] = __ldcs(src + e + u * stride);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e + u * stride < n2) dst[e + u * stride] = make_float2((float)x[u].x, (float)x[u].y);
            }
            if (g == 0 && tid == 0 && ((total - e0) & 1)) a.Af[total - 1] = (float)a.A[total - 1];
        } else {
            for (int64_t e = e0 + first; e < total; e += stride) a.Af[e] = (float)a.A[e];
        }
    }
    __threadfence();
    if (!panel_barrier(a.bar, epoch, a.wait_ns)) {
        release();
        return;
    }
    const int nbk = (N + 63) / 64;   // 64 x 64 blocks per row / column
    int p = 0;
    for (int k = kstart; k < N; k += 64, ++p) {
        const int nb = min(64, N - k);
        const int kblk = k / 64;
        const int buf = p % 3;                       // column maxima of this panel
        float *Lfp = (p & 1) ? a.Lf2 : a.Lf, *Wfp = (p & 1) ? a.Wf2 : a.Wf;
        // this panel's columns have taken every earlier panel's update
        if (p > 0 && !wait_count(&a.colcnt[kblk], 4u * (unsigned)(nbk - kblk), a.bar, a.wait_ns)) {
            release();
            return;
        }
        if (tid < 64) {
            s_cmax_blk[tid] = s_cmax_own[tid] = 0u;
            s_rc[tid] = 0.0f;
        }
        // S's diagonal of the block (for the FP64 pivots), loaded ahead of the chains
        const double adiag = tid < nb ? a.A[(int64_t)(k + tid) * (N + 1)] : 0.0;
        const int brow = N - k - nb;
        const int R = (brow + G - 1) / G;
        const int r_begin = k + nb + g * R, r_end = min(N, r_begin + R);
        for (int cb = r_begin, pass = 0; pass == 0 || cb < r_end; cb += kOwn, ++pass) {
            const int nr = max(0, min(kOwn, r_end - cb));
            const bool blk = pass == 0;   // the diagonal block is factored in the first pass
            // ---- stage: warp w takes columns w, w + 8, ..; lanes over rows
            // (block rows c..nb-1 of column c on the first pass, then own rows)
            __syncthreads();
#pragma unroll
            for (int cc = 0; cc < 64 / kWarps; ++cc) {
                const int c = wid + kWarps * cc;
                constexpr int kR = (64 + kOwn + 31) / 32;
                float v[kR];
#pragma unroll
                for (int q = 0; q < kR; ++q) {
                    const int rr = lane + 32 * q;
                    v[q] = 0.0f;
                    if (c < nb) {
                        if (rr < 64) {
                            if (blk && rr < nb && rr >= c) v[q] = a.Af[(int64_t)(k + rr) + (int64_t)(k + c) * N];
                        } else if (rr - 64 < nr) {
                            v[q] = a.Af[(int64_t)(cb + rr - 64) + (int64_t)(k + c) * N];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kR; ++q) {
                    const int rr = lane + 32 * q;
                    if ((rr < 64 && blk) || (rr >= 64 && rr - 64 < nr)) Rb[rr * kPP + c] = v[q];
                }
            }
            __syncthreads();
            // ---- the sub-panels, each followed by the update of the columns after it
            for (int c0 = 0; c0 < nb; c0 += Q) {
                persist_subpanel<Q>(Rb, s_rc, s_col, c0, min(Q, nb - c0), nb, blk, nr, !blk);
                if (c0 + Q < nb) persist_rank_q<Q>(Rb, s_rc, c0, nb, blk, nr);
            }
            if (blk) {
                // FP64 pivots, then the block's L and D and the column maxima of
                // its rows: column c by CTA c mod G, one warp per column
                if (tid < 64) {
                    double d = 0.0;
                    if (tid < nb) d = chain_w64<float>(Rb[tid * kPP + tid], adiag);
                    s_d[tid] = d;
                }
                __syncthreads();
                for (int c = g + G * wid; c < nb; c += G * kWarps) {
                    unsigned bm = 0u;
                    for (int r = c + lane; r < nb; r += 32) {
                        const int64_t o = (int64_t)(k + r) + (int64_t)(k + c) * N;
                        if (r == c) {
                            a.L[o] = 1.0;
                            a.Dd[k + c] = s_d[c];
                        } else {
                            const float w = Rb[r * kPP + c];
                            a.L[o] = (double)(w * s_rc[c]);
                            bm = max(bm, __float_as_uint(w) & 0x7fffffffu);
                        }
                    }
                    bm = __reduce_max_sync(0xffffffffu, bm);
                    if (lane == 0) s_cmax_blk[c] = bm;
                }
            }
            // own rows: L (FP64 copy), the FP32 L and W columns, column maxima
            for (int c = wid; c < nb; c += kWarps) {
                unsigned bm = 0u;
                for (int r = lane; r < nr; r += 32) {
                    const int i = cb + r;
                    const float w = Rb[(64 + r) * kPP + c], l = w * s_rc[c];
                    a.L[(int64_t)i + (int64_t)(k + c) * N] = (double)l;
                    Lfp[(int64_t)i + (int64_t)c * N] = l;
                    Wfp[(int64_t)i + (int64_t)c * N] = w;
                    bm = max(bm, __float_as_uint(w) & 0x7fffffffu);
                }
                bm = __reduce_max_sync(0xffffffffu, bm);
                if (lane == 0) s_cmax_own[c] = max(s_cmax_own[c], bm);
            }
        }
        __syncthreads();
        if (tid < 64) {
            const unsigned bm = max(s_cmax_blk[tid], s_cmax_own[tid]);
            if (bm) atomicMax(&a.cmax[buf * 64 + tid], absbits64((double)__uint_as_float(bm)));
        }
        if (!panel_barrier(a.bar, epoch, a.wait_ns)) {
            release();
            return;
        }
        if (!persist_keep(a, k, nb, buf, (p + 2) % 3, ztol, s_d)) {
            // hand over at column k: the FP64 matrix takes the FP32 updates
            for (int c = k + g; c < N; c += G)
                for (int i = c + tid; i < N; i += kPThreads) {
                    const int64_t o = i + (int64_t)c * N;
                    const double s0 = a.A[o];
                    a.A[o] = s0 + ((double)a.Af[o] - (double)(float)s0);
                }
            if (g == 0 && tid == 0) {
                a.st->k = k;
                a.st->kb = 0;
                a.st->spec = 0;
            }
            release();
            return;
        }
        if (k + nb >= N) break;
        // ---------------- trailing update on the FP32 copy.  The next panel's
        // column of 64 x 64 blocks goes first, as 4 n1 quarter blocks on the CUDA
        // cores (it is on the critical path: the next panel starts when all of
        // them have counted themselves done), then the other blocks: in
        // vertically adjacent pairs on the tensor cores, column by column,
        // while there are more than four blocks per CTA; else one per item on
        // the CUDA cores (a pair's staging and read-back cost about as much as
        // two blocks' FMAs, so pairs pay only where they halve the number of
        // items a CTA works through: measured at N = 2050 0.85 ms with blocks
        // against 0.88 ms with pairs, at N = 8003 11.4 against 9.9 ms).
        // CTA g takes items g, g + G, ...  Every block's update of the previous
        // panel finished before this panel's grid barrier, so any CTA may take
        // any block.
        {
            const int n1 = nbk - kblk - 1, m2 = nbk - kblk - 2;
            const int nwhole = m2 > 0 ? m2 * (m2 + 1) / 2 : 0;
            const bool pairs = nwhole > 4 * G;
            int npairs = 0;
            if (pairs)
                for (int J = kblk + 2; J < nbk; ++J) npairs += (nbk - J + 1) / 2;
            const int nitems = 4 * n1 + (pairs ? npairs : nwhole);
            int b = g;
            for (; b < nitems && b < 4 * n1; b += G) {
                const int I = kblk + 1 + (b >> 2), J = kblk + 1, q = b & 3;
                const int i0 = 64 * I + 32 * (q >> 1), c0 = 64 * J + 32 * (q & 1);
                if (i0 + 31 >= c0) block_update_f32<32>(i0, c0, N, nb, a.Af, Lfp, Wfp, psm);
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&a.colcnt[J]) : "memory");
                }
            }
            if (!pairs) {
                for (; b < nitems; b += G) {   // whole blocks, row-major over their triangle
                    const int lin = b - 4 * n1;
                    int r = (int)((sqrtf(8.0f * (float)lin + 1.0f) - 1.0f) * 0.5f);
                    while ((r + 1) * (r + 2) / 2 <= lin) ++r;
                    while (r * (r + 1) / 2 > lin) --r;
                    const int I = kblk + 2 + r, J = kblk + 2 + (lin - r * (r + 1) / 2);
                    block_update_f32<64>(64 * I, 64 * J, N, nb, a.Af, Lfp, Wfp, psm);
                    __syncthreads();
                }
            } else {
                int J = kblk + 2, first = 4 * n1;   // first item of column J
                for (; b < nitems; b += G) {
                    while (J < nbk - 1 && (b - first) >= (nbk - J + 1) / 2) {
                        first += (nbk - J + 1) / 2;
                        ++J;
                    }
                    const int I0 = J + 2 * (b - first);
                    if (!pair_update_tc(64 * I0, 64 * J, N, a.Af, Lfp, Wfp, psm, tmem, &s_mma_bar, mma_phase)) {
                        if (tid == 0) atomicExch(&a.bar->err, 1);
                        release();
                        return;
                    }
                }
            }
        }
    }
    release();
}

__global__ void k_bk_init(int N, int32_t *perm, PanelState *st, unsigned long long *cmax, PanelBar *bar,
                          unsigned *colcnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) perm[i] = i;
    if (blockIdx.x == 0 && threadIdx.x < 192) cmax[threadIdx.x] = 0ULL;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (N + 63) / 64 + 1; i += gridDim.x * blockDim.x)
        colcnt[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bar->count = 0u;
        bar->err = 0;
        st->k = 0;
        st->kb = 0;
        st->npos = st->nneg = st->nzero = 0;
        st->spec = 0;
        st->nacc = st->nrej = 0;
        st->done = 0u;
        st->nfail = 0;
        st->done2 = 0u;
    }
}

__global__ void k_bk_finish(const PanelState *st, int32_t *inertia, int32_t *panels) {
    pdl_wait();
    inertia[0] = st->npos;
    inertia[1] = st->nneg;
    inertia[2] = st->nzero;
    if (panels) {
        panels[0] = st->nacc;
        panels[1] = st->nrej;
    }
}

struct BlockedConfig {
    int C = 0, NB = 0, R = 0;
    size_t smem = 0;
};

size_t panel_smem(int R, int NB, bool f32) {
    const int S = NB + 1;
    return (2 * (size_t)R * S + S) * sizeof(double) + 4 * sizeof(Cand) + (f32 ? ((size_t)R * S + S) * sizeof(float) : 0) +
           64;
}

// cluster size and panel width for order N on this device (C = 0: unavailable);
// nb > 0 asks for that panel width if it fits
BlockedConfig blocked_config(int64_t N, bool f32, int nb_want = 0) {
    static std::mutex mu;
    static int clusters16[64] = {};   // 1: size 16 allowed, -1: not, 0: unknown
    int dev = 0;
    MDSIP_CUDA(cudaGetDevice(&dev));
    constexpr size_t kSmemCap = 220 * 1024;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && clusters16[dev] == 0) {
            cudaError_t e = cudaSuccess;
            for (const void *fn : {(const void *)k_bk_panel<false>, (const void *)k_bk_panel<true>}) {
                if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
                if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            }
            int ok16 = 0;
            if (e == cudaSuccess) {
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3(16);
                cfg.blockDim = dim3(kPanelThreads);
                cfg.dynamicSmemBytes = kSmemCap;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = 16;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int nclusters = 0;
                int n32 = 0;
                if (cudaOccupancyMaxActiveClusters(&nclusters, (void *)k_bk_panel<false>, &cfg) == cudaSuccess &&
                    nclusters >= 1 &&
                    cudaOccupancyMaxActiveClusters(&n32, (void *)k_bk_panel<true>, &cfg) == cudaSuccess && n32 >= 1)
                    ok16 = 1;
            }
            cudaGetLastError();
            clusters16[dev] = ok16 ? 1 : -1;
        }
    }
    BlockedConfig c;
    c.C = (dev >= 0 && dev < 64 && clusters16[dev] == 1) ? 16 : 8;
    for (int nb : {64, 32, 16, 8}) {
        const int R = (int)((N + c.C - 1) / c.C);
        if (nb_want > 0 && nb != nb_want) continue;
        if (panel_smem(R, nb, f32) <= kSmemCap) {
            c.NB = nb;
            c.R = R;
            c.smem = panel_smem(R, nb, f32);
            return c;
        }
    }
    c.C = 0;
    return c;
}

// launch with programmatic stream serialization (and a cluster when cluster > 1)
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, int cluster,
                Args... args) {
    cudaLaunchConfig_t c{};
    c.gridDim = dim3(grid);
    c.blockDim = dim3(block);
    c.dynamicSmemBytes = smem;
    c.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
    if (cluster > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = (unsigned)cluster;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = 1;
        ++na;
    }
    c.attrs = at;
    c.numAttrs = na;
    MDSIP_CUDA(cudaLaunchKernelEx(&c, kern, args...));
    count_launch();
}

// scratch layout: W of the last panel (N x 65 doubles), the panel state, the
// FP32 L and W columns of the last panel (N x 65 floats each; FP32-update
// form), and for the verified no-interchange panels the per-column maxima
// (2 x 64), the pending row tests (64) and their partial row maxima
// ((ceil(N / 32) + 2) x 64)
struct BlockedScratch {
    size_t wg, st, lf, wf, cmax, fail, rowpart, af, lf2, wf2, colcnt, total;
};

BlockedScratch blocked_scratch(int64_t N) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t n = (size_t)std::max<int64_t>(N, 1);
    BlockedScratch l{};
    l.wg = 0;
    l.st = up(n * 65 * sizeof(double));
    l.lf = l.st + 256;
    l.wf = l.lf + up(n * 65 * sizeof(float));
    l.cmax = l.wf + up(n * 65 * sizeof(float));
    l.fail = l.cmax + up(192 * sizeof(unsigned long long));
    l.rowpart = l.fail + up(64 * sizeof(RowTest));
    l.af = l.rowpart + up(((n + 31) / 32 + 2) * 64 * sizeof(unsigned long long));
    l.lf2 = l.af + up(n * n * sizeof(float));   // the FP32 copy of the persistent FP32-update kernel
    l.wf2 = l.lf2 + up(n * 64 * sizeof(float));
    l.colcnt = l.wf2 + up(n * 64 * sizeof(float));
    l.total = l.colcnt + up(((n + 63) / 64 + 1) * sizeof(unsigned));
    return l;
}

}  // namespace

// the grid barrier of the persistent kernel shares the panel state's slot
PanelBar *grid_bar(char *w, const BlockedScratch &lay) { return reinterpret_cast<PanelBar *>(w + lay.st + 128); }

// dynamic shared memory of k_bk_persist<T>: the diagonal block, or the staged
// rows of a trailing-update tile
template <typename T>
size_t persist_smem() {
    if constexpr (sizeof(T) == sizeof(float))   // k_bk_persist32: staged rows, or a trailing tile's panel rows
        return std::max({(size_t)kRowsBuf * kPP * sizeof(float), 2 * (size_t)64 * kUT * sizeof(float), kTcSmem});
    return std::max(2 * (size_t)64 * kPP * sizeof(T), 2 * (size_t)65 * kUT * sizeof(T));
}

template <typename T>
const void *persist_kernel() {
    if constexpr (sizeof(T) == sizeof(float)) return (const void *)k_bk_persist32<kPersistQ>;
    else return (const void *)k_bk_persist;
}

// Run k_bk_persist from column 0; returns the column where it stopped (N: all
// panels kept).  One cooperative launch; reads two words back (synchronises
// the stream).
template <typename T>
int run_persistent(cudaStream_t s, int num_sms, int N, const PersistArgs &pa, PanelState *st, PanelBar *bar) {
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(persist_kernel<T>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)persist_smem<T>());
    }));
    int per_sm = 0;
    MDSIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel<T>(), kPThreads,
                                                             persist_smem<T>()));
    MDSIP_REQUIRE(per_sm >= 1, MDSIP_ERR_CUDA, "ldlt: persistent factorization does not fit an SM");
    // about three trailing tiles per CTA after the first panel, at most one CTA per SM
    const int64_t nt = std::max<int64_t>(1, (N - 64 + kUT - 1) / kUT);
    const int64_t want = std::max<int64_t>(1, (nt * (nt + 1) / 2 + 2) / 3);
    const int G = (int)std::min<int64_t>(want, (int64_t)num_sms);
    PersistArgs args = pa;
    void *kargs[] = {&args};
    MDSIP_CUDA(cudaLaunchCooperativeKernel(persist_kernel<T>(), dim3(G), dim3(kPThreads), kargs,
                                           persist_smem<T>(), s));
    count_launch();
    thread_local int *h = nullptr;
    if (!h) MDSIP_CUDA(cudaMallocHost(&h, 4 * sizeof(int)));
    MDSIP_CUDA(cudaMemcpyAsync(h, &st->k, sizeof(int), cudaMemcpyDeviceToHost, s));
    MDSIP_CUDA(cudaMemcpyAsync(h + 1, &bar->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MDSIP_CUDA(cudaStreamSynchronize(s));
    MDSIP_REQUIRE(h[1] == 0, MDSIP_ERR_DEVICE, "ldlt: a bounded grid-barrier wait expired");
    return h[0];
}

size_t ldlt_blocked_scratch_bytes(int64_t N) { return blocked_scratch(N).total; }

// panel widths that fit for order N (widest first)
std::vector<int> ldlt_blocked_widths(int64_t N, bool f32) {
    std::vector<int> out;
    for (int nb : {64, 32, 16})
        if (blocked_config(N, f32, nb).C > 0) out.push_back(nb);
    return out;
}

bool ldlt_blocked_available(int64_t N) { return blocked_config(N, true).C > 0 && blocked_config(N, false).C > 0; }

// The persistent no-interchange factorization runs first (and the host reads
// back where it stopped) in mode 2, and in mode 1 from kPersistentMinOrder on
// (measured on the convex Newton-step shape, persistent against per-panel
// launches: N = 2050 FP32 updates 1.65 / 1.73 ms, FP64 8.3 / 11.1 ms; N = 4050
// 4.8 / 6.0 and 31 / 36 ms; N = 8003 27.5 / 42.9 and 179 / 194 ms) and
// wherever the pivoting panel does not fit shared memory: it needs no
// pivoting panel unless a panel fails the column test.  Below that order --
// the many small instances of a batch among them -- the per-panel launches
// (captured in a graph from their second use) stay.
bool ldlt_persistent_path(int64_t N, int spec) {
    if (spec == 0 || N <= 0 || N > (int64_t)0x7fffffff / 2) return false;
    return spec == 2 || N >= kPersistentMinOrder || !ldlt_blocked_available(N);
}

// S (lower, ld N) is overwritten.  scratch: ldlt_blocked_scratch_bytes(N),
// 256-byte aligned.  fp32_update: trailing products in FP32.  spec (with
// fp32_update): each panel first tries the verified no-interchange path.
void launch_ldlt_blocked(cudaStream_t s, int num_sms, int64_t N, double *S, const double *maxabs_dev,
                         double zero_tol, LdltOut out, void *scratch, bool fp32_update, int nb, int spec) {
    if (N <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out.inertia, 0, 3 * sizeof(int32_t), s));
        return;
    }
    BlockedConfig cfg = blocked_config(N, fp32_update, nb);
    if (cfg.C == 0) cfg = blocked_config(N, fp32_update);
    const bool persist = ldlt_persistent_path(N, spec);
    MDSIP_REQUIRE(cfg.C > 0 || persist, MDSIP_ERR_INVALID_ARG, "ldlt: N too large for the blocked factorization");
    char *w = static_cast<char *>(scratch);
    MDSIP_REQUIRE((reinterpret_cast<uintptr_t>(w) & 255) == 0, MDSIP_ERR_INVALID_ARG, "ldlt: misaligned scratch");
    const BlockedScratch lay = blocked_scratch(N);
    double *Wg = reinterpret_cast<double *>(w + lay.wg);
    PanelState *st = reinterpret_cast<PanelState *>(w + lay.st);
    PanelBar *bar = grid_bar(w, lay);
    k_bk_init<<<std::max(1, std::min(1024, ceil_div(N, 256))), 256, 0, s>>>(
        (int)N, out.perm, st, reinterpret_cast<unsigned long long *>(w + lay.cmax), bar,
        reinterpret_cast<unsigned *>(w + lay.colcnt));
    MDSIP_LAUNCHED();
    int k0 = 0;   // first column left to the panel loop below
    if (persist) {
        PersistArgs pa{};
        pa.N = (int)N;
        pa.A = S;
        pa.L = out.L;
        pa.Dd = out.Dd;
        pa.Doff = out.Doff;
        pa.kind = out.kind;
        pa.Wg = Wg;
        pa.Lf = reinterpret_cast<float *>(w + lay.lf);
        pa.Wf = reinterpret_cast<float *>(w + lay.wf);
        pa.cmax = reinterpret_cast<unsigned long long *>(w + lay.cmax);
        pa.st = st;
        pa.bar = bar;
        pa.maxabs = maxabs_dev;
        pa.zero_tol = zero_tol;
        pa.Af = reinterpret_cast<float *>(w + lay.af);
        pa.Lf2 = reinterpret_cast<float *>(w + lay.lf2);
        pa.Wf2 = reinterpret_cast<float *>(w + lay.wf2);
        pa.colcnt = reinterpret_cast<unsigned *>(w + lay.colcnt);
        pa.wait_ns = 20LL * 1000 * 1000 * 1000;   // 20 s: far above the longest phase (FP64 update at N ~ 44000)
        k0 = fp32_update ? run_persistent<float>(s, num_sms, (int)N, pa, st, bar)
                         : run_persistent<double>(s, num_sms, (int)N, pa, st, bar);
        MDSIP_REQUIRE(k0 >= N || cfg.C > 0, MDSIP_ERR_INVALID_ARG,
                      "ldlt: a panel needs interchanges and N is too large for the pivoting panel");
        // the panel loop's no-interchange kernels expect their column maxima and
        // arg-max keys at zero; the rejected panel left its maxima there
        if (k0 < N) MDSIP_CUDA(cudaMemsetAsync(w + lay.cmax, 0, 192 * sizeof(unsigned long long), s));
    }

    PanelArgs a{};
    a.N = (int)N;
    a.NB = cfg.NB;
    a.C = cfg.C;
    a.R = cfg.R;
    a.A = S;
    a.L = out.L;
    a.Dd = out.Dd;
    a.Doff = out.Doff;
    a.perm = out.perm;
    a.kind = out.kind;
    a.Wg = Wg;
    a.Lf = reinterpret_cast<float *>(w + lay.lf);
    a.Wf = reinterpret_cast<float *>(w + lay.wf);
    a.st = st;
    a.maxabs = maxabs_dev;
    a.zero_tol = zero_tol;

    const size_t usm = 2 * (size_t)(cfg.NB + 1) * kUT * (fp32_update ? sizeof(float) : sizeof(double));
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        cudaError_t e = cudaFuncSetAttribute(k_bk_trailing<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(2 * 65 * kUT * sizeof(double)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bk_trailing<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * 65 * kUT * sizeof(float)));
        return e;
    }));
    SpecArgs sa{};
    if (spec != 0 && fp32_update) {
        sa.N = (int)N;
        sa.NB = cfg.NB;
        sa.A = S;
        sa.L = out.L;
        sa.Dd = out.Dd;
        sa.Doff = out.Doff;
        sa.kind = out.kind;
        sa.Lf = a.Lf;
        sa.Wf = a.Wf;
        sa.cmax = reinterpret_cast<unsigned long long *>(w + lay.cmax);
        sa.fail = reinterpret_cast<RowTest *>(w + lay.fail);
        sa.rowpart = reinterpret_cast<unsigned long long *>(w + lay.rowpart);
        sa.st = st;
        sa.maxabs = maxabs_dev;
        sa.zero_tol = zero_tol;
        static PerDeviceOnce once_spec;
        MDSIP_CUDA(once_spec.run([] {
            return cudaFuncSetAttribute(k_bk_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem(64));
        }));
    }
    // panels from column k0 on (all of them without the persistent kernel)
    const int npanels = k0 >= N ? 0 : (int)((N - k0 + cfg.NB - 1) / cfg.NB);
    for (int p = 0; p < npanels; ++p) {
        if (spec != 0 && fp32_update) {
            // rows below the diagonal block: at most N - k0 - (p + 1) NB (every panel takes >= NB columns)
            const int64_t below = N - k0 - (int64_t)(p + 1) * cfg.NB;
            const int G = (int)std::max<int64_t>(1, (below + kSpecRB - 1) / kSpecRB);
            launch_pdl(k_bk_spec, (unsigned)G, kSpecChainThreads, spec_smem(cfg.NB), s, 1, sa);
            // rows of the active matrix: at most N - k0 - p NB
            const int G2 = (int)std::max<int64_t>(1, (N - k0 - (int64_t)p * cfg.NB + 31) / 32);
            launch_pdl(k_bk_spec_rows, (unsigned)G2, kSpecThreads, 0, s, 1, sa);
        }
        if (fp32_update)
            launch_pdl(k_bk_panel<true>, (unsigned)cfg.C, kPanelThreads, cfg.smem, s, cfg.C, a);
        else
            launch_pdl(k_bk_panel<false>, (unsigned)cfg.C, kPanelThreads, cfg.smem, s, cfg.C, a);
        // trailing matrix after panel p starts at column >= k0 + (p + 1) NB
        const int64_t rest = N - k0 - (int64_t)(p + 1) * cfg.NB;
        if (rest <= 0) continue;
        const int64_t nt = (rest + kUT - 1) / kUT;
        const unsigned tiles = (unsigned)(nt * (nt + 1) / 2);
        const float *cLf = a.Lf, *cWf = a.Wf;
        const double *cL = out.L, *cWg = Wg;
        const PanelState *cst = st;
        if (fp32_update)
            launch_pdl(k_bk_trailing<float>, tiles, kUpdThreads, usm, s, 1, (int)N, cfg.NB, S, cL, cWg, cLf, cWf, cst);
        else
            launch_pdl(k_bk_trailing<double>, tiles, kUpdThreads, usm, s, 1, (int)N, cfg.NB, S, cL, cWg, cLf, cWf, cst);
    }
    const PanelState *cst = st;
    launch_pdl(k_bk_finish, 1, 1, 0, s, 1, cst, out.inertia, out.panels);
}

}  // namespace mdsip
