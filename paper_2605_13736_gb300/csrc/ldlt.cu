// Bunch-Kaufman symmetric indefinite LDL^T with inertia (Section 2.3).
//
// The dense solver of Section 2.3 factors P K P^T = L D L^T with 1x1 and 2x2
// pivots chosen by the Bunch-Kaufman rule (alpha = (1 + sqrt 17) / 8) and
// reads the inertia from D.  This file is a GB300 design of that
// factorization for the reduced matrices of one Newton step (N up to a few
// thousand, which stay resident in the 135 MB L2):
//
//  * one persistent cooperative kernel; each CTA owns the columns j with
//    j % gridDim == blockIdx and updates them with a rank-1 or rank-2 update
//    per pivot step (right-looking, unblocked);
//  * every CTA takes the same pivot decision from the same data (colmax of
//    the pivot column, and if needed the row maximum of row r, computed
//    redundantly per CTA), so no broadcast is needed;
//  * the symmetric interchange k+kstep-1 <-> kp is folded into the update:
//    the trailing matrix is read from the old buffer through the
//    transposition and written to the other buffer (ping-pong), so a step
//    needs no separate swap phase;
//  * the CTA that owns the next pivot column updates it first, computes its
//    column maximum and publishes both with a release flag; a CTA reads only
//    its own columns and the published pivot column(s), so the other CTAs
//    wait for that flag alone (no grid barrier), except in the steps that
//    read row r of the trailing block (the row-maximum test and the
//    interchange), which are bracketed by two grid barriers;
//  * every wait is bounded (error flag instead of a hang);
//  * GB300 issues FP64 at 1/64 of the FP32 rate, so the only FP64
//    instructions per trailing element are the update FMAs: magnitudes are
//    compared as the integer bit patterns of |v| (monotone for IEEE doubles
//    >= 0), and the rank-1 and rank-2 updates have separate loops.
//
// The pivot rule, its comparisons (LAPACK ?sytf2 form: no interchange when
// |a_kk| >= alpha colmax (colmax / rowmax)) and the first-index tie-breaking
// of the column maximum are those of the published algorithm; the data
// layout, work split and synchronisation are this library's.
#include <cooperative_groups.h>

#include <mutex>

#include "internal.cuh"

namespace mdsip {

namespace {

constexpr int kBkThreads = 512;
constexpr size_t kMaxDynSmem = 200 * 1024;   // dynamic shared memory bound of the LDL^T kernels

struct BKParams {
    int N;
    int64_t ld;
    double *buf0, *buf1;           // ping-pong copies of the trailing matrix (lower, ld)
    double *L, *Dd, *Doff;
    int32_t *perm, *kind, *inertia;
    unsigned long long *slot_bits; // [N + 1] |.| bit pattern of step s's pivot-column maximum
    int *slot_idx;                 // [N + 1] its row index
    unsigned int *pub;             // number of steps whose pivot data are published
    GridBar bar;
    const double *maxabs;          // max |S| (scale of the zero-pivot test)
    double zero_tol;
};

// |v| as an unsigned integer: ordered like |v| for every non-NaN double
__device__ __forceinline__ unsigned long long absbits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// (magnitude bits, index) arg-max with first-index tie-breaking, integer ops only
__device__ __forceinline__ void argmax_combine(unsigned long long &b, int &i, unsigned long long b2, int i2) {
    if (b2 > b || (b2 == b && i2 < i)) {
        b = b2;
        i = i2;
    }
}

// result valid in thread 0
__device__ void block_argmax(unsigned long long &b, int &idx, unsigned long long *shb, int *shi) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b2 = __shfl_down_sync(0xffffffffu, b, o);
        const int i2 = __shfl_down_sync(0xffffffffu, idx, o);
        argmax_combine(b, idx, b2, i2);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        shb[wid] = b;
        shi[wid] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmax_combine(b, idx, shb[w], shi[w]);
    }
}

__device__ unsigned long long block_maxbits(unsigned long long b, unsigned long long *shb) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b2 = __shfl_down_sync(0xffffffffu, b, o);
        b = b2 > b ? b2 : b;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) shb[wid] = b;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = shb[w] > b ? shb[w] : b;
    return b;
}

// wait until *pub >= target (bounded); all threads of the CTA return the same result
__device__ __forceinline__ bool wait_published(const unsigned int *pub, unsigned int target, int *err) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile const unsigned int *vp = pub;
        if (*vp < target) {
            const long long t0 = clock64();
            while (*vp < target) {
                if (*((volatile int *)err) != 0 || clock64() - t0 > kBarrierLimitCycles) {
                    atomicExch(err, 1);
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

__global__ void __launch_bounds__(kBkThreads) k_bk_factor(BKParams p) {
    extern __shared__ double sh_dyn[];
    __shared__ unsigned long long s_redb[32];
    __shared__ int s_redi[32];
    __shared__ unsigned long long s_bcast;

    const int N = p.N;
    const int64_t ld = p.ld;
    const unsigned nb = gridDim.x;
    const int cta = blockIdx.x;
    const int tid = threadIdx.x;
    double *c0 = sh_dyn;        // pivot column(s) of the current step, rows base..N-1
    double *c1 = sh_dyn + N;
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;

    const double scale = __ldcg(p.maxabs);
    const double ztol = p.zero_tol * scale;

    // prologue: permutation, column maximum of column 0
    if (cta == 0) {
        for (int i = tid; i < N; i += blockDim.x) p.perm[i] = i;
        unsigned long long b = 0;
        int idx = 0x7fffffff;
        for (int i = 1 + tid; i < N; i += blockDim.x) argmax_combine(b, idx, absbits(__ldcg(p.buf0 + i)), i);
        block_argmax(b, idx, s_redb, s_redi);
        if (tid == 0) {
            p.slot_bits[0] = b;
            p.slot_idx[0] = idx == 0x7fffffff ? 0 : idx;
            __threadfence();
            atomicExch(p.pub, 1u);
        }
    }

    const double *cur = p.buf0;
    double *nxt = p.buf1;
    int step = 0;
    int npos = 0, nneg = 0, nzero = 0;
    int k = 0;
    while (k < N) {
        // The owner of column k+1 (the next pivot column unless this step takes
        // a 2x2 pivot or an interchange) prefetches its own, already final,
        // entries before waiting for the pivot data.
        constexpr int kPf = 4;
        double pf[kPf];
        const bool own_next = k + 1 < N && (unsigned)(k + 1) % nb == (unsigned)cta;
        if (own_next) {
#pragma unroll
            for (int u = 0; u < kPf; ++u) {
                const int i = k + 1 + tid + u * kBkThreads;
                pf[u] = i < N ? __ldcg(cur + i + (int64_t)(k + 1) * ld) : 0.0;
            }
        }
        // pivot data of this step (column k and its maximum) published by its owner
        if (!wait_published(p.pub, (unsigned)step + 1u, p.bar.err)) return;
        const double akk = __ldcg(cur + k + (int64_t)k * ld);
        const double absakk = fabs(akk);
        const double colmax = __longlong_as_double((long long)__ldcg(p.slot_bits + step));
        const int imax = __ldcg(p.slot_idx + step);
        // column k below the diagonal, loaded speculatively for the common
        // no-interchange 1x1 pivot (same round trip as the pivot value)
        for (int t = tid; t < N - k - 1; t += blockDim.x) c0[t] = __ldcg(cur + (k + 1 + t) + (int64_t)k * ld);
        int kstep = 1, kp = k;
        const bool rowtest = !(fmax(absakk, colmax) == 0.0 || absakk >= alpha * colmax);
        if (!rowtest) {
            kp = k;
        } else {
            // row r lies in every CTA's columns: all CTAs must have finished the
            // previous step before it is read
            if (!grid_barrier(p.bar, nb)) return;
            const int r = imax;
            // largest off-diagonal magnitude of row/column r in the trailing block
            unsigned long long b = 0;
            for (int t = tid; t < N - k - 1; t += blockDim.x) {
                const int idx = k + t;
                const double a = (idx < r) ? __ldcg(cur + r + (int64_t)idx * ld)
                                           : __ldcg(cur + (idx + 1) + (int64_t)r * ld);
                const unsigned long long ab = absbits(a);
                b = ab > b ? ab : b;
            }
            b = block_maxbits(b, s_redb);
            if (tid == 0) s_bcast = b;
            __syncthreads();
            const double rowmax = __longlong_as_double((long long)s_bcast);
            if (absakk >= alpha * colmax * (colmax / rowmax)) {
                kp = k;
            } else if (fabs(__ldcg(cur + r + (int64_t)r * ld)) >= alpha * rowmax) {
                kp = r;
            } else {
                kp = r;
                kstep = 2;
            }
        }
        const int kk = k + kstep - 1;
        // permuted read of the current trailing matrix (indices >= k)
        auto pi = [&](int i) { return i == kk ? kp : (i == kp ? kk : i); };
        auto get = [&](int i, int j) {
            int a = pi(i), b = pi(j);
            if (a < b) { int t = a; a = b; b = t; }
            return __ldcg(cur + a + (int64_t)b * ld);
        };
        const bool plain = kstep == 1 && kp == k;   // c0 already holds the pivot column
        const double d11 = plain ? akk : get(k, k);
        const double d21 = kstep == 2 ? get(k + 1, k) : 0.0;
        const double d22 = kstep == 2 ? get(k + 1, k + 1) : 0.0;
        const int base = k + kstep;
        const int len = N - base;
        if (!plain) {
            __syncthreads();
            for (int t = tid; t < len; t += blockDim.x) {
                c0[t] = get(base + t, k);
                if (kstep == 2) c1[t] = get(base + t, k + 1);
            }
        }
        __syncthreads();
        // with a row test the reads above may touch any CTA's columns: nobody
        // writes this buffer's columns again (next step) before all have read
        if (rowtest && !grid_barrier(p.bar, nb)) return;
        // D^-1 entries
        double e11, e21, e22;
        if (kstep == 1) {
            e11 = d11 != 0.0 ? 1.0 / d11 : 0.0;
            e21 = e22 = 0.0;
        } else {
            const double det = d11 * d22 - d21 * d21;
            e11 = d22 / det;
            e21 = -d21 / det;
            e22 = d11 / det;
        }
        // bookkeeping (CTA 0): D, kind, perm, inertia
        if (cta == 0 && tid == 0) {
            if (kstep == 1) {
                p.Dd[k] = d11;
                p.Doff[k] = 0.0;
                p.kind[k] = 1;
                if (d11 == 0.0 || fabs(d11) <= ztol) ++nzero;
                else if (d11 > 0.0) ++npos;
                else ++nneg;
            } else {
                p.Dd[k] = d11;
                p.Doff[k] = d21;
                p.Dd[k + 1] = d22;
                p.Doff[k + 1] = 0.0;
                p.kind[k] = 2;
                p.kind[k + 1] = 0;
                ++npos;
                ++nneg;
            }
            if (kp != kk) {
                const int t = p.perm[kk];
                p.perm[kk] = p.perm[kp];
                p.perm[kp] = t;
            }
        }
        // L columns k (and k+1): owner of column k
        if ((unsigned)k % nb == (unsigned)cta) {
            double *Lk = p.L + (int64_t)k * N;
            if (tid == 0) {
                Lk[k] = 1.0;
                if (kstep == 2) {
                    Lk[k + 1] = 0.0;
                    p.L[(k + 1) + (int64_t)(k + 1) * N] = 1.0;
                }
            }
            if (kstep == 1) {
                for (int t = tid; t < len; t += blockDim.x) Lk[base + t] = c0[t] * e11;
            } else {
                double *Lk1 = p.L + (int64_t)(k + 1) * N;
                for (int t = tid; t < len; t += blockDim.x) {
                    const double a = c0[t], b = c1[t];
                    Lk[base + t] = a * e11 + b * e21;
                    Lk1[base + t] = a * e21 + b * e22;
                }
            }
        }
        // interchange rows kk and kp of the finished columns of L
        if (kp != kk) {
            for (int j = cta; j < k; j += nb) {
                if (tid == 0) {
                    // written by another CTA in an earlier step: read through L2
                    double *Lj = p.L + (int64_t)j * N;
                    const double t = __ldcg(Lj + kk);
                    Lj[kk] = __ldcg(Lj + kp);
                    Lj[kp] = t;
                }
            }
        }
        // Trailing update of the owned columns.  In the trailing block
        // (indices >= base > kk) the interchange only maps row/column kp to kk.
        const double *__restrict__ C = cur;
        double *__restrict__ X = nxt;
        auto src = [&](int i, int j) -> const double * {
            const int a = (i == kp) ? kk : i;
            const int b = (j == kp) ? kk : j;
            return a >= b ? C + a + (int64_t)b * ld : C + b + (int64_t)a * ld;
        };
        const int j0 = base + (int)(((unsigned)cta + nb - (unsigned)(base % (int)nb)) % nb);
        // next pivot column: updated first, with its column maximum (integer compares)
        auto tracked = [&](int j) {
            const int tj = j - base;
            double *__restrict__ col = X + (int64_t)j * ld;
            const double f0 = kstep == 1 ? c0[tj] * e11 : c0[tj] * e11 + c1[tj] * e21;
            const double f1 = kstep == 1 ? 0.0 : c0[tj] * e21 + c1[tj] * e22;
            unsigned long long mb = 0;
            int mi = 0x7fffffff;
            int i = j + tid;
            if (plain && j == k + 1 && own_next) {
                // prefetched old values (no interchange: src(i, j) is column j itself)
#pragma unroll
                for (int u = 0; u < kPf; ++u, i += kBkThreads) {
                    if (i < N) {
                        const double v = fma(-c0[i - base], f0, pf[u]);
                        col[i] = v;
                        const unsigned long long ab = absbits(v);
                        if (i > j && ab > mb) {
                            mb = ab;
                            mi = i;
                        }
                    }
                }
            }
            for (; i < N; i += blockDim.x) {
                double v = fma(-c0[i - base], f0, __ldcg(src(i, j)));
                if (kstep == 2) v = fma(-c1[i - base], f1, v);
                col[i] = v;
                const unsigned long long ab = absbits(v);
                if (i > j && ab > mb) {
                    mb = ab;
                    mi = i;
                }
            }
            block_argmax(mb, mi, s_redb, s_redi);
            if (tid == 0) {
                p.slot_bits[step + 1] = mb;
                p.slot_idx[step + 1] = mi == 0x7fffffff ? j : mi;
                __threadfence();   // column j and the slot before the flag
                atomicExch(p.pub, (unsigned)step + 2u);
            }
        };
        if (kstep == 1 && kp == kk) {
            // common case: rank-1, no interchange; two columns (8 loads) in flight per thread
            int j = j0;
            if (j == base && j < N) {
                tracked(j);
                j += nb;
            }
            constexpr int T = kBkThreads;
            for (; j + (int)nb < N; j += 2 * nb) {
                const int j1 = j + nb;
                const double fa = c0[j - base] * e11, fb = c0[j1 - base] * e11;
                const double *__restrict__ sa = C + (int64_t)j * ld;
                const double *__restrict__ sb = C + (int64_t)j1 * ld;
                double *__restrict__ da = X + (int64_t)j * ld;
                double *__restrict__ db = X + (int64_t)j1 * ld;
                int ia = j + tid, ib = j1 + tid;
                for (; ib + 3 * T < N; ia += 4 * T, ib += 4 * T) {
                    const double a0 = __ldcg(sa + ia), a1 = __ldcg(sa + ia + T), a2 = __ldcg(sa + ia + 2 * T),
                                 a3 = __ldcg(sa + ia + 3 * T);
                    const double b0 = __ldcg(sb + ib), b1 = __ldcg(sb + ib + T), b2 = __ldcg(sb + ib + 2 * T),
                                 b3 = __ldcg(sb + ib + 3 * T);
                    da[ia] = fma(-c0[ia - base], fa, a0);
                    da[ia + T] = fma(-c0[ia + T - base], fa, a1);
                    da[ia + 2 * T] = fma(-c0[ia + 2 * T - base], fa, a2);
                    da[ia + 3 * T] = fma(-c0[ia + 3 * T - base], fa, a3);
                    db[ib] = fma(-c0[ib - base], fb, b0);
                    db[ib + T] = fma(-c0[ib + T - base], fb, b1);
                    db[ib + 2 * T] = fma(-c0[ib + 2 * T - base], fb, b2);
                    db[ib + 3 * T] = fma(-c0[ib + 3 * T - base], fb, b3);
                }
                for (; ia < N; ia += T) da[ia] = fma(-c0[ia - base], fa, __ldcg(sa + ia));
                for (; ib < N; ib += T) db[ib] = fma(-c0[ib - base], fb, __ldcg(sb + ib));
            }
            for (; j < N; j += nb) {
                const double f0 = c0[j - base] * e11;
                const double *__restrict__ scol = C + (int64_t)j * ld;
                double *__restrict__ col = X + (int64_t)j * ld;
                int i = j + tid;
                for (; i + 3 * T < N; i += 4 * T) {
                    const double v0 = __ldcg(scol + i), v1 = __ldcg(scol + i + T), v2 = __ldcg(scol + i + 2 * T),
                                 v3 = __ldcg(scol + i + 3 * T);
                    col[i] = fma(-c0[i - base], f0, v0);
                    col[i + T] = fma(-c0[i + T - base], f0, v1);
                    col[i + 2 * T] = fma(-c0[i + 2 * T - base], f0, v2);
                    col[i + 3 * T] = fma(-c0[i + 3 * T - base], f0, v3);
                }
                for (; i < N; i += T) col[i] = fma(-c0[i - base], f0, __ldcg(scol + i));
            }
        } else {
            for (int j = j0; j < N; j += nb) {
                if (j == base) {
                    tracked(j);
                    continue;
                }
                const int tj = j - base;
                double *__restrict__ col = X + (int64_t)j * ld;
                // new = old - [c0_i c1_i] D^-1 [c0_j c1_j]^T = old - c0_i f0 - c1_i f1
                const double f0 = kstep == 1 ? c0[tj] * e11 : c0[tj] * e11 + c1[tj] * e21;
                const double f1 = kstep == 1 ? 0.0 : c0[tj] * e21 + c1[tj] * e22;
                if (kstep == 1) {
                    int i = j + tid;
                    for (; i + kBkThreads < N; i += 2 * kBkThreads) {
                        const double v0 = __ldcg(src(i, j)), v1 = __ldcg(src(i + kBkThreads, j));
                        col[i] = fma(-c0[i - base], f0, v0);
                        col[i + kBkThreads] = fma(-c0[i + kBkThreads - base], f0, v1);
                    }
                    for (; i < N; i += kBkThreads) col[i] = fma(-c0[i - base], f0, __ldcg(src(i, j)));
                } else {
                    int i = j + tid;
                    for (; i + kBkThreads < N; i += 2 * kBkThreads) {
                        const double v0 = __ldcg(src(i, j)), v1 = __ldcg(src(i + kBkThreads, j));
                        col[i] = fma(-c1[i - base], f1, fma(-c0[i - base], f0, v0));
                        col[i + kBkThreads] =
                            fma(-c1[i + kBkThreads - base], f1, fma(-c0[i + kBkThreads - base], f0, v1));
                    }
                    for (; i < N; i += kBkThreads)
                        col[i] = fma(-c1[i - base], f1, fma(-c0[i - base], f0, __ldcg(src(i, j))));
                }
            }
        }
        const double *t = cur;
        cur = nxt;
        nxt = const_cast<double *>(t);
        ++step;
        k += kstep;
    }
    if (cta == 0 && tid == 0) {
        p.inertia[0] = npos;
        p.inertia[1] = nneg;
        p.inertia[2] = nzero;
    }
}

// ---------------------------------------------------------------------------
// Solve P^T L D L^T P x = b, one CTA per right-hand side, vector in shared
// memory; blocked by 32 columns (a warp solves each diagonal block).
// ---------------------------------------------------------------------------
constexpr int kSolveThreads = 1024;

__global__ void __launch_bounds__(kSolveThreads)
k_ldlt_solve(int N, const double *__restrict__ L, const double *__restrict__ Dd,
             const double *__restrict__ Doff, const int32_t *__restrict__ perm, double *B,
             int64_t ldb) {
    extern __shared__ double y[];
    double *b = B + (int64_t)blockIdx.x * ldb;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < N; i += blockDim.x) y[i] = b[perm[i]];
    __syncthreads();
    // forward: L y = P b
    for (int jb = 0; jb < N; jb += 32) {
        const int nbk = min(32, N - jb);
        if (wid == 0) {
            double yi = lane < nbk ? y[jb + lane] : 0.0;
            for (int j = 0; j < nbk; ++j) {
                const double yj = __shfl_sync(0xffffffffu, yi, j);
                if (lane > j && lane < nbk) yi -= L[(jb + lane) + (int64_t)(jb + j) * N] * yj;
            }
            if (lane < nbk) y[jb + lane] = yi;
        }
        __syncthreads();
        for (int i = jb + nbk + tid; i < N; i += blockDim.x) {
            double acc = 0.0;
            for (int j = 0; j < nbk; ++j) acc += L[i + (int64_t)(jb + j) * N] * y[jb + j];
            y[i] -= acc;
        }
        __syncthreads();
    }
    // block diagonal D
    for (int k = tid; k < N; k += blockDim.x) {
        const double off = Doff[k];
        if (off != 0.0) {
            const double a = Dd[k], c = Dd[k + 1];
            const double det = a * c - off * off;
            const double u = y[k], v = y[k + 1];
            y[k] = (c * u - off * v) / det;
            y[k + 1] = (a * v - off * u) / det;
        } else if (k == 0 || Doff[k - 1] == 0.0) {
            y[k] = y[k] / Dd[k];
        }
    }
    __syncthreads();
    // backward: L^T z = y
    const int nblk = (N + 31) / 32;
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int jb = bi * 32;
        const int nbk = min(32, N - jb);
        // y[j] -= sum_{i >= jb + nbk} L[i][j] y[i]   (warp per column j)
        if (wid < nbk) {
            const int j = jb + wid;
            double acc = 0.0;
            for (int i = jb + nbk + lane; i < N; i += 32) acc += L[i + (int64_t)j * N] * y[i];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) y[j] -= acc;
        }
        __syncthreads();
        if (wid == 0) {
            double yi = lane < nbk ? y[jb + lane] : 0.0;
            for (int j = nbk - 1; j >= 0; --j) {
                const double yj = __shfl_sync(0xffffffffu, yi, j);
                if (lane < j) yi -= L[(jb + j) + (int64_t)(jb + lane) * N] * yj;
            }
            if (lane < nbk) y[jb + lane] = yi;
        }
        __syncthreads();
    }
    for (int i = tid; i < N; i += blockDim.x) b[perm[i]] = y[i];
}

__global__ void k_maxabs_lower(int64_t N, const double *S, int64_t ld, double *partial) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int64_t j = blockIdx.x; j < N; j += gridDim.x)
        for (int64_t i = j + threadIdx.x; i < N; i += blockDim.x) v = fmax(v, fabs(S[i + j * ld]));
    v = block_max<kRedThreads>(v, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

}  // namespace

static constexpr size_t ldlt_unblocked_scratch_bytes(int64_t N) {
    // ping-pong buffer (N x N), then 64 bytes of barrier/flag words, then the
    // per-step pivot slots (N + 1 maxima and indices)
    const size_t b = (size_t)N * (size_t)N * sizeof(double) + 64 +
                     (size_t)(N + 1) * (sizeof(unsigned long long) + sizeof(int)) + 256;
    return (b + 255) / 256 * 256;  // callers place 8-byte data right after it
}

size_t ldlt_scratch_bytes(int64_t N) {
    // the unblocked kernel keeps 2 N doubles in shared memory: beyond that order
    // only the blocked scratch is ever used
    if (2 * (size_t)N * sizeof(double) > kMaxDynSmem) return ldlt_blocked_scratch_bytes(N);
    return std::max(ldlt_unblocked_scratch_bytes(N), ldlt_blocked_scratch_bytes(N));
}

void launch_maxabs_lower(cudaStream_t s, int64_t N, const double *S, int64_t ld, double *partial,
                         double *out) {
    k_maxabs_lower<<<kRedBlocks, kRedThreads, 0, s>>>(N, S, ld, partial);
    MDSIP_LAUNCHED();
    launch_finalize_max(s, partial, 1, out);
}

// S: lower triangle with leading dimension ld, overwritten.  scratch:
// ldlt_scratch_bytes(N) bytes of device memory.  err_dev: device int set to 1
// when a bounded wait expires (must be 0 on entry).
static void launch_ldlt_unblocked(cudaStream_t s, int num_sms, int64_t N, const double *S, int64_t ld,
                                  const double *maxabs_dev, double zero_tol, LdltOut out, void *scratch,
                                  int *err_dev) {
    if (N <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out.inertia, 0, 3 * sizeof(int32_t), s));
        return;
    }
    char *w = static_cast<char *>(scratch);
    MDSIP_REQUIRE((reinterpret_cast<uintptr_t>(w) & 255) == 0, MDSIP_ERR_INVALID_ARG, "ldlt: misaligned scratch");
    BKParams p{};
    p.N = (int)N;
    p.buf0 = const_cast<double *>(S);
    p.buf1 = reinterpret_cast<double *>(w);
    // the ping-pong copy uses the leading dimension N
    MDSIP_REQUIRE(ld == N, MDSIP_ERR_INVALID_ARG, "ldlt: leading dimension must equal N");
    p.ld = ld;
    char *tail = w + (size_t)N * (size_t)N * sizeof(double);
    p.bar.count = reinterpret_cast<unsigned int *>(tail);
    p.bar.gen = reinterpret_cast<unsigned int *>(tail + 4);
    p.pub = reinterpret_cast<unsigned int *>(tail + 8);
    p.bar.err = err_dev;
    MDSIP_CUDA(cudaMemsetAsync(tail, 0, 64, s));
    p.slot_bits = reinterpret_cast<unsigned long long *>(tail + 64);
    p.slot_idx = reinterpret_cast<int *>(tail + 64 + (size_t)(N + 1) * sizeof(unsigned long long));
    p.L = out.L;
    p.Dd = out.Dd;
    p.Doff = out.Doff;
    p.perm = out.perm;
    p.kind = out.kind;
    p.inertia = out.inertia;
    p.maxabs = maxabs_dev;
    p.zero_tol = zero_tol;

    const size_t smem = 2 * (size_t)N * sizeof(double);
    MDSIP_REQUIRE(smem <= kMaxDynSmem, MDSIP_ERR_INVALID_ARG, "ldlt: N too large for this kernel");
    // The attribute is global to the kernel: set once to the bound every launch
    // respects (launches of different N may run concurrently from several threads).
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(k_bk_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    }));
    int per_sm = 0;
    MDSIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bk_factor, kBkThreads, smem));
    MDSIP_REQUIRE(per_sm >= 1, MDSIP_ERR_INVALID_ARG, "ldlt: kernel does not fit on an SM");
    int grid = (int)std::min<int64_t>((int64_t)num_sms * per_sm, std::min<int64_t>(num_sms, std::max<int64_t>(1, N / 12)));
    void *args[] = {&p};
    MDSIP_CUDA(cudaLaunchCooperativeKernel((const void *)k_bk_factor, dim3(grid), dim3(kBkThreads),
                                           args, smem, s));
    count_launch();
}

// The factorization of the Newton step: the blocked kernels (ldlt_blocked.cu)
// when this device can run their thread-block cluster, else the unblocked
// persistent kernel.  fp32_update: trailing products of the blocked form in
// FP32 (refined mixed-precision path).
void launch_ldlt(cudaStream_t s, int num_sms, int64_t N, const double *S, int64_t ld,
                 const double *maxabs_dev, double zero_tol, LdltOut out, void *scratch,
                 int *err_dev, bool fp32_update, int nb, int spec) {
    if (N > 0 && ld == N && (ldlt_blocked_available(N) || ldlt_persistent_path(N, spec))) {
        launch_ldlt_blocked(s, num_sms, N, const_cast<double *>(S), maxabs_dev, zero_tol, out, scratch,
                            fp32_update, nb, spec);
        return;
    }
    launch_ldlt_unblocked(s, num_sms, N, S, ld, maxabs_dev, zero_tol, out, scratch, err_dev);
}

void launch_ldlt_solve(cudaStream_t s, int64_t N, const double *L, const double *Dd,
                       const double *Doff, const int32_t *perm, int64_t nrhs, double *B,
                       int64_t ldb) {
    if (N <= 0 || nrhs <= 0) return;
    const size_t smem = (size_t)N * sizeof(double);
    MDSIP_REQUIRE(smem <= kMaxDynSmem, MDSIP_ERR_INVALID_ARG, "ldlt_solve: N too large");
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(k_ldlt_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    }));
    k_ldlt_solve<<<(unsigned)nrhs, kSolveThreads, smem, s>>>((int)N, L, Dd, Doff, perm, B, ldb);
    MDSIP_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the factorization.
//
// Some callers cannot call cudaMalloc: a host whose device memory is owned in
// full by another allocator (a framework's caching allocator, a pre-sized
// arena of a real-time controller), or a loop that must not pay the implicit
// device synchronisation that allocating and freeing can cause.  For them
// the factorization's scratch (the ping-pong copy of the trailing matrix, the
// pivot hand-off slots, the barrier words, the error flag and the reduction
// partials of the zero-pivot scale) lives in this fixed device array, which
// every GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocMaxN = 1024;
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxN * kNoAllocMaxN * sizeof(double) + 16384;
// the layout below: [factor scratch, rounded up to 256 | error flag (256) |
// kRedBlocks partials | max |S|], for the largest accepted order
static_assert(ldlt_unblocked_scratch_bytes(kNoAllocMaxN) + 256 + (size_t)(kRedBlocks + 1) * sizeof(double) <=
                  kNoAllocBytes,
              "fixed scratch too small for the factorization's layout");
static __device__ __align__(256) unsigned char g_ldlt_fixed_scratch[kNoAllocBytes];

namespace {
std::mutex g_fixed_mu;
void *g_fixed_addr[256] = {};  // device address of the array, per device ordinal
}  // namespace

// Host-side address of the fixed array on `device` (which must be current).
// The array's name in host code is only a stand-in; the device address comes
// from cudaGetSymbolAddress, looked up once per device and kept for the
// process: after cudaDeviceReset (which unloads the module with the array)
// the kept address is stale, so the entry point must not be called again in
// that process.
static void *fixed_scratch_address(int device) {
    MDSIP_REQUIRE(device >= 0 && device < 256, MDSIP_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_fixed_mu);
    if (!g_fixed_addr[device]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_ldlt_fixed_scratch);
        MDSIP_REQUIRE(e == cudaSuccess && ptr != nullptr, MDSIP_ERR_CUDA,
                      std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_fixed_addr[device] = ptr;
    }
    return g_fixed_addr[device];
}

int64_t ldlt_fixed_scratch_max_n() { return kNoAllocMaxN; }

void ldlt_factor_fixed_scratch(cudaStream_t s, int device, int num_sms, int64_t N, double *S,
                               int64_t ld, double zero_tol, LdltOut out) {
    MDSIP_REQUIRE(N >= 0 && ld == N, MDSIP_ERR_INVALID_ARG, "ldlt: need ld == N");
    MDSIP_REQUIRE(N <= kNoAllocMaxN, MDSIP_ERR_INVALID_ARG,
                  "ldlt (fixed scratch): N exceeds the limit of 1024");
    MDSIP_REQUIRE(out.inertia, MDSIP_ERR_INVALID_ARG, "ldlt: null inertia");
    if (N == 0) {
        MDSIP_CUDA(cudaMemsetAsync(out.inertia, 0, 3 * sizeof(int32_t), s));
        return;
    }
    MDSIP_REQUIRE(S && out.L && out.Dd && out.Doff && out.perm && out.kind, MDSIP_ERR_INVALID_ARG,
                  "ldlt: null pointer");
    char *base = static_cast<char *>(fixed_scratch_address(device));
    // layout: [unblocked factor scratch | error flag | partials | max |S|]
    const size_t fs = ldlt_unblocked_scratch_bytes(N);
    int *err = reinterpret_cast<int *>(base + fs);
    double *partial = reinterpret_cast<double *>(base + fs + 256);
    double *maxabs = partial + kRedBlocks;
    MDSIP_REQUIRE(((reinterpret_cast<uintptr_t>(partial) | reinterpret_cast<uintptr_t>(base)) & 255) == 0,
                  MDSIP_ERR_INVALID_ARG, "ldlt (fixed scratch): misaligned layout");
    // every call shares the array: clear what must start at zero (the factor
    // launch clears its own slots and barrier words)
    MDSIP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    launch_maxabs_lower(s, N, S, ld, partial, maxabs);
    launch_ldlt_unblocked(s, num_sms, N, S, ld, maxabs, zero_tol, out, base, err);
    int herr = 0;
    MDSIP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MDSIP_CUDA(cudaStreamSynchronize(s));
    MDSIP_REQUIRE(herr == 0, MDSIP_ERR_DEVICE, "ldlt: a bounded device wait expired");
}

}  // namespace mdsip
