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
//  * the CTA that owns the next pivot column computes its column maximum
//    while updating it, so each pivot step costs exactly one grid barrier;
//  * the barrier's wait is bounded (error flag instead of a hang);
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

struct BKParams {
    int N;
    int64_t ld;
    double *buf0, *buf1;           // ping-pong copies of the trailing matrix (lower, ld)
    double *L, *Dd, *Doff;
    int32_t *perm, *kind, *inertia;
    unsigned long long *slot_bits; // [2] |.| bit pattern of the next pivot column's maximum
    int *slot_idx;                 // [2] its row index
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
        }
    }
    if (!grid_barrier(p.bar, nb)) return;

    const double *cur = p.buf0;
    double *nxt = p.buf1;
    int parity = 0;
    int npos = 0, nneg = 0, nzero = 0;
    int k = 0;
    while (k < N) {
        const double akk = __ldcg(cur + k + (int64_t)k * ld);
        const double absakk = fabs(akk);
        const double colmax = __longlong_as_double((long long)__ldcg(p.slot_bits + parity));
        const int imax = __ldcg(p.slot_idx + parity);
        int kstep = 1, kp = k;
        if (fmax(absakk, colmax) == 0.0 || absakk >= alpha * colmax) {
            kp = k;
        } else {
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
        const double d11 = get(k, k);
        const double d21 = kstep == 2 ? get(k + 1, k) : 0.0;
        const double d22 = kstep == 2 ? get(k + 1, k + 1) : 0.0;
        const int base = k + kstep;
        const int len = N - base;
        for (int t = tid; t < len; t += blockDim.x) {
            c0[t] = get(base + t, k);
            if (kstep == 2) c1[t] = get(base + t, k + 1);
        }
        __syncthreads();
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
        for (int j = j0; j < N; j += nb) {
            const int tj = j - base;
            double *__restrict__ col = X + (int64_t)j * ld;
            // new = old - [c0_i c1_i] D^-1 [c0_j c1_j]^T = old - c0_i f0 - c1_i f1
            const double f0 = kstep == 1 ? c0[tj] * e11 : c0[tj] * e11 + c1[tj] * e21;
            const double f1 = kstep == 1 ? 0.0 : c0[tj] * e21 + c1[tj] * e22;
            const bool simple_col = (j != kp) || kp == kk;
            if (j == base) {
                // next pivot column: also its column maximum (integer compares)
                unsigned long long mb = 0;
                int mi = 0x7fffffff;
                for (int i = j + tid; i < N; i += blockDim.x) {
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
                    p.slot_bits[parity ^ 1] = mb;
                    p.slot_idx[parity ^ 1] = mi == 0x7fffffff ? j : mi;
                }
            } else if (kstep == 1 && simple_col && kp == kk) {
                // common case: no interchange, rank-1, four loads in flight per thread
                const double *__restrict__ scol = C + (int64_t)j * ld;
                int i = j + tid;
                for (; i + 3 * kBkThreads < N; i += 4 * kBkThreads) {
                    const double v0 = __ldcg(scol + i), v1 = __ldcg(scol + i + kBkThreads),
                                 v2 = __ldcg(scol + i + 2 * kBkThreads), v3 = __ldcg(scol + i + 3 * kBkThreads);
                    col[i] = fma(-c0[i - base], f0, v0);
                    col[i + kBkThreads] = fma(-c0[i + kBkThreads - base], f0, v1);
                    col[i + 2 * kBkThreads] = fma(-c0[i + 2 * kBkThreads - base], f0, v2);
                    col[i + 3 * kBkThreads] = fma(-c0[i + 3 * kBkThreads - base], f0, v3);
                }
                for (; i < N; i += kBkThreads) col[i] = fma(-c0[i - base], f0, __ldcg(scol + i));
            } else if (kstep == 1) {
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
                    col[i + kBkThreads] = fma(-c1[i + kBkThreads - base], f1, fma(-c0[i + kBkThreads - base], f0, v1));
                }
                for (; i < N; i += kBkThreads)
                    col[i] = fma(-c1[i - base], f1, fma(-c0[i - base], f0, __ldcg(src(i, j))));
            }
        }
        if (!grid_barrier(p.bar, nb)) return;
        const double *t = cur;
        cur = nxt;
        nxt = const_cast<double *>(t);
        parity ^= 1;
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

size_t ldlt_scratch_bytes(int64_t N) {
    // ping-pong buffer (N x N), slots, barrier words
    return (size_t)N * (size_t)N * sizeof(double) + 256;
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
void launch_ldlt(cudaStream_t s, int num_sms, int64_t N, const double *S, int64_t ld,
                 const double *maxabs_dev, double zero_tol, LdltOut out, void *scratch,
                 int *err_dev) {
    if (N <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out.inertia, 0, 3 * sizeof(int32_t), s));
        return;
    }
    char *w = static_cast<char *>(scratch);
    BKParams p{};
    p.N = (int)N;
    p.buf0 = const_cast<double *>(S);
    p.buf1 = reinterpret_cast<double *>(w);
    // the ping-pong copy uses the leading dimension N
    MDSIP_REQUIRE(ld == N, MDSIP_ERR_INVALID_ARG, "ldlt: leading dimension must equal N");
    p.ld = ld;
    char *tail = w + (size_t)N * (size_t)N * sizeof(double);
    p.slot_bits = reinterpret_cast<unsigned long long *>(tail);
    p.slot_idx = reinterpret_cast<int *>(tail + 16);
    p.bar.count = reinterpret_cast<unsigned int *>(tail + 32);
    p.bar.gen = reinterpret_cast<unsigned int *>(tail + 36);
    p.bar.err = err_dev;
    MDSIP_CUDA(cudaMemsetAsync(tail, 0, 64, s));
    p.L = out.L;
    p.Dd = out.Dd;
    p.Doff = out.Doff;
    p.perm = out.perm;
    p.kind = out.kind;
    p.inertia = out.inertia;
    p.maxabs = maxabs_dev;
    p.zero_tol = zero_tol;

    const size_t smem = 2 * (size_t)N * sizeof(double);
    MDSIP_REQUIRE(smem <= 200 * 1024, MDSIP_ERR_INVALID_ARG, "ldlt: N too large for this kernel");
    MDSIP_CUDA(cudaFuncSetAttribute(k_bk_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    int per_sm = 0;
    MDSIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bk_factor, kBkThreads, smem));
    MDSIP_REQUIRE(per_sm >= 1, MDSIP_ERR_INVALID_ARG, "ldlt: kernel does not fit on an SM");
    int grid = (int)std::min<int64_t>((int64_t)num_sms * per_sm, std::min<int64_t>(num_sms, std::max<int64_t>(1, N / 12)));
    void *args[] = {&p};
    MDSIP_CUDA(cudaLaunchCooperativeKernel((const void *)k_bk_factor, dim3(grid), dim3(kBkThreads),
                                           args, smem, s));
    count_launch();
}

void launch_ldlt_solve(cudaStream_t s, int64_t N, const double *L, const double *Dd,
                       const double *Doff, const int32_t *perm, int64_t nrhs, double *B,
                       int64_t ldb) {
    if (N <= 0 || nrhs <= 0) return;
    const size_t smem = (size_t)N * sizeof(double);
    MDSIP_REQUIRE(smem <= 200 * 1024, MDSIP_ERR_INVALID_ARG, "ldlt_solve: N too large");
    MDSIP_CUDA(cudaFuncSetAttribute(k_ldlt_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
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
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxN * kNoAllocMaxN * sizeof(double) + 4096;
static __device__ __align__(256) unsigned char g_ldlt_fixed_scratch[kNoAllocBytes];

namespace {
std::mutex g_fixed_mu;
void *g_fixed_addr[256] = {};  // device address of the array, per device ordinal
}  // namespace

// Host-side address of the fixed array on `device` (which must be current).
// The array's name in host code is only a stand-in; the device address comes
// from cudaGetSymbolAddress, looked up once per device.
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
    // layout: [factor scratch | error flag | partials | max |S|]
    const size_t fs = ldlt_scratch_bytes(N);
    int *err = reinterpret_cast<int *>(base + fs);
    double *partial = reinterpret_cast<double *>(base + fs + 256);
    double *maxabs = partial + kRedBlocks;
    // every call shares the array: clear what must start at zero (the factor
    // launch clears its own slots and barrier words)
    MDSIP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    launch_maxabs_lower(s, N, S, ld, partial, maxabs);
    launch_ldlt(s, num_sms, N, S, ld, maxabs, zero_tol, out, base, err);
    int herr = 0;
    MDSIP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MDSIP_CUDA(cudaStreamSynchronize(s));
    MDSIP_REQUIRE(herr == 0, MDSIP_ERR_DEVICE, "ldlt: a bounded device wait expired");
}

}  // namespace mdsip
