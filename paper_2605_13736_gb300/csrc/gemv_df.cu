// Passes over the dense Jacobian block A in double-float arithmetic.
//
// On GB300 an FP64 pass over A (2 flop per 8 bytes) is bound by the FP64
// FMA rate, 1/64 of the FP32 rate, before HBM.  Here A is kept a second
// time as two FP32 arrays, A = A_hi + A_lo (A_hi = fl32(A), A_lo =
// fl32(A - A_hi), 8 bytes per entry like FP64, exact to 2^-48 relative), the
// vector likewise, and every product is formed on the FP32 pipes:
//
//   a x = a_hi x_hi + (a_hi x_lo + a_lo x_hi) + O(2^-48 |a x|),
//
// a_hi x_hi exactly as p + e (p = fl(a_hi x_hi), e = fma(a_hi, x_hi, -p)),
// accumulated with Knuth's two-sum into a double-float (s, c); each thread
// folds its (s, c) into an FP64 sum every 16 terms.  The error per 16-term
// block is a few 2^-48 of its sum of |terms|, so the result has the accuracy
// of an FP64 dot product (whose rounding is n 2^-53 of the sum of |terms|);
// the FP64 instructions left are two conversions and two additions per 16
// terms, and the pass is bound by reading A_hi and A_lo from HBM.
//
// The iterative refinement of the mixed-precision path and that path's
// constraint and gradient passes use these; the plain FP64 path keeps FP64.
#include "internal.cuh"

namespace mdsip {

namespace {

constexpr int NT = 256;

// (s, c) += a x in double-float, a = (ah, al), x = (xh, xl)
__device__ __forceinline__ void df_acc(float ah, float al, float xh, float xl, float &s, float &c) {
    const float p = ah * xh;
    const float pe = fmaf(ah, xh, -p);                 // exact error of the product
    const float sm = fmaf(ah, xl, fmaf(al, xh, pe));   // the small terms (al xl dropped: 2^-48)
    const float t = s + p;                             // two-sum (Knuth): s + p = t + e exactly
    const float bb = t - s;
    const float e = (s - (t - bb)) + (p - bb);
    s = t;
    c += e + sm;
}

// rows by block, columns by thread; the padding columns n .. lda - 1 become zeros
__global__ void k_split_matrix(const double *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                               float *__restrict__ hi, float *__restrict__ lo) {
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const double *row = A + i * lda;
        float *rh = hi + i * lda, *rl = lo + i * lda;
        for (int64_t c = threadIdx.x; c < lda; c += blockDim.x) {
            const double a = c < n ? __ldcs(row + c) : 0.0;
            const float h = (float)a;
            rh[c] = h;
            rl[c] = (float)(a - (double)h);
        }
    }
}

__global__ void k_split_vector(const double *__restrict__ v, int64_t n, float2 *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = v[i];
        const float h = (float)a;
        out[i] = make_float2(h, (float)(a - (double)h));
    }
}

// out[i] = sum_p A[i][p] x[p]: two threads per row, each taking alternate
// 16-byte chunks of A_hi and A_lo; x (split) staged in shared memory
__global__ void __launch_bounds__(NT) k_gemv_rows_df(const float *__restrict__ Ahi, const float *__restrict__ Alo,
                                                     int64_t m, int64_t n, int64_t lda,
                                                     const float2 *__restrict__ xs, double *__restrict__ out) {
    extern __shared__ float2 xsh[];    // n rounded up to a multiple of 16, zero padded
    const int64_t n16 = (n + 15) / 16 * 16;
    for (int64_t k = threadIdx.x; k < n16; k += NT) xsh[k] = k < n ? xs[k] : make_float2(0.0f, 0.0f);
    __syncthreads();
    const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t i = gt >> 1;
    const int h = (int)(gt & 1);
    const bool live = i < m;
    const float4 *rh = reinterpret_cast<const float4 *>(Ahi + (live ? i : 0) * lda);
    const float4 *rl = reinterpret_cast<const float4 *>(Alo + (live ? i : 0) * lda);
    double acc = 0.0;
    float s = 0.0f, c = 0.0f;
    const int64_t full = live ? n / 16 : 0;   // groups of 16 columns: 4 chunks, 2 per thread
    for (int64_t g = 0; g < full; ++g) {
        float4 ah[2], al[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            ah[u] = __ldg(rh + 4 * g + h + 2 * u);
            al[u] = __ldg(rl + 4 * g + h + 2 * u);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t col = 16 * g + 4 * (h + 2 * u);
            float2 x;
            x = xsh[col + 0]; df_acc(ah[u].x, al[u].x, x.x, x.y, s, c);
            x = xsh[col + 1]; df_acc(ah[u].y, al[u].y, x.x, x.y, s, c);
            x = xsh[col + 2]; df_acc(ah[u].z, al[u].z, x.x, x.y, s, c);
            x = xsh[col + 3]; df_acc(ah[u].w, al[u].w, x.x, x.y, s, c);
        }
        if (g & 1) {   // every 16 terms of this thread
            acc += (double)s;
            acc += (double)c;
            s = c = 0.0f;
        }
    }
    if (live && h == 0) {
        const float *rhs = Ahi + i * lda, *rls = Alo + i * lda;
        for (int64_t col = 16 * full; col < n; ++col) {   // ragged tail (fewer than 16 columns)
            const float2 x = xsh[col];
            df_acc(rhs[col], rls[col], x.x, x.y, s, c);
        }
    }
    acc += (double)s;
    acc += (double)c;
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);   // the pair's halves (every lane reaches this)
    if (live && h == 0) out[i] = acc;
}

// partial[b][p] = sum over the rows of block b of A[i][p] y[i] (y split)
constexpr int kCols = 8;   // columns per thread per pass
__global__ void __launch_bounds__(NT) k_gemv_t_df(const float *__restrict__ Ahi, const float *__restrict__ Alo,
                                                  int64_t m, int64_t n, int64_t lda,
                                                  const float2 *__restrict__ ys, double *__restrict__ partial) {
    const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(m, r0 + rows_per);
    for (int64_t c0 = 0; c0 < n; c0 += (int64_t)NT * kCols) {
        float s[kCols], cc[kCols];
        double acc[kCols];
#pragma unroll
        for (int q = 0; q < kCols; ++q) {
            s[q] = cc[q] = 0.0f;
            acc[q] = 0.0;
        }
        int cnt = 0;
        for (int64_t i = r0; i < r1; ++i) {
            const float2 y = ys[i];
            const float *rh = Ahi + i * lda, *rl = Alo + i * lda;
            float ah[kCols], al[kCols];
#pragma unroll
            for (int q = 0; q < kCols; ++q) {
                const int64_t p = c0 + threadIdx.x + (int64_t)q * NT;
                ah[q] = p < n ? __ldg(rh + p) : 0.0f;
                al[q] = p < n ? __ldg(rl + p) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < kCols; ++q) df_acc(ah[q], al[q], y.x, y.y, s[q], cc[q]);
            if (++cnt == 16) {
#pragma unroll
                for (int q = 0; q < kCols; ++q) {
                    acc[q] += (double)s[q];
                    acc[q] += (double)cc[q];
                    s[q] = cc[q] = 0.0f;
                }
                cnt = 0;
            }
        }
#pragma unroll
        for (int q = 0; q < kCols; ++q) {
            const int64_t p = c0 + threadIdx.x + (int64_t)q * NT;
            if (p < n) partial[(size_t)blockIdx.x * n + p] = acc[q] + (double)s[q] + (double)cc[q];
        }
    }
}

// Both products of the residual in one read of A: out[i] = sum_p A[i][p] x[p]
// for this block's rows and partial[b][p] = sum_{i of block b} A[i][p] y[i].
// Thread t owns columns 4t .. 4t + 3 and 1024 + 4t .. 1024 + 4t + 3 of each
// 2048-column pass (16-byte loads of A_hi and A_lo); rows go in batches of
// eight, whose per-thread row sums are reduced over the block as
// double-float pairs (warp shuffles, then one slot per warp).
constexpr int kBothCols = 8 * NT;   // columns per pass
__device__ __forceinline__ void df_add(float &s, float &c, float s2, float c2) {
    const float t = s + s2, bb = t - s;
    const float e = (s - (t - bb)) + (s2 - bb);
    s = t;
    c = c + c2 + e;
}
__global__ void __launch_bounds__(NT, 1) k_gemv_both_df(const float *__restrict__ Ahi, const float *__restrict__ Alo,
                                                     int64_t m, int64_t n, int64_t lda,
                                                     const float2 *__restrict__ xs, const float2 *__restrict__ ys,
                                                     double *__restrict__ out, double *__restrict__ partial) {
    __shared__ float2 red[2][8][NT / 32];   // [batch parity][row][warp]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(m, r0 + rows_per);
    int parity = 0;
    for (int64_t cp = 0; cp < n; cp += kBothCols) {
        int64_t p[2];
        bool on[2];
        float xh[8], xl[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            p[h] = cp + 4 * tid + (int64_t)h * (kBothCols / 2);
            on[h] = p[h] < n && p[h] < lda;   // lda is a multiple of 4: the 16-byte chunk stays in the row
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 x = (p[h] + q < n) ? xs[p[h] + q] : make_float2(0.0f, 0.0f);
                xh[4 * h + q] = x.x;
                xl[4 * h + q] = x.y;
            }
        }
        float cs[8], cc[8];
        double cacc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            cs[q] = cc[q] = 0.0f;
            cacc[q] = 0.0;
        }
        int cnt = 0;
        for (int64_t i0 = r0; i0 < r1; i0 += 8) {
            // all 32 16-byte loads of the batch in flight before the arithmetic
            float4 ah[8][2], al[8][2];
            float2 y[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const int64_t i = i0 + rr;
                const bool live = i < r1;
                y[rr] = live ? ys[i] : make_float2(0.0f, 0.0f);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    ah[rr][h] = al[rr][h] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (live && on[h]) {
                        ah[rr][h] = __ldcs(reinterpret_cast<const float4 *>(Ahi + i * lda + p[h]));
                        al[rr][h] = __ldcs(reinterpret_cast<const float4 *>(Alo + i * lda + p[h]));
                    }
                }
            }
            float rs[8], rc[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                rs[rr] = rc[rr] = 0.0f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float a_h[4] = {ah[rr][h].x, ah[rr][h].y, ah[rr][h].z, ah[rr][h].w};
                    const float a_l[4] = {al[rr][h].x, al[rr][h].y, al[rr][h].z, al[rr][h].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {   // zero entries (dead rows, columns past n) add nothing
                        df_acc(a_h[q], a_l[q], xh[4 * h + q], xl[4 * h + q], rs[rr], rc[rr]);
                        df_acc(a_h[q], a_l[q], y[rr].x, y[rr].y, cs[4 * h + q], cc[4 * h + q]);
                    }
                }
            }
            if (++cnt == 2) {   // every 16 rows: the column sums into FP64
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    cacc[q] += (double)cs[q];
                    cacc[q] += (double)cc[q];
                    cs[q] = cc[q] = 0.0f;
                }
                cnt = 0;
            }
            // the eight row sums over the block
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, rs[rr], o);
                    const float c2 = __shfl_xor_sync(0xffffffffu, rc[rr], o);
                    df_add(rs[rr], rc[rr], s2, c2);
                }
                if (lane == 0) red[parity][rr][wid] = make_float2(rs[rr], rc[rr]);
            }
            __syncthreads();
            if (tid < 8 && i0 + tid < r1) {
                float s = 0.0f, c = 0.0f;
#pragma unroll
                for (int w = 0; w < NT / 32; ++w) df_add(s, c, red[parity][tid][w].x, red[parity][tid][w].y);
                const double v = (double)s + (double)c;
                out[i0 + tid] = cp == 0 ? v : out[i0 + tid] + v;
            }
            parity ^= 1;   // the other slot set next batch: one barrier per batch
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t c = p[h] + q;
                if (c < n) partial[(size_t)blockIdx.x * n + c] = cacc[4 * h + q] + (double)cs[4 * h + q] + (double)cc[4 * h + q];
            }
    }
}

// out[i] = sum_p A_hi[i][p] x[p] in FP32 (the approximate solves' product)
__global__ void __launch_bounds__(NT) k_gemv_rows_f32(const float *__restrict__ Ahi, int64_t m, int64_t n,
                                                      int64_t lda, const double *__restrict__ x,
                                                      double *__restrict__ out) {
    extern __shared__ float xf[];   // n rounded up to a multiple of 8, zero padded
    const int64_t n8 = (n + 7) / 8 * 8;
    for (int64_t k = threadIdx.x; k < n8; k += NT) xf[k] = k < n ? (float)x[k] : 0.0f;
    __syncthreads();
    const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t i = gt >> 1;
    const int h = (int)(gt & 1);
    const bool live = i < m;
    const float4 *rh = reinterpret_cast<const float4 *>(Ahi + (live ? i : 0) * lda);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int64_t full = live ? n / 8 : 0;   // groups of 8 columns: 2 chunks, 1 per thread
#pragma unroll 4
    for (int64_t g = 0; g < full; ++g) {
        const float4 a = __ldcs(rh + 2 * g + h);
        const int64_t col = 8 * g + 4 * h;
        acc[0] = fmaf(a.x, xf[col + 0], acc[0]);
        acc[1] = fmaf(a.y, xf[col + 1], acc[1]);
        acc[2] = fmaf(a.z, xf[col + 2], acc[2]);
        acc[3] = fmaf(a.w, xf[col + 3], acc[3]);
    }
    if (live && h == 0)
        for (int64_t col = 8 * full; col < n; ++col) acc[0] = fmaf(Ahi[i * lda + col], xf[col], acc[0]);
    float s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (live && h == 0) out[i] = (double)s;
}

}  // namespace

// out_rows = A x, out_cols = A^T y in one pass (double-float); xs: n float2,
// ys: m float2 of scratch; partial: kRedBlocks x n doubles (at most one row
// per SM is used)
void launch_gemv_both_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                         const double *x, const double *y, float2 *xs, float2 *ys, double *partial,
                         double *out_rows, double *out_cols) {
    if (n <= 0) {
        if (m > 0) MDSIP_CUDA(cudaMemsetAsync(out_rows, 0, m * sizeof(double), s));
        return;
    }
    if (m <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out_cols, 0, n * sizeof(double), s));
        return;
    }
    MDSIP_REQUIRE((lda & 3) == 0 && ((reinterpret_cast<uintptr_t>(Ahi) | reinterpret_cast<uintptr_t>(Alo)) & 15) == 0,
                  MDSIP_ERR_INVALID_ARG, "gemv (double-float): rows of A must be 16-byte aligned");
    k_split_vector<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (n + NT - 1) / NT)), NT, 0, s>>>(x, n, xs);
    MDSIP_LAUNCHED();
    k_split_vector<<<(unsigned)std::min<int64_t>(4096, (m + NT - 1) / NT), NT, 0, s>>>(y, m, ys);
    MDSIP_LAUNCHED();
    // one CTA per SM (the batch's loads take most of the registers)
    int dev = 0, sms = 0;
    MDSIP_CUDA(cudaGetDevice(&dev));
    MDSIP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(sms, kRedBlocks));
    k_gemv_both_df<<<grid, NT, 0, s>>>(Ahi, Alo, m, n, lda, xs, ys, out_rows, partial);
    MDSIP_LAUNCHED();
    launch_colsum(s, partial, grid, n, out_cols);
}

// out = A_hi x with FP32 products and sums (approximate solves)
void launch_gemv_rows_f32(cudaStream_t s, const float *Ahi, int64_t m, int64_t n, int64_t lda, const double *x,
                          double *out) {
    if (m <= 0) return;
    MDSIP_REQUIRE((lda & 3) == 0 && (reinterpret_cast<uintptr_t>(Ahi) & 15) == 0, MDSIP_ERR_INVALID_ARG,
                  "gemv (FP32): rows of A must be 16-byte aligned");
    const size_t smem = (size_t)((n + 7) / 8) * 8 * sizeof(float);
    MDSIP_REQUIRE(smem <= 192 * 1024, MDSIP_ERR_INVALID_ARG, "gemv (FP32): n too large");
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(k_gemv_rows_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 * 1024);
    }));
    const int64_t grid = (2 * m + NT - 1) / NT;
    MDSIP_REQUIRE(grid <= 0x7fffffff, MDSIP_ERR_INVALID_ARG, "gemv (FP32): m too large");
    k_gemv_rows_f32<<<(unsigned)grid, NT, smem, s>>>(Ahi, m, n, lda, x, out);
    MDSIP_LAUNCHED();
}

void launch_split_matrix(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda, float *hi,
                         float *lo) {
    if (m <= 0 || lda <= 0) return;
    k_split_matrix<<<(unsigned)std::min<int64_t>(65535, m), NT, 0, s>>>(A, m, n, lda, hi, lo);
    MDSIP_LAUNCHED();
}

// out = A x; xs: scratch of n float2
void launch_gemv_rows_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                         const double *x, float2 *xs, double *out) {
    if (m <= 0) return;
    MDSIP_REQUIRE((lda & 3) == 0 && ((reinterpret_cast<uintptr_t>(Ahi) | reinterpret_cast<uintptr_t>(Alo)) & 15) == 0,
                  MDSIP_ERR_INVALID_ARG, "gemv (double-float): rows of A must be 16-byte aligned");
    const size_t smem = (size_t)((n + 15) / 16) * 16 * sizeof(float2);
    MDSIP_REQUIRE(smem <= 192 * 1024, MDSIP_ERR_INVALID_ARG, "gemv (double-float): n too large");
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(k_gemv_rows_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 * 1024);
    }));
    if (n > 0) {
        k_split_vector<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (n + NT - 1) / NT)), NT, 0, s>>>(
            x, n, xs);
        MDSIP_LAUNCHED();
    }
    const int64_t grid = (2 * m + NT - 1) / NT;   // two threads per row
    MDSIP_REQUIRE(grid <= 0x7fffffff, MDSIP_ERR_INVALID_ARG, "gemv (double-float): m too large");
    k_gemv_rows_df<<<(unsigned)grid, NT, smem, s>>>(Ahi, Alo, m, n, lda, xs, out);
    MDSIP_LAUNCHED();
}

// out = A^T y; ys: scratch of m float2; partial: kRedBlocks x n doubles
void launch_gemv_t_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                      const double *y, float2 *ys, double *partial, double *out) {
    if (n <= 0) return;
    if (m <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out, 0, n * sizeof(double), s));
        return;
    }
    k_split_vector<<<(unsigned)std::min<int64_t>(4096, (m + NT - 1) / NT), NT, 0, s>>>(y, m, ys);
    MDSIP_LAUNCHED();
    k_gemv_t_df<<<kRedBlocks, NT, 0, s>>>(Ahi, Alo, m, n, lda, ys, partial);
    MDSIP_LAUNCHED();
    launch_colsum(s, partial, kRedBlocks, n, out);
}

}  // namespace mdsip
