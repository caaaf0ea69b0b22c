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
#include "tc.cuh"

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

__global__ void k_round_vector(const double *__restrict__ v, int64_t n, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)v[i];
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
// One CTA of 512 threads per SM.  Rows stream through shared memory in
// batches of kBR rows (a 2048-column slice of A_hi and of A_lo per row, by
// bulk asynchronous copies into a kBS-stage ring completed on mbarriers), so
// the copies of the next batches are in flight while the current one is
// computed.  Thread t owns columns 4t .. 4t + 3 of each slice (16 warps per
// SM: the double-float arithmetic, not the memory, sets the pace, and it
// needs the warps for its dependent chains); the per-thread row sums of a
// batch are reduced over the block as double-float pairs (warp shuffles,
// then one slot per warp).  Waits are bounded: on expiry the kernel sets
// *err and stops.  The fused form (kFuse, one slice) also takes the first
// half of the refinement's next approximate solve: each finished row sum
// gives v_i (BothNext), and A_hi^T v accumulates in FP32 one batch behind,
// from the previous batch's A_hi chunk kept in registers (its stage is
// already being refilled), so the batch keeps its single barrier.
constexpr int kBothThreads = 512;
constexpr int kBothCols = 4 * kBothThreads;   // columns per slice
constexpr int kBR = 4;                        // rows per stage
constexpr int kBS = 3;                        // stages
constexpr size_t kBothSmem = (size_t)kBS * kBR * 2 * kBothCols * sizeof(float) + 256;
__device__ __forceinline__ void df_add(float &s, float &c, float s2, float c2) {
    const float t = s + s2, bb = t - s;
    const float e = (s - (t - bb)) + (s2 - bb);
    s = t;
    c = c + c2 + e;
}
// df_acc on two lanes at once with the packed FP32 instructions (each lane
// rounded exactly as the scalar form; a - b as fma(b, -1, a))
__device__ __forceinline__ void df_acc2(float2 ah, float2 al, float2 xh, float2 xl, float2 &s, float2 &c) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 p = __fmul2_rn(ah, xh);
    const float2 pe = __ffma2_rn(ah, xh, __fmul2_rn(p, m1));           // exact error of the product
    const float2 sm = __ffma2_rn(ah, xl, __ffma2_rn(al, xh, pe));       // the small terms
    const float2 t = __fadd2_rn(s, p);                                  // two-sum: s + p = t + e
    const float2 bb = __ffma2_rn(s, m1, t);
    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, t), m1, s), __ffma2_rn(bb, m1, p));
    s = t;
    c = __fadd2_rn(c, __fadd2_rn(e, sm));
}
// Operands of the fused form, which also takes the first half of the next
// approximate solve: from the row sum (A x)_i = s + c (double-float) it forms
// v_i = fl32(bt_i wf_i), bt_i = (cw_i.x + cw_i.y) - (s + c) in double-float
// (cw = cpre split into FP32 halves, wf = fl32(winv)), and accumulates
// A_hi^T v in FP32 into vpart (one row of n per block).  One slice only
// (n <= kBothCols): v_i needs the whole row.
struct BothNext {
    const float2 *cw;
    const float *wf;
    double *vpart;
};
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}
template <bool kFuse>
__global__ void __launch_bounds__(kBothThreads, 1)
    k_gemv_both_df(const float *__restrict__ Ahi, const float *__restrict__ Alo, int64_t m, int64_t n, int64_t lda,
                   const float2 *__restrict__ xs, const float2 *__restrict__ ys, double *__restrict__ out,
                   double *__restrict__ partial, int *err, BothNext nx) {
    extern __shared__ __align__(128) unsigned char bsm[];
    float *ring = reinterpret_cast<float *>(bsm);   // [kBS][kBR][2][kBothCols]
    uint64_t *full = reinterpret_cast<uint64_t *>(bsm + (size_t)kBS * kBR * 2 * kBothCols * sizeof(float));
    constexpr int kW = kBothThreads / 32;
    __shared__ float2 red[2][kBR][kW];   // [batch parity][row][warp]
    __shared__ float4 s_v[2];            // fused form: v of the batch's kBR rows, [batch parity]
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(m, r0 + rows_per);
    const int nbat = r1 > r0 ? (int)((r1 - r0 + kBR - 1) / kBR) : 0;
    if (tid == 0) {
        for (int st = 0; st < kBS; ++st) tc::mbar_init(&full[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_stop = 0;
        s_v[0] = s_v[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    int gb = 0;   // batches issued/consumed over all slices (stage and phase)
    int parity = 0;
    for (int64_t cp = 0; cp < n; cp += kBothCols) {
        const uint32_t width = (uint32_t)min((int64_t)kBothCols, lda - cp);   // a multiple of 4 floats
        // thread 0 fills stage (gb + b) % kBS with batch b of this slice
        auto issue = [&](int b) {
            const int st = (gb + b) % kBS;
            uint32_t bytes = 0;
            for (int rr = 0; rr < kBR; ++rr)
                if (r0 + (int64_t)b * kBR + rr < r1) bytes += 2 * width * (uint32_t)sizeof(float);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_expect_tx(&full[st], bytes);
            for (int rr = 0; rr < kBR; ++rr) {
                const int64_t i = r0 + (int64_t)b * kBR + rr;
                if (i >= r1) break;
                float *dst = ring + ((size_t)st * kBR + rr) * 2 * kBothCols;
                bulk_g2s(dst, Ahi + i * lda + cp, width * (uint32_t)sizeof(float), &full[st]);
                bulk_g2s(dst + kBothCols, Alo + i * lda + cp, width * (uint32_t)sizeof(float), &full[st]);
            }
        };
        if (tid == 0)
            for (int b = 0; b < min(kBS, nbat); ++b) issue(b);
        // this thread's chunk: inside the copied width whenever it starts below n
        // (lda is a multiple of 4), with A's padding columns n .. lda - 1 zero
        const int64_t p0 = cp + 4 * tid;
        const bool on = p0 < n;
        float xh[4], xl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 x = (p0 + q < n) ? xs[p0 + q] : make_float2(0.0f, 0.0f);
            xh[q] = x.x;
            xl[q] = x.y;
        }
        // column sums: a double-float pair per 16 rows, added into a second
        // pair, which goes into FP64 every 256 rows (the FP64 pipe runs at
        // 1/64 of the FP32 rate)
        float cs[4], cc[4], CS[4], CC[4];
        double cacc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cs[q] = cc[q] = CS[q] = CC[q] = 0.0f;
            cacc[q] = 0.0;
        }
        // fused form: A_hi^T v in FP32, v known one batch late (after the
        // batch's row sums), so each batch's A_hi chunk is kept for one batch
        // (a chunk array only ever holds A_hi values or zero: a row past the
        // block's end keeps a stale chunk, which meets v = 0)
        float2 cv01 = make_float2(0.0f, 0.0f), cv23 = make_float2(0.0f, 0.0f);
        float4 ahA[kBR], ahB[kBR];   // fused form: A_hi chunks of alternate batches
#pragma unroll
        for (int rr = 0; rr < kBR; ++rr) ahA[rr] = ahB[rr] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int cnt = 0, cnt2 = 0;
        // one batch: its chunk into cur, the previous batch's chunk in prev;
        // true when a bounded wait expired (every thread then stops)
        auto batch = [&](int b, float4(&cur)[kBR], float4(&prev)[kBR]) -> bool {
            const int st = (gb + b) % kBS;
            const uint32_t ph = (uint32_t)(((gb + b) / kBS) & 1);
            const int64_t i0 = r0 + (int64_t)b * kBR;
            // fused form: the row's cw and wf, loaded now so that their
            // latency passes under the batch's products
            [[maybe_unused]] float2 cw_i = make_float2(0.0f, 0.0f);
            [[maybe_unused]] float wf_i = 0.0f;
            if constexpr (kFuse) {
                if (tid < kBR && i0 + tid < r1) {
                    cw_i = nx.cw[i0 + tid];
                    wf_i = nx.wf[i0 + tid];
                }
            }
            if (!tc::mbar_wait(&full[st], ph)) {   // bounded; every thread stops at the barrier below
                atomicExch(err, 1);
                s_stop = 1;
            }
            float rs[kBR], rc[kBR];
#pragma unroll
            for (int rr = 0; rr < kBR; ++rr) {
                rs[rr] = rc[rr] = 0.0f;
                if (!on || i0 + rr >= r1) continue;
                const float2 y = ys[i0 + rr];
                const float2 yh = make_float2(y.x, y.x), yl = make_float2(y.y, y.y);
                const float *row = ring + ((size_t)st * kBR + rr) * 2 * kBothCols;
                const float4 ah = *reinterpret_cast<const float4 *>(row + 4 * tid);
                const float4 al = *reinterpret_cast<const float4 *>(row + kBothCols + 4 * tid);
                if constexpr (kFuse) cur[rr] = ah;
                // columns (0, 1) and (2, 3) as lane pairs: the row sum in two
                // partial pairs, the column sums in their own pairs
                float2 rsp = make_float2(0.0f, 0.0f), rcp = make_float2(0.0f, 0.0f);
                df_acc2(make_float2(ah.x, ah.y), make_float2(al.x, al.y), make_float2(xh[0], xh[1]),
                        make_float2(xl[0], xl[1]), rsp, rcp);
                df_acc2(make_float2(ah.z, ah.w), make_float2(al.z, al.w), make_float2(xh[2], xh[3]),
                        make_float2(xl[2], xl[3]), rsp, rcp);
                float2 c01s = make_float2(cs[0], cs[1]), c01c = make_float2(cc[0], cc[1]);
                float2 c23s = make_float2(cs[2], cs[3]), c23c = make_float2(cc[2], cc[3]);
                df_acc2(make_float2(ah.x, ah.y), make_float2(al.x, al.y), yh, yl, c01s, c01c);
                df_acc2(make_float2(ah.z, ah.w), make_float2(al.z, al.w), yh, yl, c23s, c23c);
                cs[0] = c01s.x;
                cs[1] = c01s.y;
                cs[2] = c23s.x;
                cs[3] = c23s.y;
                cc[0] = c01c.x;
                cc[1] = c01c.y;
                cc[2] = c23c.x;
                cc[3] = c23c.y;
                rs[rr] = rsp.x;
                rc[rr] = rcp.x;
                df_add(rs[rr], rc[rr], rsp.y, rcp.y);
            }
            if (++cnt == 4) {   // every 16 rows
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    df_add(CS[q], CC[q], cs[q], cc[q]);
                    cs[q] = cc[q] = 0.0f;
                }
                cnt = 0;
                if (++cnt2 == 16) {   // every 256 rows
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        cacc[q] += (double)CS[q];
                        cacc[q] += (double)CC[q];
                        CS[q] = CC[q] = 0.0f;
                    }
                    cnt2 = 0;
                }
            }
            // the four row sums over the warp by halving exchanges: after the
            // xor-16 and xor-8 steps each lane holds one row (row 2 bit4 +
            // bit3 of the lane), summed over its 8 lanes by three more steps
            {
                static_assert(kBR == 4, "the exchange below is written for four rows");
                const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
                float sa = u16 ? rs[0] : rs[2], ca = u16 ? rc[0] : rc[2];
                float sb = u16 ? rs[1] : rs[3], cb = u16 ? rc[1] : rc[3];
                float ka = u16 ? rs[2] : rs[0], kc = u16 ? rc[2] : rc[0];
                float kb = u16 ? rs[3] : rs[1], kd = u16 ? rc[3] : rc[1];
                sa = __shfl_xor_sync(0xffffffffu, sa, 16);
                ca = __shfl_xor_sync(0xffffffffu, ca, 16);
                sb = __shfl_xor_sync(0xffffffffu, sb, 16);
                cb = __shfl_xor_sync(0xffffffffu, cb, 16);
                df_add(ka, kc, sa, ca);   // row 0 (lower half) or 2 (upper)
                df_add(kb, kd, sb, cb);   // row 1 or 3
                float ss = u8 ? ka : kb, sc = u8 ? kc : kd;
                float vs = u8 ? kb : ka, vc = u8 ? kd : kc;
                ss = __shfl_xor_sync(0xffffffffu, ss, 8);
                sc = __shfl_xor_sync(0xffffffffu, sc, 8);
                df_add(vs, vc, ss, sc);
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {
                    const float s2 = __shfl_xor_sync(0xffffffffu, vs, o);
                    const float c2 = __shfl_xor_sync(0xffffffffu, vc, o);
                    df_add(vs, vc, s2, c2);
                }
                if ((lane & 7) == 0) red[parity][2 * (lane >> 4) + ((lane >> 3) & 1)][wid] = make_float2(vs, vc);
            }
            __syncthreads();   // the stage is consumed, the batch's row sums are in red
            if (s_stop) return true;
            if (tid == 0 && b + kBS < nbat) issue(b + kBS);
            if constexpr (kFuse) {   // the previous batch's v is in s_v[parity ^ 1]
                const float4 v4 = s_v[parity ^ 1];
                const float vr[kBR] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int rr = 0; rr < kBR; ++rr) {
                    const float2 v2 = make_float2(vr[rr], vr[rr]);
                    cv01 = __ffma2_rn(make_float2(prev[rr].x, prev[rr].y), v2, cv01);
                    cv23 = __ffma2_rn(make_float2(prev[rr].z, prev[rr].w), v2, cv23);
                }
            }
            if (tid < kBR) {
                [[maybe_unused]] float vf = 0.0f;
                if (i0 + tid < r1) {
                    float s = 0.0f, c = 0.0f;
#pragma unroll
                    for (int w = 0; w < kW; ++w) df_add(s, c, red[parity][tid][w].x, red[parity][tid][w].y);
                    const double v = (double)s + (double)c;
                    out[i0 + tid] = cp == 0 ? v : out[i0 + tid] + v;
                    if constexpr (kFuse) {   // one slice: (s, c) is the whole row sum
                        float bs = cw_i.x, bc = cw_i.y;
                        df_add(bs, bc, -s, -c);
                        vf = (bs + bc) * wf_i;
                    }
                }
                if constexpr (kFuse) reinterpret_cast<float *>(&s_v[parity])[tid] = vf;
            }
            parity ^= 1;   // the other slot set next batch: one barrier per batch
            return false;
        };
        bool stopped = false;
        if constexpr (kFuse) {   // two batches per trip: the chunk arrays swap roles without copies
            int b = 0;
            for (; b + 1 < nbat && !stopped; b += 2) stopped = batch(b, ahA, ahB) || batch(b + 1, ahB, ahA);
            if (!stopped && b < nbat) stopped = batch(b, ahA, ahB);
        } else {
            for (int b = 0; b < nbat && !stopped; ++b) stopped = batch(b, ahA, ahB);
        }
        if constexpr (kFuse) {   // the last batch's v
            __syncthreads();
            if (!s_stop && nbat > 0) {   // the last batch's chunk: ahA for an even index, ahB for odd
                const bool odd = ((nbat - 1) & 1) != 0;
                const float4 v4 = s_v[parity ^ 1];
                const float vr[kBR] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int rr = 0; rr < kBR; ++rr) {
                    const float4 a = odd ? ahB[rr] : ahA[rr];
                    const float2 v2 = make_float2(vr[rr], vr[rr]);
                    cv01 = __ffma2_rn(make_float2(a.x, a.y), v2, cv01);
                    cv23 = __ffma2_rn(make_float2(a.z, a.w), v2, cv23);
                }
            }
        }
        if (s_stop) return;
        gb += nbat;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t c = p0 + q;
            if (c < n) {
                partial[(size_t)blockIdx.x * n + c] =
                    cacc[q] + (double)CS[q] + (double)CC[q] + (double)cs[q] + (double)cc[q];
                if constexpr (kFuse) {
                    const float cvq = q == 0 ? cv01.x : q == 1 ? cv01.y : q == 2 ? cv23.x : cv23.y;
                    nx.vpart[(size_t)blockIdx.x * n + c] = (double)cvq;
                }
            }
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

bool gemv_both_fusable(int64_t n) { return n > 0 && n <= kBothCols; }

// out_rows = A x, out_cols = A^T y in one pass (double-float); xs: n float2,
// ys: m float2 of scratch; partial: kRedBlocks x n doubles (at most two rows
// per SM are used); err: device int set to 1 when a bounded wait expires.
// With nx (cw non-null; gemv_both_fusable(n)) the same pass also writes
// out_v = A_hi^T v (FP32 products and block sums, see BothNext).
void launch_gemv_both_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                         const double *x, const double *y, float2 *xs, float2 *ys, double *partial,
                         double *out_rows, double *out_cols, int *err, const BothNextArgs *nx) {
    const bool fuse = nx != nullptr && nx->cw != nullptr;
    MDSIP_REQUIRE(!fuse || gemv_both_fusable(n), MDSIP_ERR_INVALID_ARG,
                  "gemv (double-float, fused): n must be in 1 .. 2048");
    if (n <= 0) {
        if (m > 0) MDSIP_CUDA(cudaMemsetAsync(out_rows, 0, m * sizeof(double), s));
        return;
    }
    if (m <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out_cols, 0, n * sizeof(double), s));
        if (fuse) MDSIP_CUDA(cudaMemsetAsync(nx->out_v, 0, n * sizeof(double), s));
        return;
    }
    MDSIP_REQUIRE((lda & 3) == 0 && ((reinterpret_cast<uintptr_t>(Ahi) | reinterpret_cast<uintptr_t>(Alo)) & 15) == 0,
                  MDSIP_ERR_INVALID_ARG, "gemv (double-float): rows of A must be 16-byte aligned");
    k_split_vector<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (n + NT - 1) / NT)), NT, 0, s>>>(x, n, xs);
    MDSIP_LAUNCHED();
    k_split_vector<<<(unsigned)std::min<int64_t>(4096, (m + NT - 1) / NT), NT, 0, s>>>(y, m, ys);
    MDSIP_LAUNCHED();
    // one CTA per SM (the staging ring takes most of the shared memory)
    int dev = 0, sms = 0;
    MDSIP_CUDA(cudaGetDevice(&dev));
    MDSIP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(sms, kRedBlocks / 2));   // rows grid .. 2 grid - 1: A_hi^T v
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        cudaError_t e = cudaFuncSetAttribute(k_gemv_both_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kBothSmem);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_gemv_both_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kBothSmem);
    }));
    if (fuse) {
        double *vpart = partial + (size_t)grid * n;
        k_gemv_both_df<true><<<grid, kBothThreads, kBothSmem, s>>>(Ahi, Alo, m, n, lda, xs, ys, out_rows, partial,
                                                                   err, BothNext{nx->cw, nx->wf, vpart});
        MDSIP_LAUNCHED();
        launch_colsum(s, vpart, grid, n, nx->out_v);
    } else {
        k_gemv_both_df<false><<<grid, kBothThreads, kBothSmem, s>>>(Ahi, Alo, m, n, lda, xs, ys, out_rows, partial,
                                                                    err, BothNext{});
        MDSIP_LAUNCHED();
    }
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

void launch_split_vector(cudaStream_t s, const double *v, int64_t n, float2 *out) {
    if (n <= 0) return;
    k_split_vector<<<(unsigned)std::min<int64_t>(4096, (n + NT - 1) / NT), NT, 0, s>>>(v, n, out);
    MDSIP_LAUNCHED();
}

void launch_round_vector(cudaStream_t s, const double *v, int64_t n, float *out) {
    if (n <= 0) return;
    k_round_vector<<<(unsigned)std::min<int64_t>(4096, (n + NT - 1) / NT), NT, 0, s>>>(v, n, out);
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
