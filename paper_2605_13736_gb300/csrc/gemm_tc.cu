// BF16 GEMM on the 5th-generation tensor cores for the warm-start network:
//
//     C[m][n] = sum_k A[m][k] B[n][k]          (FP32 accumulation)
//
// with A (M x K) and B (N x K) both K-major in BF16, C FP32 row-major.  Every
// layer of the network, forward and backward, is this one contraction with
// the operands stored in the needed orientation (the producers write
// transposed copies alongside).
//
// One CTA computes a 128 x 128 tile over one K range: warp 0 lane 0 streams
// 64-element K slabs of A and B by TMA (128-byte swizzle, out-of-range rows
// and columns read as zero) into a 3-stage ring, warp 1 lane 0 issues
// tcgen05.mma into a 128-column FP32 accumulator in tensor memory, and the
// four warps move the accumulator out with tcgen05.ld.  When the tile grid is
// smaller than the GPU, K is split and the partial tiles are summed in a
// fixed order by a second kernel.  Waits are bounded and raise an error flag.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"
#include "tc.cuh"

namespace mdsip {

namespace {

constexpr int G_TILE = 128;
constexpr int G_THREADS = 128;
constexpr int G_STAGES = 3;
constexpr int G_SLAB = 64;                       // BF16 elements (128 bytes) of K per stage
constexpr int G_TILE_BYTES = G_TILE * G_SLAB * 2;
constexpr uint32_t G_TMEM_COLS = 128;
constexpr size_t kGemmSmemBytes = 1024 + 2 * G_STAGES * G_TILE_BYTES + 256;

struct GemmArgs {
    int64_t M, N;
    int total_slabs, slabs_per_split;
    float *out;       // nsplit == 1: C; else partials [split][M][N]
    int64_t ldo;
    int64_t split_stride;
    int *err;
};

__global__ void __launch_bounds__(G_THREADS, 2)
    k_gemm_bf16(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap, GemmArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + G_STAGES * G_TILE_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 2 * G_STAGES * G_TILE_BYTES);
    uint64_t *empty = full + G_STAGES;
    uint64_t *accum = empty + G_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * G_TILE, m0 = blockIdx.y * G_TILE;
    const int split = blockIdx.z;
    const int s0 = split * a.slabs_per_split;
    const int nslab = max(0, min(a.total_slabs, s0 + a.slabs_per_split) - s0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < G_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bmap)) : "memory");
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, G_TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        for (int it = 0; it < nslab; ++it) {
            const int st = it % G_STAGES, rnd = it / G_STAGES;
            if (!tc::mbar_wait(&empty[st], (rnd & 1) ^ 1)) {
                atomicExch(a.err, 1);
                break;
            }
            tc::mbar_expect_tx(&full[st], 2 * G_TILE_BYTES);
            const int kx = (s0 + it) * G_SLAB;
            tc::tma_load_2d(sA + st * G_TILE_BYTES, &amap, &full[st], kx, m0);
            tc::tma_load_2d(sB + st * G_TILE_BYTES, &bmap, &full[st], kx, n0);
        }
    } else if (warp == 1 && lane == 0) {
        for (int it = 0; it < nslab; ++it) {
            const int st = it % G_STAGES, rnd = it / G_STAGES;
            if (!tc::mbar_wait(&full[st], rnd & 1)) {
                atomicExch(a.err, 1);
                break;
            }
            tc::fence_after();
            const uint32_t ab = tc::smem_u32(sA + st * G_TILE_BYTES), bb = tc::smem_u32(sB + st * G_TILE_BYTES);
#pragma unroll
            for (int k = 0; k < 4; ++k)   // four K steps of 16 elements (32 bytes)
                tc::mma<false, tc::instr_desc(false, G_TILE, G_TILE)>(tmem, tc::sw128_kmajor_desc(ab + 32 * k),
                                                                      tc::sw128_kmajor_desc(bb + 32 * k),
                                                                      (it > 0 || k > 0) ? 1u : 0u);
            tc::commit(&empty[st]);
        }
        tc::commit(accum);
    }
    __syncwarp();
    const bool ok = nslab == 0 || tc::mbar_wait(accum, 0);
    tc::fence_after();
    if (!ok) atomicExch(a.err, 1);
    float *out = a.out + (size_t)split * a.split_stride;
    const int64_t m = m0 + warp * 32 + lane;   // TMEM lane = tile row
    const bool vec = (a.ldo % 4 == 0) && (reinterpret_cast<uintptr_t>(a.out) % 16 == 0);
#pragma unroll 1
    for (int c = 0; c < G_TILE / 32; ++c) {
        const int64_t nb = n0 + 32 * c;
        if (nb >= a.N) break;   // uniform across the CTA
        uint32_t r[32];
        if (ok && nslab > 0) {
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) r[j] = 0u;
        }
        if (m >= a.M) continue;
        float *row = out + m * a.ldo + nb;
        if (vec && nb + 32 <= a.N) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4 *>(row + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                                   __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (nb + j < a.N) row[j] = __uint_as_float(r[j]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, G_TMEM_COLS);
}

// ---------------------------------------------------------------------------
// M <= 256 and many column tiles (the network's output layer, M = batch):
// persistent CTAs, one per SM, each walking its 128-column tiles of C.  Per
// tile one tcgen05.mma of shape 128 x 256 per K step computes the transposed
// tile C^T[n][m] = sum_k B[n][k] A[m][k] (B's rows as the instruction's A
// operand, all 256 rows of A as its B operand), so every slab of B is read
// once from HBM and A (at most 256 x K) is re-read from L2.  Warp roles:
// warp 0 lane 0 streams K slabs by TMA into a 4-stage ring; warp 1 lane 0
// issues the MMAs into one of two 256-column TMEM accumulators; warps 4-7
// drain the other accumulator (TMEM lane = column n of C, so each store of a
// warp writes 32 consecutive floats of one row of C) while the next tile
// accumulates.  Waits are bounded and raise the error flag.
constexpr int W_THREADS = 256;
constexpr int W_STAGES = 4;
constexpr int W_BN = 128;                          // columns of C per tile (rows of B)
constexpr int W_BM = 256;                          // rows of C (A) held per tile
constexpr int W_B_BYTES = W_BN * G_SLAB * 2;       // 16 KB
constexpr int W_A_BYTES = W_BM * G_SLAB * 2;       // 32 KB
constexpr uint32_t W_TMEM_COLS = 512;              // two 256-column accumulators
constexpr size_t kGemmWideSmemBytes = 1024 + (size_t)W_STAGES * (W_A_BYTES + W_B_BYTES) + 256;

struct GemmWideArgs {
    int64_t M, N;
    int ntiles, nslab;
    float *C;
    int64_t ldc;
    int *err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(W_THREADS, 1)
    k_gemm_bf16_wide(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                     GemmWideArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;                                  // [stage][256 rows][64 K]
    uint8_t *sB = smem + W_STAGES * W_A_BYTES;           // [stage][128 rows][64 K]
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + W_STAGES * W_B_BYTES);
    uint64_t *empty = full + W_STAGES;
    uint64_t *tfull = empty + W_STAGES;                  // [2]: accumulator ready for the epilogue
    uint64_t *tempty = tfull + 2;                        // [2]: accumulator drained
    uint64_t *done = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < W_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 4);   // one arrival per epilogue warp
        }
        tc::mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bmap)) : "memory");
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, W_TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {   // producer
        int it = 0;
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
            for (int ks = 0; ks < a.nslab; ++ks, ++it) {
                const int st = it % W_STAGES, rnd = it / W_STAGES;
                if (!tc::mbar_wait(&empty[st], (rnd & 1) ^ 1)) {
                    ok = false;
                    break;
                }
                tc::mbar_expect_tx(&full[st], W_A_BYTES + W_B_BYTES);
                tc::tma_load_2d(sA + st * W_A_BYTES, &amap, &full[st], ks * G_SLAB, 0);
                tc::tma_load_2d(sB + st * W_B_BYTES, &bmap, &full[st], ks * G_SLAB, t * W_BN);
            }
        }
    } else if (warp == 1 && lane == 0) {   // MMA issuer
        int it = 0, tl = 0;
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tl) {
            const int b = tl & 1, use = tl >> 1;
            if (!tc::mbar_wait(&tempty[b], (use & 1) ^ 1)) {
                ok = false;
                break;
            }
            tc::fence_after();
            const uint32_t acc = tmem + (uint32_t)(b * W_BM);
            for (int ks = 0; ks < a.nslab; ++ks, ++it) {
                const int st = it % W_STAGES, rnd = it / W_STAGES;
                if (!tc::mbar_wait(&full[st], rnd & 1)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const uint32_t ab = tc::smem_u32(sB + st * W_B_BYTES), bb = tc::smem_u32(sA + st * W_A_BYTES);
#pragma unroll
                for (int k = 0; k < 4; ++k)   // four K steps of 16 elements (32 bytes)
                    tc::mma<false, tc::instr_desc(false, W_BN, W_BM)>(acc, tc::sw128_kmajor_desc(ab + 32 * k),
                                                                      tc::sw128_kmajor_desc(bb + 32 * k),
                                                                      (ks > 0 || k > 0) ? 1u : 0u);
                tc::commit(&empty[st]);
            }
            if (!ok) break;
            tc::commit(&tfull[b]);
        }
        tc::commit(done);   // every MMA this CTA issued has completed when `done` flips
        if (!tc::mbar_wait(done, 0)) ok = false;
    } else if (warp >= 4) {   // epilogue: TMEM lanes 32 q .. 32 q + 31 = columns n of the tile
        const int q = warp & 3;
        int tl = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++tl) {
            const int b = tl & 1, use = tl >> 1;
            if (!tc::mbar_wait(&tfull[b], use & 1)) {
                ok = false;
                break;
            }
            tc::fence_after();
            const int64_t n = (int64_t)t * W_BN + 32 * q + lane;
#pragma unroll 1
            for (int c = 0; c < W_BM / 32; ++c) {
                const int64_t m0 = 32 * c;
                if (m0 >= a.M) break;   // uniform across the warp
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * W_BM + 32 * c), r);
                if (n < a.N) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (m0 + j < a.M) a.C[(m0 + j) * a.ldc + n] = __uint_as_float(r[j]);
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    if (!ok) atomicExch(a.err, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, W_TMEM_COLS);
}

// C[m][n] = sum_s part[s][m][n]  (fixed order)
__global__ void k_gemm_reduce(int64_t M, int64_t N, int nsplit, const float *__restrict__ part, float *__restrict__ C,
                              int64_t ldc) {
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * total + e];
        C[(e / N) * ldc + e % N] = s;
    }
}

struct GemmPlan {
    int64_t tm, tn;
    int total_slabs, nsplit, slabs_per_split;
};

GemmPlan gemm_plan(int64_t M, int64_t N, int64_t K, int num_sms) {
    GemmPlan p{};
    p.tm = (M + G_TILE - 1) / G_TILE;
    p.tn = (N + G_TILE - 1) / G_TILE;
    p.total_slabs = (int)((K + G_SLAB - 1) / G_SLAB);
    const int64_t tiles = p.tm * p.tn;
    int s = 1;
    if (tiles < 2LL * num_sms && p.total_slabs >= 8)
        s = (int)std::min<int64_t>((2LL * num_sms + tiles - 1) / tiles, p.total_slabs / 4);
    s = std::max(1, s);
    p.slabs_per_split = (p.total_slabs + s - 1) / s;
    p.nsplit = p.slabs_per_split > 0 ? (p.total_slabs + p.slabs_per_split - 1) / p.slabs_per_split : 1;
    p.nsplit = std::max(1, p.nsplit);
    return p;
}

// the persistent wide-M kernel: all rows of A in one tile, at least one
// column tile per SM, K of at least one slab
bool gemm_wide(int64_t M, int64_t N, int64_t K, int num_sms) {
    return M <= W_BM && K >= 1 && (N + W_BN - 1) / W_BN >= num_sms && (N + W_BN - 1) / W_BN < (1LL << 31);
}

}  // namespace

size_t gemm_bf16_ws_bytes(int64_t M, int64_t N, int64_t K, int num_sms) {
    if (gemm_wide(M, N, K, num_sms)) return 0;
    const GemmPlan p = gemm_plan(M, N, K, num_sms);
    return p.nsplit > 1 ? (size_t)p.nsplit * M * N * sizeof(float) : 0;
}

// C = A B^T.  A: M x K BF16 (row stride lda elements), B: N x K BF16 (ldb);
// both 16-byte aligned with lda, ldb multiples of 8.  C: FP32, row stride ldc.
// ws: gemm_bf16_ws_bytes(M, N, K, num_sms) bytes.  err_dev: device int.
void launch_gemm_bf16(cudaStream_t s, int num_sms, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                      int64_t ldb, int64_t M, int64_t N, int64_t K, float *C, int64_t ldc, void *ws, int *err_dev) {
    if (M <= 0 || N <= 0) return;
    MDSIP_REQUIRE(K >= 0 && lda >= K && ldb >= K && ldc >= N, MDSIP_ERR_INVALID_ARG, "gemm: bad leading dimension");
    MDSIP_REQUIRE(M < (1LL << 31) / G_TILE * G_TILE && N < (1LL << 31) / G_TILE * G_TILE, MDSIP_ERR_INVALID_ARG,
                  "gemm: dimension too large");
    const GemmPlan p = gemm_plan(M, N, K, num_sms);
    MDSIP_REQUIRE(p.tm <= 65535, MDSIP_ERR_INVALID_ARG, "gemm: M too large");
    if (gemm_wide(M, N, K, num_sms)) {
        CUtensorMap amap, bmap;
        tc::encode_2d(&amap, A, false, (uint64_t)K, (uint64_t)M, (uint64_t)std::max<int64_t>(lda, 8), G_SLAB, W_BM);
        tc::encode_2d(&bmap, B, false, (uint64_t)K, (uint64_t)N, (uint64_t)std::max<int64_t>(ldb, 8), G_SLAB, W_BN);
        GemmWideArgs wa{};
        wa.M = M;
        wa.N = N;
        wa.ntiles = (int)((N + W_BN - 1) / W_BN);
        wa.nslab = (int)((K + G_SLAB - 1) / G_SLAB);
        wa.C = C;
        wa.ldc = ldc;
        wa.err = err_dev;
        static PerDeviceOnce once_w;
        MDSIP_CUDA(once_w.run([] {
            return cudaFuncSetAttribute(k_gemm_bf16_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kGemmWideSmemBytes);
        }));
        const int grid = std::min(wa.ntiles, num_sms);
        k_gemm_bf16_wide<<<grid, W_THREADS, kGemmWideSmemBytes, s>>>(amap, bmap, wa);
        MDSIP_LAUNCHED();
        return;
    }
    CUtensorMap amap, bmap;
    tc::encode_2d(&amap, A, false, (uint64_t)std::max<int64_t>(K, 1), (uint64_t)M, (uint64_t)std::max<int64_t>(lda, 8),
                  G_SLAB, G_TILE);
    tc::encode_2d(&bmap, B, false, (uint64_t)std::max<int64_t>(K, 1), (uint64_t)N, (uint64_t)std::max<int64_t>(ldb, 8),
                  G_SLAB, G_TILE);
    GemmArgs a{};
    a.M = M;
    a.N = N;
    a.total_slabs = p.total_slabs;
    a.slabs_per_split = p.slabs_per_split;
    a.err = err_dev;
    if (p.nsplit > 1) {
        MDSIP_REQUIRE(ws != nullptr, MDSIP_ERR_INVALID_ARG, "gemm: missing split workspace");
        a.out = static_cast<float *>(ws);
        a.ldo = N;
        a.split_stride = M * N;
    } else {
        a.out = C;
        a.ldo = ldc;
        a.split_stride = 0;
    }
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmemBytes);
    }));
    const dim3 grid((unsigned)p.tn, (unsigned)p.tm, (unsigned)p.nsplit);
    k_gemm_bf16<<<grid, G_THREADS, kGemmSmemBytes, s>>>(amap, bmap, a);
    MDSIP_LAUNCHED();
    if (p.nsplit > 1) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms * 8, ceil_div(M * N, 256)));
        k_gemm_reduce<<<g, 256, 0, s>>>(M, N, p.nsplit, a.out, C, ldc);
        MDSIP_LAUNCHED();
    }
}

}  // namespace mdsip

extern "C" mdsip_status mdsip_gemm_bf16(mdsip_ctx *hctx, int64_t M, int64_t N, int64_t K, const uint16_t *A,
                                        int64_t lda, const uint16_t *B, int64_t ldb, float *C, int64_t ldc) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    mdsip::Ctx *ctx = reinterpret_cast<mdsip::Ctx *>(hctx);
    return mdsip::guarded(ctx, [&] {
        mdsip::DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(M >= 0 && N >= 0 && K >= 0, MDSIP_ERR_INVALID_ARG, "gemm: negative size");
        if (M == 0 || N == 0) return;
        MDSIP_REQUIRE(A && B && C, MDSIP_ERR_INVALID_ARG, "gemm: null pointer");
        MDSIP_REQUIRE(lda % 8 == 0 && ldb % 8 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0 &&
                          reinterpret_cast<uintptr_t>(B) % 16 == 0,
                      MDSIP_ERR_INVALID_ARG, "gemm: A and B need 16-byte aligned rows (lda, ldb multiples of 8)");
        const size_t ws = mdsip::gemm_bf16_ws_bytes(M, N, K, ctx->num_sms);
        const size_t wsa = (ws + 255) / 256 * 256;
        char *base = static_cast<char *>(ctx->scratch_at_least(wsa + 256));
        int *err = reinterpret_cast<int *>(base + wsa);
        MDSIP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
        mdsip::launch_gemm_bf16(ctx->stream, ctx->num_sms, reinterpret_cast<const __nv_bfloat16 *>(A), lda,
                                reinterpret_cast<const __nv_bfloat16 *>(B), ldb, M, N, K, C, ldc,
                                ws ? base : nullptr, err);
        int herr = 0;
        MDSIP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
        MDSIP_REQUIRE(herr == 0, MDSIP_ERR_DEVICE, "gemm: a bounded device wait expired");
    });
}
