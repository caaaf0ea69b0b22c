// Condensation product on the 5th-generation tensor cores (mixed precision):
//
//     C[p][q] = beta C[p][q] + sum_i A[i][p] A[i][q] / w_i       (p >= q)
//
// computed as C = At At^T with At = (diag(w^-1/2) A)^T in BF16 (kind::f16) or
// FP32 read as TF32 (kind::tf32), FP32 accumulation in tensor memory, the
// split-K partials summed in FP32 and their total added to the FP64 matrix
// with one conversion per entry.  The FP64 caller wins the accuracy back with
// iterative refinement of the Newton system.
//
// Structure (one CTA = one 128x128 lower-triangle tile x one K range):
//   * warp 0 lane 0 streams 128-byte-wide K slabs of the two row blocks of
//     At with TMA (128-byte swizzle) into a 3-stage shared-memory ring;
//   * warp 1 lane 0 issues tcgen05.mma (M = N = 128, four K steps per slab)
//     into a 128-column FP32 accumulator in TMEM and releases each stage with
//     tcgen05.commit on its mbarrier;
//   * all four warps read the accumulator with tcgen05.ld (32 lanes each)
//     and write the partial tile, transposed for coalesced reduction.
// Every mbarrier wait is bounded; on expiry the kernel raises an error flag
// instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "internal.cuh"
#include "tc.cuh"

namespace mdsip {

namespace {

constexpr int TC_TILE = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_STAGES = 3;
constexpr int SLAB_BYTES = 128;                        // K bytes per row and stage
constexpr int TILE_BYTES = TC_TILE * SLAB_BYTES;       // 16 KiB per operand and stage
constexpr uint32_t TMEM_COLS = 128;
using tc::commit;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::smem_u32;
using tc::sw128_kmajor_desc;
using tc::tma_load_2d;
using tc::tmem_ld32;
using tc::fence_after;
using tc::fence_before;

__device__ __forceinline__ void tile_of(int t, int &tp, int &tq) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    tp = r;
    tq = t - r * (r + 1) / 2;
}

struct TcArgs {
    int tiles;            // lower-triangle tiles
    int slabs_per_split;  // K slabs per split
    int total_slabs;      // K slabs overall
    int elems_per_slab;   // 64 (BF16) or 32 (TF32)
    float *work;          // [split][tile][128 q][128 p] partial tiles
    int *err;
};

constexpr size_t kTcSmemBytes = 1024 + 2 * TC_STAGES * TILE_BYTES + 256;

template <bool TF32>
__global__ void __launch_bounds__(TC_THREADS, 2) k_syrk_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + TC_STAGES * TILE_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 2 * TC_STAGES * TILE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *accum = empty + TC_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tp, tq;
    tile_of(blockIdx.x, tp, tq);
    const int split = blockIdx.y;
    const int s0 = split * a.slabs_per_split;
    const int s1 = min(a.total_slabs, s0 + a.slabs_per_split);
    const int nslab = max(0, s1 - s0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the two 128-row blocks of At for each K slab
        for (int it = 0; it < nslab; ++it) {
            const int st = it % TC_STAGES, rnd = it / TC_STAGES;
            if (!mbar_wait(&empty[st], (rnd & 1) ^ 1)) {
                atomicExch(a.err, 1);
                break;
            }
            mbar_expect_tx(&full[st], 2 * TILE_BYTES);
            const int kx = (s0 + it) * a.elems_per_slab;
            tma_load_2d(sA + st * TILE_BYTES, &tmap, &full[st], kx, tp * TC_TILE);
            tma_load_2d(sB + st * TILE_BYTES, &tmap, &full[st], kx, tq * TC_TILE);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: 4 K steps of 32 bytes per slab
        for (int it = 0; it < nslab; ++it) {
            const int st = it % TC_STAGES, rnd = it / TC_STAGES;
            if (!mbar_wait(&full[st], rnd & 1)) {
                atomicExch(a.err, 1);
                break;
            }
            fence_after();
            const uint32_t ab = smem_u32(sA + st * TILE_BYTES), bb = smem_u32(sB + st * TILE_BYTES);
#pragma unroll
            for (int k = 0; k < SLAB_BYTES / 32; ++k)
                tc::mma<TF32, tc::instr_desc(TF32, TC_TILE, TC_TILE)>(
                    tmem, sw128_kmajor_desc(ab + 32 * k), sw128_kmajor_desc(bb + 32 * k), (it > 0 || k > 0) ? 1u : 0u);
            commit(&empty[st]);
        }
        commit(accum);
    }
    __syncwarp();
    // epilogue: TMEM lanes 32w..32w+31 are rows p of the tile
    const bool ok = mbar_wait(accum, 0);
    fence_after();
    float *out = a.work + ((size_t)split * a.tiles + blockIdx.x) * (TC_TILE * TC_TILE);
    const int row = warp * 32 + lane;
    if (ok && nslab > 0) {
#pragma unroll 1
        for (int c = 0; c < TC_TILE / 32; ++c) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) out[(size_t)(c * 32 + j) * TC_TILE + row] = __uint_as_float(r[j]);
        }
    } else {
        if (!ok) atomicExch(a.err, 1);
        for (int c = 0; c < TC_TILE; ++c) out[(size_t)c * TC_TILE + row] = 0.0f;
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        tc::tmem_dealloc(tmem, TMEM_COLS);
}

// AfT[p][i] = (float) A[i][p]  (transposed FP32 copy, zero padded to ldt)
__global__ void k_transpose_f32(const double *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                float *__restrict__ AfT, int64_t ldt) {
    __shared__ float t[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, p0 = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, p = p0 + threadIdx.x;
        t[r][threadIdx.x] = (i < m && p < n) ? (float)A[i * lda + p] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t p = p0 + r, i = i0 + threadIdx.x;
        if (p < n && i < ldt) AfT[p * ldt + i] = t[threadIdx.x][r];
    }
}

// rs[i] = w_i^-1/2 in FP32 (zero beyond m)
__global__ void k_rsqrt_w(int64_t m, int64_t mp, const double *__restrict__ w, float *__restrict__ rs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mp; i += (int64_t)gridDim.x * blockDim.x)
        rs[i] = i < m ? rsqrtf((float)w[i]) : 0.0f;
}

// At[p][i] = AfT[p][i] * rs[i], BF16 or FP32, 4 elements per thread
template <bool TF32>
__global__ void k_scale_rows(int64_t n, int64_t ldt, const float *__restrict__ AfT, const float *__restrict__ rs,
                             void *__restrict__ At) {
    const int64_t total4 = n * ldt / 4;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (e * 4) % ldt;
        const float4 v = reinterpret_cast<const float4 *>(AfT)[e];
        const float4 s = *reinterpret_cast<const float4 *>(rs + i);
        const float4 o = make_float4(v.x * s.x, v.y * s.y, v.z * s.z, v.w * s.w);
        if constexpr (TF32) {
            reinterpret_cast<float4 *>(At)[e] = o;
        } else {
            __nv_bfloat162 lo = __floats2bfloat162_rn(o.x, o.y), hi = __floats2bfloat162_rn(o.z, o.w);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t *>(&lo);
            pk.y = *reinterpret_cast<uint32_t *>(&hi);
            reinterpret_cast<uint2 *>(At)[e] = pk;
        }
    }
}

// C[p][q] = beta C[p][q] + sum_split work[split][tile(p,q)][q % 128][p % 128]   (p >= q)
// The split partials are FP32 tensor-core sums; they are added in FP32 (their
// own rounding, 2^-24 per addition, is far below the operands' BF16/TF32
// rounding) and the total enters the FP64 matrix with one conversion and one
// FP64 addition per entry: GB300 runs FP64 adds and conversions at 1/64 of the
// FP32 rate, which made an all-FP64 sum of ~20 partials the kernel's cost.
__global__ void k_tc_reduce(int64_t n, int tiles, int nsplit, const float *__restrict__ work, double beta,
                            double *__restrict__ C, int64_t ldc) {
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
        const int tq = (int)(q / TC_TILE);
        for (int64_t p = q + threadIdx.x; p < n; p += blockDim.x) {
            const int tp = (int)(p / TC_TILE);
            const int t = tp * (tp + 1) / 2 + tq;
            const size_t off = (size_t)(q % TC_TILE) * TC_TILE + (size_t)(p % TC_TILE);
            const size_t stride = (size_t)tiles * (TC_TILE * TC_TILE);
            const float *w = work + (size_t)t * (TC_TILE * TC_TILE) + off;
            float s0 = 0.0f, s1 = 0.0f;
            int k = 0;
            for (; k + 1 < nsplit; k += 2) {
                s0 += w[(size_t)k * stride];
                s1 += w[(size_t)(k + 1) * stride];
            }
            if (k < nsplit) s0 += w[(size_t)k * stride];
            double *c = C + p + q * ldc;
            *c = (beta != 0.0 ? *c : 0.0) + (double)(s0 + s1);
        }
    }
}

// vf[i] = (float) v[i] for i < m, 0 up to ldt
__global__ void k_to_f32_padded(int64_t m, int64_t ldt, const double *__restrict__ v, float *__restrict__ vf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ldt; i += (int64_t)gridDim.x * blockDim.x)
        vf[i] = i < m ? (float)v[i] : 0.0f;
}

// out[p] = sum_i AfT[p][i] vf[i] (FP32 products and sums, one block per row of
// AfT, i.e. per column of A; 16-byte loads)
__global__ void __launch_bounds__(256) k_aft_dot(const float *__restrict__ AfT, int64_t ldt, int64_t n,
                                                 const float *__restrict__ vf, double *__restrict__ out) {
    __shared__ float red[8];
    const int64_t q = ldt / 4;
    const float4 *v4 = reinterpret_cast<const float4 *>(vf);
    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const float4 *row = reinterpret_cast<const float4 *>(AfT + p * ldt);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int64_t k = threadIdx.x;
        for (; k + 768 < q; k += 1024) {   // four 16-byte loads of the row in flight per thread
            float4 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = __ldg(row + k + 256 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = __ldg(v4 + k + 256 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s0 = fmaf(a[u].x, b[u].x, s0);
                s1 = fmaf(a[u].y, b[u].y, s1);
                s2 = fmaf(a[u].z, b[u].z, s2);
                s3 = fmaf(a[u].w, b[u].w, s3);
            }
        }
        for (; k < q; k += 256) {
            const float4 a = __ldg(row + k), b = __ldg(v4 + k);
            s0 = fmaf(a.x, b.x, s0);
            s1 = fmaf(a.y, b.y, s1);
            s2 = fmaf(a.z, b.z, s2);
            s3 = fmaf(a.w, b.w, s3);
        }
        float t = (s0 + s1) + (s2 + s3);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            float u = 0.f;
            for (int w = 0; w < 8; ++w) u += red[w];
            out[p] = (double)u;
        }
        __syncthreads();
    }
}

}  // namespace

// out = A^T v in FP32 from the transposed copy AfT (n x ldt, zero padded
// beyond m): the approximate products of the refined path.  vf: ldt floats.
void launch_aft_dot(cudaStream_t s, int num_sms, const float *AfT, int64_t ldt, int64_t m, int64_t n,
                    const double *v, float *vf, double *out) {
    if (n <= 0) return;
    k_to_f32_padded<<<std::max(1, std::min(4096, ceil_div(ldt, 256))), 256, 0, s>>>(m, ldt, v, vf);
    MDSIP_LAUNCHED();
    k_aft_dot<<<(unsigned)std::min<int64_t>(n, (int64_t)num_sms * 8), 256, 0, s>>>(AfT, ldt, n, vf, out);
    MDSIP_LAUNCHED();
}

int64_t syrk_tc_ld(int64_t m) { return (std::max<int64_t>(m, 1) + 63) / 64 * 64; }

void launch_transpose_f32(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda, float *AfT,
                          int64_t ldt) {
    if (n <= 0) return;
    const dim3 grid((unsigned)ceil_div(ldt, 32), (unsigned)ceil_div(n, 32));
    k_transpose_f32<<<grid, dim3(32, 8), 0, s>>>(A, m, n, lda, AfT, ldt);
    MDSIP_LAUNCHED();
}

TcPlan syrk_tc_plan(int64_t m, int64_t n, int num_sms, int precision) {
    TcPlan pl{};
    const int64_t ldt = syrk_tc_ld(m);
    const int64_t nt = (n + TC_TILE - 1) / TC_TILE;
    pl.tiles = (int)(nt * (nt + 1) / 2);
    pl.elems_per_slab = precision == MDSIP_PREC_TF32 ? 32 : 64;
    pl.total_slabs = (int)(ldt / pl.elems_per_slab);
    // split-K so that (tile, split) items fill whole waves of two CTAs per SM
    double best = 0.0;
    pl.nsplit = 1;
    for (int s = 1; s <= 64; ++s) {
        if (s > 1 && pl.total_slabs / s < 8) break;
        const double waves = (double)pl.tiles * s / (2.0 * num_sms);
        const double eff = waves / std::ceil(waves);
        if (eff > best + 0.005) {
            best = eff;
            pl.nsplit = s;
        }
        if (eff >= 0.985) break;
    }
    pl.slabs_per_split = (pl.total_slabs + pl.nsplit - 1) / pl.nsplit;
    pl.nsplit = (pl.total_slabs + pl.slabs_per_split - 1) / pl.slabs_per_split;  // no empty split
    pl.ldt = ldt;
    pl.work_floats = (size_t)pl.nsplit * pl.tiles * TC_TILE * TC_TILE;
    return pl;
}

// AfT: n x ldt FP32 transposed copy of A (launch_transpose_f32).  ws holds
// rs (ldt floats), At (n x ldt BF16/FP32) and the split partials, laid out by
// syrk_tc_workspace_bytes.  err_dev: device int, must be 0 on entry.
size_t syrk_tc_workspace_bytes(const TcPlan &pl, int64_t n, int precision) {
    const size_t esz = precision == MDSIP_PREC_TF32 ? 4 : 2;
    auto al = [](size_t b) { return (b + 1023) / 1024 * 1024; };
    return al(pl.ldt * 4) + al((size_t)n * pl.ldt * esz) + al(pl.work_floats * 4);
}

void launch_syrk_tc(cudaStream_t s, int num_sms, int precision, const float *AfT, int64_t m, int64_t n,
                    const double *w, double beta, double *C, int64_t ldc, void *ws, int *err_dev) {
    if (n <= 0) return;
    MDSIP_REQUIRE(precision == MDSIP_PREC_TF32 || precision == MDSIP_PREC_BF16, MDSIP_ERR_INVALID_ARG,
                  "syrk_tc: precision must be TF32 or BF16");
    const bool tf32 = precision == MDSIP_PREC_TF32;
    const TcPlan pl = syrk_tc_plan(m, n, num_sms, precision);
    auto al = [](size_t b) { return (b + 1023) / 1024 * 1024; };
    char *base = static_cast<char *>(ws);
    float *rs = reinterpret_cast<float *>(base);
    void *At = base + al(pl.ldt * 4);
    float *work = reinterpret_cast<float *>(base + al(pl.ldt * 4) + al((size_t)n * pl.ldt * (tf32 ? 4 : 2)));

    k_rsqrt_w<<<std::max(1, std::min(4096, ceil_div(pl.ldt, 256))), 256, 0, s>>>(m, pl.ldt, w, rs);
    MDSIP_LAUNCHED();
    const int64_t total4 = n * pl.ldt / 4;
    const int sg = std::max(1, std::min(num_sms * 16, ceil_div(total4, 256)));
    if (tf32)
        k_scale_rows<true><<<sg, 256, 0, s>>>(n, pl.ldt, AfT, rs, At);
    else
        k_scale_rows<false><<<sg, 256, 0, s>>>(n, pl.ldt, AfT, rs, At);
    MDSIP_LAUNCHED();

    // tensor map over At: inner dimension K (ldt elements), outer n rows
    CUtensorMap tmap;
    tc::encode_2d(&tmap, At, tf32, (uint64_t)pl.ldt, (uint64_t)n, (uint64_t)pl.ldt, (uint32_t)pl.elems_per_slab,
                  (uint32_t)TC_TILE);

    TcArgs a{};
    a.tiles = pl.tiles;
    a.slabs_per_split = pl.slabs_per_split;
    a.total_slabs = pl.total_slabs;
    a.elems_per_slab = pl.elems_per_slab;
    a.work = work;
    a.err = err_dev;
    const dim3 grid((unsigned)pl.tiles, (unsigned)pl.nsplit);
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        cudaError_t e =
            cudaFuncSetAttribute(k_syrk_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_syrk_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmemBytes);
        return e;
    }));
    if (tf32)
        k_syrk_tc<true><<<grid, TC_THREADS, kTcSmemBytes, s>>>(tmap, a);
    else
        k_syrk_tc<false><<<grid, TC_THREADS, kTcSmemBytes, s>>>(tmap, a);
    MDSIP_LAUNCHED();
    k_tc_reduce<<<(unsigned)std::min<int64_t>(n, 4096), 256, 0, s>>>(n, pl.tiles, pl.nsplit, work, beta, C, ldc);
    MDSIP_LAUNCHED();
}

namespace tc {

// driver entry point for tensor-map encoding (no link-time libcuda dependency)
namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    MDSIP_REQUIRE(fn != nullptr, MDSIP_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    return fn;
}
}  // namespace

void encode_2d(CUtensorMap *map, const void *base, bool f32, uint64_t inner, uint64_t outer, uint64_t ld,
               uint32_t box_inner, uint32_t box_outer) {
    const size_t esz = f32 ? 4 : 2;
    MDSIP_REQUIRE(reinterpret_cast<uintptr_t>(base) % 16 == 0 && (ld * esz) % 16 == 0 && ld >= inner,
                  MDSIP_ERR_INVALID_ARG, "tensor map: base or row stride not 16-byte aligned");
    const cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t gstride[1] = {(cuuint64_t)(ld * esz)};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = encode_fn()(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                   const_cast<void *>(base), gdim, gstride, box, estride,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    MDSIP_REQUIRE(r == CUDA_SUCCESS, MDSIP_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

}  // namespace tc

}  // namespace mdsip
