// Condensation product of the two-stage elimination, FP64 (Section 2.2/2.3:
// the K3-type update M := M + A D B^T with A = B dense and D = W^-1 diagonal):
//
//     C[p][q] = beta C[p][q] + sum_i A[i][p] A[i][q] / w_i        (p >= q)
//
// A is m x n row-major (the dense Jacobian block J_{x_d} g), C column-major.
// GB300 FP64 runs on the SIMT DFMA pipe only (about 2 DFMA per clock per SM),
// so the kernel is arranged to keep that pipe saturated: 64x64 output tiles of
// the lower triangle, 4x4 accumulators per thread, 16-row K slabs staged in
// shared memory with 16-byte loads and register prefetch, and split-K chosen
// so that the number of (tile, split) work items fills whole waves of the
// 152 SMs.  Split partials are summed in fixed order (deterministic).
#include <algorithm>

#include "internal.cuh"

namespace mdsip {

namespace {

constexpr int BM = 64;   // tile edge
constexpr int KB = 16;   // K rows per slab
constexpr int SYRK_THREADS = 256;

struct SyrkArgs {
    const double *A;
    int64_t m, n, lda;
    const double *w;
    int nsplit;
    int64_t kchunk;   // rows of A per split (multiple of KB)
    double beta;
    double *C;        // final output (nsplit == 1)
    int64_t ldc;
    double *work;     // nsplit x n x n partials (nsplit > 1)
};

__device__ __forceinline__ void tile_of(int t, int &tp, int &tq) {
    int r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    tp = r;
    tq = t - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(SYRK_THREADS, 2) k_syrk_fp64(SyrkArgs a) {
    __shared__ __align__(16) double As[KB][BM];   // p side, scaled by 1/w
    __shared__ __align__(16) double Bs[KB][BM];   // q side
    int tp, tq;
    tile_of(blockIdx.x, tp, tq);
    const int64_t p0 = (int64_t)tp * BM, q0 = (int64_t)tq * BM;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t kbeg = (int64_t)blockIdx.y * a.kchunk;
    const int64_t kend = min(a.m, kbeg + a.kchunk);

    // loader mapping: row lr = tid / 16 of the slab, column pairs lc and lc + 16
    const int lr = tid >> 4;
    const int lc = tid & 15;

    double2 pa0, pa1, pb0, pb1;
    double rw;
    auto load = [&](int64_t k0) {
        const int64_t i = k0 + lr;
        pa0 = pa1 = pb0 = pb1 = make_double2(0.0, 0.0);
        rw = 0.0;
        if (i < kend) {
            rw = 1.0 / a.w[i];
            const double *row = a.A + i * a.lda;
            const int64_t c0 = 2 * lc, c1 = 2 * lc + 32;
            auto ld2 = [&](int64_t col) {
                double2 v = make_double2(0.0, 0.0);
                if (col + 1 < a.lda) {
                    v = __ldg(reinterpret_cast<const double2 *>(row + col));
                    if (col >= a.n) v.x = 0.0;
                    if (col + 1 >= a.n) v.y = 0.0;
                } else if (col < a.n) {
                    v.x = row[col];
                }
                return v;
            };
            pa0 = ld2(p0 + c0);
            pa1 = ld2(p0 + c1);
            pb0 = ld2(q0 + c0);
            pb1 = ld2(q0 + c1);
        }
    };
    auto store = [&]() {
        *reinterpret_cast<double2 *>(&As[lr][2 * lc]) = make_double2(pa0.x * rw, pa0.y * rw);
        *reinterpret_cast<double2 *>(&As[lr][2 * lc + 32]) = make_double2(pa1.x * rw, pa1.y * rw);
        *reinterpret_cast<double2 *>(&Bs[lr][2 * lc]) = pb0;
        *reinterpret_cast<double2 *>(&Bs[lr][2 * lc + 32]) = pb1;
    };

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    if (kbeg < kend) load(kbeg);
    for (int64_t k0 = kbeg; k0 < kend; k0 += KB) {
        __syncthreads();
        store();
        __syncthreads();
        if (k0 + KB < kend) load(k0 + KB);
#pragma unroll
        for (int kk = 0; kk < KB; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
    }
    // epilogue: lower triangle only
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t q = q0 + ty + 16 * j;
        if (q >= a.n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t p = p0 + tx + 16 * i;
            if (p >= a.n || p < q) continue;
            if (a.nsplit == 1) {
                double *c = a.C + p + q * a.ldc;
                *c = (a.beta != 0.0 ? a.beta * *c : 0.0) + acc[i][j];
            } else {
                a.work[(size_t)blockIdx.y * a.n * a.n + p + q * a.n] = acc[i][j];
            }
        }
    }
}

__global__ void k_syrk_reduce(int64_t n, int nsplit, const double *__restrict__ work, double beta,
                              double *__restrict__ C, int64_t ldc) {
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
        for (int64_t p = q + threadIdx.x; p < n; p += blockDim.x) {
            double s = 0.0;
            for (int k = 0; k < nsplit; ++k) s += work[(size_t)k * n * n + p + q * n];
            double *c = C + p + q * ldc;
            *c = (beta != 0.0 ? beta * *c : 0.0) + s;
        }
    }
}

int choose_split(int64_t m, int64_t n, int num_sms) {
    const int64_t nt = (n + BM - 1) / BM;
    const int64_t T = nt * (nt + 1) / 2;
    const int64_t slots = (int64_t)num_sms * 2;
    int best = 1;
    double best_eff = 0.0;
    for (int s = 1; s <= 8; ++s) {
        if (s > 1 && m / s < 256) break;
        const double waves = (double)(T * s) / (double)slots;
        const double eff = waves / std::ceil(waves);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = s;
        }
        if (eff >= 0.95) break;
    }
    return best;
}

}  // namespace

size_t syrk_fp64_scratch_bytes(int64_t m, int64_t n, int num_sms) {
    const int s = choose_split(m, n, num_sms);
    return s > 1 ? (size_t)s * (size_t)n * (size_t)n * sizeof(double) : 0;
}

void launch_syrk_fp64_ws(cudaStream_t st, int num_sms, const double *A, int64_t m, int64_t n,
                         int64_t lda, const double *w, double beta, double *C, int64_t ldc,
                         double *work) {
    if (n <= 0) return;
    SyrkArgs a{};
    a.A = A;
    a.m = m;
    a.n = n;
    a.lda = lda;
    a.w = w;
    a.beta = beta;
    a.C = C;
    a.ldc = ldc;
    a.nsplit = m > 0 ? choose_split(m, n, num_sms) : 1;
    a.kchunk = ((std::max<int64_t>(m, 1) + a.nsplit - 1) / a.nsplit + KB - 1) / KB * KB;
    a.work = work;
    const int64_t nt = (n + BM - 1) / BM;
    const int64_t T = nt * (nt + 1) / 2;
    MDSIP_REQUIRE(T < (1LL << 31), MDSIP_ERR_INVALID_ARG, "syrk: n too large");
    k_syrk_fp64<<<dim3((unsigned)T, (unsigned)a.nsplit), SYRK_THREADS, 0, st>>>(a);
    MDSIP_LAUNCHED();
    if (a.nsplit > 1) {
        k_syrk_reduce<<<(unsigned)std::min<int64_t>(n, 4096), 256, 0, st>>>(n, a.nsplit, work, beta, C,
                                                                            ldc);
        MDSIP_LAUNCHED();
    }
}

void launch_syrk_fp64(Ctx *ctx, const double *A, int64_t m, int64_t n, int64_t lda, const double *w,
                      double beta, double *C, int64_t ldc) {
    const size_t ws = syrk_fp64_scratch_bytes(m, n, ctx->num_sms);
    double *work = ws ? static_cast<double *>(ctx->scratch_at_least(ws)) : nullptr;
    launch_syrk_fp64_ws(ctx->stream, ctx->num_sms, A, m, n, lda, w, beta, C, ldc, work);
}

}  // namespace mdsip
