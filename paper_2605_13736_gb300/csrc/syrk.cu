// Condensation product of the two-stage elimination, FP64 (Section 2.2/2.3:
// the K3-type update M := M + A D B^T with A = B dense and D = W^-1 diagonal):
//
//     C[p][q] = beta C[p][q] + sum_i A[i][p] A[i][q] / w_i        (p >= q)
//
// A is m x n row-major (the dense Jacobian block J_{x_d} g), C column-major.
// GB300 FP64 runs on the SIMT DFMA pipe only (about 2 DFMA per clock per SM),
// so the kernel is arranged to keep that pipe saturated with useful FMAs:
// 64x64 or 80x80 output tiles of the lower triangle (whichever executes the
// fewest FMAs on the ragged edge and the diagonal tiles), 4x4 or 5x5
// accumulators per thread, 16-row K slabs staged in shared memory with
// 16-byte loads and register prefetch, the reciprocals 1/w computed once per
// call, diagonal tiles skipping the accumulators that hold only entries above
// the diagonal, and split-K chosen so that the (tile, split) work items fill
// whole waves of the 152 SMs.  Split partials are summed in fixed order
// (deterministic).
#include <algorithm>

#include "internal.cuh"

namespace mdsip {

namespace {

constexpr int KB = 16;   // K rows per slab
constexpr int SYRK_THREADS = 256;

struct SyrkArgs {
    const double *A;
    int64_t m, n, lda;
    const double *rw;  // 1 / w, m entries
    int nsplit;
    int64_t kchunk;    // rows of A per split (multiple of KB)
    double beta;
    double *C;         // final output (nsplit == 1)
    int64_t ldc;
    double *work;      // nsplit x n x n partials (nsplit > 1)
};

__device__ __forceinline__ void tile_of(int t, int &tp, int &tq) {
    int r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    tp = r;
    tq = t - r * (r + 1) / 2;
}

// BM x BM tile of the lower triangle; thread (tx, ty) owns rows tx + 16 i and
// columns ty + 16 j of the tile (TM x TM accumulators, TM = BM / 16).
template <int BM>
__global__ void __launch_bounds__(SYRK_THREADS, 2) k_syrk_fp64(SyrkArgs a) {
    constexpr int TM = BM / 16;
    constexpr int VROW = BM / 2;                 // 16-byte vectors per slab row
    constexpr int VTOT = KB * VROW;
    constexpr int LPT = (VTOT + SYRK_THREADS - 1) / SYRK_THREADS;
    __shared__ __align__(16) double As[KB][BM];  // p side, scaled by 1/w
    __shared__ __align__(16) double Bs[KB][BM];  // q side
    int tp, tq;
    tile_of(blockIdx.x, tp, tq);
    const int64_t p0 = (int64_t)tp * BM, q0 = (int64_t)tq * BM;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t kbeg = (int64_t)blockIdx.y * a.kchunk;
    const int64_t kend = min(a.m, kbeg + a.kchunk);

    double2 ra[LPT], rb[LPT];
    double rs[LPT];
    auto ld2 = [&](const double *row, int64_t col) {
        double2 v = make_double2(0.0, 0.0);
        if (col < a.lda) {   // lda even and col even: both elements inside the row
            v = __ldg(reinterpret_cast<const double2 *>(row + col));
            if (col >= a.n) v.x = 0.0;
            if (col + 1 >= a.n) v.y = 0.0;
        }
        return v;
    };
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int e = tid + u * SYRK_THREADS;
            ra[u] = rb[u] = make_double2(0.0, 0.0);
            rs[u] = 0.0;
            if (e < VTOT) {
                const int r = e / VROW, c = 2 * (e % VROW);
                const int64_t i = k0 + r;
                if (i < kend) {
                    const double *row = a.A + i * a.lda;
                    rs[u] = __ldg(a.rw + i);
                    ra[u] = ld2(row, p0 + c);
                    rb[u] = ld2(row, q0 + c);
                }
            }
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int e = tid + u * SYRK_THREADS;
            if (e < VTOT) {
                const int r = e / VROW, c = 2 * (e % VROW);
                *reinterpret_cast<double2 *>(&As[r][c]) = make_double2(ra[u].x * rs[u], ra[u].y * rs[u]);
                *reinterpret_cast<double2 *>(&Bs[r][c]) = rb[u];
            }
        }
    };

    double acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;

    // On a diagonal tile (p0 == q0) the accumulators (i, j > i) hold only
    // entries above the diagonal (q - p = ty - tx + 16 (j - i) > 0): they are
    // skipped for every thread alike, 40% of the tile's FMAs at TM = 5.
    const bool diag = tp == tq;
    if (kbeg < kend) load(kbeg);
    for (int64_t k0 = kbeg; k0 < kend; k0 += KB) {
        __syncthreads();
        store();
        __syncthreads();
        if (k0 + KB < kend) load(k0 + KB);
        if (diag) {
#pragma unroll
            for (int kk = 0; kk < KB; ++kk) {
                double av[TM], bv[TM];
#pragma unroll
                for (int i = 0; i < TM; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
                for (int j = 0; j < TM; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j <= i; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < KB; ++kk) {
                double av[TM], bv[TM];
#pragma unroll
                for (int i = 0; i < TM; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
                for (int j = 0; j < TM; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TM; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
        }
    }
    // epilogue: lower triangle only
#pragma unroll
    for (int j = 0; j < TM; ++j) {
        const int64_t q = q0 + ty + 16 * j;
        if (q >= a.n) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t p = p0 + tx + 16 * i;
            if (p >= a.n || p < q) continue;
            if (a.nsplit == 1) {
                double *c = a.C + p + q * a.ldc;
                *c = (a.beta != 0.0 ? *c : 0.0) + acc[i][j];
            } else {
                a.work[(size_t)blockIdx.y * a.n * a.n + p + q * a.n] = acc[i][j];
            }
        }
    }
}

__global__ void k_recip(int64_t m, const double *__restrict__ w, double *__restrict__ rw) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        rw[i] = 1.0 / w[i];
}

__global__ void k_syrk_reduce(int64_t n, int nsplit, const double *__restrict__ work, double beta,
                              double *__restrict__ C, int64_t ldc) {
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
        for (int64_t p = q + threadIdx.x; p < n; p += blockDim.x) {
            double s = 0.0;
            for (int k = 0; k < nsplit; ++k) s += work[(size_t)k * n * n + p + q * n];
            double *c = C + p + q * ldc;
            *c = (beta != 0.0 ? *c : 0.0) + s;
        }
    }
}

struct Plan {
    int bm;
    int64_t tiles;
    int nsplit;
};

// Tile edge with the least executed work (ragged edge + diagonal tiles), or
// bm_force (64 or 80) when given, then the split count whose (tile, split)
// items fill whole waves of 2 CTAs per SM.
Plan plan_for(int64_t m, int64_t n, int num_sms, int bm_force = 0) {
    Plan best{64, 0, 1};
    double best_work = 0;
    for (int bm : {64, 80}) {
        if (bm_force && bm != bm_force) continue;
        const int64_t nt = (n + bm - 1) / bm;
        const int64_t T = nt * (nt + 1) / 2;
        const double work = (double)T * bm * bm;
        if (best.tiles == 0 || work < best_work * 0.995) {
            best = Plan{bm, T, 1};
            best_work = work;
        }
    }
    const int64_t slots = (int64_t)num_sms * 2;
    const size_t cap = (size_t)1 << 30;  // split partials at most 1 GiB
    double best_eff = 0.0;
    for (int s = 1; s <= 32; ++s) {
        if (s > 1 && (m / s < 512 || (size_t)s * n * n * sizeof(double) > cap)) break;
        const double waves = (double)(best.tiles * s) / (double)slots;
        const double eff = waves / std::ceil(waves);
        if (eff > best_eff + 0.005) {
            best_eff = eff;
            best.nsplit = s;
        }
        if (eff >= 0.99) break;
    }
    return best;
}

}  // namespace

// enough for either tile edge
size_t syrk_fp64_scratch_bytes(int64_t m, int64_t n, int num_sms) {
    size_t part = 0;
    for (int bm : {64, 80}) {
        const Plan pl = plan_for(m, n, num_sms, bm);
        if (pl.nsplit > 1) part = std::max(part, (size_t)pl.nsplit * (size_t)n * (size_t)n * sizeof(double));
    }
    return part + ((size_t)std::max<int64_t>(m, 1) * sizeof(double) + 255) / 256 * 256;
}

// work: syrk_fp64_scratch_bytes(m, n, num_sms) bytes (split partials, then 1/w)
void launch_syrk_fp64_ws(cudaStream_t st, int num_sms, const double *A, int64_t m, int64_t n,
                         int64_t lda, const double *w, double beta, double *C, int64_t ldc,
                         double *work, int bm) {
    if (n <= 0) return;
    const Plan pl = plan_for(m, n, num_sms, bm == 64 || bm == 80 ? bm : 0);
    SyrkArgs a{};
    a.A = A;
    a.m = m;
    a.n = n;
    a.lda = lda;
    a.beta = beta;
    a.C = C;
    a.ldc = ldc;
    a.nsplit = m > 0 ? pl.nsplit : 1;
    a.kchunk = ((std::max<int64_t>(m, 1) + a.nsplit - 1) / a.nsplit + KB - 1) / KB * KB;
    a.work = work;
    double *rw = work + (pl.nsplit > 1 ? (size_t)pl.nsplit * n * n : 0);
    a.rw = rw;
    if (m > 0) {
        k_recip<<<std::max(1, std::min(4096, ceil_div(m, 256))), 256, 0, st>>>(m, w, rw);
        MDSIP_LAUNCHED();
    }
    MDSIP_REQUIRE(pl.tiles < (1LL << 31), MDSIP_ERR_INVALID_ARG, "syrk: n too large");
    const dim3 grid((unsigned)pl.tiles, (unsigned)a.nsplit);
    if (pl.bm == 80)
        k_syrk_fp64<80><<<grid, SYRK_THREADS, 0, st>>>(a);
    else
        k_syrk_fp64<64><<<grid, SYRK_THREADS, 0, st>>>(a);
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
    double *work = static_cast<double *>(ctx->scratch_at_least(ws));
    launch_syrk_fp64_ws(ctx->stream, ctx->num_sms, A, m, n, lda, w, beta, C, ldc, work);
}

}  // namespace mdsip
