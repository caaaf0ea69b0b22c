// Solve with the Bunch-Kaufman factor P K P^T = L D L^T (Section 2.3):
//
//     x = L^-1 P b,   w = D^-1 x,   z = L^-T w,   b <- P^T z.
//
// N is a few thousand at most, so the time of a solve is its dependency
// chain, not its 2 N^2 flops.  The layout and schedule are built around that
// chain:
//
//  * once per factorization, L is copied into 64 x 64 tiles (column-major
//    inside a tile, in FP64 or, for the refined mixed-precision path, FP32):
//    F(I, J) = L_IJ for J < I and F(I, I) = inv(L_II) for the forward sweep,
//    and their transposes for the backward sweep, so that every tile
//    product in both sweeps reads its tile with lanes along contiguous rows;
//  * one CTA per 64-row block row (cooperative launch, so all are resident).
//    The CTA of block row I accumulates L_IJ x_J for J < I as soon as block J
//    has published x_J (a per-block release flag tagged with the launch's
//    epoch, no grid-wide barrier), loads the next tile into registers before
//    it waits for the next flag, and finishes with inv(L_II); the backward
//    sweep runs the same way from the last block up;
//  * D^-1 (1x1 and 2x2 blocks) is applied per block row between the sweeps;
//    a 2x2 block that straddles two block rows waits for the neighbour's
//    forward result.
//
// Flags hold the epoch of the launch that set them, so no reset is needed
// between solves; the last CTA to finish advances the epoch.  Every wait is
// bounded and sets the error flag on expiry.
#include <algorithm>

#include "internal.cuh"

namespace mdsip {

namespace {

constexpr int kBS = 64;            // block rows and tile edge
constexpr int kThreads = 256;      // 64 rows x 4 column quarters
constexpr int kTile = kBS * kBS;

__host__ __device__ inline int64_t tile_index(int64_t I, int64_t J) { return I * (I + 1) / 2 + J; }  // J <= I

struct Layout {
    int nblk = 0;
    int64_t ntile = 0;
    size_t off_flags_f = 0, off_flags_b = 0, off_x = 0, off_z = 0, off_F = 0, off_B = 0, total = 0;
};

Layout layout_for(int64_t N) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    Layout l;
    l.nblk = (int)((std::max<int64_t>(N, 1) + kBS - 1) / kBS);
    l.ntile = (int64_t)l.nblk * (l.nblk + 1) / 2;
    size_t o = 256;                                    // epoch, done counter
    l.off_flags_f = o; o += al((size_t)l.nblk * 4);
    l.off_flags_b = o; o += al((size_t)l.nblk * 4);
    l.off_x = o; o += al((size_t)l.nblk * kBS * sizeof(double));
    l.off_z = o; o += al((size_t)l.nblk * kBS * sizeof(double));
    l.off_F = o; o += al((size_t)l.ntile * kTile * sizeof(double));
    l.off_B = o; o += al((size_t)l.ntile * kTile * sizeof(double));
    l.total = o;
    return l;
}

// Tiles of one factorization.  Block (bx): tile t = tile_index(I, J), J <= I.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_solve_tiles(int N, const double *__restrict__ L, T *__restrict__ F,
                                                          T *__restrict__ Bk) {
    __shared__ double s[kBS][kBS + 1];
    const int64_t t = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
    while ((int64_t)I * (I + 1) / 2 > t) --I;
    const int J = (int)(t - (int64_t)I * (I + 1) / 2);
    const int tid = threadIdx.x;
    T *f = F + t * kTile, *bk = Bk + t * kTile;
    if (J < I) {
        // s[r][c] = L[64I + r][64J + c]  (read along r: L is column-major)
        for (int e = tid; e < kTile; e += kThreads) {
            const int r = e & (kBS - 1), c = e >> 6;
            const int64_t gr = (int64_t)I * kBS + r, gc = (int64_t)J * kBS + c;
            const double v = (gr < N && gc < N) ? L[gr + gc * (int64_t)N] : 0.0;
            s[r][c] = v;
            f[c * kBS + r] = (T)v;
        }
        __syncthreads();
        for (int e = tid; e < kTile; e += kThreads) {
            const int r = e & (kBS - 1), c = e >> 6;   // Bk(r = j, c = i) = L[64I + i][64J + j]
            bk[c * kBS + r] = (T)s[c][r];
        }
        return;
    }
    // diagonal block: inverse of the unit lower triangle, column c by forward substitution
    const int jb = I * kBS, bw = min(kBS, N - jb);
    if constexpr (sizeof(T) == sizeof(float)) {
        // FP32 tiles (the refined path's approximate solves): the inverse in FP32 arithmetic,
        // four partial sums per entry.  On the FP64 pipe (1/64 of the FP32 rate) the 2016
        // dependent products of a column made this launch take about 0.1 ms at N = 2050.
        float(*sf)[kBS + 1] = reinterpret_cast<float(*)[kBS + 1]>(&s[0][0]);   // s's storage
        for (int e = tid; e < kTile; e += kThreads) {
            const int r = e & (kBS - 1), c = e >> 6;
            sf[r][c] = (r < bw && c < bw) ? (float)L[(jb + r) + (int64_t)(jb + c) * N] : 0.0f;
        }
        __syncthreads();
        float xf[kBS];
        const int c = tid;
        if (c < kBS) {
#pragma unroll
            for (int i = 0; i < kBS; ++i) {
                float v[4] = {(i == c) ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int j = 0; j < i; ++j) v[j & 3] = fmaf(-sf[i][j], xf[j], v[j & 3]);
                xf[i] = i < c ? 0.0f : (v[0] + v[1]) + (v[2] + v[3]);
            }
        }
        __syncthreads();
        if (c < kBS) {
#pragma unroll
            for (int i = 0; i < kBS; ++i) sf[i][c] = (i < bw && c < bw) ? xf[i] : 0.0f;
        }
        __syncthreads();
        for (int e = tid; e < kTile; e += kThreads) {
            const int r = e & (kBS - 1), cc = e >> 6;
            f[cc * kBS + r] = (T)sf[r][cc];    // F(I, I)(r, c) = inv(L_II)[r][c]
            bk[cc * kBS + r] = (T)sf[cc][r];   // B(I, I)(r, c) = inv(L_II)[c][r]
        }
        return;
    }
    for (int e = tid; e < kTile; e += kThreads) {
        const int r = e & (kBS - 1), c = e >> 6;
        s[r][c] = (r < bw && c < bw) ? L[(jb + r) + (int64_t)(jb + c) * N] : 0.0;
    }
    __syncthreads();
    double x[kBS];
    const int c = tid;
    if (c < kBS) {
#pragma unroll
        for (int i = 0; i < kBS; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
#pragma unroll
            for (int j = 0; j < kBS; ++j)
                if (j < i) v = fma(-s[i][j], x[j], v);
            x[i] = i < c ? 0.0 : v;
        }
    }
    __syncthreads();
    // s[i][c] = inv(L_II)[i][c]
    if (c < kBS) {
#pragma unroll
        for (int i = 0; i < kBS; ++i) s[i][c] = (i < bw && c < bw) ? x[i] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < kTile; e += kThreads) {
        const int r = e & (kBS - 1), cc = e >> 6;
        f[cc * kBS + r] = (T)s[r][cc];    // F(I, I)(r, c) = inv(L_II)[r][c]
        bk[cc * kBS + r] = (T)s[cc][r];   // B(I, I)(r, c) = inv(L_II)[c][r]
    }
}

template <typename T>
struct FlagSolve {
    int N, nblk;
    const T *F, *Bk;
    const double *Dd, *Doff;
    const int32_t *perm;
    double *b;
    T *x, *z;
    unsigned *fwd, *bwd, *epoch, *done;
    int *err;
};

// all threads: wait until *flag == e (bounded); uniform result
__device__ __forceinline__ bool wait_flag(const unsigned *flag, unsigned e, int *err, int *s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile const unsigned *vp = flag;
        if (*vp != e) {
            const long long t0 = clock64();
            while (*vp != e) {
                if (*((volatile int *)err) != 0 || clock64() - t0 > kBarrierLimitCycles) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// partial of (tile * v)[r] over the column quarter q, tile in registers
template <typename T>
__device__ __forceinline__ void load_quarter(const T *tile, int r, int q, T (&reg)[16]) {
    const T *p = tile + (16 * q) * kBS + r;
#pragma unroll
    for (int c = 0; c < 16; ++c) reg[c] = __ldg(p + c * kBS);
}

template <typename T>
__device__ __forceinline__ T dot_quarter(const T (&reg)[16], const T *sv, int q, T acc) {
#pragma unroll
    for (int c = 0; c < 16; ++c) acc = fma(reg[c], sv[16 * q + c], acc);
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ldlt_solve_flags(FlagSolve<T> p) {
    __shared__ T sv[kBS];
    __shared__ T spart[4][kBS];
    __shared__ unsigned s_e;
    __shared__ int s_ok;
    const int tid = threadIdx.x, r = tid & (kBS - 1), q = tid >> 6;
    const int G = (int)gridDim.x, N = p.N, nblk = p.nblk;
    if (tid == 0) s_e = *((volatile unsigned *)p.epoch) + 1u;
    __syncthreads();
    const unsigned e = s_e;
    bool ok = true;
    T reg[16];

    // ---------------- forward: x_I = inv(L_II) (P b - sum_J<I L_IJ x_J) ----------------
    for (int I = blockIdx.x; I < nblk && ok; I += G) {
        T acc = (T)0;
        for (int J = 0; J < I; ++J) {
            load_quarter(p.F + tile_index(I, J) * kTile, r, q, reg);
            if (!wait_flag(p.fwd + J, e, p.err, &s_ok)) {
                ok = false;
                break;
            }
            if (tid < kBS) sv[tid] = __ldcg(p.x + (int64_t)J * kBS + tid);
            __syncthreads();
            acc = dot_quarter(reg, sv, q, acc);
            __syncthreads();
        }
        if (!ok) break;
        load_quarter(p.F + tile_index(I, I) * kTile, r, q, reg);
        spart[q][r] = acc;
        __syncthreads();
        if (tid < kBS) {
            const int row = I * kBS + tid;
            const T y0 = row < N ? (T)p.b[p.perm[row]] : (T)0;
            sv[tid] = y0 - (spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid]);
        }
        __syncthreads();
        const T a2 = dot_quarter(reg, sv, q, (T)0);
        __syncthreads();
        spart[q][r] = a2;
        __syncthreads();
        if (tid < kBS) {
            p.x[(int64_t)I * kBS + tid] = spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid];
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) atomicExch(p.fwd + I, e);
    }

    // ---------------- w = D^-1 x, then z_I = inv(L_II)^T (w_I - sum_J>I L_JI^T z_J) ----------------
    int last = (int)blockIdx.x;
    while (last + G < nblk) last += G;
    for (int I = last; I >= 0 && ok && (int)blockIdx.x < nblk; I -= G) {
        // a 2x2 block straddling into block row I+1 needs its forward result
        const int lr = I * kBS + kBS - 1;
        if (I + 1 < nblk && lr + 1 < N && p.Doff[lr] != 0.0) {
            if (!wait_flag(p.fwd + I + 1, e, p.err, &s_ok)) {
                ok = false;
                break;
            }
        }
        T w = (T)0;
        if (tid < kBS) {
            const int k = I * kBS + tid;
            if (k < N) {
                const double off = p.Doff[k];
                if (off != 0.0) {
                    const double a = p.Dd[k], c = p.Dd[k + 1];
                    const double u = (double)__ldcg(p.x + k), v = (double)__ldcg(p.x + k + 1);
                    w = (T)((c * u - off * v) / (a * c - off * off));
                } else if (k > 0 && p.Doff[k - 1] != 0.0) {
                    const double a = p.Dd[k - 1], c = p.Dd[k], o2 = p.Doff[k - 1];
                    const double u = (double)__ldcg(p.x + k - 1), v = (double)__ldcg(p.x + k);
                    w = (T)((a * v - o2 * u) / (a * c - o2 * o2));
                } else {
                    w = (T)((double)__ldcg(p.x + k) / p.Dd[k]);
                }
            }
        }
        T acc = (T)0;
        for (int J = nblk - 1; J > I; --J) {
            load_quarter(p.Bk + tile_index(J, I) * kTile, r, q, reg);
            if (!wait_flag(p.bwd + J, e, p.err, &s_ok)) {
                ok = false;
                break;
            }
            if (tid < kBS) sv[tid] = __ldcg(p.z + (int64_t)J * kBS + tid);
            __syncthreads();
            acc = dot_quarter(reg, sv, q, acc);
            __syncthreads();
        }
        if (!ok) break;
        load_quarter(p.Bk + tile_index(I, I) * kTile, r, q, reg);
        spart[q][r] = acc;
        __syncthreads();
        if (tid < kBS) sv[tid] = w - (spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid]);
        __syncthreads();
        const T a2 = dot_quarter(reg, sv, q, (T)0);
        __syncthreads();
        spart[q][r] = a2;
        __syncthreads();
        if (tid < kBS) {
            const T zi = spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid];
            p.z[(int64_t)I * kBS + tid] = zi;
            const int row = I * kBS + tid;
            if (row < N) p.b[p.perm[row]] = (double)zi;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) atomicExch(p.bwd + I, e);
    }

    // the last CTA to finish advances the epoch (every CTA has read it by then:
    // none can finish before all have published their backward blocks)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned d = atomicAdd(p.done, 1u);
        if (d == (unsigned)G - 1u) {
            atomicExch(p.done, 0u);
            __threadfence();
            atomicAdd(p.epoch, 1u);
        }
    }
}

// FP32 form (the refined mixed-precision path): a block's result travels as
// 64-bit words (value bits | epoch << 32), so one load both tests that block J
// is published and delivers x_J, and a CTA fetches up to four published blocks
// per round trip.  No separate flags, no fences between value and flag.
struct TagSolve {
    int N, nblk;
    const float *F, *Bk;
    const double *Dd, *Doff;
    const int32_t *perm;
    double *b;
    unsigned long long *xw, *zw;   // tagged block results
    unsigned *epoch, *done;
    int *err;
};

__device__ __forceinline__ unsigned long long tag_word(float v, unsigned e) {
    return ((unsigned long long)e << 32) | (unsigned long long)__float_as_uint(v);
}

// value of a tagged word once it carries epoch e (bounded wait; false on expiry)
__device__ __forceinline__ bool tag_wait(const unsigned long long *w, unsigned e, int *err, float &v) {
    volatile const unsigned long long *vp = w;
    unsigned long long x = *vp;
    if ((unsigned)(x >> 32) != e) {
        const long long t0 = clock64();
        do {
            if (*((volatile int *)err) != 0 || clock64() - t0 > kBarrierLimitCycles) {
                atomicExch(err, 1);
                return false;
            }
            x = *vp;
        } while ((unsigned)(x >> 32) != e);
    }
    v = __uint_as_float((unsigned)x);
    return true;
}

constexpr int kTagBatch = 4;   // published blocks fetched per round trip

__global__ void __launch_bounds__(kThreads) k_ldlt_solve_tagged(TagSolve p) {
    __shared__ float sv[kTagBatch][kBS];
    __shared__ float spart[4][kBS];
    __shared__ unsigned s_e;
    __shared__ int s_ok;
    const int tid = threadIdx.x, r = tid & (kBS - 1), q = tid >> 6;
    const int G = (int)gridDim.x, N = p.N, nblk = p.nblk;
    if (tid == 0) {
        s_e = *((volatile unsigned *)p.epoch) + 1u;
        s_ok = 1;
    }
    __syncthreads();
    const unsigned e = s_e;
    float reg[kTagBatch][16];

    // sum over J in [J0, J1) of tile(J) * v_J, tiles at tile_of(J), results in words w
    auto accumulate = [&](auto tile_of, const unsigned long long *w, int J0, int J1, int step, float acc) {
        for (int J = J0; J != J1 && s_ok;) {
            const int nbat = min(kTagBatch, (J1 - J) * step);
#pragma unroll
            for (int bq = 0; bq < kTagBatch; ++bq)
                if (bq < nbat) load_quarter(tile_of(J + bq * step), r, q, reg[bq]);
            {   // thread t fetches word t % 64 of block t / 64
                const int bq = tid >> 6;
                if (bq < nbat) {
                    float v = 0.0f;
                    if (!tag_wait(w + (int64_t)(J + bq * step) * kBS + r, e, p.err, v)) atomicExch(&s_ok, 0);
                    sv[bq][r] = v;
                }
            }
            __syncthreads();
            if (!s_ok) break;
#pragma unroll
            for (int bq = 0; bq < kTagBatch; ++bq)
                if (bq < nbat) acc = dot_quarter(reg[bq], sv[bq], q, acc);
            __syncthreads();
            J += nbat * step;
        }
        return acc;
    };

    // ---------------- forward: x_I = inv(L_II) (P b - sum_J<I L_IJ x_J) ----------------
    for (int I = blockIdx.x; I < nblk && s_ok; I += G) {
        float acc = accumulate([&](int J) { return p.F + tile_index(I, J) * kTile; }, p.xw, 0, I, 1, 0.0f);
        if (!s_ok) break;
        load_quarter(p.F + tile_index(I, I) * kTile, r, q, reg[0]);
        spart[q][r] = acc;
        __syncthreads();
        if (tid < kBS) {
            const int row = I * kBS + tid;
            const float y0 = row < N ? (float)p.b[p.perm[row]] : 0.0f;
            sv[0][tid] = y0 - (spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid]);
        }
        __syncthreads();
        const float a2 = dot_quarter(reg[0], sv[0], q, 0.0f);
        __syncthreads();
        spart[q][r] = a2;
        __syncthreads();
        if (tid < kBS)
            p.xw[(int64_t)I * kBS + tid] = tag_word(spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid], e);
        __syncthreads();
    }

    // ---------------- w = D^-1 x, then z_I = inv(L_II)^T (w_I - sum_J>I L_JI^T z_J) ----------------
    int last = (int)blockIdx.x;
    while (last + G < nblk) last += G;
    for (int I = last; I >= 0 && s_ok && (int)blockIdx.x < nblk; I -= G) {
        float w = 0.0f;
        if (tid < kBS) {
            const int k = I * kBS + tid;
            if (k < N) {
                // x of rows k and k + 1 (a 2x2 block may straddle into block I + 1)
                auto xval = [&](int kk) {
                    float v = 0.0f;
                    if (!tag_wait(p.xw + kk, e, p.err, v)) atomicExch(&s_ok, 0);
                    return (double)v;
                };
                const double off = p.Doff[k];
                if (off != 0.0) {
                    const double a = p.Dd[k], c = p.Dd[k + 1];
                    const double u = xval(k), v = xval(k + 1);
                    w = (float)((c * u - off * v) / (a * c - off * off));
                } else if (k > 0 && p.Doff[k - 1] != 0.0) {
                    const double a = p.Dd[k - 1], c = p.Dd[k], o2 = p.Doff[k - 1];
                    const double u = xval(k - 1), v = xval(k);
                    w = (float)((a * v - o2 * u) / (a * c - o2 * o2));
                } else {
                    w = (float)(xval(k) / p.Dd[k]);
                }
            }
        }
        __syncthreads();
        if (!s_ok) break;
        float acc = accumulate([&](int J) { return p.Bk + tile_index(J, I) * kTile; }, p.zw, nblk - 1, I, -1, 0.0f);
        if (!s_ok) break;
        load_quarter(p.Bk + tile_index(I, I) * kTile, r, q, reg[0]);
        spart[q][r] = acc;
        __syncthreads();
        if (tid < kBS) sv[0][tid] = w - (spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid]);
        __syncthreads();
        const float a2 = dot_quarter(reg[0], sv[0], q, 0.0f);
        __syncthreads();
        spart[q][r] = a2;
        __syncthreads();
        if (tid < kBS) {
            const float zi = spart[0][tid] + spart[1][tid] + spart[2][tid] + spart[3][tid];
            p.zw[(int64_t)I * kBS + tid] = tag_word(zi, e);
            const int row = I * kBS + tid;
            if (row < N) p.b[p.perm[row]] = (double)zi;
        }
        __syncthreads();
    }

    // the last CTA to finish advances the epoch (every CTA has read it by then)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned d = atomicAdd(p.done, 1u);
        if (d == (unsigned)G - 1u) {
            atomicExch(p.done, 0u);
            __threadfence();
            atomicAdd(p.epoch, 1u);
        }
    }
}

void launch_solve_tagged(cudaStream_t s, int num_sms, int64_t N, const double *Dd, const double *Doff,
                         const int32_t *perm, int64_t nrhs, double *B, int64_t ldb, char *w, int *err_dev) {
    const Layout l = layout_for(N);
    TagSolve p{};
    p.N = (int)N;
    p.nblk = l.nblk;
    p.F = reinterpret_cast<const float *>(w + l.off_F);
    p.Bk = reinterpret_cast<const float *>(w + l.off_B);
    p.Dd = Dd;
    p.Doff = Doff;
    p.perm = perm;
    p.xw = reinterpret_cast<unsigned long long *>(w + l.off_x);
    p.zw = reinterpret_cast<unsigned long long *>(w + l.off_z);
    p.epoch = reinterpret_cast<unsigned *>(w);
    p.done = reinterpret_cast<unsigned *>(w + 4);
    p.err = err_dev;
    int per_sm = 0;
    MDSIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ldlt_solve_tagged, kThreads, 0));
    MDSIP_REQUIRE(per_sm >= 1, MDSIP_ERR_INVALID_ARG, "ldlt_solve: kernel does not fit on an SM");
    const int grid = (int)std::min<int64_t>(l.nblk, (int64_t)num_sms * per_sm);
    for (int64_t rr = 0; rr < nrhs; ++rr) {
        p.b = B + rr * ldb;
        void *args[] = {&p};
        MDSIP_CUDA(cudaLaunchCooperativeKernel((const void *)k_ldlt_solve_tagged, dim3(grid), dim3(kThreads), args,
                                               0, s));
        count_launch();
    }
}

template <typename T>
void launch_solve_t(cudaStream_t s, int num_sms, int64_t N, const double *Dd, const double *Doff,
                    const int32_t *perm, int64_t nrhs, double *B, int64_t ldb, char *w, int *err_dev) {
    const Layout l = layout_for(N);
    FlagSolve<T> p{};
    p.N = (int)N;
    p.nblk = l.nblk;
    p.F = reinterpret_cast<const T *>(w + l.off_F);
    p.Bk = reinterpret_cast<const T *>(w + l.off_B);
    p.Dd = Dd;
    p.Doff = Doff;
    p.perm = perm;
    p.x = reinterpret_cast<T *>(w + l.off_x);
    p.z = reinterpret_cast<T *>(w + l.off_z);
    p.epoch = reinterpret_cast<unsigned *>(w);
    p.done = reinterpret_cast<unsigned *>(w + 4);
    p.fwd = reinterpret_cast<unsigned *>(w + l.off_flags_f);
    p.bwd = reinterpret_cast<unsigned *>(w + l.off_flags_b);
    p.err = err_dev;
    int per_sm = 0;
    MDSIP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ldlt_solve_flags<T>, kThreads, 0));
    MDSIP_REQUIRE(per_sm >= 1, MDSIP_ERR_INVALID_ARG, "ldlt_solve: kernel does not fit on an SM");
    const int grid = (int)std::min<int64_t>(l.nblk, (int64_t)num_sms * per_sm);
    for (int64_t rr = 0; rr < nrhs; ++rr) {
        p.b = B + rr * ldb;
        void *args[] = {&p};
        MDSIP_CUDA(cudaLaunchCooperativeKernel((const void *)k_ldlt_solve_flags<T>, dim3(grid), dim3(kThreads),
                                               args, 0, s));
        count_launch();
    }
}

}  // namespace

size_t ldlt_solve_scratch_bytes(int64_t N) { return layout_for(N).total; }

// Tiles of L (FP64, or FP32 when fp32) and reset flags; once per factorization.
void launch_ldlt_solve_prepare(cudaStream_t s, int64_t N, const double *L, void *scratch, bool fp32) {
    if (N <= 0) return;
    char *w = static_cast<char *>(scratch);
    MDSIP_REQUIRE((reinterpret_cast<uintptr_t>(w) & 255) == 0, MDSIP_ERR_INVALID_ARG,
                  "ldlt_solve: misaligned scratch");
    const Layout l = layout_for(N);
    // epoch, done counter, flags, and the tagged results (a stale word must
    // not carry an epoch of the new series)
    MDSIP_CUDA(cudaMemsetAsync(w, 0, l.off_F, s));
    if (fp32)
        k_solve_tiles<float><<<(unsigned)l.ntile, kThreads, 0, s>>>(
            (int)N, L, reinterpret_cast<float *>(w + l.off_F), reinterpret_cast<float *>(w + l.off_B));
    else
        k_solve_tiles<double><<<(unsigned)l.ntile, kThreads, 0, s>>>(
            (int)N, L, reinterpret_cast<double *>(w + l.off_F), reinterpret_cast<double *>(w + l.off_B));
    MDSIP_LAUNCHED();
}

// b_r <- K^-1 b_r for nrhs right-hand sides (columns of B, ld ldb), with the
// tiles of the last launch_ldlt_solve_prepare (same fp32 flag).  err_dev: set
// to 1 when a bounded wait expires.
void launch_ldlt_solve_coop(cudaStream_t s, int num_sms, int64_t N, const double *Dd, const double *Doff,
                            const int32_t *perm, int64_t nrhs, double *B, int64_t ldb, void *scratch, int *err_dev,
                            bool fp32) {
    if (N <= 0 || nrhs <= 0) return;
    char *w = static_cast<char *>(scratch);
    if (fp32)
        launch_solve_tagged(s, num_sms, N, Dd, Doff, perm, nrhs, B, ldb, w, err_dev);
    else
        launch_solve_t<double>(s, num_sms, N, Dd, Doff, perm, nrhs, B, ldb, w, err_dev);
}

}  // namespace mdsip
