// Fused vector kernels of one Newton step (Section 2.3, kernel classes K1 and
// K2) and the evaluation of the benchmark model family (Section 2 problem
// class).  All FP64.  Reductions are two-pass and deterministic: every
// reduction kernel runs on kRedBlocks blocks and writes one partial per block;
// a finalize kernel combines the partials in block order.
#include "internal.cuh"
#include "vec.cuh"

namespace mdsip {

namespace {

constexpr int NT = kRedThreads;

__device__ __forceinline__ bool fin(double v) { return isfinite(v); }

// partial slot of quantity q for this block
__device__ __forceinline__ double *slot(double *partial, int q) {
    return partial + (size_t)q * kRedBlocks + blockIdx.x;
}

__global__ void k_finalize(const double *partial, int nq, double *out, int op) {
    // one warp per quantity; fixed order inside the warp reduction
    const int q = blockIdx.x;
    if (q >= nq) return;
    const double *p = partial + (size_t)q * kRedBlocks;
    double v = op == 0 ? 0.0 : (op == 1 ? -INFINITY : INFINITY);
    for (int b = threadIdx.x; b < kRedBlocks; b += 32) {
        const double x = p[b];
        v = op == 0 ? v + x : (op == 1 ? fmax(v, x) : fmin(v, x));
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double x = __shfl_down_sync(0xffffffffu, v, o);
        v = op == 0 ? v + x : (op == 1 ? fmax(v, x) : fmin(v, x));
    }
    if (threadIdx.x == 0) out[q] = v;
}

// ---------------------------------------------------------------------------
// Model: f and grad f.  f = 1/2 x_d^T Q x_d + sum 1/4 x_s^4 + c^T x
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_eval_f(Dims D, ModelView M, const double *__restrict__ x,
                                               double *__restrict__ grad, double *partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * NT;
    for (int64_t i = gtid; i < D.n_s; i += gsz) {
        const double v = x[i];
        const double v2 = v * v;
        acc += 0.25 * v2 * v2 + M.c[i] * v;
        if (grad) grad[i] = v2 * v + M.c[i];
    }
    // x_d part: one warp per row of Q
    const int lane = threadIdx.x & 31;
    const int64_t gw = gtid >> 5, nw = gsz >> 5;
    const double *xd = x + D.n_s;
    for (int64_t p = gw; p < D.n_d; p += nw) {
        const double *row = M.Q + p * D.n_d;
        double s = 0.0;
        for (int64_t k = lane; k < D.n_d; k += 32) s += row[k] * xd[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double cp = M.c[D.n_s + p];
            acc += 0.5 * xd[p] * s + cp * xd[p];
            if (grad) grad[D.n_s + p] = s + cp;
        }
    }
    const double r = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) *slot(partial, 0) = r;
}

// ---------------------------------------------------------------------------
// Model: constraint residuals cg = g(x) - g_E (warp per row: sparse part plus
// the dense row of A), ch = h(x) - d.  Reductions: sum |c|, max |c|.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_eval_cons(Dims D, ModelView M, const double *__restrict__ x,
                                                  const double *__restrict__ Axd, const double *__restrict__ d,
                                                  double *__restrict__ cg, double *__restrict__ ch,
                                                  double *partial) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * NT) >> 5;
    const double *xd = x + D.n_s;
    double s1 = 0.0, mx = 0.0;
    // equalities: the dense part A x_d comes from the row-block pass (Axd)
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < D.m_E; i += (int64_t)gridDim.x * NT) {
        double s = Axd[i];
        for (int e = M.csr_ptr[i]; e < M.csr_ptr[i + 1]; ++e) s += M.csr_val[e] * x[M.csr_col[e]];
        const double r = s - M.gE[i];
        cg[i] = r;
        s1 += fabs(r);
        mx = fmax(mx, fabs(r));
    }
    for (int64_t j = gw; j < D.m_I; j += nw) {
        double s = 0.0;
        for (int64_t k = lane; k < D.n_d; k += 32)
            if (M.h_set[k] == j) s += xd[k] * xd[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (M.hsr_ptr)   // the sparse x_s part of the inequality (J_sh x_s)_j
                for (int e = M.hsr_ptr[j]; e < M.hsr_ptr[j + 1]; ++e) s += M.hsr_val[e] * x[M.hsr_col[e]];
            const double r = s - d[j];
            ch[j] = r;
            s1 += fabs(r);
            mx = fmax(mx, fabs(r));
        }
    }
    const double a = block_sum<NT>(s1, sh);
    if (threadIdx.x == 0) *slot(partial, 0) = a;
    const double b = block_max<NT>(mx, sh);
    if (threadIdx.x == 0) *slot(partial, 1) = b;
}

// Jacobian of h (dense m_I x n_d row-major) and the Hessian blocks:
// Hss = 3 x_s^2 (diagonal), Hdd = Q + 2 diag(y_h[h_set[k]]).
__global__ void k_jac_hess(Dims D, ModelView M, const double *__restrict__ x,
                           const double *__restrict__ yh, double *__restrict__ Jdh,
                           double *__restrict__ Hss, double *__restrict__ Hdd) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const double *xd = x + D.n_s;
    for (int64_t i = gtid; i < D.n_s; i += gsz) Hss[i] = 3.0 * x[i] * x[i];
    for (int64_t e = gtid; e < D.m_I * D.n_d; e += gsz) {
        const int64_t j = e / D.n_d, k = e % D.n_d;
        Jdh[e] = M.h_set[k] == j ? 2.0 * xd[k] : 0.0;
    }
    for (int64_t e = gtid; e < D.n_d * D.n_d; e += gsz) {
        const int64_t p = e / D.n_d, q = e % D.n_d;
        double v = M.Q[e];
        if (p == q && M.h_set[p] >= 0) v += 2.0 * yh[M.h_set[p]];
        Hdd[e] = v;
    }
}

// ---------------------------------------------------------------------------
// A passes
// ---------------------------------------------------------------------------
// out = A v: two threads per row, v staged in shared memory.  The pair reads
// alternate 16-byte chunks of its row, so each warp load fills 16 whole
// 32-byte sectors; each thread keeps eight independent FP64 accumulators and
// loads the next group of its row before using the current one (a pass over A
// is bound by memory latency at the ~20 rows per SM that one-thread-per-row
// occupancy gives, and on GB300 by the DFMA rate next: 2 flop per 8 bytes).
__global__ void __launch_bounds__(NT) k_gemv_rows(const double *__restrict__ A, int64_t m, int64_t n,
                                                  int64_t lda, const double *__restrict__ v,
                                                  double *__restrict__ out) {
    extern __shared__ double vs[];   // n rounded up to a multiple of 16, zero padded
    const int64_t n16 = (n + 15) / 16 * 16;
    for (int64_t k = threadIdx.x; k < n16; k += NT) vs[k] = k < n ? v[k] : 0.0;
    __syncthreads();
    const int64_t gt = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t i = gt >> 1;
    const int h = (int)(gt & 1);
    const bool live = i < m;
    const double2 *r = reinterpret_cast<const double2 *>(A + (live ? i : 0) * lda);
    const double2 *x2 = reinterpret_cast<const double2 *>(vs);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    const int64_t full = live ? n / 16 : 0;   // groups of 16 columns (8 chunks; 4 per thread)
    double2 cur[4], nxt[4] = {};
    if (full > 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = __ldg(r + h + 2 * u);
    }
    for (int64_t g = 0; g < full; ++g) {
        if (g + 1 < full) {
#pragma unroll
            for (int u = 0; u < 4; ++u) nxt[u] = __ldg(r + 8 * (g + 1) + h + 2 * u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 b = x2[8 * g + h + 2 * u];
            acc[2 * u] = fma(cur[u].x, b.x, acc[2 * u]);
            acc[2 * u + 1] = fma(cur[u].y, b.y, acc[2 * u + 1]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = nxt[u];
    }
    if (live && h == 0) {
        const double *rd = A + i * lda;
#pragma unroll
        for (int t = 0; t < 16; ++t) {   // ragged tail (fewer than 16 columns)
            const int64_t c = 16 * full + t;
            if (c < n) acc[t & 7] = fma(rd[c], vs[c], acc[t & 7]);
        }
    }
    double sum = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);   // the pair's halves (every lane reaches this)
    if (live && h == 0) out[i] = sum;
}

// partial[b][p] = sum over the rows of block b of A[i][p] u[i]
constexpr int kGtCols = 8;  // columns per thread per pass
__global__ void __launch_bounds__(NT) k_gemv_t(const double *__restrict__ A, int64_t m, int64_t n,
                                               int64_t lda, const double *__restrict__ u,
                                               double *__restrict__ partial) {
    const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(m, r0 + rows_per);
    for (int64_t c0 = 0; c0 < n; c0 += (int64_t)NT * kGtCols) {
        double acc[kGtCols];
#pragma unroll
        for (int c = 0; c < kGtCols; ++c) acc[c] = 0.0;
        int64_t i = r0;
        for (; i + 1 < r1; i += 2) {
            const double u0 = u[i], u1 = u[i + 1];
            const double *row0 = A + i * lda, *row1 = row0 + lda;
            double a0[kGtCols], a1[kGtCols];
#pragma unroll
            for (int c = 0; c < kGtCols; ++c) {
                const int64_t p = c0 + threadIdx.x + (int64_t)c * NT;
                a0[c] = p < n ? __ldg(row0 + p) : 0.0;
                a1[c] = p < n ? __ldg(row1 + p) : 0.0;
            }
#pragma unroll
            for (int c = 0; c < kGtCols; ++c) acc[c] = fma(a1[c], u1, fma(a0[c], u0, acc[c]));
        }
        for (; i < r1; ++i) {
            const double ui = u[i];
            const double *row = A + i * lda;
#pragma unroll
            for (int c = 0; c < kGtCols; ++c) {
                const int64_t p = c0 + threadIdx.x + (int64_t)c * NT;
                if (p < n) acc[c] = fma(__ldg(row + p), ui, acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < kGtCols; ++c) {
            const int64_t p = c0 + threadIdx.x + (int64_t)c * NT;
            if (p < n) partial[(size_t)blockIdx.x * n + p] = acc[c];
        }
    }
}

// out[p] = sum_b partial[b][p]: a block per 32 columns, warp w summing the
// partials b = w, w + 8, ... in order (coalesced 32-column rows, eight rows in
// flight per warp), then the eight warp sums in order (deterministic).
__global__ void __launch_bounds__(256) k_colsum(const double *__restrict__ partial, int nparts, int64_t n,
                                                double *__restrict__ out) {
    __shared__ double sp[8][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * 32 + lane;
    double s = 0.0;
    if (p < n) {
        int b = wid;
        for (; b + 24 < nparts; b += 32) {
            const double a0 = partial[(size_t)b * n + p], a1 = partial[(size_t)(b + 8) * n + p];
            const double a2 = partial[(size_t)(b + 16) * n + p], a3 = partial[(size_t)(b + 24) * n + p];
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; b < nparts; b += 8) s += partial[(size_t)b * n + p];
    }
    sp[wid][lane] = s;
    __syncthreads();
    if (wid == 0 && p < n) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += sp[w][lane];
        out[p] = t;
    }
}

// ---------------------------------------------------------------------------
// Gradient of the Lagrangian: gl = grad f + J_g^T y_g + J_h^T y_h
// ---------------------------------------------------------------------------
__global__ void k_lagrangian_grad(Dims D, ModelView M, const double *__restrict__ grad,
                                  const double *__restrict__ yg, const double *__restrict__ yh,
                                  const double *__restrict__ Jdh, const double *__restrict__ ATy,
                                  double *__restrict__ gl) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.n_s; i += gsz) {
        double s = grad[i];
        for (int e = M.csc_ptr[i]; e < M.csc_ptr[i + 1]; ++e) s += M.csc_val[e] * yg[M.csc_row[e]];
        if (M.hsc_ptr)
            for (int e = M.hsc_ptr[i]; e < M.hsc_ptr[i + 1]; ++e) s += M.hsc_val[e] * yh[M.hsc_row[e]];
        gl[i] = s;
    }
    for (int64_t k = gtid; k < D.n_d; k += gsz) {
        double s = grad[D.n_s + k] + ATy[k];
        for (int64_t j = 0; j < D.m_I; ++j) s += Jdh[j * D.n_d + k] * yh[j];
        gl[D.n_s + k] = s;
    }
}

// ---------------------------------------------------------------------------
// Optimality error components (W&B scaled KKT error) and the log-barrier sum.
// quantities: 0 max|dual| (max), 1 max|c| (max), 2 max s*z (max),
//             3 min s*z (min), 4 ||y||_1 (sum), 5 ||z||_1 (sum), 6 sum log s (sum)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_errors(Dims D, ModelView M, IterView I,
                                               const double *__restrict__ gl,
                                               const double *__restrict__ cg,
                                               const double *__restrict__ ch, double *partial) {
    __shared__ double sh[32];
    double du = 0.0, pr = 0.0, cmax = -INFINITY, cmin = INFINITY, y1 = 0.0, z1 = 0.0, lg = 0.0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * NT;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double xi = I.x[i];
        du = fmax(du, fabs(gl[i] - I.zl[i] + I.zu[i]));
        if (isfinite(M.xl[i])) {
            const double s = xi - M.xl[i];
            const double p = s * I.zl[i];
            cmax = fmax(cmax, p);
            cmin = fmin(cmin, p);
            z1 += fabs(I.zl[i]);
            lg += log(s);
        }
        if (isfinite(M.xu[i])) {
            const double s = M.xu[i] - xi;
            const double p = s * I.zu[i];
            cmax = fmax(cmax, p);
            cmin = fmin(cmin, p);
            z1 += fabs(I.zu[i]);
            lg += log(s);
        }
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        du = fmax(du, fabs(-I.yh[j] - I.vl[j] + I.vu[j]));
        pr = fmax(pr, fabs(ch[j]));
        y1 += fabs(I.yh[j]);
        const double dj = I.d[j];
        if (isfinite(M.hl[j])) {
            const double s = dj - M.hl[j];
            const double p = s * I.vl[j];
            cmax = fmax(cmax, p);
            cmin = fmin(cmin, p);
            z1 += fabs(I.vl[j]);
            lg += log(s);
        }
        if (isfinite(M.hu[j])) {
            const double s = M.hu[j] - dj;
            const double p = s * I.vu[j];
            cmax = fmax(cmax, p);
            cmin = fmin(cmin, p);
            z1 += fabs(I.vu[j]);
            lg += log(s);
        }
    }
    for (int64_t i = gtid; i < D.m_E; i += gsz) {
        pr = fmax(pr, fabs(cg[i]));
        y1 += fabs(I.yg[i]);
    }
    double r;
    r = block_max<NT>(du, sh);   if (threadIdx.x == 0) *slot(partial, 0) = r;
    r = block_max<NT>(pr, sh);   if (threadIdx.x == 0) *slot(partial, 1) = r;
    r = block_max<NT>(cmax, sh); if (threadIdx.x == 0) *slot(partial, 2) = r;
    r = block_min<NT>(cmin, sh); if (threadIdx.x == 0) *slot(partial, 3) = r;
    r = block_sum<NT>(y1, sh);   if (threadIdx.x == 0) *slot(partial, 4) = r;
    r = block_sum<NT>(z1, sh);   if (threadIdx.x == 0) *slot(partial, 5) = r;
    r = block_sum<NT>(lg, sh);   if (threadIdx.x == 0) *slot(partial, 6) = r;
}

// ---------------------------------------------------------------------------
// Diagonal scaling (Section 2.1 barrier diagonals) and the diagonal W of the
// two-stage elimination.  q = H_ss + Sigma_xs + dw; Sigma_d; w = J_sg^2 q^-1 + dc.
// quantities: 0..2 inertia of Q_s (pos, neg, zero), 3..5 inertia of -W.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sigma_x(const ModelView &M, const IterView &I, int64_t i) {
    double s = 0.0;
    if (isfinite(M.xl[i])) s += I.zl[i] / (I.x[i] - M.xl[i]);
    if (isfinite(M.xu[i])) s += I.zu[i] / (M.xu[i] - I.x[i]);
    return s;
}

__global__ void __launch_bounds__(NT) k_newton_diag(Dims D, ModelView M, IterView I,
                                                    const double *__restrict__ Hss, double dw,
                                                    double dc, int want_w, double *__restrict__ sig_x,
                                                    double *__restrict__ q, double *__restrict__ sig_d,
                                                    double *__restrict__ w, double *partial) {
    __shared__ double sh[32];
    double qp = 0, qn = 0, qz = 0, wp = 0, wn = 0, wz = 0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * NT;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double s = sigma_x(M, I, i);
        sig_x[i] = s;
        if (i < D.n_s) {
            const double qi = Hss[i] + s + dw;
            q[i] = qi;
            qp += qi > 0.0;
            qn += qi < 0.0;
            qz += qi == 0.0;
        }
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        double s = 0.0;
        if (isfinite(M.hl[j])) s += I.vl[j] / (I.d[j] - M.hl[j]);
        if (isfinite(M.hu[j])) s += I.vu[j] / (M.hu[j] - I.d[j]);
        sig_d[j] = s;
    }
    if (want_w) {
        for (int64_t i = gtid; i < D.m_E; i += gsz) {
            double s = dc;
            for (int e = M.csr_ptr[i]; e < M.csr_ptr[i + 1]; ++e) {
                const int64_t c = M.csr_col[e];
                const double qc = Hss[c] + sigma_x(M, I, c) + dw;
                s += M.csr_val[e] * M.csr_val[e] / qc;
            }
            w[i] = s;
            // inertia of -W
            wp += s < 0.0;
            wn += s > 0.0;
            wz += s == 0.0;
        }
    }
    double r;
    r = block_sum<NT>(qp, sh); if (threadIdx.x == 0) *slot(partial, 0) = r;
    r = block_sum<NT>(qn, sh); if (threadIdx.x == 0) *slot(partial, 1) = r;
    r = block_sum<NT>(qz, sh); if (threadIdx.x == 0) *slot(partial, 2) = r;
    r = block_sum<NT>(wp, sh); if (threadIdx.x == 0) *slot(partial, 3) = r;
    r = block_sum<NT>(wn, sh); if (threadIdx.x == 0) *slot(partial, 4) = r;
    r = block_sum<NT>(wz, sh); if (threadIdx.x == 0) *slot(partial, 5) = r;
}

// barrier gradient of the Lagrangian at x: rN_i = gl_i - mu/s_l + mu/s_u
__device__ __forceinline__ double rN_x(const ModelView &M, const IterView &I, const double *gl,
                                       double mu, int64_t i) {
    double r = gl[i];
    if (isfinite(M.xl[i])) r -= mu / (I.x[i] - M.xl[i]);
    if (isfinite(M.xu[i])) r += mu / (M.xu[i] - I.x[i]);
    return r;
}

// r_d = grad_d phi - y_h = -mu/(d - hl) + mu/(hu - d) - y_h
__device__ __forceinline__ double r_dslack(const ModelView &M, const IterView &I, double mu,
                                           int64_t j) {
    double r = -I.yh[j];
    if (isfinite(M.hl[j])) r -= mu / (I.d[j] - M.hl[j]);
    if (isfinite(M.hu[j])) r += mu / (M.hu[j] - I.d[j]);
    return r;
}

// ---------------------------------------------------------------------------
// Right-hand sides.  b = -[rN_x; c_g; c_h + Dh^-1 r_d] (Eq. (linsys4x4) rows).
// Path P2: bt_g = b_g - J_sg (b_s / q);  u = bt_g / w;  rhs_S = [b_d + A^T u; b_h]
// Path P1: rhs_M = [b_d; b_y - J_s (b_s / q)]
// ---------------------------------------------------------------------------
__global__ void k_rhs_y(Dims D, ModelView M, IterView I, const double *__restrict__ gl,
                        const double *__restrict__ cg, const double *__restrict__ q,
                        const double *__restrict__ w, double mu, double *__restrict__ bt_g,
                        double *__restrict__ u) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.m_E; i += gsz) {
        double s = -cg[i];
        for (int e = M.csr_ptr[i]; e < M.csr_ptr[i + 1]; ++e) {
            const int64_t c = M.csr_col[e];
            s += M.csr_val[e] * rN_x(M, I, gl, mu, c) / q[c];   // -J_sg (b_s/q), b_s = -rN_s
        }
        bt_g[i] = s;
        if (u) u[i] = s / w[i];
    }
}

// P2: rhs_S[0:n_d] = -rN_xd + ATu ; rhs_S[n_d + j] = -(ch + r_d / Dh)
// P1: rhs_M[0:n_d] = -rN_xd ; rhs_M[n_d + i] = bt_g[i] ; rhs_M[n_d + m_E + j] = -(ch + r_d/Dh)
// (with J_sh != 0, P1's h rows also take -J_sh (b_s / q))
__global__ void k_rhs_reduced(Dims D, ModelView M, IterView I, const double *__restrict__ gl,
                              const double *__restrict__ ch, const double *__restrict__ sig_d,
                              const double *__restrict__ ATu, const double *__restrict__ bt_g,
                              const double *__restrict__ q, double mu, double dw, int p1,
                              double *__restrict__ rhs) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = gtid; k < D.n_d; k += gsz) {
        double r = -rN_x(M, I, gl, mu, D.n_s + k);
        if (!p1) r += ATu[k];
        rhs[k] = r;
    }
    const int64_t off_h = p1 ? D.n_d + D.m_E : D.n_d;
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        double r = -(ch[j] + r_dslack(M, I, mu, j) / (sig_d[j] + dw));
        if (p1 && M.hsr_ptr)
            for (int e = M.hsr_ptr[j]; e < M.hsr_ptr[j + 1]; ++e) {
                const int64_t c = M.hsr_col[e];
                r += M.hsr_val[e] * rN_x(M, I, gl, mu, c) / q[c];   // -J_sh (b_s/q), b_s = -rN_s
            }
        rhs[off_h + j] = r;
    }
    if (p1)
        for (int64_t i = gtid; i < D.m_E; i += gsz) rhs[D.n_d + i] = bt_g[i];
}

// P2: dy_g = (A dx_d - bt_g) / w
__global__ void k_dyg_p2(int64_t m_E, const double *__restrict__ Adx, const double *__restrict__ bt_g,
                         const double *__restrict__ w, double *__restrict__ dyg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_E;
         i += (int64_t)gridDim.x * blockDim.x)
        dyg[i] = (Adx[i] - bt_g[i]) / w[i];
}

// Common back-substitution: dx_s = (b_s - J_sg^T dy_g)/q, dx_d, dy_h from the
// reduced solution, dd = (dy_h - r_d)/Dh, and the bound-multiplier steps
// dz = mu/s - z - (z/s) ds (W&B eq. (11)).
__global__ void k_backsub(Dims D, ModelView M, IterView I, DirView Dir, const double *__restrict__ gl,
                          const double *__restrict__ q, const double *__restrict__ sig_d,
                          const double *__restrict__ sol_dxd, const double *__restrict__ sol_dyh,
                          double mu, double dw) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        double dx;
        if (i < D.n_s) {
            double s = -rN_x(M, I, gl, mu, i);
            for (int e = M.csc_ptr[i]; e < M.csc_ptr[i + 1]; ++e)
                s -= M.csc_val[e] * Dir.dyg[M.csc_row[e]];
            if (M.hsc_ptr)   // J_sh^T dy_h (dy_h from the reduced solution: Dir.dyh is written below)
                for (int e = M.hsc_ptr[i]; e < M.hsc_ptr[i + 1]; ++e) s -= M.hsc_val[e] * sol_dyh[M.hsc_row[e]];
            dx = s / q[i];
        } else {
            dx = sol_dxd[i - D.n_s];
        }
        Dir.dx[i] = dx;
        const double xi = I.x[i];
        if (isfinite(M.xl[i])) {
            const double s = xi - M.xl[i];
            Dir.dzl[i] = mu / s - I.zl[i] - I.zl[i] / s * dx;
        } else {
            Dir.dzl[i] = 0.0;
        }
        if (isfinite(M.xu[i])) {
            const double s = M.xu[i] - xi;
            Dir.dzu[i] = mu / s - I.zu[i] + I.zu[i] / s * dx;
        } else {
            Dir.dzu[i] = 0.0;
        }
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double dyh = sol_dyh[j];
        Dir.dyh[j] = dyh;
        const double dd = (dyh - r_dslack(M, I, mu, j)) / (sig_d[j] + dw);
        Dir.dd[j] = dd;
        const double dj = I.d[j];
        if (isfinite(M.hl[j])) {
            const double s = dj - M.hl[j];
            Dir.dvl[j] = mu / s - I.vl[j] - I.vl[j] / s * dd;
        } else {
            Dir.dvl[j] = 0.0;
        }
        if (isfinite(M.hu[j])) {
            const double s = M.hu[j] - dj;
            Dir.dvu[j] = mu / s - I.vu[j] + I.vu[j] / s * dd;
        } else {
            Dir.dvu[j] = 0.0;
        }
    }
}

// Distance between two packed directions: quantities 0 = sum (a - b)^2,
// 1 = sum b^2 over the eight blocks (dx, dd, dyg, dyh, dzl, dzu, dvl, dvu).
__global__ void __launch_bounds__(NT) k_dir_diff(Dims D, DirView a, DirView b, double *partial) {
    __shared__ double sh[32];
    const double *pa[8] = {a.dx, a.dd, a.dyg, a.dyh, a.dzl, a.dzu, a.dvl, a.dvu};
    const double *pb[8] = {b.dx, b.dd, b.dyg, b.dyh, b.dzl, b.dzu, b.dvl, b.dvu};
    const int64_t len[8] = {D.n, D.m_I, D.m_E, D.m_I, D.n, D.n, D.m_I, D.m_I};
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * NT;
    double dd = 0.0, bb = 0.0;
    for (int k = 0; k < 8; ++k)
        for (int64_t i = gtid; i < len[k]; i += gsz) {
            const double y = pb[k][i], e = pa[k][i] - y;
            dd += e * e;
            bb += y * y;
        }
    double r;
    r = block_sum<NT>(dd, sh); if (threadIdx.x == 0) *slot(partial, 0) = r;
    r = block_sum<NT>(bb, sh); if (threadIdx.x == 0) *slot(partial, 1) = r;
}

__global__ void k_copy(const double *__restrict__ src, double *__restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Line-search scalars: fraction-to-boundary (Section 2.1: the search starts at
// the farthest bound-feasible point) and grad phi^T d.
// quantities: 0 alpha_max (min), 1 alpha_z (min), 2 gphi (sum)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ftb(double v, double dv, double tau) {
    return dv < 0.0 ? -tau * v / dv : INFINITY;
}

__global__ void __launch_bounds__(NT) k_step_scalars(Dims D, ModelView M, IterView I, DirView Dir,
                                                     const double *__restrict__ grad, double tau,
                                                     double mu, double *partial) {
    __shared__ double sh[32];
    double ap = INFINITY, az = INFINITY, gp = 0.0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * NT;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double dx = Dir.dx[i];
        double g = grad[i];
        if (isfinite(M.xl[i])) {
            const double s = I.x[i] - M.xl[i];
            ap = fmin(ap, ftb(s, dx, tau));
            az = fmin(az, ftb(I.zl[i], Dir.dzl[i], tau));
            g -= mu / s;
        }
        if (isfinite(M.xu[i])) {
            const double s = M.xu[i] - I.x[i];
            ap = fmin(ap, ftb(s, -dx, tau));
            az = fmin(az, ftb(I.zu[i], Dir.dzu[i], tau));
            g += mu / s;
        }
        gp += g * dx;
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double dd = Dir.dd[j];
        double g = 0.0;
        if (isfinite(M.hl[j])) {
            const double s = I.d[j] - M.hl[j];
            ap = fmin(ap, ftb(s, dd, tau));
            az = fmin(az, ftb(I.vl[j], Dir.dvl[j], tau));
            g -= mu / s;
        }
        if (isfinite(M.hu[j])) {
            const double s = M.hu[j] - I.d[j];
            ap = fmin(ap, ftb(s, -dd, tau));
            az = fmin(az, ftb(I.vu[j], Dir.dvu[j], tau));
            g += mu / s;
        }
        gp += g * dd;
    }
    double r;
    r = block_min<NT>(ap, sh); if (threadIdx.x == 0) *slot(partial, 0) = r;
    r = block_min<NT>(az, sh); if (threadIdx.x == 0) *slot(partial, 1) = r;
    r = block_sum<NT>(gp, sh); if (threadIdx.x == 0) *slot(partial, 2) = r;
}

// Trial point x_t = x + alpha dx, d_t = d + alpha dd; sum of log slacks and
// "strictly inside" count at the trial point.
// quantities: 0 sum log s (sum), 1 number of non-positive slacks (sum)
__global__ void __launch_bounds__(NT) k_trial(Dims D, ModelView M, IterView I, DirView Dir,
                                              double alpha, double *__restrict__ xt,
                                              double *__restrict__ dt, double *partial) {
    __shared__ double sh[32];
    double lg = 0.0, bad = 0.0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * NT;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double v = I.x[i] + alpha * Dir.dx[i];
        xt[i] = v;
        if (isfinite(M.xl[i])) {
            const double s = v - M.xl[i];
            if (s > 0.0) lg += log(s); else bad += 1.0;
        }
        if (isfinite(M.xu[i])) {
            const double s = M.xu[i] - v;
            if (s > 0.0) lg += log(s); else bad += 1.0;
        }
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double v = I.d[j] + alpha * Dir.dd[j];
        dt[j] = v;
        if (isfinite(M.hl[j])) {
            const double s = v - M.hl[j];
            if (s > 0.0) lg += log(s); else bad += 1.0;
        }
        if (isfinite(M.hu[j])) {
            const double s = M.hu[j] - v;
            if (s > 0.0) lg += log(s); else bad += 1.0;
        }
    }
    double r;
    r = block_sum<NT>(lg, sh);  if (threadIdx.x == 0) *slot(partial, 0) = r;
    r = block_sum<NT>(bad, sh); if (threadIdx.x == 0) *slot(partial, 1) = r;
}

// Accept: y += alpha dy, z += alpha_z dz, then the kappa_Sigma safeguard
// (W&B eq. (16)) against the new slacks (x, d already hold the new point).
__global__ void k_accept(Dims D, ModelView M, IterView I, DirView Dir, double alpha,
                         double alpha_z, double mu, double ks) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    auto guard = [&](double z, double s) { return fmax(fmin(z, ks * mu / s), mu / (ks * s)); };
    for (int64_t i = gtid; i < D.m_E; i += gsz) I.yg[i] += alpha * Dir.dyg[i];
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        I.yh[j] += alpha * Dir.dyh[j];
        const double dj = I.d[j];
        if (isfinite(M.hl[j])) I.vl[j] = guard(I.vl[j] + alpha_z * Dir.dvl[j], dj - M.hl[j]);
        if (isfinite(M.hu[j])) I.vu[j] = guard(I.vu[j] + alpha_z * Dir.dvu[j], M.hu[j] - dj);
    }
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double xi = I.x[i];
        if (isfinite(M.xl[i])) I.zl[i] = guard(I.zl[i] + alpha_z * Dir.dzl[i], xi - M.xl[i]);
        if (isfinite(M.xu[i])) I.zu[i] = guard(I.zu[i] + alpha_z * Dir.dzu[i], M.xu[i] - xi);
    }
}

// W&B Section 3.6 starting point: push x0 (and d0 = h(x0)) inside the bounds;
// multipliers of finite bounds 1, y = 0.
__device__ double push_inside(double v, double lo, double hi, double k1, double k2) {
    const bool hl = isfinite(lo), hu = isfinite(hi);
    const double width = (hl && hu) ? hi - lo : INFINITY;
    if (hl) {
        const double pl = fmin(k1 * fmax(1.0, fabs(lo)), k2 * width);
        v = fmax(v, lo + pl);
    }
    if (hu) {
        const double pu = fmin(k1 * fmax(1.0, fabs(hi)), k2 * width);
        v = fmin(v, hi - pu);
    }
    return v;
}

__global__ void k_init_x(Dims D, ModelView M, const double *__restrict__ x0, double k1, double k2,
                         IterView I) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        I.x[i] = push_inside(x0 ? x0[i] : 0.0, M.xl[i], M.xu[i], k1, k2);
        I.zl[i] = isfinite(M.xl[i]) ? 1.0 : 0.0;
        I.zu[i] = isfinite(M.xu[i]) ? 1.0 : 0.0;
    }
    for (int64_t i = gtid; i < D.m_E; i += gsz) I.yg[i] = 0.0;
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        I.yh[j] = 0.0;
        I.d[j] = 0.0;
        I.vl[j] = isfinite(M.hl[j]) ? 1.0 : 0.0;
        I.vu[j] = isfinite(M.hu[j]) ? 1.0 : 0.0;
    }
}

// d0 = push(h(x0)); ch currently holds h(x0) - 0
__global__ void k_init_d(Dims D, ModelView M, const double *__restrict__ ch, double k1, double k2,
                         IterView I) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < D.m_I;
         j += (int64_t)gridDim.x * blockDim.x)
        I.d[j] = push_inside(ch[j], M.hl[j], M.hu[j], k1, k2);
}

// Warm start from a prediction in the packed layout [x | d | y_g | y_h | z_l |
// z_u | v_l | v_u]: primal values pushed inside the bounds (the Section 3.6
// rule of W&B with kappa_1 = kappa_2 = push), each finite-bound multiplier
// raised to at least mu0 / (its slack), so that every complementarity
// product is at least mu0; multipliers of infinite bounds are 0.
__global__ void k_start_predicted(Dims D, ModelView M, const float *__restrict__ pred, double push, double mu0,
                                  IterView I) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t o_d = D.n, o_yg = o_d + D.m_I, o_yh = o_yg + D.m_E, o_zl = o_yh + D.m_I, o_zu = o_zl + D.n,
                  o_vl = o_zu + D.n, o_vu = o_vl + D.m_I;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double lo = M.xl[i], hi = M.xu[i];
        const double x = push_inside((double)pred[i], lo, hi, push, push);
        I.x[i] = x;
        I.zl[i] = isfinite(lo) ? fmax((double)pred[o_zl + i], mu0 / (x - lo)) : 0.0;
        I.zu[i] = isfinite(hi) ? fmax((double)pred[o_zu + i], mu0 / (hi - x)) : 0.0;
    }
    for (int64_t i = gtid; i < D.m_E; i += gsz) I.yg[i] = (double)pred[o_yg + i];
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double lo = M.hl[j], hi = M.hu[j];
        const double d = push_inside((double)pred[o_d + j], lo, hi, push, push);
        I.d[j] = d;
        I.yh[j] = (double)pred[o_yh + j];
        I.vl[j] = isfinite(lo) ? fmax((double)pred[o_vl + j], mu0 / (d - lo)) : 0.0;
        I.vu[j] = isfinite(hi) ? fmax((double)pred[o_vu + j], mu0 / (hi - d)) : 0.0;
    }
}

__global__ void __launch_bounds__(NT) k_cons_from_values(Dims D, ModelView M, const double *__restrict__ g,
                                                         const double *__restrict__ h, const double *__restrict__ d,
                                                         double *__restrict__ cg, double *__restrict__ ch,
                                                         double *partial) {
    __shared__ double sh[32];
    double s1 = 0.0, mx = 0.0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x, gsz = (int64_t)gridDim.x * NT;
    for (int64_t i = gtid; i < D.m_E; i += gsz) {
        const double r = g[i] - M.gE[i];
        cg[i] = r;
        s1 += fabs(r);
        mx = fmax(mx, fabs(r));
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double r = h[j] - d[j];
        ch[j] = r;
        s1 += fabs(r);
        mx = fmax(mx, fabs(r));
    }
    const double a = block_sum<NT>(s1, sh);
    if (threadIdx.x == 0) *slot(partial, 0) = a;
    const double b = block_max<NT>(mx, sh);
    if (threadIdx.x == 0) *slot(partial, 1) = b;
}

__global__ void k_gather(int64_t n, const double *__restrict__ src, const int32_t *__restrict__ idx,
                         double *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_finalize_sum(cudaStream_t s, const double *partial, int nq, double *out) {
    k_finalize<<<nq, 32, 0, s>>>(partial, nq, out, 0);
    MDSIP_LAUNCHED();
}
void launch_finalize_max(cudaStream_t s, const double *partial, int nq, double *out) {
    k_finalize<<<nq, 32, 0, s>>>(partial, nq, out, 1);
    MDSIP_LAUNCHED();
}
void launch_finalize_min(cudaStream_t s, const double *partial, int nq, double *out) {
    k_finalize<<<nq, 32, 0, s>>>(partial, nq, out, 2);
    MDSIP_LAUNCHED();
}

static int elem_grid(int64_t n) { return std::max(1, std::min(4096, ceil_div(n, 256))); }

// A: rows 16-byte aligned (lda even, A 16-byte aligned); n <= 24560 (v staged in shared memory)
void launch_gemv_rows(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda,
                      const double *v, double *out) {
    if (m <= 0) return;
    MDSIP_REQUIRE((lda & 1) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0, MDSIP_ERR_INVALID_ARG,
                  "gemv: rows of A must be 16-byte aligned");
    const size_t smem = (size_t)((n + 15) / 16) * 16 * sizeof(double);
    MDSIP_REQUIRE(smem <= 192 * 1024, MDSIP_ERR_INVALID_ARG, "gemv: n too large");
    static PerDeviceOnce once;
    MDSIP_CUDA(once.run([] {
        return cudaFuncSetAttribute(k_gemv_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 * 1024);
    }));
    const int64_t grid = (2 * m + NT - 1) / NT;   // two threads per row
    MDSIP_REQUIRE(grid <= 0x7fffffff, MDSIP_ERR_INVALID_ARG, "gemv: m too large");
    k_gemv_rows<<<(unsigned)grid, NT, smem, s>>>(A, m, n, lda, v, out);
    MDSIP_LAUNCHED();
}

void launch_colsum(cudaStream_t s, const double *partial, int nparts, int64_t n, double *out) {
    if (n <= 0) return;
    k_colsum<<<(unsigned)ceil_div(n, 32), 256, 0, s>>>(partial, nparts, n, out);
    MDSIP_LAUNCHED();
}

void launch_gemv_t(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda,
                   const double *u, double *partial, double *out) {
    if (n <= 0) return;
    if (m <= 0) {
        MDSIP_CUDA(cudaMemsetAsync(out, 0, n * sizeof(double), s));
        return;
    }
    k_gemv_t<<<kRedBlocks, NT, 0, s>>>(A, m, n, lda, u, partial);
    MDSIP_LAUNCHED();
    k_colsum<<<(unsigned)ceil_div(n, 32), 256, 0, s>>>(partial, kRedBlocks, n, out);
    MDSIP_LAUNCHED();
}

void VecOps::eval_f(const double *x, double *grad, double *out_scalar) {
    k_eval_f<<<kRedBlocks, NT, 0, st>>>(D, M, x, grad, partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 1, out_scalar);
}

void VecOps::eval_cons(const double *x, const double *d, double *cg, double *ch, double *out2) {
    if (D.m_E > 0) {
        if (Ahi) launch_gemv_rows_df(st, Ahi, Alo, D.m_E, D.n_d, D.lda, x + D.n_s, split, rowtmp);
        else launch_gemv_rows(st, M.A, D.m_E, D.n_d, D.lda, x + D.n_s, rowtmp);
    }
    k_eval_cons<<<kRedBlocks, NT, 0, st>>>(D, M, x, rowtmp, d, cg, ch, partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 1, out2);
    launch_finalize_max(st, partial + kRedBlocks, 1, out2 + 1);
}

void VecOps::eval_cons_ax(const double *x, const double *Ax, const double *d, double *cg, double *ch,
                          double *out2) {
    k_eval_cons<<<kRedBlocks, NT, 0, st>>>(D, M, x, Ax, d, cg, ch, partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 1, out2);
    launch_finalize_max(st, partial + kRedBlocks, 1, out2 + 1);
}

namespace {
__global__ void k_axpby(int64_t n, const double *__restrict__ a, double alpha, const double *__restrict__ b,
                        double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a[i] + alpha * b[i];
}
}  // namespace

void VecOps::axpby(int64_t n, const double *a, double alpha, const double *b, double *y) {
    if (n <= 0) return;
    k_axpby<<<elem_grid(n), 256, 0, st>>>(n, a, alpha, b, y);
    MDSIP_LAUNCHED();
}

void VecOps::jac_hess(const double *x, const double *yh, double *Jdh, double *Hss, double *Hdd) {
    k_jac_hess<<<elem_grid(std::max(D.n_s, D.n_d * D.n_d)), 256, 0, st>>>(D, M, x, yh, Jdh, Hss, Hdd);
    MDSIP_LAUNCHED();
}

void VecOps::lagrangian_grad(const IterView &I, const double *grad, const double *Jdh, double *ATy,
                             double *gl) {
    if (Ahi) launch_gemv_t_df(st, Ahi, Alo, D.m_E, D.n_d, D.lda, I.yg, split, colpart, ATy);
    else launch_gemv_t(st, M.A, D.m_E, D.n_d, D.lda, I.yg, colpart, ATy);
    k_lagrangian_grad<<<elem_grid(std::max(D.n_s, D.n_d)), 256, 0, st>>>(D, M, grad, I.yg, I.yh, Jdh,
                                                                         ATy, gl);
    MDSIP_LAUNCHED();
}

void VecOps::lagrangian_grad_aty(const IterView &I, const double *grad, const double *Jdh, const double *ATy,
                                 double *gl) {
    k_lagrangian_grad<<<elem_grid(std::max(D.n_s, D.n_d)), 256, 0, st>>>(D, M, grad, I.yg, I.yh, Jdh,
                                                                         ATy, gl);
    MDSIP_LAUNCHED();
}

void VecOps::errors(const IterView &I, const double *gl, const double *cg, const double *ch,
                    double *out7) {
    k_errors<<<kRedBlocks, NT, 0, st>>>(D, M, I, gl, cg, ch, partial);
    MDSIP_LAUNCHED();
    launch_finalize_max(st, partial, 3, out7);                       // 0,1,2
    launch_finalize_min(st, partial + 3 * kRedBlocks, 1, out7 + 3);  // 3
    launch_finalize_sum(st, partial + 4 * kRedBlocks, 3, out7 + 4);  // 4,5,6
}

void VecOps::newton_diag(const IterView &I, const double *Hss, double dw, double dc, bool want_w,
                         double *sig_x, double *q, double *sig_d, double *w, double *out6) {
    k_newton_diag<<<kRedBlocks, NT, 0, st>>>(D, M, I, Hss, dw, dc, want_w ? 1 : 0, sig_x, q, sig_d, w,
                                             partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 6, out6);
}

void VecOps::rhs_y(const IterView &I, const double *gl, const double *cg, const double *q,
                   const double *w, double mu, double *bt_g, double *u) {
    k_rhs_y<<<elem_grid(D.m_E), 256, 0, st>>>(D, M, I, gl, cg, q, w, mu, bt_g, u);
    MDSIP_LAUNCHED();
}

void VecOps::rhs_reduced(const IterView &I, const double *gl, const double *ch, const double *sig_d,
                         const double *ATu, const double *bt_g, const double *q, double mu, double dw, bool p1,
                         double *rhs) {
    k_rhs_reduced<<<elem_grid(std::max(D.n_d, D.m_E)), 256, 0, st>>>(D, M, I, gl, ch, sig_d, ATu, bt_g, q,
                                                                     mu, dw, p1 ? 1 : 0, rhs);
    MDSIP_LAUNCHED();
}

void VecOps::dyg_p2(const double *Adx, const double *bt_g, const double *w, double *dyg) {
    k_dyg_p2<<<elem_grid(D.m_E), 256, 0, st>>>(D.m_E, Adx, bt_g, w, dyg);
    MDSIP_LAUNCHED();
}

void VecOps::copy(const double *src, double *dst, int64_t n) {
    if (n <= 0) return;
    k_copy<<<elem_grid(n), 256, 0, st>>>(src, dst, n);
    MDSIP_LAUNCHED();
}

void VecOps::backsub(const IterView &I, const DirView &Dir, const double *gl, const double *q,
                     const double *sig_d, const double *sol_dxd, const double *sol_dyh, double mu,
                     double dw) {
    k_backsub<<<elem_grid(D.n), 256, 0, st>>>(D, M, I, Dir, gl, q, sig_d, sol_dxd, sol_dyh, mu, dw);
    MDSIP_LAUNCHED();
}

void VecOps::step_scalars(const IterView &I, const DirView &Dir, const double *grad, double tau,
                          double mu, double *out3) {
    k_step_scalars<<<kRedBlocks, NT, 0, st>>>(D, M, I, Dir, grad, tau, mu, partial);
    MDSIP_LAUNCHED();
    launch_finalize_min(st, partial, 2, out3);
    launch_finalize_sum(st, partial + 2 * kRedBlocks, 1, out3 + 2);
}

void VecOps::trial(const IterView &I, const DirView &Dir, double alpha, double *xt, double *dt,
                   double *out2) {
    k_trial<<<kRedBlocks, NT, 0, st>>>(D, M, I, Dir, alpha, xt, dt, partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 2, out2);
}

void VecOps::accept(const IterView &I, const DirView &Dir, double alpha, double alpha_z, double mu,
                    double ks) {
    k_accept<<<elem_grid(std::max(D.n, D.m_E)), 256, 0, st>>>(D, M, I, Dir, alpha, alpha_z, mu, ks);
    MDSIP_LAUNCHED();
}

void VecOps::init_x(const double *x0, double k1, double k2, const IterView &I) {
    k_init_x<<<elem_grid(std::max(D.n, D.m_E)), 256, 0, st>>>(D, M, x0, k1, k2, I);
    MDSIP_LAUNCHED();
}

void VecOps::init_d(const double *ch, double k1, double k2, const IterView &I) {
    k_init_d<<<elem_grid(D.m_I), 256, 0, st>>>(D, M, ch, k1, k2, I);
    MDSIP_LAUNCHED();
}

void VecOps::start_predicted(const float *pred, double push, double mu0, const IterView &I) {
    k_start_predicted<<<elem_grid(std::max(D.n, D.m_E)), 256, 0, st>>>(D, M, pred, push, mu0, I);
    MDSIP_LAUNCHED();
}

void VecOps::cons_from_values(const double *g, const double *h, const double *d, double *cg, double *ch,
                              double *out2) {
    k_cons_from_values<<<kRedBlocks, NT, 0, st>>>(D, M, g, h, d, cg, ch, partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 1, out2);
    launch_finalize_max(st, partial + kRedBlocks, 1, out2 + 1);
}

void VecOps::dir_diff(const DirView &a, const DirView &b, double *out2) {
    k_dir_diff<<<kRedBlocks, NT, 0, st>>>(D, a, b, partial);
    MDSIP_LAUNCHED();
    launch_finalize_sum(st, partial, 2, out2);
}

void VecOps::copy_dir(const DirView &src, const DirView &dst) {
    copy(src.dx, dst.dx, D.n);
    copy(src.dd, dst.dd, D.m_I);
    copy(src.dyg, dst.dyg, D.m_E);
    copy(src.dyh, dst.dyh, D.m_I);
    copy(src.dzl, dst.dzl, D.n);
    copy(src.dzu, dst.dzu, D.n);
    copy(src.dvl, dst.dvl, D.m_I);
    copy(src.dvu, dst.dvu, D.m_I);
}

void VecOps::gather(int64_t n, const double *src, const int32_t *idx, double *dst) {
    if (n <= 0) return;
    k_gather<<<elem_grid(n), 256, 0, st>>>(n, src, idx, dst);
    MDSIP_LAUNCHED();
}

}  // namespace mdsip
