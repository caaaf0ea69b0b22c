// Iterative refinement of the Newton direction on the unreduced system of
// Eq. (linsys4x4), in FP64 (path P2).
//
// The reduced matrix S may be factored from a low-precision condensation
// product; the direction is then refined: u <- u + S~^-1 (b - K u), where the
// residual b - K u is formed in FP64 from the blocks of the 4x4 matrix
// (diagonal Q_s, dense Q_d, sparse J_sg, dense A and J_dh) and the
// approximate solve S~^-1 is the same two-stage elimination used for the
// direction itself.  Vectors are packed as [u_s (n_s) | u_d (n_d) | u_g (m_E) | u_h (m_I)].
// With a tensor-core factor and n_d <= 2048 the residual's double-float pass
// over A also forms the FP32 A^T (bt_g / w) of the approximate solve that
// follows it, so that solve reads A once (for A sol_d) instead of twice.
#include "refine.cuh"

namespace mdsip {

namespace {

constexpr int NT = kRedThreads;

__device__ __forceinline__ double *slot(double *partial, int q) {
    return partial + (size_t)q * kRedBlocks + blockIdx.x;
}

__device__ __forceinline__ double rN_x(const ModelView &M, const IterView &I, const double *gl, double mu,
                                       int64_t i) {
    double r = gl[i];
    if (isfinite(M.xl[i])) r -= mu / (I.x[i] - M.xl[i]);
    if (isfinite(M.xu[i])) r += mu / (M.xu[i] - I.x[i]);
    return r;
}

__device__ __forceinline__ double r_dslack(const ModelView &M, const IterView &I, double mu, int64_t j) {
    double r = -I.yh[j];
    if (isfinite(M.hl[j])) r -= mu / (I.d[j] - M.hl[j]);
    if (isfinite(M.hu[j])) r += mu / (M.hu[j] - I.d[j]);
    return r;
}

// b = -[rN_x; c_g; c_h + Dh^-1 r_d]
__global__ void k_rhs_full(Dims D, ModelView M, IterView I, const double *__restrict__ gl,
                           const double *__restrict__ cg, const double *__restrict__ ch,
                           const double *__restrict__ sig_d, double mu, double dw, double *__restrict__ b) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.n; i += gsz) b[i] = -rN_x(M, I, gl, mu, i);
    for (int64_t i = gtid; i < D.m_E; i += gsz) b[D.n + i] = -cg[i];
    for (int64_t j = gtid; j < D.m_I; j += gsz)
        b[D.n + D.m_E + j] = -(ch[j] + r_dslack(M, I, mu, j) / (sig_d[j] + dw));
}

// bt_g = b_g - J_sg (b_s / q);  u = bt_g / w
__global__ void k_prep_g(Dims D, ModelView M, const double *__restrict__ b, const double *__restrict__ q,
                         const double *__restrict__ w, double *__restrict__ bt_g, double *__restrict__ u) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D.m_E; i += (int64_t)gridDim.x * blockDim.x) {
        double s = b[D.n + i];
        for (int e = M.csr_ptr[i]; e < M.csr_ptr[i + 1]; ++e) {
            const int c = M.csr_col[e];
            s -= M.csr_val[e] * b[c] / q[c];
        }
        bt_g[i] = s;
        u[i] = s / w[i];
    }
}

// The part of bt_g that does not involve A, for the residual r = b - K u that
// the next pass forms: with r_s = b_s - Q_s u_s - J_sg^T u_g,
// bt_g = r_g - J_sg (r_s / q) = cpre - A u_d, where
// cpre = b_g + dc u_g - J_sg u_s - J_sg (r_s / q); also cpre as FP32 halves
// (cw) and wf = fl32(1 / w) for the pass
__global__ void k_pre_bt(Dims D, ModelView M, const double *__restrict__ b, const double *__restrict__ u,
                         const double *__restrict__ q, const double *__restrict__ w, double dc,
                         double *__restrict__ cpre, float2 *__restrict__ cw, float *__restrict__ wf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D.m_E; i += (int64_t)gridDim.x * blockDim.x) {
        double s = b[D.n + i] + dc * u[D.n + i];
        for (int e = M.csr_ptr[i]; e < M.csr_ptr[i + 1]; ++e) {
            const int c = M.csr_col[e];
            double Ku = q[c] * u[c];
            for (int f = M.csc_ptr[c]; f < M.csc_ptr[c + 1]; ++f) Ku += M.csc_val[f] * u[D.n + M.csc_row[f]];
            const double rs = b[c] - Ku;
            s -= M.csr_val[e] * u[c];
            s -= M.csr_val[e] * rs / q[c];
        }
        cpre[i] = s;
        const float h = (float)s;
        cw[i] = make_float2(h, (float)(s - (double)h));
        wf[i] = (float)(1.0 / w[i]);
    }
}

// rhs_S = [b_d + A^T u; b_h]
__global__ void k_rhs_S(Dims D, const double *__restrict__ b, const double *__restrict__ ATu,
                        double *__restrict__ rhsS) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = gtid; k < D.n_d; k += gsz) rhsS[k] = b[D.n_s + k] + ATu[k];
    for (int64_t j = gtid; j < D.m_I; j += gsz) rhsS[D.n_d + j] = b[D.n + D.m_E + j];
}

// sol_g = (A sol_d - bt_g) / w ; sol_d, sol_h from the reduced solution
__global__ void k_sol_gdh(Dims D, const double *__restrict__ Adx, const double *__restrict__ bt_g,
                          const double *__restrict__ w, const double *__restrict__ rhsS, double *__restrict__ sol) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.m_E; i += gsz) sol[D.n + i] = (Adx[i] - bt_g[i]) / w[i];
    for (int64_t k = gtid; k < D.n_d; k += gsz) sol[D.n_s + k] = rhsS[k];
    for (int64_t j = gtid; j < D.m_I; j += gsz) sol[D.n + D.m_E + j] = rhsS[D.n_d + j];
}

// k_sol_gdh after the fused residual pass, with bt_g = cpre - A u_d formed here
__global__ void k_sol_gdh_pre(Dims D, const double *__restrict__ Adx, const double *__restrict__ cpre,
                              const double *__restrict__ Au, const double *__restrict__ w,
                              const double *__restrict__ rhsS, double *__restrict__ sol) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.m_E; i += gsz) sol[D.n + i] = (Adx[i] - (cpre[i] - Au[i])) / w[i];
    for (int64_t k = gtid; k < D.n_d; k += gsz) sol[D.n_s + k] = rhsS[k];
    for (int64_t j = gtid; j < D.m_I; j += gsz) sol[D.n + D.m_E + j] = rhsS[D.n_d + j];
}

// sol_s = (b_s - J_sg^T sol_g) / q
__global__ void k_sol_s(Dims D, ModelView M, const double *__restrict__ b, const double *__restrict__ q,
                        double *__restrict__ sol) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < D.n_s; k += (int64_t)gridDim.x * blockDim.x) {
        double s = b[k];
        for (int e = M.csc_ptr[k]; e < M.csc_ptr[k + 1]; ++e) s -= M.csc_val[e] * sol[D.n + M.csc_row[e]];
        sol[k] = s / q[k];
    }
}

// Hu = H_dd u_d (warp per row)
// Hu[p] = (H_dd u_d)[p] for p < n_d and (J_dh u_d)[p - n_d] for p < n_d + m_I
// (one warp per row)
__global__ void k_hdd_gemv(int64_t n_d, int64_t m_I, const double *__restrict__ Hdd,
                           const double *__restrict__ Jdh, const double *__restrict__ ud,
                           double *__restrict__ Hu) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = gw; p < n_d + m_I; p += nw) {
        double s0 = 0.0, s1 = 0.0;
        const double *row = p < n_d ? Hdd + p * n_d : Jdh + (p - n_d) * n_d;
        int64_t k = lane;
        for (; k + 32 < n_d; k += 64) {
            s0 = fma(row[k], ud[k], s0);
            s1 = fma(row[k + 32], ud[k + 32], s1);
        }
        if (k < n_d) s0 = fma(row[k], ud[k], s0);
        double s = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) Hu[p] = s;
    }
}

// r = b - K u, with Au = A u_d, ATug = A^T u_g and Hu = [H_dd u_d; J_dh u_d] precomputed.
// Reductions: 0 ||r||_inf, 1 ||b||_inf, 2 ||b - r||_inf (= ||K u||_inf), 3 ||u||_inf
__global__ void __launch_bounds__(NT) k_residual(Dims D, ModelView M, const double *__restrict__ b,
                                                 const double *__restrict__ u, const double *__restrict__ q,
                                                 const double *__restrict__ sig_xd, const double *__restrict__ sig_d,
                                                 const double *__restrict__ Jdh, const double *__restrict__ Au,
                                                 const double *__restrict__ ATug, const double *__restrict__ Hu,
                                                 double dw, double dc, double *__restrict__ r, double *partial) {
    __shared__ double sh[32];
    double rm = 0.0, bm = 0.0, km = 0.0, um = 0.0;
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x, gsz = (int64_t)gridDim.x * NT;
    const double *us = u, *ud = u + D.n_s, *ug = u + D.n, *uh = u + D.n + D.m_E;
    auto put = [&](int64_t idx, double Ku) {
        const double bi = b[idx];
        const double ri = bi - Ku;
        r[idx] = ri;
        rm = fmax(rm, fabs(ri));
        bm = fmax(bm, fabs(bi));
        km = fmax(km, fabs(Ku));
        um = fmax(um, fabs(u[idx]));
    };
    for (int64_t k = gtid; k < D.n_s; k += gsz) {
        double Ku = q[k] * us[k];
        for (int e = M.csc_ptr[k]; e < M.csc_ptr[k + 1]; ++e) Ku += M.csc_val[e] * ug[M.csc_row[e]];
        put(k, Ku);
    }
    for (int64_t k = gtid; k < D.n_d; k += gsz) {
        double Ku = Hu[k] + (sig_xd[k] + dw) * ud[k] + ATug[k];
        for (int64_t j = 0; j < D.m_I; ++j) Ku += Jdh[j * D.n_d + k] * uh[j];
        put(D.n_s + k, Ku);
    }
    for (int64_t i = gtid; i < D.m_E; i += gsz) {
        double Ku = Au[i] - dc * ug[i];
        for (int e = M.csr_ptr[i]; e < M.csr_ptr[i + 1]; ++e) Ku += M.csr_val[e] * us[M.csr_col[e]];
        put(D.n + i, Ku);
    }
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double Ku = -(1.0 / (sig_d[j] + dw) + dc) * uh[j] + Hu[D.n_d + j];   // + (J_dh u_d)_j
        put(D.n + D.m_E + j, Ku);
    }
    double x;
    x = block_max<NT>(rm, sh); if (threadIdx.x == 0) *slot(partial, 0) = x;
    x = block_max<NT>(bm, sh); if (threadIdx.x == 0) *slot(partial, 1) = x;
    x = block_max<NT>(km, sh); if (threadIdx.x == 0) *slot(partial, 2) = x;
    x = block_max<NT>(um, sh); if (threadIdx.x == 0) *slot(partial, 3) = x;
}

__global__ void k_axpy(int64_t n, const double *__restrict__ x, double *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

// Direction from the packed solution: dx, dy, dd = (dy_h - r_d)/Dh, dz, dv.
__global__ void k_dir_from_sol(Dims D, ModelView M, IterView I, DirView Dir, const double *__restrict__ u,
                               const double *__restrict__ sig_d, double mu, double dw) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < D.n; i += gsz) {
        const double dx = u[i];
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
    for (int64_t i = gtid; i < D.m_E; i += gsz) Dir.dyg[i] = u[D.n + i];
    for (int64_t j = gtid; j < D.m_I; j += gsz) {
        const double dyh = u[D.n + D.m_E + j];
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

int grid_for(int64_t n) { return std::max(1, std::min(4096, ceil_div(std::max<int64_t>(n, 1), 256))); }

}  // namespace

void Refiner::rhs(const IterView &I, const double *gl, const double *cg, const double *ch, const double *sig_d,
                  double mu, double dw, double *b) {
    k_rhs_full<<<grid_for(std::max(D.n, D.m_E)), 256, 0, st>>>(D, M, I, gl, cg, ch, sig_d, mu, dw, b);
    MDSIP_LAUNCHED();
}

bool Refiner::fuse_pass() const { return cpre && Ahi && solve_fp32 && AfT && gemv_both_fusable(D.n_d); }

void Refiner::approx_solve(const double *b, double *sol) {
    const double *ATu = tmp_nd;
    const bool pre = pre_for != nullptr && pre_for == b;
    if (pre) {   // A_hi^T (bt_g / w) came with the residual b; bt_g = cpre - A u_d (tmp_m)
        ATu = ATv;
    } else {
        k_prep_g<<<grid_for(D.m_E), 256, 0, st>>>(D, M, b, q, w, bt_g, tmp_m);
        MDSIP_LAUNCHED();
        if (solve_fp32 && AfT)   // approximate solve of a low-precision factor: FP32 A^T product
            launch_aft_dot(st, num_sms, AfT, ldt, D.m_E, D.n_d, tmp_m, vf, tmp_nd);
        else
            launch_gemv_t(st, M.A, D.m_E, D.n_d, D.lda, tmp_m, colpart, tmp_nd);
    }
    pre_for = nullptr;
    k_rhs_S<<<grid_for(std::max(D.n_d, D.m_I)), 256, 0, st>>>(D, b, ATu, rhsS);
    MDSIP_LAUNCHED();
    launch_ldlt_solve_coop(st, num_sms, N, Dd, Doff, perm, 1, rhsS, N, solve_ws, solve_err, solve_fp32);
    if (pre) {
        launch_gemv_rows_f32(st, Ahi, D.m_E, D.n_d, D.lda, rhsS, Asd);
        k_sol_gdh_pre<<<grid_for(std::max(D.m_E, D.n_d)), 256, 0, st>>>(D, Asd, cpre, tmp_m, w, rhsS, sol);
    } else {
        if (Ahi) launch_gemv_rows_f32(st, Ahi, D.m_E, D.n_d, D.lda, rhsS, tmp_m);
        else launch_gemv_rows(st, M.A, D.m_E, D.n_d, D.lda, rhsS, tmp_m);
        k_sol_gdh<<<grid_for(std::max(D.m_E, D.n_d)), 256, 0, st>>>(D, tmp_m, bt_g, w, rhsS, sol);
    }
    MDSIP_LAUNCHED();
    k_sol_s<<<grid_for(D.n_s), 256, 0, st>>>(D, M, b, q, sol);
    MDSIP_LAUNCHED();
}

void Refiner::track_Au(bool init) {
    if (Ahi) return;   // the residual forms A u_d itself
    if (init) {
        MDSIP_CUDA(cudaMemcpyAsync(Au_run, tmp_m, D.m_E * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        axpy(D.m_E, tmp_m, Au_run);
    }
}

void Refiner::residual(const double *b, const double *u, double dw, double dc, double *r, double *out4) {
    const double *Au = Au_run;
    pre_for = nullptr;
    if (Ahi) {   // A u_d and A^T u_g from one double-float pass
        const bool fuse = fuse_pass();
        BothNextArgs nx{cw, wf, ATv};
        if (fuse) {
            k_pre_bt<<<grid_for(D.m_E), 256, 0, st>>>(D, M, b, u, q, w, dc, cpre, cw, wf);
            MDSIP_LAUNCHED();
        }
        launch_gemv_both_df(st, Ahi, Alo, D.m_E, D.n_d, D.lda, u + D.n_s, u + D.n, split, split + D.n_d, colpart,
                            tmp_m, tmp_nd, solve_err, fuse ? &nx : nullptr);
        Au = tmp_m;
        if (fuse) pre_for = r;
    } else {
        launch_gemv_t(st, M.A, D.m_E, D.n_d, D.lda, u + D.n, colpart, tmp_nd);   // A^T u_g
    }
    k_hdd_gemv<<<std::max(1, std::min(4096, ceil_div((D.n_d + D.m_I) * 32, 256))), 256, 0, st>>>(
        D.n_d, D.m_I, Hdd, Jdh, u + D.n_s, tmp_nd2);
    MDSIP_LAUNCHED();
    k_residual<<<kRedBlocks, NT, 0, st>>>(D, M, b, u, q, sig_xd, sig_d, Jdh, Au, tmp_nd, tmp_nd2, dw, dc,
                                          r, partial);
    MDSIP_LAUNCHED();
    launch_finalize_max(st, partial, 4, out4);
}

void Refiner::axpy(int64_t n, const double *x, double *y) {
    k_axpy<<<grid_for(n), 256, 0, st>>>(n, x, y);
    MDSIP_LAUNCHED();
}

void Refiner::direction(const IterView &I, const DirView &Dir, const double *u, double mu, double dw) {
    k_dir_from_sol<<<grid_for(std::max(D.n, D.m_E)), 256, 0, st>>>(D, M, I, Dir, u, sig_d, mu, dw);
    MDSIP_LAUNCHED();
}

}  // namespace mdsip
