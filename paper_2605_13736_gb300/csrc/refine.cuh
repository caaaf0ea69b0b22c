// Iterative refinement of the Newton direction (refine.cu).
#pragma once
#include "vec.cuh"

namespace mdsip {

struct Refiner {
    Dims D;
    ModelView M;
    cudaStream_t st;
    // factor of the reduced matrix
    int64_t N;
    const double *L, *Dd, *Doff;
    const int32_t *perm;
    int num_sms;
    void *solve_ws;   // ldlt_solve_scratch_bytes(N)
    bool solve_fp32;  // the prepared tiles are FP32 (tensor-core factor)
    // FP32 transposed copy of A (n_d x ldt) and an ldt-float scratch: with a
    // tensor-core factor the approximate solve forms its A^T products from it
    const float *AfT;
    int64_t ldt;
    float *vf;
    int *solve_err;
    // Newton quantities of the current attempt
    const double *q, *w, *sig_xd, *sig_d, *Jdh, *Hdd;
    // scratch: bt_g, tmp_m (m_E), tmp_nd (n_d), tmp_nd2 (n_d + m_I), rhsS (N), colpart, partial
    double *bt_g, *tmp_m, *tmp_nd, *tmp_nd2, *rhsS, *colpart, *partial;
    double *Au_run;   // A u_d of the current solution, kept as a running sum (m_E)
    // A as an FP32 pair (null: FP64 passes).  With it the approximate solves
    // take FP32 products with A_hi and the residual takes A u_d and A^T u_g
    // from one double-float pass over (A_hi, A_lo)
    const float *Ahi, *Alo;
    float2 *split;    // m_E + n_d float2
    // With a tensor-core factor and n_d <= 2048 (one slice of the pass), the
    // residual's pass over A also forms A_hi^T (bt_g / w) for the approximate
    // solve of that residual, bt_g = cpre - A u_d: cpre (m_E), its FP32 halves
    // cw (m_E), wf = fl32(1 / w) (m_E), the product ATv (n_d) and that solve's
    // A sol_d in Asd (m_E); null cpre: separate passes
    double *cpre, *ATv, *Asd;
    float2 *cw;
    float *wf;
    const double *pre_for;   // the residual whose first solve half is ready (else null)

    // b = right-hand side of Eq. (linsys4x4), packed [s | d | g | h]
    void rhs(const IterView &I, const double *gl, const double *cg, const double *ch, const double *sig_d,
             double mu, double dw, double *b);
    // sol = S~^-1-based solve of K sol = b (two-stage elimination with the factor);
    // b the last residual: its first half came with that residual's pass (fuse_pass)
    void approx_solve(const double *b, double *sol);
    bool fuse_pass() const;
    // after approx_solve: Au_run = A sol_d (init) or Au_run += A sol_d (FP64 passes only)
    void track_Au(bool init);
    // r = b - K u in FP64 (A u_d from Au_run, or from the double-float pass);
    // out4 = (||r||inf, ||b||inf, ||K u||inf, ||u||inf).  The approximate solve
    // of r that may follow has to come next (its first half is in cpre / ATv)
    void residual(const double *b, const double *u, double dw, double dc, double *r, double *out4);
    void axpy(int64_t n, const double *x, double *y);
    // full direction (incl. dd and the bound-multiplier steps) from the packed solution
    void direction(const IterView &I, const DirView &Dir, const double *u, double mu, double dw);
};

}  // namespace mdsip
