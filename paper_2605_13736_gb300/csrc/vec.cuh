// Launch wrappers of the fused vector kernels (vec.cu).
#pragma once
#include "internal.cuh"

namespace mdsip {

struct IterView {
    double *x, *d, *yg, *yh, *zl, *zu, *vl, *vu;
};

struct DirView {
    double *dx, *dd, *dyg, *dyh, *dzl, *dzu, *dvl, *dvu;
};

// All launches on one stream; `partial` holds kRedBlocks x 8 doubles and
// `colpart` kRedBlocks x n_d doubles of reduction scratch, `rowtmp` m_E doubles.
struct VecOps {
    Dims D;
    ModelView M;
    cudaStream_t st;
    double *partial;
    double *colpart;
    double *rowtmp;   // m_E doubles: A x_d of the constraint evaluation
    // mixed-precision path: A as an FP32 pair (A_hi + A_lo) for the passes over A
    // in double-float arithmetic, and their vector scratch (max(m_E, n_d) float2);
    // null on the plain FP64 path
    const float *Ahi = nullptr, *Alo = nullptr;
    float2 *split = nullptr;

    void eval_f(const double *x, double *grad, double *out_scalar);
    void eval_cons(const double *x, const double *d, double *cg, double *ch, double *out2);
    // the same with A x_d given (Ax, m_E doubles) instead of formed from x
    void eval_cons_ax(const double *x, const double *Ax, const double *d, double *cg, double *ch, double *out2);
    // y = a + alpha b (n doubles)
    void axpby(int64_t n, const double *a, double alpha, const double *b, double *y);
    void jac_hess(const double *x, const double *yh, double *Jdh, double *Hss, double *Hdd);
    void lagrangian_grad(const IterView &I, const double *grad, const double *Jdh, double *ATy,
                         double *gl);
    // the same with ATy = A^T y_g already in place
    void lagrangian_grad_aty(const IterView &I, const double *grad, const double *Jdh, const double *ATy,
                             double *gl);
    void errors(const IterView &I, const double *gl, const double *cg, const double *ch,
                double *out7);
    void newton_diag(const IterView &I, const double *Hss, double dw, double dc, bool want_w,
                     double *sig_x, double *q, double *sig_d, double *w, double *out6);
    void rhs_y(const IterView &I, const double *gl, const double *cg, const double *q,
               const double *w, double mu, double *bt_g, double *u);
    void rhs_reduced(const IterView &I, const double *gl, const double *ch, const double *sig_d,
                     const double *ATu, const double *bt_g, const double *q, double mu, double dw, bool p1,
                     double *rhs);
    void dyg_p2(const double *Adx, const double *bt_g, const double *w, double *dyg);
    void copy(const double *src, double *dst, int64_t n);
    void backsub(const IterView &I, const DirView &Dir, const double *gl, const double *q,
                 const double *sig_d, const double *sol_dxd, const double *sol_dyh, double mu,
                 double dw);
    void step_scalars(const IterView &I, const DirView &Dir, const double *grad, double tau,
                      double mu, double *out3);
    void trial(const IterView &I, const DirView &Dir, double alpha, double *xt, double *dt,
               double *out2);
    void accept(const IterView &I, const DirView &Dir, double alpha, double alpha_z, double mu,
                double ks);
    void init_x(const double *x0, double k1, double k2, const IterView &I);
    void init_d(const double *ch, double k1, double k2, const IterView &I);
    // Warm start from a predicted packed point `pred` (FP32): x and d pushed
    // inside their bounds by `push`, bound multipliers at least mu0 / slack.
    void start_predicted(const float *pred, double push, double mu0, const IterView &I);
    // residuals from model values given by a callback: cg = g - g_E, ch = h - d
    void cons_from_values(const double *g, const double *h, const double *d, double *cg, double *ch,
                          double *out2);
    // dst[i] = src[idx[i]]
    void gather(int64_t n, const double *src, const int32_t *idx, double *dst);
    // out2 = (sum (a - b)^2, sum b^2) over every block of two directions
    void dir_diff(const DirView &a, const DirView &b, double *out2);
    void copy_dir(const DirView &src, const DirView &dst);
};

// Reduced-matrix assembly (assemble.cu).
// P2:  S = [[Hdd + diag(sig_xd + dw), Jdh^T], [Jdh, -1/(sig_d + dw) - dc]]  (lower, col-major, ld = N)
//      (the A^T W^-1 A term is added by the SYRK afterwards)
void launch_assemble_S(cudaStream_t s, const Dims &D, const double *Hdd, const double *sig_xd,
                       const double *Jdh, const double *sig_d, double dw, double dc, double *S);
// P1:  M of Eq. (compressed) (lower, col-major, ld = N = n_d + m)
void launch_assemble_M(cudaStream_t s, const Dims &D, const ModelView &Mv, const double *Hdd,
                       const double *sig_xd, const double *Jdh, const double *sig_d, const double *q,
                       double dw, double dc, double *Mat);

}  // namespace mdsip
