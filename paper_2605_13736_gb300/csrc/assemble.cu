// Assembly of the reduced matrices of one Newton step.
//
// Path P1: the compressed 3x3 block matrix of Eq. (compressed) (Section 2.2),
// with the inertia-correction shifts of Section 2.1:
//
//   M = [ Q_d    A^T                          Jdh^T                              ]
//       [ A      -J_sg Q_s^-1 J_sg^T - dc I   -J_sg Q_s^-1 J_sh^T                ]
//       [ Jdh    -J_sh Q_s^-1 J_sg^T          -J_sh Q_s^-1 J_sh^T - Dh^-1 - dc I ]
//
// Q_d = H_dd + Sigma_xd + dw I, Dh = Sigma_d + dw; the J_sh blocks vanish in
// the benchmark family.  The sparse product J_s Q_s^-1 J_s^T (J_s = [J_sg;
// J_sh]) is the K3 kernel of Section 2.3, here computed row by row from the
// CSR/CSC indices (each thread owns one output row, so the accumulation
// order is fixed).
//
// Path P2: S = [[Q_d, Jdh^T], [Jdh, -Dh^-1 - dc I]]; the SYRK adds A^T W^-1 A.
//
// Storage: lower triangle, column-major, leading dimension N.
#include "vec.cuh"

namespace mdsip {

namespace {

__global__ void k_assemble_S(Dims D, const double *__restrict__ Hdd, const double *__restrict__ sig_xd,
                             const double *__restrict__ Jdh, const double *__restrict__ sig_d,
                             double dw, double dc, double *__restrict__ S) {
    const int64_t N = D.n_d + D.m_I;
    for (int64_t q = blockIdx.x; q < N; q += gridDim.x) {
        for (int64_t p = q + threadIdx.x; p < N; p += blockDim.x) {
            double v;
            if (q < D.n_d) {
                if (p < D.n_d)
                    v = Hdd[p * D.n_d + q] + (p == q ? sig_xd[p] + dw : 0.0);
                else
                    v = Jdh[(p - D.n_d) * D.n_d + q];
            } else {
                v = p == q ? -1.0 / (sig_d[p - D.n_d] + dw) - dc : 0.0;
            }
            S[p + q * N] = v;
        }
    }
}

__global__ void k_assemble_M_dense(Dims D, ModelView Mv, const double *__restrict__ Hdd,
                                   const double *__restrict__ sig_xd, const double *__restrict__ Jdh,
                                   const double *__restrict__ sig_d, double dw, double dc,
                                   double *__restrict__ Mat) {
    const int64_t N = D.n_d + D.m;
    const int64_t h0 = D.n_d + D.m_E;
    for (int64_t q = blockIdx.x; q < N; q += gridDim.x) {
        for (int64_t p = q + threadIdx.x; p < N; p += blockDim.x) {
            double v;
            if (q < D.n_d) {
                if (p < D.n_d)
                    v = Hdd[p * D.n_d + q] + (p == q ? sig_xd[p] + dw : 0.0);
                else if (p < h0)
                    v = Mv.A[(p - D.n_d) * D.lda + q];
                else
                    v = Jdh[(p - h0) * D.n_d + q];
            } else {
                v = 0.0;
                if (p == q) {
                    v = -dc;
                    if (p >= h0) v -= 1.0 / (sig_d[p - h0] + dw);
                }
            }
            Mat[p + q * N] = v;
        }
    }
}

// M[n_d + r1][n_d + r2] -= sum_k J[r1,k] J[r2,k] / q_k  for r2 <= r1
__global__ void k_assemble_M_sparse(Dims D, ModelView Mv, const double *__restrict__ q,
                                    double *__restrict__ Mat) {
    const int64_t N = D.n_d + D.m;
    for (int64_t r1 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r1 < D.m_E;
         r1 += (int64_t)gridDim.x * blockDim.x) {
        for (int e = Mv.csr_ptr[r1]; e < Mv.csr_ptr[r1 + 1]; ++e) {
            const int k = Mv.csr_col[e];
            const double f = Mv.csr_val[e] / q[k];
            for (int e2 = Mv.csc_ptr[k]; e2 < Mv.csc_ptr[k + 1]; ++e2) {
                const int64_t r2 = Mv.csc_row[e2];
                if (r2 > r1) continue;
                Mat[(D.n_d + r1) + (D.n_d + r2) * N] -= f * Mv.csc_val[e2];
            }
        }
    }
}

// the h rows of J_s Q_s^-1 J_s^T: for each entry (j, k) of J_sh, with
// f = J_sh[j,k] / q_k, M[h0 + j][n_d + r] -= f J_sg[r,k] for every r of column
// k of J_sg, and M[h0 + j][h0 + j2] -= f J_sh[j2,k] for j2 <= j
__global__ void k_assemble_M_sparse_h(Dims D, ModelView Mv, const double *__restrict__ q,
                                      double *__restrict__ Mat) {
    const int64_t N = D.n_d + D.m;
    const int64_t h0 = D.n_d + D.m_E;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < D.m_I;
         j += (int64_t)gridDim.x * blockDim.x) {
        for (int e = Mv.hsr_ptr[j]; e < Mv.hsr_ptr[j + 1]; ++e) {
            const int k = Mv.hsr_col[e];
            const double f = Mv.hsr_val[e] / q[k];
            for (int e2 = Mv.csc_ptr[k]; e2 < Mv.csc_ptr[k + 1]; ++e2)
                Mat[(h0 + j) + (D.n_d + (int64_t)Mv.csc_row[e2]) * N] -= f * Mv.csc_val[e2];
            for (int e2 = Mv.hsc_ptr[k]; e2 < Mv.hsc_ptr[k + 1]; ++e2) {
                const int64_t j2 = Mv.hsc_row[e2];
                if (j2 > j) continue;
                Mat[(h0 + j) + (h0 + j2) * N] -= f * Mv.hsc_val[e2];
            }
        }
    }
}

}  // namespace

void launch_assemble_S(cudaStream_t s, const Dims &D, const double *Hdd, const double *sig_xd,
                       const double *Jdh, const double *sig_d, double dw, double dc, double *S) {
    const int64_t N = D.n_d + D.m_I;
    if (N <= 0) return;
    k_assemble_S<<<(unsigned)std::min<int64_t>(N, 8192), 256, 0, s>>>(D, Hdd, sig_xd, Jdh, sig_d, dw,
                                                                      dc, S);
    MDSIP_LAUNCHED();
}

void launch_assemble_M(cudaStream_t s, const Dims &D, const ModelView &Mv, const double *Hdd,
                       const double *sig_xd, const double *Jdh, const double *sig_d, const double *q,
                       double dw, double dc, double *Mat) {
    const int64_t N = D.n_d + D.m;
    if (N <= 0) return;
    k_assemble_M_dense<<<(unsigned)std::min<int64_t>(N, 8192), 256, 0, s>>>(D, Mv, Hdd, sig_xd, Jdh,
                                                                            sig_d, dw, dc, Mat);
    MDSIP_LAUNCHED();
    if (D.m_E > 0) {
        k_assemble_M_sparse<<<std::max(1, std::min(4096, ceil_div(D.m_E, 256))), 256, 0, s>>>(D, Mv, q,
                                                                                              Mat);
        MDSIP_LAUNCHED();
    }
    if (D.m_I > 0 && Mv.hsr_ptr) {
        k_assemble_M_sparse_h<<<std::max(1, std::min(4096, ceil_div(D.m_I, 128))), 128, 0, s>>>(D, Mv, q, Mat);
        MDSIP_LAUNCHED();
    }
}

}  // namespace mdsip
