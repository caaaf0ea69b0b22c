// Internal declarations of libmdsip: context, problem state, device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/mdsip.h"

namespace mdsip {

// ---------------------------------------------------------------------------
// Error handling: every CUDA call is checked; failures become statuses.
// ---------------------------------------------------------------------------
struct Error {
    mdsip_status status;
    std::string msg;
};

#define MDSIP_CUDA(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::mdsip::Error{e_ == cudaErrorMemoryAllocation ? MDSIP_ERR_OOM           \
                                                                 : MDSIP_ERR_CUDA,         \
                                 std::string(#call) + ": " + cudaGetErrorString(e_)};      \
    } while (0)

#define MDSIP_REQUIRE(cond, st, text)                                                      \
    do {                                                                                   \
        if (!(cond)) throw ::mdsip::Error{st, text};                                       \
    } while (0)

void count_launch();
#define MDSIP_LAUNCHED()                   \
    do {                                   \
        ::mdsip::count_launch();           \
        MDSIP_CUDA(cudaGetLastError());    \
    } while (0)

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mdsip_alloc_hooks hooks{};
    bool has_hooks = false;
    int num_sms = 0;
    std::string last_error;
    int32_t ldlt_panels[2] = {0, 0};   // of the last mdsip_ldlt_factor* call
    // grow-only scratch arena for kernel-level calls
    void *scratch = nullptr;
    size_t scratch_bytes = 0;

    void *alloc(size_t bytes);
    void release(void *p, size_t bytes);
    void *scratch_at_least(size_t bytes);
};

// Makes `dev` current for the scope of the object.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        MDSIP_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Runs fn, turning exceptions into a status and the context's last error.
template <class F>
inline mdsip_status guarded(Ctx *ctx, F &&fn) {
    try {
        fn();
        return MDSIP_OK;
    } catch (const Error &e) {
        if (ctx) ctx->last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->last_error = "host allocation failed";
        return MDSIP_ERR_OOM;
    } catch (...) {
        if (ctx) ctx->last_error = "unknown error";
        return MDSIP_ERR_CUDA;
    }
}

// A device buffer owned through the context's allocator.
struct DBuf {
    Ctx *ctx = nullptr;
    void *ptr = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { reset(); }
    void reset() {
        if (ptr && ctx) ctx->release(ptr, bytes);
        ptr = nullptr;
        bytes = 0;
    }
    template <class T>
    T *get(Ctx *c, size_t count) {
        reset();
        ctx = c;
        bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
        ptr = c->alloc(bytes);
        return static_cast<T *>(ptr);
    }
    template <class T>
    T *as() const { return static_cast<T *>(ptr); }
};

// ---------------------------------------------------------------------------
// Options: constants of the method (Section 2.1, with the readings of the
// filter line search and inertia correction it delegates).
// ---------------------------------------------------------------------------
struct Options {
    double tol = 1e-8;
    int64_t max_iter = 200;
    double mu0 = 0.1;
    double kappa_eps = 10.0, kappa_mu = 0.2, theta_mu = 1.5, tau_min = 0.99;
    double s_max = 100.0, kappa_1 = 1e-2, kappa_2 = 1e-2, kappa_sigma = 1e10;
    double gamma_theta = 1e-5, gamma_phi = 1e-8, delta = 1.0, s_theta = 1.1, s_phi = 2.3;
    double eta_phi = 1e-8, gamma_alpha = 0.05;
    double theta_max_fact = 1e4, theta_min_fact = 1e-4;
    int64_t max_ls = 60;
    double dw0 = 1e-4, dw_min = 1e-20, dw_max = 1e40, kw_minus = 1.0 / 3.0, kw_plus = 8.0,
           kw_plus_bar = 100.0, dc_bar = 1e-8, kappa_c = 0.25;
    double zero_tol = 1e-14;
    int64_t path = MDSIP_PATH_AUTO;
    int64_t refine_max = -1;          // -1: 0 for FP64, 30 for tensor-core products
    int64_t precision = MDSIP_PREC_FP64;
    double refine_tol = 1e-14;
    double refine_fallback_tol = 1e-10;
    double time_limit_s = 0.0;
    int64_t graphs = 1;               // 1: replay the factorization phase as a CUDA graph
    int64_t autotune = 1;             // 1: time tile-shape candidates at first use per shape
    int64_t ldlt_spec = 1;            // 1: mixed-precision LDL^T panels try the verified no-interchange path
    int64_t direction_check = 0;      // 1: each mixed-precision step also forms the FP64 direction and logs the gap
};

// ---------------------------------------------------------------------------
// Device views passed to kernels by value.
// ---------------------------------------------------------------------------
struct Dims {
    int64_t n_s, n_d, m_E, m_I, n, m;
    int64_t lda;  // leading dimension of A (row-major, padded to a multiple of 4)
};

struct ModelView {
    const double *Q, *c, *A, *gE, *hl, *hu, *xl, *xu;
    const int32_t *h_set;
    const int32_t *csr_ptr, *csr_col;  // J_sg by rows (m_E + 1, nnz)
    const double *csr_val;
    const int32_t *csc_ptr, *csc_row;  // J_sg by columns (n_s + 1, nnz)
    const double *csc_val;
    // J_sh (the inequalities' sparse block): by rows (m_I + 1) and by columns
    // (n_s + 1); all null when J_sh = 0 (the benchmark family)
    const int32_t *hsr_ptr, *hsr_col;
    const double *hsr_val;
    const int32_t *hsc_ptr, *hsc_row;
    const double *hsc_val;
};

// Number of per-block partial slots used by the reduction kernels.
constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

// Scalars written by reduction kernels and read by the host control.
enum Scalar : int {
    S_F = 0,          // objective
    S_THETA,          // ||c||_1
    S_INF_PR,         // ||c||_inf
    S_INF_DU,         // ||grad L - z||_inf (x and d parts)
    S_COMP_MAX,       // max over finite bounds of s*z
    S_COMP_MIN,       // min over finite bounds of s*z
    S_Y1,             // ||y||_1
    S_Z1,             // ||z||_1 + ||v||_1
    S_LOGSUM,         // sum of log slacks at the current point
    S_GPHI,           // grad phi_mu^T (dx, dd)
    S_AMAX,           // fraction-to-boundary alpha for the primal
    S_AZ,             // fraction-to-boundary alpha for the multipliers
    S_QPOS, S_QNEG, S_QZERO,   // inertia of Q_s
    S_WPOS, S_WNEG, S_WZERO,   // inertia of -W (path P2)
    S_T_F, S_T_THETA, S_T_LOGSUM, S_T_INSIDE, S_T_FINITE,  // trial point
    S_MAXABS,         // max |reduced matrix| (zero-pivot scale)
    S_NONFINITE,      // count of non-finite model values
    S_RES_INF, S_RHS_INF, S_SOL_INF,  // refinement: ||r||_inf, ||rhs||_inf, ||dir||_inf
    S_COUNT
};

// ---------------------------------------------------------------------------
// Block-level reductions (deterministic for a fixed launch shape).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) r += sh[i];
    }
    return r;  // valid in thread 0
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = -INFINITY;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) r = fmax(r, sh[i]);
    }
    return r;
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double *sh) {
    return -block_max<NT>(-v, sh);
}

// ---------------------------------------------------------------------------
// Grid barrier with a bounded wait.  Used only in cooperative launches (all
// blocks co-resident).  On expiry it raises *err and returns false; callers
// leave their loops at once, so a lost block never hangs the GPU.
// ---------------------------------------------------------------------------
struct GridBar {
    unsigned int *count;
    unsigned int *gen;
    int *err;
};

constexpr long long kBarrierLimitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ bool grid_barrier(const GridBar &b, unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vgen = b.gen;
        const unsigned int my = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(b.count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(b.count, 0u);
            __threadfence();
            atomicAdd(b.gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == my) {
                if (*((volatile int *)b.err) != 0 || clock64() - t0 > kBarrierLimitCycles) {
                    atomicExch(b.err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Runs a configuration call (e.g. a kernel attribute, which is global to the
// kernel on a device) once per device, thread-safely; returns its result.
struct PerDeviceOnce {
    std::mutex mu;
    bool done[64] = {};
    cudaError_t err[64] = {};
    template <class F>
    cudaError_t run(F &&f) {
        int dev = 0;
        const cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return f();
        std::lock_guard<std::mutex> lk(mu);
        if (!done[dev]) {
            err[dev] = f();
            done[dev] = true;
        }
        return err[dev];
    }
};

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
// reductions: partial[k * kRedBlocks + b] -> scalars[first + k] (sum / max / min)
// probe.cu: blocks x 256 threads, each iters x 8 independent FP64 FMAs; sink
// holds blocks x 256 doubles
void launch_fp64_fma_probe(cudaStream_t s, int blocks, int64_t iters, double *sink);
void launch_finalize_sum(cudaStream_t s, const double *partial, int nq, double *out);
void launch_finalize_max(cudaStream_t s, const double *partial, int nq, double *out);
void launch_finalize_min(cudaStream_t s, const double *partial, int nq, double *out);

// A passes (row-major A, m x n, leading dimension lda)
void launch_gemv_rows(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda,
                      const double *v, double *out);  // out = A v
// out[p] = sum_b partial[b][p] (fixed order); partial: nparts x n
void launch_colsum(cudaStream_t s, const double *partial, int nparts, int64_t n, double *out);
// gemv_df.cu: passes over A = A_hi + A_lo (FP32 pair, m x lda) in double-float
// arithmetic with FP64 accuracy; xs / ys: scratch of n / m float2
void launch_split_matrix(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda, float *hi,
                         float *lo);
void launch_gemv_rows_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                         const double *x, float2 *xs, double *out);
void launch_gemv_t_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                      const double *y, float2 *ys, double *partial, double *out);
// out_rows = A x and out_cols = A^T y from one read of A.  With nx, the same
// read also gives out_v = A_hi^T v, v_i = fl32((cpre_i - (A x)_i) wf_i) with
// the difference in double-float (FP32 products and sums): the first half of
// the refinement's next approximate solve.  cw = cpre as FP32 halves
// (launch_split_vector), wf = fl32(1 / w) (launch_round_vector).  The fused
// form needs the whole row in one slice: gemv_both_fusable(n).
struct BothNextArgs {
    const float2 *cw;   // m
    const float *wf;    // m
    double *out_v;      // n
};
void launch_split_vector(cudaStream_t s, const double *v, int64_t n, float2 *out);   // out = (fl32(v), fl32(v - hi))
void launch_round_vector(cudaStream_t s, const double *v, int64_t n, float *out);    // out = fl32(v)
bool gemv_both_fusable(int64_t n);
void launch_gemv_both_df(cudaStream_t s, const float *Ahi, const float *Alo, int64_t m, int64_t n, int64_t lda,
                         const double *x, const double *y, float2 *xs, float2 *ys, double *partial,
                         double *out_rows, double *out_cols, int *err, const BothNextArgs *nx = nullptr);
// out = A_hi x with FP32 products and sums
void launch_gemv_rows_f32(cudaStream_t s, const float *Ahi, int64_t m, int64_t n, int64_t lda, const double *x,
                          double *out);
void launch_gemv_t(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda,
                   const double *u, double *partial, double *out);  // out = A^T u

// SYRK: C (column-major, ldc) = beta C + A^T diag(1/w) A (lower)
void launch_syrk_fp64(Ctx *ctx, const double *A, int64_t m, int64_t n, int64_t lda, const double *w,
                      double beta, double *C, int64_t ldc);
size_t syrk_fp64_scratch_bytes(int64_t m, int64_t n, int num_sms);
void launch_syrk_fp64_ws(cudaStream_t s, int num_sms, const double *A, int64_t m, int64_t n,
                         int64_t lda, const double *w, double beta, double *C, int64_t ldc,
                         double *work, int bm = 0);

// Tensor-core SYRK (syrk_tc.cu)
struct TcPlan {
    int tiles, nsplit, slabs_per_split, total_slabs, elems_per_slab;
    int64_t ldt;
    size_t work_floats;
};
int64_t syrk_tc_ld(int64_t m);
void launch_aft_dot(cudaStream_t s, int num_sms, const float *AfT, int64_t ldt, int64_t m, int64_t n,
                    const double *v, float *vf, double *out);
TcPlan syrk_tc_plan(int64_t m, int64_t n, int num_sms, int precision);
size_t syrk_tc_workspace_bytes(const TcPlan &pl, int64_t n, int precision);
void launch_transpose_f32(cudaStream_t s, const double *A, int64_t m, int64_t n, int64_t lda, float *AfT,
                          int64_t ldt);
void launch_syrk_tc(cudaStream_t s, int num_sms, int precision, const float *AfT, int64_t m, int64_t n,
                    const double *w, double beta, double *C, int64_t ldc, void *ws, int *err_dev);

// Bunch-Kaufman LDL^T
struct LdltOut {
    double *L, *Dd, *Doff;
    int32_t *perm, *kind, *inertia;
    int32_t *panels = nullptr;   // optional: panels taken by the no-interchange path, and handed back
};
size_t ldlt_scratch_bytes(int64_t N);
void launch_ldlt(cudaStream_t s, int num_sms, int64_t N, const double *S, int64_t ld,
                 const double *maxabs_dev, double zero_tol, LdltOut out, void *scratch,
                 int *err_dev, bool fp32_update = false, int nb = 0, int spec = 1);
size_t ldlt_blocked_scratch_bytes(int64_t N);
bool ldlt_blocked_available(int64_t N);
// Speculation mode of the blocked factorization: 0 every panel pivots; 1 (auto)
// no-interchange panels, the persistent kernel from order kPersistentMinOrder
// on or where the pivoting panel does not fit; 2 the persistent kernel at any
// order.  The persistent kernel reads back where it stopped (synchronises the
// stream).
constexpr int64_t kPersistentMinOrder = 2048;
bool ldlt_persistent_path(int64_t N, int spec);
std::vector<int> ldlt_blocked_widths(int64_t N, bool f32);
void launch_ldlt_blocked(cudaStream_t s, int num_sms, int64_t N, double *S, const double *maxabs_dev,
                         double zero_tol, LdltOut out, void *scratch, bool fp32_update, int nb = 0,
                         int spec = 1);
void launch_ldlt_solve(cudaStream_t s, int64_t N, const double *L, const double *Dd,
                       const double *Doff, const int32_t *perm, int64_t nrhs, double *B,
                       int64_t ldb);
void launch_maxabs_lower(cudaStream_t s, int64_t N, const double *S, int64_t ld, double *partial,
                         double *out);
size_t ldlt_solve_scratch_bytes(int64_t N);
// tiles of L for the solve (FP64, or FP32 when fp32), into the solve scratch; after each factorization
void launch_ldlt_solve_prepare(cudaStream_t s, int64_t N, const double *L, void *scratch, bool fp32);
// b_r <- K^-1 b_r with the prepared tiles (same fp32 flag)
void launch_ldlt_solve_coop(cudaStream_t s, int num_sms, int64_t N, const double *Dd, const double *Doff,
                            const int32_t *perm, int64_t nrhs, double *B, int64_t ldb, void *scratch, int *err_dev,
                            bool fp32);
// LDL^T with its scratch in a fixed device array (no allocation); N <= the limit.
int64_t ldlt_fixed_scratch_max_n();
void ldlt_factor_fixed_scratch(cudaStream_t s, int device, int num_sms, int64_t N, double *S,
                               int64_t ld, double zero_tol, LdltOut out);

}  // namespace mdsip
