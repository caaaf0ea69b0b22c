// Host control of the interior-point method and the C ABI of libmdsip.
//
// The control logic of the method is sequential (Section 3): the host runs
// the filter line-search loop of Section 2.1 (Waechter-Biegler Algorithm A
// with inertia correction, no second-order correction, no restoration) and
// launches the device kernels; per step it reads back only scalars (norms,
// inertia counts, step lengths, trial merit values).  All vectors and
// matrices stay on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <tuple>
#include <atomic>
#include <map>
#include <thread>

#include "internal.cuh"
#include "refine.cuh"
#include "vec.cuh"

namespace mdsip {

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;   // this thread's launches (graph capture bookkeeping)
void count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}
static void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
void *Ctx::alloc(size_t bytes) {
    void *p = nullptr;
    if (has_hooks) {
        p = hooks.alloc(bytes, stream, hooks.user);
        if (!p) throw Error{MDSIP_ERR_OOM, "allocation hook returned NULL"};
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{MDSIP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
        }
    }
    return p;
}

void Ctx::release(void *p, size_t bytes) {
    if (!p) return;
    if (has_hooks)
        hooks.free(p, bytes, stream, hooks.user);
    else
        cudaFree(p);
}

void *Ctx::scratch_at_least(size_t bytes) {
    if (bytes <= scratch_bytes) return scratch;
    if (scratch) {
        MDSIP_CUDA(cudaStreamSynchronize(stream));
        release(scratch, scratch_bytes);
        scratch = nullptr;
        scratch_bytes = 0;
    }
    scratch = alloc(bytes);
    scratch_bytes = bytes;
    return scratch;
}


// ---------------------------------------------------------------------------
// Problem state
// ---------------------------------------------------------------------------
enum : int {
    SC_F = 0, SC_THETA = 1, SC_CMAX = 2,
    SC_E = 3,        // 7: max|dual|, max|c|, max sz, min sz, ||y||_1, ||z||_1, sum log s
    SC_DIAG = 10,    // 6: In(Q_s) pos/neg/zero, In(-W) pos/neg/zero
    SC_STEP = 16,    // 3: alpha_max, alpha_z, gphi
    SC_TF = 19, SC_TTHETA = 20, SC_TCMAX = 21,
    SC_TRIAL = 22,   // 2: sum log s, #non-positive slacks
    SC_MAXABS = 24,
    SC_REF = 25,     // 4: ||r||inf, ||b||inf, ||K u||inf, ||u||inf
    SC_DCHK = 29,    // 2: sum (mixed - FP64 direction)^2, sum (FP64 direction)^2
    SC_COUNT = 32
};

struct Problem {
    Ctx *ctx = nullptr;
    Dims D{};
    ModelView Mv{};
    Options opt;
    int path = MDSIP_PATH_P2;
    bool p2_ok = false;
    bool sparse_dup = false;
    int64_t n_bounds = 0;
    int64_t N = 0;  // reduced matrix size

    // model data
    DBuf bQ, bc, bA, bgE, bhl, bhu, bxl, bxu, bx0, bhset;
    DBuf bcsr_ptr, bcsr_col, bcsr_val, bcsc_ptr, bcsc_row, bcsc_val;
    // iterate, trial, direction
    DBuf bx, bd, byg, byh, bzl, bzu, bvl, bvu, bxt, bdt;
    DBuf bdx, bdd, bdyg, bdyh, bdzl, bdzu, bdvl, bdvu;
    DBuf bcx, bcd, bcyg, bcyh, bczl, bczu, bcvl, bcvu;   // saved direction of the FP64 check
    DBuf bhsr_ptr, bhsr_col, bhsr_val, bhsc_ptr, bhsc_row, bhsc_val;   // J_sh by rows and by columns
    int64_t nnz_jsh = 0;
    DirView Dchk{};
    // model values and Newton quantities
    DBuf bgrad, bgrad_t, bcg, bcg_t, bch, bch_t, bgl, bATy, bJdh, bHss, bHdd;
    DBuf bsig_x, bq, bsig_d, bw, bbt_g, bu, bATu, brhs, bAdx;
    // reduced matrix and factors
    DBuf bS, bL, bDd, bDoff, bperm, bkind, binertia, bldlt_ws, berr, bsyrk_ws, btune;
    // tensor-core condensation and refinement
    DBuf bAfT, bvf, btc_ws, btc_err, bref_b, bref_u, bref_r, bref_d, btmp_nd2, bsolve_ws, bsolve_err, bAu_run;
    DBuf bcpre, bcw, bwf, bATv, bAsd;   // the refinement's fused residual pass
    bool aft_ready = false;
    DBuf bAhi, bAlo, bsplit;   // A as an FP32 pair (mixed path's double-float passes) and vector scratch
    // Products with A carried from step to step on the mixed path of a data-given
    // problem, whose constraints are linear in x_d: A x_d of the iterate and of
    // the trial, A dx_d and A^T dy_g of the direction (from the refinement's last
    // residual pass); A^T y_g of the iterate lives in bATy.
    DBuf bAx_a, bAx_b, bdAx, bdATy;
    double *ax_cur = nullptr, *ax_t = nullptr;
    bool lin_ax = false;    // ax_cur holds A x_d of the iterate
    bool lin_aty = false;   // bATy holds A^T y_g of the iterate
    bool dir_prod = false;  // bAdx / bATu hold A dx_d and A^T dy_g of the direction just computed
    bool df_ready = false;
    int64_t tc_prec = -1;
    DBuf bscal, bpartial, bcolpart, browtmp;
    double *hscal = nullptr;  // pinned mirror of the scalars
    int32_t *hint = nullptr;  // pinned: inertia (3) + device error flag

    IterView I{};
    DirView Dir{};
    VecOps V{};
    double *xt = nullptr, *dt = nullptr, *grad = nullptr, *grad_t = nullptr, *cg = nullptr,
           *cg_t = nullptr, *ch = nullptr, *ch_t = nullptr;

    // model: 0 = the built-in benchmark family, 1 = user callbacks
    int model_kind = 0;
    mdsip_callbacks cb{};
    void *user = nullptr;
    bool bounds_set = true;
    DBuf bJsg_user, bperm_csr, bperm_csc, bg_raw, bh_raw;
    int64_t nnz = 0;

    bool has_start = false;
    bool solve_fp32 = false;  // tiles of the current factor are FP32 (refined tensor-core path)
    double start_mu0 = -1.0;
    std::vector<mdsip_iter_rec> log;
    mdsip_stats stats{};
    cudaEvent_t ev[12]{};
    // The factorization phase (scale of S, the LDL^T's kernels, the solve's
    // tiles: about 70 launches with fixed arguments for a given order and
    // precision) as a CUDA graph: captured on its second use, replayed after.
    struct FactorGraph {
        cudaGraphExec_t exec = nullptr;
        int64_t N = -1;
        double zero_tol = -1.0;
        int uses = 0;
        long long launches = 0;
        bool disabled = false;
    } fgraph[2];   // [0] FP64 updates, [1] FP32 updates

    void drop_graphs() {
        for (auto &g : fgraph) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = FactorGraph{};
        }
    }

    ~Problem() {
        drop_graphs();
        if (hscal) cudaFreeHost(hscal);
        if (hint) cudaFreeHost(hint);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }

    double *scal() const { return bscal.as<double>(); }

    void sync_scalars() {
        MDSIP_CUDA(cudaMemcpyAsync(hscal, scal(), SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
    }
};

// ---------------------------------------------------------------------------
// Creation
// ---------------------------------------------------------------------------
template <class T>
static std::vector<T> fetch(const T *src, int64_t count, int mem) {
    std::vector<T> out((size_t)std::max<int64_t>(count, 0));
    if (count <= 0) return out;
    MDSIP_REQUIRE(src != nullptr, MDSIP_ERR_INVALID_ARG, "null data pointer");
    if (mem == MDSIP_MEM_HOST)
        std::memcpy(out.data(), src, count * sizeof(T));
    else
        MDSIP_CUDA(cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
    return out;
}

template <class T>
static T *upload(Ctx *ctx, DBuf &buf, const std::vector<T> &v, int64_t count) {
    T *p = buf.get<T>(ctx, (size_t)std::max<int64_t>(count, 1));
    if (count > 0)
        MDSIP_CUDA(cudaMemcpyAsync(p, v.data(), count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return p;
}

// copy into an existing allocation (pointers held elsewhere stay valid)
template <class T>
static void fill(Ctx *ctx, DBuf &buf, const std::vector<T> &v, int64_t count) {
    MDSIP_REQUIRE(buf.ptr != nullptr && (size_t)std::max<int64_t>(count, 0) * sizeof(T) <= buf.bytes,
                  MDSIP_ERR_INVALID_ARG, "internal: buffer too small");
    if (count > 0)
        MDSIP_CUDA(cudaMemcpyAsync(buf.ptr, v.data(), count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
}

static double *dvec(Ctx *ctx, DBuf &b, int64_t n) {
    double *p = b.get<double>(ctx, (size_t)std::max<int64_t>(n, 1));
    MDSIP_CUDA(cudaMemsetAsync(p, 0, std::max<int64_t>(n, 1) * sizeof(double), ctx->stream));
    return p;
}

// Sparse indices of J_sg: CSR and CSC (int32), duplicates summed; perm_csr /
// perm_csc map each stored position to the index of its triplet (used to
// refresh the values of a callback model; duplicates are rejected there).
struct SparseBuild {
    std::vector<int32_t> csr_ptr, csr_col, csc_ptr, csc_row, perm_csr, perm_csc;
    std::vector<double> csr_val, csc_val;
    bool has_dup = false;
    bool p2_ok = true;
};

// (nrows x n_s block: J_sg with nrows = m_E, J_sh with nrows = m_I)
static SparseBuild build_sparse(const Dims &D, const std::vector<int32_t> &rows, const std::vector<int32_t> &cols,
                                const std::vector<double> &vals, int64_t nrows = -1, const char *what = "J_sg") {
    SparseBuild b;
    if (nrows < 0) nrows = D.m_E;
    const int64_t n_in = (int64_t)rows.size();
    for (int64_t e = 0; e < n_in; ++e)
        MDSIP_REQUIRE(rows[e] >= 0 && rows[e] < nrows && cols[e] >= 0 && cols[e] < D.n_s, MDSIP_ERR_INVALID_ARG,
                      std::string(what) + " index out of range");
    std::vector<int64_t> order((size_t)n_in);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
        return std::tie(rows[a], cols[a], a) < std::tie(rows[c], cols[c], c);
    });
    std::vector<int32_t> r2, c2, src;
    for (int64_t t = 0; t < n_in; ++t) {
        const int64_t e = order[t];
        if (!r2.empty() && r2.back() == rows[e] && c2.back() == cols[e]) {
            b.csr_val.back() += vals[e];
            b.has_dup = true;
        } else {
            r2.push_back(rows[e]);
            c2.push_back(cols[e]);
            b.csr_val.push_back(vals[e]);
            src.push_back((int32_t)e);
        }
    }
    const int64_t nnz = (int64_t)r2.size();
    b.csr_ptr.assign(nrows + 1, 0);
    b.csc_ptr.assign(D.n_s + 1, 0);
    b.csc_row.resize(nnz);
    b.csc_val.resize(nnz);
    b.perm_csc.resize(nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        b.csr_ptr[r2[e] + 1]++;
        b.csc_ptr[c2[e] + 1]++;
    }
    for (int64_t i = 0; i < nrows; ++i) b.csr_ptr[i + 1] += b.csr_ptr[i];
    for (int64_t k = 0; k < D.n_s; ++k) b.csc_ptr[k + 1] += b.csc_ptr[k];
    std::vector<int32_t> fill(b.csc_ptr.begin(), b.csc_ptr.end() - 1);
    for (int64_t e = 0; e < nnz; ++e) {  // rows ascending within each column
        const int32_t pos = fill[c2[e]]++;
        b.csc_row[pos] = r2[e];
        b.csc_val[pos] = b.csr_val[e];
        b.perm_csc[pos] = src[e];
    }
    for (int64_t k = 0; k < D.n_s; ++k)
        if (b.csc_ptr[k + 1] - b.csc_ptr[k] > 1) b.p2_ok = false;
    b.csr_col = std::move(c2);
    b.perm_csr = std::move(src);
    return b;
}

// Common part of both problem kinds: dimensions, sparse indices, iterate and
// work vectors.  Bounds, g_E and x0 buffers are allocated (filled by the caller).
static Problem *create_common(Ctx *ctx, int64_t n_d, int64_t n_s, int64_t m_E, int64_t m_I,
                              const std::vector<int32_t> &rows, const std::vector<int32_t> &cols,
                              const std::vector<double> &vals) {
    MDSIP_REQUIRE(n_d >= 0 && n_s >= 0 && m_E >= 0 && m_I >= 0, MDSIP_ERR_INVALID_ARG, "negative size");
    MDSIP_REQUIRE(n_s + n_d > 0, MDSIP_ERR_INVALID_ARG, "no variables");
    MDSIP_REQUIRE((int64_t)rows.size() < (1LL << 31) && m_E < (1LL << 31) && n_s < (1LL << 31),
                  MDSIP_ERR_INVALID_ARG, "sparse block too large for 32-bit indices");
    auto P = new Problem();
    try {
        P->ctx = ctx;
        Dims &D = P->D;
        D.n_s = n_s;
        D.n_d = n_d;
        D.m_E = m_E;
        D.m_I = m_I;
        D.n = D.n_s + D.n_d;
        D.m = D.m_E + D.m_I;
        D.lda = std::max<int64_t>(4, (D.n_d + 3) / 4 * 4);
        cudaStream_t st = ctx->stream;
        SparseBuild sb = build_sparse(D, rows, cols, vals);
        P->p2_ok = sb.p2_ok;
        P->nnz = (int64_t)sb.csr_val.size();
        P->sparse_dup = sb.has_dup;
        ModelView &M = P->Mv;
        M.csr_ptr = upload(ctx, P->bcsr_ptr, sb.csr_ptr, D.m_E + 1);
        M.csr_col = upload(ctx, P->bcsr_col, sb.csr_col, P->nnz);
        M.csr_val = upload(ctx, P->bcsr_val, sb.csr_val, P->nnz);
        M.csc_ptr = upload(ctx, P->bcsc_ptr, sb.csc_ptr, D.n_s + 1);
        M.csc_row = upload(ctx, P->bcsc_row, sb.csc_row, P->nnz);
        M.csc_val = upload(ctx, P->bcsc_val, sb.csc_val, P->nnz);
        upload(ctx, P->bperm_csr, sb.perm_csr, P->nnz);
        upload(ctx, P->bperm_csc, sb.perm_csc, P->nnz);
        M.c = dvec(ctx, P->bc, D.n);
        M.gE = dvec(ctx, P->bgE, D.m_E);
        M.hl = dvec(ctx, P->bhl, D.m_I);
        M.hu = dvec(ctx, P->bhu, D.m_I);
        M.xl = dvec(ctx, P->bxl, D.n);
        M.xu = dvec(ctx, P->bxu, D.n);
        dvec(ctx, P->bx0, D.n);
        M.Q = dvec(ctx, P->bQ, 0);
        M.h_set = P->bhset.get<int32_t>(ctx, std::max<int64_t>(D.n_d, 1));
        MDSIP_CUDA(cudaMemsetAsync(P->bhset.ptr, 0xff, std::max<int64_t>(D.n_d, 1) * sizeof(int32_t), st));
        M.A = dvec(ctx, P->bA, D.m_E * D.lda);

        // iterate and work vectors
        IterView &I = P->I;
        I.x = dvec(ctx, P->bx, D.n);
        I.d = dvec(ctx, P->bd, D.m_I);
        I.yg = dvec(ctx, P->byg, D.m_E);
        I.yh = dvec(ctx, P->byh, D.m_I);
        I.zl = dvec(ctx, P->bzl, D.n);
        I.zu = dvec(ctx, P->bzu, D.n);
        I.vl = dvec(ctx, P->bvl, D.m_I);
        I.vu = dvec(ctx, P->bvu, D.m_I);
        P->xt = dvec(ctx, P->bxt, D.n);
        P->dt = dvec(ctx, P->bdt, D.m_I);
        DirView &R = P->Dir;
        R.dx = dvec(ctx, P->bdx, D.n);
        R.dd = dvec(ctx, P->bdd, D.m_I);
        R.dyg = dvec(ctx, P->bdyg, D.m_E);
        R.dyh = dvec(ctx, P->bdyh, D.m_I);
        R.dzl = dvec(ctx, P->bdzl, D.n);
        R.dzu = dvec(ctx, P->bdzu, D.n);
        R.dvl = dvec(ctx, P->bdvl, D.m_I);
        R.dvu = dvec(ctx, P->bdvu, D.m_I);
        P->grad = dvec(ctx, P->bgrad, D.n);
        P->grad_t = dvec(ctx, P->bgrad_t, D.n);
        P->cg = dvec(ctx, P->bcg, D.m_E);
        P->cg_t = dvec(ctx, P->bcg_t, D.m_E);
        P->ch = dvec(ctx, P->bch, D.m_I);
        P->ch_t = dvec(ctx, P->bch_t, D.m_I);
        dvec(ctx, P->bgl, D.n);
        dvec(ctx, P->bATy, D.n_d);
        dvec(ctx, P->bJdh, D.m_I * D.n_d);
        dvec(ctx, P->bHss, D.n_s);
        dvec(ctx, P->bHdd, D.n_d * D.n_d);
        dvec(ctx, P->bsig_x, D.n);
        dvec(ctx, P->bq, D.n_s);
        dvec(ctx, P->bsig_d, D.m_I);
        dvec(ctx, P->bw, D.m_E);
        dvec(ctx, P->bbt_g, D.m_E);
        dvec(ctx, P->bu, D.m_E);
        dvec(ctx, P->bATu, D.n_d);
        dvec(ctx, P->bAdx, D.m_E);
        dvec(ctx, P->bscal, SC_COUNT);
        dvec(ctx, P->bpartial, (int64_t)kRedBlocks * 8);
        dvec(ctx, P->bcolpart, (int64_t)kRedBlocks * std::max<int64_t>(D.n_d, 1));
        dvec(ctx, P->browtmp, std::max<int64_t>(D.m_E, 1));
        P->berr.get<int>(ctx, 4);
        MDSIP_CUDA(cudaMallocHost(&P->hscal, SC_COUNT * sizeof(double)));
        MDSIP_CUDA(cudaMallocHost(&P->hint, 8 * sizeof(int32_t)));
        for (auto &e : P->ev) MDSIP_CUDA(cudaEventCreate(&e));
        P->V.D = D;
        P->V.M = M;
        P->V.st = st;
        P->V.partial = P->bpartial.as<double>();
        P->V.colpart = P->bcolpart.as<double>();
        P->V.rowtmp = P->browtmp.as<double>();
    } catch (...) {
        delete P;
        throw;
    }
    return P;
}

// bounds, g_E, x0 from host vectors (validated); counts the finite bounds
static void set_bounds_host(Problem *P, const std::vector<double> &xl, const std::vector<double> &xu,
                            const std::vector<double> &hl, const std::vector<double> &hu,
                            const std::vector<double> &gE, const std::vector<double> &x0) {
    const Dims &D = P->D;
    int64_t nb = 0;
    for (int64_t i = 0; i < D.n; ++i) {
        MDSIP_REQUIRE(!(xl[i] > xu[i]), MDSIP_ERR_INVALID_ARG, "xl > xu");
        nb += std::isfinite(xl[i]) + std::isfinite(xu[i]);
    }
    for (int64_t j = 0; j < D.m_I; ++j) {
        MDSIP_REQUIRE(hl[j] < hu[j], MDSIP_ERR_INVALID_ARG, "need hl < hu");
        MDSIP_REQUIRE(std::isfinite(hl[j]) || std::isfinite(hu[j]), MDSIP_ERR_INVALID_ARG,
                      "every inequality needs a finite bound");
        nb += std::isfinite(hl[j]) + std::isfinite(hu[j]);
    }
    P->n_bounds = nb;
    Ctx *ctx = P->ctx;
    fill(ctx, P->bxl, xl, D.n);
    fill(ctx, P->bxu, xu, D.n);
    fill(ctx, P->bhl, hl, D.m_I);
    fill(ctx, P->bhu, hu, D.m_I);
    fill(ctx, P->bgE, gE, D.m_E);
    fill(ctx, P->bx0, x0, D.n);
    MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
    P->bounds_set = true;
}

static Problem *create_synthetic(Ctx *ctx, const mdsip_synth_data *dat, int mem) {
    MDSIP_REQUIRE(dat, MDSIP_ERR_INVALID_ARG, "null data");
    MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
    MDSIP_REQUIRE(dat->n_d >= 0 && dat->n_s >= 0 && dat->m_E >= 0 && dat->m_I >= 0 && dat->nnz_Jsg >= 0,
                  MDSIP_ERR_INVALID_ARG, "negative size");
    const int64_t n = dat->n_s + dat->n_d;
    auto rows = fetch(dat->Jsg_rows, dat->nnz_Jsg, mem);
    auto cols = fetch(dat->Jsg_cols, dat->nnz_Jsg, mem);
    auto vals = fetch(dat->Jsg_vals, dat->nnz_Jsg, mem);
    Problem *P = create_common(ctx, dat->n_d, dat->n_s, dat->m_E, dat->m_I, rows, cols, vals);
    try {
        const Dims &D = P->D;
        cudaStream_t st = ctx->stream;
        auto c = fetch(dat->c, n, mem);
        auto gE = fetch(dat->gE, D.m_E, mem);
        auto hl = fetch(dat->hl, D.m_I, mem);
        auto hu = fetch(dat->hu, D.m_I, mem);
        auto xl = fetch(dat->xl, n, mem);
        auto xu = fetch(dat->xu, n, mem);
        std::vector<double> x0 = dat->x0 ? fetch(dat->x0, n, mem) : std::vector<double>(n, 0.0);
        auto hset = fetch(dat->h_set, D.n_d, mem);
        for (int64_t k = 0; k < D.n_d; ++k)
            MDSIP_REQUIRE(hset[k] >= -1 && hset[k] < D.m_I, MDSIP_ERR_INVALID_ARG, "h_set out of range");
        ModelView &M = P->Mv;
        MDSIP_REQUIRE(dat->nnz_Jsh >= 0, MDSIP_ERR_INVALID_ARG, "negative nnz_Jsh");
        if (dat->nnz_Jsh > 0) {   // the inequalities' sparse block: P2's precondition no longer holds
            MDSIP_REQUIRE(dat->Jsh_rows && dat->Jsh_cols && dat->Jsh_vals, MDSIP_ERR_INVALID_ARG, "null J_sh");
            auto hr = fetch(dat->Jsh_rows, dat->nnz_Jsh, mem);
            auto hc = fetch(dat->Jsh_cols, dat->nnz_Jsh, mem);
            auto hv = fetch(dat->Jsh_vals, dat->nnz_Jsh, mem);
            SparseBuild hb = build_sparse(D, hr, hc, hv, D.m_I, "J_sh");
            const int64_t nz = (int64_t)hb.csr_val.size();
            P->nnz_jsh = nz;
            M.hsr_ptr = upload(ctx, P->bhsr_ptr, hb.csr_ptr, D.m_I + 1);
            M.hsr_col = upload(ctx, P->bhsr_col, hb.csr_col, nz);
            M.hsr_val = upload(ctx, P->bhsr_val, hb.csr_val, nz);
            M.hsc_ptr = upload(ctx, P->bhsc_ptr, hb.csc_ptr, D.n_s + 1);
            M.hsc_row = upload(ctx, P->bhsc_row, hb.csc_row, nz);
            M.hsc_val = upload(ctx, P->bhsc_val, hb.csc_val, nz);
            P->p2_ok = false;
        }
        fill(ctx, P->bc, c, n);
        fill(ctx, P->bhset, hset, D.n_d);
        const auto kind = mem == MDSIP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        double *Q = P->bQ.get<double>(ctx, std::max<int64_t>(D.n_d * D.n_d, 1));
        if (D.n_d > 0) {
            MDSIP_REQUIRE(dat->Q, MDSIP_ERR_INVALID_ARG, "null Q");
            MDSIP_CUDA(cudaMemcpyAsync(Q, dat->Q, D.n_d * D.n_d * sizeof(double), kind, st));
        }
        M.Q = Q;
        if (D.m_E > 0 && D.n_d > 0) {
            MDSIP_REQUIRE(dat->A, MDSIP_ERR_INVALID_ARG, "null A");
            MDSIP_CUDA(cudaMemcpy2DAsync(P->bA.ptr, D.lda * sizeof(double), dat->A, D.n_d * sizeof(double),
                                         D.n_d * sizeof(double), D.m_E, kind, st));
        }
        P->V.M = M;
        set_bounds_host(P, xl, xu, hl, hu, gE, x0);
    } catch (...) {
        delete P;
        throw;
    }
    return P;
}

static Problem *create_callbacks(Ctx *ctx, const mdsip_dims *dims, const int32_t *rows_p, const int32_t *cols_p,
                                 const mdsip_callbacks *cb, void *user, int mem) {
    MDSIP_REQUIRE(dims && cb, MDSIP_ERR_INVALID_ARG, "null dims or callbacks");
    MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
    MDSIP_REQUIRE(cb->eval_f && cb->eval_grad_f && cb->eval_cons && cb->eval_jac && cb->eval_hess,
                  MDSIP_ERR_INVALID_ARG, "every callback is required");
    MDSIP_REQUIRE(dims->nnz_Jsg >= 0, MDSIP_ERR_INVALID_ARG, "negative nnz");
    auto rows = fetch(rows_p, dims->nnz_Jsg, mem);
    auto cols = fetch(cols_p, dims->nnz_Jsg, mem);
    std::vector<double> zeros((size_t)dims->nnz_Jsg, 0.0);
    Problem *P = create_common(ctx, dims->n_d, dims->n_s, dims->m_E, dims->m_I, rows, cols, zeros);
    if (P->sparse_dup) {
        delete P;
        throw Error{MDSIP_ERR_INVALID_ARG, "duplicate J_sg triplets"};
    }
    P->model_kind = 1;
    P->cb = *cb;
    P->user = user;
    P->bounds_set = false;
    dvec(ctx, P->bJsg_user, P->nnz);
    dvec(ctx, P->bg_raw, P->D.m_E);
    dvec(ctx, P->bh_raw, P->D.m_I);
    MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
    return P;
}

// ---------------------------------------------------------------------------
// Model evaluation: built-in family or callbacks
// ---------------------------------------------------------------------------
static void cb_check(int rc, const char *what) {
    if (rc != 0) throw Error{MDSIP_ERR_CALLBACK, std::string("callback ") + what + " returned " + std::to_string(rc)};
}

static void model_f(Problem *P, const double *x, double *grad, double *fout) {
    if (P->model_kind == 0) {
        P->V.eval_f(x, grad, fout);
        return;
    }
    void *st = static_cast<void *>(P->ctx->stream);
    cb_check(P->cb.eval_f(P->user, st, x, fout), "eval_f");
    cb_check(P->cb.eval_grad_f(P->user, st, x, grad), "eval_grad_f");
}

static void model_cons(Problem *P, const double *x, const double *d, double *cg, double *ch, double *out2) {
    if (P->model_kind == 0) {
        P->V.eval_cons(x, d, cg, ch, out2);
        return;
    }
    cb_check(P->cb.eval_cons(P->user, static_cast<void *>(P->ctx->stream), x, P->bg_raw.as<double>(),
                             P->bh_raw.as<double>()),
             "eval_cons");
    P->V.cons_from_values(P->bg_raw.as<double>(), P->bh_raw.as<double>(), d, cg, ch, out2);
}

static void model_jac_hess(Problem *P, const double *x, const double *yg, const double *yh) {
    if (P->model_kind == 0) {
        P->V.jac_hess(x, yh, P->bJdh.as<double>(), P->bHss.as<double>(), P->bHdd.as<double>());
        return;
    }
    const Dims &D = P->D;
    void *st = static_cast<void *>(P->ctx->stream);
    cb_check(P->cb.eval_jac(P->user, st, x, P->bJsg_user.as<double>(), P->bA.as<double>(), D.lda,
                            P->bJdh.as<double>(), D.n_d),
             "eval_jac");
    P->V.gather(P->nnz, P->bJsg_user.as<double>(), P->bperm_csr.as<int32_t>(), P->bcsr_val.as<double>());
    P->V.gather(P->nnz, P->bJsg_user.as<double>(), P->bperm_csc.as<int32_t>(), P->bcsc_val.as<double>());
    cb_check(P->cb.eval_hess(P->user, st, x, yg, yh, P->bHss.as<double>(), P->bHdd.as<double>(), D.n_d),
             "eval_hess");
    P->aft_ready = false;  // the tensor-core copy of A follows the Jacobian
    if (P->df_ready)       // so does its FP32 pair
        launch_split_matrix(P->ctx->stream, P->bA.as<double>(), D.m_E, D.n_d, D.lda, P->bAhi.as<float>(),
                            P->bAlo.as<float>());
}

// allocate the reduced matrix and factor storage for the chosen path
static void prepare_path(Problem *P) {
    const Dims &D = P->D;
    int path = (int)P->opt.path;
    if (path == MDSIP_PATH_AUTO) path = P->p2_ok ? MDSIP_PATH_P2 : MDSIP_PATH_P1;
    MDSIP_REQUIRE(path != MDSIP_PATH_P2 || P->p2_ok, MDSIP_ERR_PRECONDITION,
                  P->nnz_jsh > 0 ? "path P2 needs J_sh = 0" : "path P2 needs J_sg rows with disjoint column supports");
    const int64_t N = path == MDSIP_PATH_P2 ? D.n_d + D.m_I : D.n_d + D.m;
    MDSIP_REQUIRE(2 * N * (int64_t)sizeof(double) <= 200 * 1024 || ldlt_blocked_available(N), MDSIP_ERR_INVALID_ARG,
                  "reduced matrix too large for the dense factorization");
    if (path == P->path && N == P->N && P->bS.ptr) return;
    P->drop_graphs();   // the captured factorizations point at the old buffers
    P->path = path;
    P->N = N;
    Ctx *ctx = P->ctx;
    dvec(ctx, P->bS, N * N);
    dvec(ctx, P->bL, N * N);
    dvec(ctx, P->bDd, N);
    dvec(ctx, P->bDoff, N);
    P->bperm.get<int32_t>(ctx, std::max<int64_t>(N, 1));
    P->bkind.get<int32_t>(ctx, std::max<int64_t>(N, 1));
    P->binertia.get<int32_t>(ctx, 4);
    P->bldlt_ws.get<char>(ctx, ldlt_scratch_bytes(N));
    P->bsolve_ws.get<char>(ctx, ldlt_solve_scratch_bytes(N));
    P->bsolve_err.get<int>(ctx, 4);
    MDSIP_CUDA(cudaMemsetAsync(P->bsolve_err.ptr, 0, sizeof(int), ctx->stream));
    dvec(ctx, P->brhs, std::max<int64_t>(N, 1) * 2);
    const size_t sw = path == MDSIP_PATH_P2 ? syrk_fp64_scratch_bytes(D.m_E, D.n_d, ctx->num_sms) : 0;
    if (sw) P->bsyrk_ws.get<char>(ctx, sw);
    else P->bsyrk_ws.reset();
    if (path == MDSIP_PATH_P2) {
        const int64_t nm = D.n + D.m;
        dvec(ctx, P->bref_b, nm);
        dvec(ctx, P->bref_u, nm);
        dvec(ctx, P->bref_r, nm);
        dvec(ctx, P->bref_d, nm);
        dvec(ctx, P->btmp_nd2, D.n_d + D.m_I);
        dvec(ctx, P->bAu_run, D.m_E);
        dvec(ctx, P->bcpre, D.m_E);
        dvec(ctx, P->bcw, D.m_E);    // m_E float2
        dvec(ctx, P->bwf, D.m_E);    // m_E floats (room for m_E doubles)
        dvec(ctx, P->bATv, D.n_d);
        dvec(ctx, P->bAsd, D.m_E);
    }
}

// Tensor-core condensation: FP32 transposed copy of A (once; A is constant
// for the model family) and the per-call workspace.
static void prepare_tc(Problem *P) {
    const int prec = (int)P->opt.precision;
    P->V.Ahi = P->V.Alo = nullptr;
    P->V.split = nullptr;
    if (prec == MDSIP_PREC_FP64 || P->path != MDSIP_PATH_P2) return;
    Ctx *ctx = P->ctx;
    const Dims &D = P->D;
    if (!P->df_ready && D.m_E > 0 && D.n_d > 0) {   // A as an FP32 pair (once: A follows the Jacobian)
        P->bAhi.get<float>(ctx, (size_t)D.m_E * D.lda);
        P->bAlo.get<float>(ctx, (size_t)D.m_E * D.lda);
        P->bsplit.get<float2>(ctx, (size_t)(D.m_E + D.n_d));
        launch_split_matrix(ctx->stream, P->Mv.A, D.m_E, D.n_d, D.lda, P->bAhi.as<float>(), P->bAlo.as<float>());
        P->df_ready = true;
    }
    if (P->df_ready) {
        P->V.Ahi = P->bAhi.as<float>();
        P->V.Alo = P->bAlo.as<float>();
        P->V.split = P->bsplit.as<float2>();
    }
    const TcPlan pl = syrk_tc_plan(D.m_E, D.n_d, ctx->num_sms, prec);
    if (!P->bAfT.ptr) P->bAfT.get<float>(ctx, (size_t)std::max<int64_t>(D.n_d, 1) * pl.ldt);
    if (!P->bvf.ptr) P->bvf.get<float>(ctx, (size_t)pl.ldt);
    if (P->tc_prec != prec) {
        P->btc_ws.get<char>(ctx, syrk_tc_workspace_bytes(pl, D.n_d, prec));
        P->btc_err.get<int>(ctx, 4);
        P->tc_prec = prec;
    }
}

// ---------------------------------------------------------------------------
// One factorization attempt with shifts (dw, dc): condensation, LDL^T and
// the inertia of the 4x4 matrix by Haynsworth additivity (Section 2.3).
// ---------------------------------------------------------------------------
struct Inertia {
    int64_t pos = 0, neg = 0, zero = 0;
    bool operator==(const Inertia &o) const { return pos == o.pos && neg == o.neg && zero == o.zero; }
};

// ---------------------------------------------------------------------------
// Autotuning: tile shapes chosen by timing the candidates once per device and
// shape (CUDA events on the problem's stream, one warm and one timed run each)
// and remembered for the process.
// ---------------------------------------------------------------------------
enum TuneKind { TUNE_LDLT_PANEL = 0, TUNE_SYRK_TILE = 1 };
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int64_t, int64_t>, int> g_tune;

static bool tune_get(int kind, int64_t a, int64_t b, int *v) {
    int dev = 0;
    MDSIP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, kind, a, b));
    if (it == g_tune.end()) return false;
    *v = it->second;
    return true;
}

static void tune_put(int kind, int64_t a, int64_t b, int v) {
    int dev = 0;
    MDSIP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(dev, kind, a, b)] = v;
}

// best of `cands` by the CUDA-event time of run(c) (after one warm run)
template <class F>
static int tune_pick(Problem *P, const std::vector<int> &cands, F &&run) {
    cudaStream_t st = P->ctx->stream;
    int best = cands.empty() ? 0 : cands[0];
    float best_ms = INFINITY;
    for (int c : cands) {
        run(c);
        MDSIP_CUDA(cudaEventRecord(P->ev[11], st));
        run(c);
        MDSIP_CUDA(cudaEventRecord(P->ev[7], st));
        MDSIP_CUDA(cudaEventSynchronize(P->ev[7]));
        float ms = 0.0f;
        MDSIP_CUDA(cudaEventElapsedTime(&ms, P->ev[11], P->ev[7]));
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    return best;
}

// Tile edge of the FP64 condensation product for this problem's A (tuned when
// the product is small enough for the extra runs not to matter: the many-
// instance setting, where the analytic choice is least reliable).
static int tuned_syrk_tile(Problem *P) {
    const Dims &D = P->D;
    if (!P->opt.autotune || (double)D.m_E * D.n_d * D.n_d > 4e10) return 0;
    int v = 0;
    if (tune_get(TUNE_SYRK_TILE, D.m_E, D.n_d, &v)) return v;
    double *C = P->btune.get<double>(P->ctx, (size_t)std::max<int64_t>(D.n_d * D.n_d, 1));
    v = tune_pick(P, {64, 80}, [&](int bm) {
        launch_syrk_fp64_ws(P->ctx->stream, P->ctx->num_sms, P->Mv.A, D.m_E, D.n_d, D.lda, P->bw.as<double>(),
                            0.0, C, D.n_d, P->bsyrk_ws.as<double>(), bm);
    });
    P->btune.reset();
    tune_put(TUNE_SYRK_TILE, D.m_E, D.n_d, v);
    return v;
}

// Run the factorization phase `enqueue` on the problem's stream: eagerly on
// its first use for an order, captured into a CUDA graph on the second (only
// with the blocked factorization's panel loop, whose launches need no host
// state; the persistent factorization is a few launches and reads back where
// it stopped, so it runs eagerly), and as one graph launch afterwards.  A
// capture that fails falls back to eager launches for good.
template <class F>
static void run_factor_phase(Problem *P, int slot, F &&enqueue) {
    Problem::FactorGraph &g = P->fgraph[slot];
    cudaStream_t st = P->ctx->stream;
    if (g.N != P->N || g.zero_tol != P->opt.zero_tol) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = Problem::FactorGraph{};
        g.N = P->N;
        g.zero_tol = P->opt.zero_tol;
    }
    if (g.exec) {
        MDSIP_CUDA(cudaGraphLaunch(g.exec, st));
        count_launches(g.launches);
        return;
    }
    ++g.uses;
    // the persistent factorization reads back where it stopped: nothing to capture
    if (!P->opt.graphs || g.disabled || g.uses < 2 || !ldlt_blocked_available(P->N) ||
        ldlt_persistent_path(P->N, (int)P->opt.ldlt_spec)) {
        enqueue();
        return;
    }
    const long long before = t_launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {   // e.g. legacy stream
        cudaGetLastError();
        g.disabled = true;
        enqueue();
        return;
    }
    try {
        enqueue();
    } catch (...) {
        cudaStreamEndCapture(st, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        g.disabled = true;
        throw;
    }
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        g.exec = exec;
        g.launches = t_launches - before;
        g_launches.fetch_sub(g.launches, std::memory_order_relaxed);   // counted at replay
    } else {
        g.disabled = true;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (g.exec) {
        MDSIP_CUDA(cudaGraphLaunch(g.exec, st));
        count_launches(g.launches);
    } else {
        enqueue();
    }
}

// Panel width of the blocked LDL^T for this order and update precision, tuned
// on a copy of the current S (the trial factorizations overwrite S, L, D).
static int tuned_ldlt_width(Problem *P, bool fp32) {
    const int64_t N = P->N;
    if (!P->opt.autotune || !ldlt_blocked_available(N)) return 0;
    int v = 0;
    if (tune_get(TUNE_LDLT_PANEL, N, fp32 ? 1 : 0, &v)) return v;
    const std::vector<int> cands = ldlt_blocked_widths(N, fp32);
    if (cands.size() < 2) {
        v = cands.empty() ? 0 : cands[0];
    } else {
        cudaStream_t st = P->ctx->stream;
        double *S = P->bS.as<double>(), *Ssave = P->btune.get<double>(P->ctx, (size_t)N * N);
        double *sc = P->scal();
        MDSIP_CUDA(cudaMemcpyAsync(Ssave, S, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        v = tune_pick(P, cands, [&](int nb) {
            MDSIP_CUDA(cudaMemcpyAsync(S, Ssave, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
            launch_maxabs_lower(st, N, S, N, P->V.partial, sc + SC_MAXABS);
            LdltOut o{P->bL.as<double>(), P->bDd.as<double>(), P->bDoff.as<double>(), P->bperm.as<int32_t>(),
                      P->bkind.as<int32_t>(), P->binertia.as<int32_t>()};
            launch_ldlt(st, P->ctx->num_sms, N, S, N, sc + SC_MAXABS, P->opt.zero_tol, o, P->bldlt_ws.ptr,
                        P->berr.as<int>(), fp32, nb, (int)P->opt.ldlt_spec);
        });
        MDSIP_CUDA(cudaMemcpyAsync(S, Ssave, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        MDSIP_CUDA(cudaStreamSynchronize(st));
        P->btune.reset();
    }
    tune_put(TUNE_LDLT_PANEL, N, fp32 ? 1 : 0, v);
    return v;
}

static Inertia factor_attempt(Problem *P, double dw, double dc, bool force_fp64 = false) {
    const Dims &D = P->D;
    cudaStream_t st = P->ctx->stream;
    double *sc = P->scal();
    const bool p2 = P->path == MDSIP_PATH_P2;
    double *sig_x = P->bsig_x.as<double>(), *q = P->bq.as<double>(), *sig_d = P->bsig_d.as<double>(),
           *w = P->bw.as<double>(), *S = P->bS.as<double>();
    MDSIP_CUDA(cudaEventRecord(P->ev[0], st));
    P->V.newton_diag(P->I, P->bHss.as<double>(), dw, dc, p2, sig_x, q, sig_d, w, sc + SC_DIAG);
    if (p2) {
        launch_assemble_S(st, D, P->bHdd.as<double>(), sig_x + D.n_s, P->bJdh.as<double>(), sig_d, dw, dc,
                          S);
        MDSIP_CUDA(cudaEventRecord(P->ev[8], st));
        if (P->opt.precision != MDSIP_PREC_FP64 && !force_fp64) {
            if (!P->aft_ready) {  // FP32 transposed copy of the current A
                const TcPlan pl = syrk_tc_plan(D.m_E, D.n_d, P->ctx->num_sms, (int)P->opt.precision);
                launch_transpose_f32(st, P->Mv.A, D.m_E, D.n_d, D.lda, P->bAfT.as<float>(), pl.ldt);
                P->aft_ready = true;
            }
            MDSIP_CUDA(cudaMemsetAsync(P->btc_err.ptr, 0, sizeof(int), st));
            launch_syrk_tc(st, P->ctx->num_sms, (int)P->opt.precision, P->bAfT.as<float>(), D.m_E, D.n_d, w,
                           1.0, S, P->N, P->btc_ws.ptr, P->btc_err.as<int>());
        } else {
            const int bm = tuned_syrk_tile(P);
            MDSIP_CUDA(cudaEventRecord(P->ev[8], st));   // the tile choice's trial runs are not the product
            launch_syrk_fp64_ws(st, P->ctx->num_sms, P->Mv.A, D.m_E, D.n_d, D.lda, w, 1.0, S, P->N,
                                P->bsyrk_ws.as<double>(), bm);
        }
        MDSIP_CUDA(cudaEventRecord(P->ev[9], st));
    } else {
        launch_assemble_M(st, D, P->Mv, P->bHdd.as<double>(), sig_x + D.n_s, P->bJdh.as<double>(), sig_d,
                          q, dw, dc, S);
    }
    MDSIP_CUDA(cudaEventRecord(P->ev[1], st));
    MDSIP_CUDA(cudaEventRecord(P->ev[10], st));
    const bool tc_factor = p2 && P->opt.precision != MDSIP_PREC_FP64 && !force_fp64;
    // the refined tensor-core path solves with FP32 tiles of L; the FP64 path with FP64 tiles
    P->solve_fp32 = tc_factor;
    const int nb = tuned_ldlt_width(P, tc_factor);
    MDSIP_CUDA(cudaEventRecord(P->ev[10], st));   // the width's trial runs are not the factorization
    auto factor_phase = [&] {
        launch_maxabs_lower(st, P->N, S, P->N, P->V.partial, sc + SC_MAXABS);
        MDSIP_CUDA(cudaMemsetAsync(P->berr.ptr, 0, sizeof(int), st));
        LdltOut o{P->bL.as<double>(), P->bDd.as<double>(), P->bDoff.as<double>(), P->bperm.as<int32_t>(),
                  P->bkind.as<int32_t>(), P->binertia.as<int32_t>()};
        launch_ldlt(st, P->ctx->num_sms, P->N, S, P->N, sc + SC_MAXABS, P->opt.zero_tol, o, P->bldlt_ws.ptr,
                    P->berr.as<int>(), tc_factor, nb, (int)P->opt.ldlt_spec);
        launch_ldlt_solve_prepare(st, P->N, P->bL.as<double>(), P->bsolve_ws.ptr, P->solve_fp32);
    };
    run_factor_phase(P, tc_factor ? 1 : 0, factor_phase);
    MDSIP_CUDA(cudaEventRecord(P->ev[2], st));
    MDSIP_CUDA(cudaMemcpyAsync(P->hint, P->binertia.ptr, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MDSIP_CUDA(cudaMemcpyAsync(P->hint + 4, P->berr.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    const bool tc = p2 && P->opt.precision != MDSIP_PREC_FP64 && !force_fp64;
    if (tc) MDSIP_CUDA(cudaMemcpyAsync(P->hint + 5, P->btc_err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    P->sync_scalars();
    MDSIP_REQUIRE(P->hint[4] == 0, MDSIP_ERR_DEVICE, "LDL^T: a bounded device wait expired");
    MDSIP_REQUIRE(!tc || P->hint[5] == 0, MDSIP_ERR_DEVICE, "tensor-core product: a bounded device wait expired");
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, P->ev[0], P->ev[1]);
    cudaEventElapsedTime(&b, P->ev[1], P->ev[2]);
    P->stats.t_condense_ms += a;
    P->stats.t_factor_ms += b;
    P->stats.n_factorizations++;
    if (p2) {
        cudaEventElapsedTime(&c, P->ev[8], P->ev[9]);
        P->stats.t_syrk_ms += c;
        P->stats.n_syrk++;
    }
    cudaEventElapsedTime(&c, P->ev[10], P->ev[2]);
    P->stats.t_ldlt_ms += c;
    P->stats.n_ldlt++;
    const double *h = P->hscal;
    Inertia in;
    in.pos = (int64_t)h[SC_DIAG + 0] + P->hint[0];
    in.neg = (int64_t)h[SC_DIAG + 1] + P->hint[1];
    in.zero = (int64_t)h[SC_DIAG + 2] + P->hint[2];
    if (p2) {
        in.pos += (int64_t)h[SC_DIAG + 3];
        in.neg += (int64_t)h[SC_DIAG + 4];
        in.zero += (int64_t)h[SC_DIAG + 5];
    }
    return in;
}

// Solve with the current factorization and back-substitute to the full
// direction (Eq. (linsys4x4) unknowns plus dd and the bound multipliers).
static void solve_direction(Problem *P, double mu, double dw) {
    const Dims &D = P->D;
    cudaStream_t st = P->ctx->stream;
    const bool p2 = P->path == MDSIP_PATH_P2;
    double *gl = P->bgl.as<double>(), *q = P->bq.as<double>(), *w = P->bw.as<double>(),
           *sig_d = P->bsig_d.as<double>(), *bt_g = P->bbt_g.as<double>(), *u = P->bu.as<double>(),
           *ATu = P->bATu.as<double>(), *rhs = P->brhs.as<double>(), *Adx = P->bAdx.as<double>();
    MDSIP_CUDA(cudaEventRecord(P->ev[3], st));
    P->V.rhs_y(P->I, gl, P->cg, q, p2 ? w : nullptr, mu, bt_g, p2 ? u : nullptr);
    if (p2) launch_gemv_t(st, P->Mv.A, D.m_E, D.n_d, D.lda, u, P->V.colpart, ATu);
    P->V.rhs_reduced(P->I, gl, P->ch, sig_d, ATu, bt_g, q, mu, dw, !p2, rhs);
    launch_ldlt_solve_coop(st, P->ctx->num_sms, P->N, P->bDd.as<double>(), P->bDoff.as<double>(),
                           P->bperm.as<int32_t>(), 1, rhs, P->N, P->bsolve_ws.ptr, P->bsolve_err.as<int>(),
                           P->solve_fp32);
    if (p2) {
        launch_gemv_rows(st, P->Mv.A, D.m_E, D.n_d, D.lda, rhs, Adx);
        P->V.dyg_p2(Adx, bt_g, w, P->Dir.dyg);
        P->V.backsub(P->I, P->Dir, gl, q, sig_d, rhs, rhs + D.n_d, mu, dw);
    } else {
        P->V.copy(rhs + D.n_d, P->Dir.dyg, D.m_E);
        P->V.backsub(P->I, P->Dir, gl, q, sig_d, rhs, rhs + D.n_d + D.m_E, mu, dw);
    }
    MDSIP_CUDA(cudaEventRecord(P->ev[4], st));
}

struct RefineResult {
    bool ok;
    int sweeps;
    double res;              // ||b - K u||inf / (||b||inf + ||K u||inf)
    bool fell_back = false;  // re-factored with the FP64 product after refinement stalled
};

// Direction through the FP64 residual of the unreduced system, refined with
// the current factor (path P2).  ok = false when the residual stays above
// refine_fallback_tol (the caller then re-factors with the FP64 product).
static RefineResult solve_direction_refined(Problem *P, double mu, double dw, double dc, int max_sweeps) {
    const Dims &D = P->D;
    cudaStream_t st = P->ctx->stream;
    Refiner R{};
    R.D = D;
    R.M = P->Mv;
    R.st = st;
    R.N = P->N;
    R.L = P->bL.as<double>();
    R.Dd = P->bDd.as<double>();
    R.Doff = P->bDoff.as<double>();
    R.perm = P->bperm.as<int32_t>();
    R.num_sms = P->ctx->num_sms;
    R.solve_ws = P->bsolve_ws.ptr;
    R.solve_err = P->bsolve_err.as<int>();
    R.solve_fp32 = P->solve_fp32;
    R.AfT = P->aft_ready ? P->bAfT.as<float>() : nullptr;
    R.ldt = syrk_tc_ld(D.m_E);
    R.vf = P->bvf.as<float>();
    R.q = P->bq.as<double>();
    R.w = P->bw.as<double>();
    R.sig_xd = P->bsig_x.as<double>() + D.n_s;
    R.sig_d = P->bsig_d.as<double>();
    R.Jdh = P->bJdh.as<double>();
    R.Hdd = P->bHdd.as<double>();
    R.bt_g = P->bbt_g.as<double>();
    R.tmp_m = P->bAdx.as<double>();
    R.tmp_nd = P->bATu.as<double>();
    R.tmp_nd2 = P->btmp_nd2.as<double>();
    R.rhsS = P->brhs.as<double>();
    R.colpart = P->V.colpart;
    R.partial = P->V.partial;
    R.Au_run = P->bAu_run.as<double>();
    R.Ahi = P->V.Ahi;
    R.Alo = P->V.Alo;
    R.split = P->V.split;
    R.cpre = P->bcpre.as<double>();
    R.cw = P->bcw.as<float2>();
    R.wf = P->bwf.as<float>();
    R.ATv = P->bATv.as<double>();
    R.Asd = P->bAsd.as<double>();
    double *b = P->bref_b.as<double>(), *u = P->bref_u.as<double>(), *r = P->bref_r.as<double>(),
           *d = P->bref_d.as<double>();
    const double *h = P->hscal;
    MDSIP_CUDA(cudaEventRecord(P->ev[3], st));
    R.rhs(P->I, P->bgl.as<double>(), P->cg, P->ch, R.sig_d, mu, dw, b);
    R.approx_solve(b, u);
    R.track_Au(true);
    RefineResult out{false, 0, INFINITY};
    double rprev = INFINITY;
    while (true) {
        R.residual(b, u, dw, dc, r, P->scal() + SC_REF);
        P->sync_scalars();
        const double rinf = h[SC_REF], scale = h[SC_REF + 1] + h[SC_REF + 2];
        out.res = scale > 0 ? rinf / scale : 0.0;
        if (!std::isfinite(out.res)) break;
        if (rinf <= P->opt.refine_tol * scale) break;
        if (out.sweeps >= max_sweeps || (out.sweeps > 0 && rinf > 0.5 * rprev)) break;
        R.approx_solve(r, d);
        R.track_Au(false);
        R.axpy(D.n + D.m, d, u);
        out.sweeps++;
        rprev = rinf;
    }
    out.ok = std::isfinite(out.res) && out.res <= P->opt.refine_fallback_tol;
    // the loop ends right after a residual, whose double-float pass left A u_d in
    // tmp_m and A^T u_g in tmp_nd for the final u: the direction's products
    P->dir_prod = R.Ahi != nullptr;
    R.direction(P->I, P->Dir, u, mu, dw);
    MDSIP_CUDA(cudaEventRecord(P->ev[4], st));
    P->stats.n_refine += out.sweeps;
    return out;
}

static int refine_sweeps(const Problem *P) {
    if (P->opt.refine_max >= 0) return (int)P->opt.refine_max;
    return P->opt.precision == MDSIP_PREC_FP64 ? 0 : 30;
}

static bool use_refined(const Problem *P) {
    return P->path == MDSIP_PATH_P2 && (P->opt.precision != MDSIP_PREC_FP64 || refine_sweeps(P) > 0);
}

// Direction with the current factor; with a tensor-core product that does
// not refine to tolerance, re-factor with the FP64 product and solve again.
static void check_solve_flag(Problem *P) {
    MDSIP_CUDA(cudaMemcpyAsync(P->hint + 6, P->bsolve_err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               P->ctx->stream));
    MDSIP_CUDA(cudaStreamSynchronize(P->ctx->stream));
    MDSIP_REQUIRE(P->hint[6] == 0, MDSIP_ERR_DEVICE,
                  "LDL^T solve or residual pass: a bounded device wait expired");
}

static RefineResult direction_step_(Problem *P, double mu, double dw, double dc, bool fp64, Inertia *used);

// `used` holds the inertia of the current factor on entry; after an FP64
// re-factorization it receives that factor's inertia, which the caller checks
// against the target before taking the direction.
static RefineResult direction_step(Problem *P, double mu, double dw, double dc, bool fp64, Inertia *used) {
    const RefineResult r = direction_step_(P, mu, dw, dc, fp64, used);
    check_solve_flag(P);
    return r;
}

static RefineResult direction_step_(Problem *P, double mu, double dw, double dc, bool fp64, Inertia *used) {
    if (!use_refined(P)) {
        solve_direction(P, mu, dw);
        return RefineResult{true, 0, 0.0};
    }
    RefineResult rr = solve_direction_refined(P, mu, dw, dc, refine_sweeps(P));
    if (!rr.ok && P->opt.precision != MDSIP_PREC_FP64 && !fp64) {
        *used = factor_attempt(P, dw, dc, true);
        P->stats.n_fp64_fallback++;
        RefineResult r2 = solve_direction_refined(P, mu, dw, dc, std::max(refine_sweeps(P), 3));
        r2.sweeps += rr.sweeps;
        r2.ok = false;  // marks the fallback in the log
        r2.fell_back = true;
        return r2;
    }
    return rr;
}

// model derivatives and the Lagrangian gradient at the current point
// (A^T y_g taken from bATy when it is carried for this iterate)
static void eval_derivatives(Problem *P) {
    model_jac_hess(P, P->I.x, P->I.yg, P->I.yh);
    if (P->lin_aty) {
        P->V.lagrangian_grad_aty(P->I, P->grad, P->bJdh.as<double>(), P->bATy.as<double>(), P->bgl.as<double>());
        return;
    }
    P->V.lagrangian_grad(P->I, P->grad, P->bJdh.as<double>(), P->bATy.as<double>(), P->bgl.as<double>());
}

// Data-given problems on the mixed path: the constraints are linear in x_d and
// the refinement's last residual pass forms A dx_d and A^T dy_g of the
// direction anyway, so the line search's trial constraints (A x_t = A x +
// alpha A dx) and the next iterate's A^T y_g need no pass over A.
static bool carry_products(const Problem *P) { return P->model_kind == 0 && P->V.Ahi != nullptr && P->D.m_E > 0; }

struct Errs {
    double E, dual, primal, comp;
};

static Errs kkt_error(const Problem *P, double mu) {
    const double *e = P->hscal + SC_E;
    const Options &o = P->opt;
    const double nm = (double)(P->D.m + P->n_bounds);
    const double s_d = nm > 0 ? std::max(o.s_max, (e[4] + e[5]) / nm) / o.s_max : 1.0;
    const double s_c = P->n_bounds > 0 ? std::max(o.s_max, e[5] / (double)P->n_bounds) / o.s_max : 1.0;
    const double comp = P->n_bounds > 0 ? std::max(std::fabs(e[2] - mu), std::fabs(e[3] - mu)) : 0.0;
    Errs r;
    r.dual = e[0];
    r.primal = e[1];
    r.comp = comp;
    r.E = std::max(std::max(r.dual / s_d, r.primal), comp / s_c);
    return r;
}

static void swap_trial(Problem *P) {
    std::swap(P->I.x, P->xt);
    std::swap(P->I.d, P->dt);
    std::swap(P->grad, P->grad_t);
    std::swap(P->cg, P->cg_t);
    std::swap(P->ch, P->ch_t);
}

// Relative distance ||D_mixed - D_fp64||_2 / ||D_fp64||_2 between the
// direction just computed with the low-precision factor and the FP64 direction
// (FP64 product and factorization, same iterate and shifts).  P->Dir keeps the
// low-precision direction: the solve goes on exactly as without the check.
static double fp64_direction_error(Problem *P, double mu, double dw, double dc) {
    const Dims &D = P->D;
    if (!P->Dchk.dx) {
        DirView &C = P->Dchk;
        C.dx = dvec(P->ctx, P->bcx, D.n);
        C.dd = dvec(P->ctx, P->bcd, D.m_I);
        C.dyg = dvec(P->ctx, P->bcyg, D.m_E);
        C.dyh = dvec(P->ctx, P->bcyh, D.m_I);
        C.dzl = dvec(P->ctx, P->bczl, D.n);
        C.dzu = dvec(P->ctx, P->bczu, D.n);
        C.dvl = dvec(P->ctx, P->bcvl, D.m_I);
        C.dvu = dvec(P->ctx, P->bcvu, D.m_I);
    }
    P->V.copy_dir(P->Dir, P->Dchk);
    Inertia in64 = factor_attempt(P, dw, dc, true);
    direction_step(P, mu, dw, dc, true, &in64);
    P->V.dir_diff(P->Dchk, P->Dir, P->scal() + SC_DCHK);
    P->V.copy_dir(P->Dchk, P->Dir);
    P->sync_scalars();
    const double *h = P->hscal;
    return h[SC_DCHK + 1] > 0 ? std::sqrt(h[SC_DCHK] / h[SC_DCHK + 1]) : 0.0;
}

static mdsip_status run_ipm(Problem *P) {
    MDSIP_REQUIRE(P->bounds_set, MDSIP_ERR_INVALID_ARG, "bounds not set (mdsip_set_bounds)");
    prepare_path(P);
    prepare_tc(P);
    const Dims &D = P->D;
    const Options &o = P->opt;
    cudaStream_t st = P->ctx->stream;
    double *sc = P->scal();
    const double *h = P->hscal;
    const auto t_start = std::chrono::steady_clock::now();
    P->stats = mdsip_stats{};
    P->stats.path = P->path;
    P->stats.precision = (P->path == MDSIP_PATH_P2) ? (int32_t)P->opt.precision : MDSIP_PREC_FP64;
    P->log.clear();
    MDSIP_CUDA(cudaEventRecord(P->ev[6], st));

    if (!P->has_start) {
        P->V.init_x(P->bx0.as<double>(), o.kappa_1, o.kappa_2, P->I);
        model_cons(P, P->I.x, P->I.d, P->cg, P->ch, sc + SC_THETA);  // ch = h(x0) - 0
        P->V.init_d(P->ch, o.kappa_1, o.kappa_2, P->I);
    }
    double mu = (P->has_start && P->start_mu0 > 0) ? P->start_mu0 : o.mu0;
    double tau = std::max(o.tau_min, 1.0 - mu);
    model_f(P, P->I.x, P->grad, sc + SC_F);
    model_cons(P, P->I.x, P->I.d, P->cg, P->ch, sc + SC_THETA);
    P->lin_ax = P->lin_aty = P->dir_prod = false;
    if (carry_products(P)) {
        P->ax_cur = P->bAx_a.get<double>(P->ctx, D.m_E);
        P->ax_t = P->bAx_b.get<double>(P->ctx, D.m_E);
        P->bdAx.get<double>(P->ctx, D.m_E);
        P->bdATy.get<double>(P->ctx, std::max<int64_t>(D.n_d, 1));
        P->V.copy(P->V.rowtmp, P->ax_cur, D.m_E);   // A x_d of the start, from the evaluation above
        P->lin_ax = true;
    }
    P->sync_scalars();
    double f = h[SC_F], th = h[SC_THETA];
    const double theta_max = o.theta_max_fact * std::max(1.0, th);
    const double theta_min = o.theta_min_fact * std::max(1.0, th);
    std::vector<std::pair<double, double>> filt;
    double dw_last = 0.0;
    const Inertia target{D.n, D.m, 0};
    int64_t k = 0;
    mdsip_status status = MDSIP_MAX_ITER;

    while (true) {
        eval_derivatives(P);
        if (carry_products(P)) P->lin_aty = true;   // bATy now holds A^T y_g of this iterate
        P->V.errors(P->I, P->bgl.as<double>(), P->cg, P->ch, sc + SC_E);
        P->sync_scalars();
        Errs e0 = kkt_error(P, 0.0);
        mdsip_iter_rec rec{};
        rec.dir_err_fp64 = -1.0;
        rec.iter = (int32_t)k;
        rec.mu = mu;
        rec.f = f;
        rec.theta = th;
        rec.E0 = e0.E;
        rec.inf_pr = e0.primal;
        rec.inf_du = e0.dual;
        if (!std::isfinite(e0.E)) { status = MDSIP_ERR_NONFINITE; P->log.push_back(rec); break; }
        if (e0.E <= o.tol) { status = MDSIP_OK; P->log.push_back(rec); break; }
        if (k >= o.max_iter) { status = MDSIP_MAX_ITER; P->log.push_back(rec); break; }
        if (o.time_limit_s > 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (el > o.time_limit_s) { status = MDSIP_TIMEOUT; P->log.push_back(rec); break; }
        }
        // A.3 barrier update
        while (true) {
            const double Emu = kkt_error(P, mu).E;
            if (Emu <= o.kappa_eps * mu) {
                const double mu_new = std::max(o.tol / 10.0, std::min(o.kappa_mu * mu, std::pow(mu, o.theta_mu)));
                if (mu_new == mu) break;
                mu = mu_new;
                tau = std::max(o.tau_min, 1.0 - mu);
                filt.clear();
                if (k == 0) continue;
            }
            break;
        }
        rec.mu = mu;
        const double logsum = h[SC_E + 6];
        // A.4 direction with inertia correction
        double dw = 0.0, dc = 0.0;
        auto record = [&](const Inertia &in) {
            if (rec.n_ic < MDSIP_MAX_IC) {
                rec.ic_dw[rec.n_ic] = dw;
                rec.ic_dc[rec.n_ic] = dc;
                rec.ic_inertia[rec.n_ic][0] = (int32_t)in.pos;
                rec.ic_inertia[rec.n_ic][1] = (int32_t)in.neg;
                rec.ic_inertia[rec.n_ic][2] = (int32_t)in.zero;
            }
            rec.n_ic++;
        };
        // A low-precision factor whose refined direction stalls is replaced by the
        // FP64 factor with the same shifts; if that one misses the target inertia,
        // Algorithm IC runs again for this iteration on FP64 factors alone.
        bool ic_failed = false, fp64 = false;
        const double dw_last0 = dw_last;
        Inertia used{};
        RefineResult rr{};
        P->dir_prod = false;
        while (true) {
            dw = 0.0;
            dc = 0.0;
            Inertia in = factor_attempt(P, dw, dc, fp64);
            record(in);
            if (!(in == target)) {
                if (in.zero > 0) dc = o.dc_bar * std::pow(mu, o.kappa_c);
                dw = dw_last == 0.0 ? o.dw0 : std::max(o.dw_min, o.kw_minus * dw_last);
                while (true) {
                    in = factor_attempt(P, dw, dc, fp64);
                    record(in);
                    if (in == target) { dw_last = dw; break; }
                    dw = dw_last == 0.0 ? o.kw_plus_bar * dw : o.kw_plus * dw;
                    if (dw > o.dw_max) { ic_failed = true; break; }
                }
            }
            if (ic_failed) break;
            used = in;
            rr = direction_step(P, mu, dw, dc, fp64, &used);
            if (rr.fell_back && !(used == target)) {
                record(used);           // the FP64 factor that missed the target
                fp64 = true;
                dw_last = dw_last0;     // as an FP64 run would start this iteration
                continue;
            }
            break;
        }
        if (rec.n_ic > MDSIP_MAX_IC) rec.n_ic = MDSIP_MAX_IC;
        if (ic_failed) { status = MDSIP_ERR_INERTIA; P->log.push_back(rec); break; }
        rec.factor_inertia[0] = (int32_t)used.pos;
        rec.factor_inertia[1] = (int32_t)used.neg;
        rec.factor_inertia[2] = (int32_t)used.zero;
        rec.n_refine = rr.sweeps;
        rec.fp64_fallback = (rr.ok && !fp64) ? 0 : 1;
        rec.refine_res = rr.res;
        // the direction's products with A, kept before anything else uses the
        // refinement's buffers (the FP64 check below computes a direction of its own)
        const bool lin_step = carry_products(P) && P->lin_ax && P->dir_prod;
        if (lin_step) {
            P->V.copy(P->bAdx.as<double>(), P->bdAx.as<double>(), D.m_E);
            P->V.copy(P->bATu.as<double>(), P->bdATy.as<double>(), D.n_d);
        }
        if (o.direction_check && use_refined(P) && P->opt.precision != MDSIP_PREC_FP64 && !fp64 && !rr.fell_back)
            rec.dir_err_fp64 = fp64_direction_error(P, mu, dw, dc);
        // A.5 line search
        P->V.step_scalars(P->I, P->Dir, P->grad, tau, mu, sc + SC_STEP);
        P->sync_scalars();
        {
            float a = 0;
            cudaEventElapsedTime(&a, P->ev[3], P->ev[4]);
            P->stats.t_solve_ms += a;
            P->stats.t_refine_ms += a;
        }
        const double alpha_max = std::min(1.0, h[SC_STEP + 0]);
        const double alpha_z = std::min(1.0, h[SC_STEP + 1]);
        const double gphi = h[SC_STEP + 2];
        const double phi_k = f - mu * logsum;
        const double th_k = th;
        double a_min;
        if (gphi < 0 && th_k <= theta_min)
            a_min = o.gamma_alpha * std::min({o.gamma_theta, o.gamma_phi * th_k / (-gphi),
                                              o.delta * std::pow(th_k, o.s_theta) / std::pow(-gphi, o.s_phi)});
        else if (gphi < 0)
            a_min = o.gamma_alpha * std::min(o.gamma_theta, o.gamma_phi * th_k / (-gphi));
        else
            a_min = o.gamma_alpha * o.gamma_theta;
        double alpha = alpha_max;
        int64_t n_ls = 0;
        bool accepted = false, ftype = false, armijo = false;
        double f_t = 0, th_t = 0;
        MDSIP_CUDA(cudaEventRecord(P->ev[5], st));
        while (true) {
            P->V.trial(P->I, P->Dir, alpha, P->xt, P->dt, sc + SC_TRIAL);
            model_f(P, P->xt, P->grad_t, sc + SC_TF);
            if (lin_step) {   // A x_t = A x + alpha A dx (the same trial point)
                P->V.axpby(D.m_E, P->ax_cur, alpha, P->bdAx.as<double>(), P->ax_t);
                P->V.eval_cons_ax(P->xt, P->ax_t, P->dt, P->cg_t, P->ch_t, sc + SC_TTHETA);
            } else {
                model_cons(P, P->xt, P->dt, P->cg_t, P->ch_t, sc + SC_TTHETA);
            }
            P->sync_scalars();
            f_t = h[SC_TF];
            th_t = h[SC_TTHETA];
            const bool inside = h[SC_TRIAL + 1] == 0.0;
            const double phi_t = inside ? f_t - mu * h[SC_TRIAL] : INFINITY;
            ftype = gphi < 0 && alpha * std::pow(-gphi, o.s_phi) > o.delta * std::pow(th_k, o.s_theta);
            armijo = phi_t <= phi_k + o.eta_phi * alpha * gphi;
            bool ok = false;
            if (inside && std::isfinite(phi_t) && std::isfinite(th_t)) {
                if (th_k <= theta_min && ftype)
                    ok = armijo;
                else
                    ok = th_t <= (1 - o.gamma_theta) * th_k || phi_t <= phi_k - o.gamma_phi * th_k;
                if (ok) {
                    ok = th_t < theta_max;
                    for (auto &fe : filt)
                        if (th_t >= fe.first && phi_t >= fe.second) ok = false;
                }
            }
            P->stats.n_ls_trials++;
            if (ok) { accepted = true; break; }
            n_ls++;
            alpha *= 0.5;
            if (alpha < a_min || n_ls >= o.max_ls) break;
        }
        {
            MDSIP_CUDA(cudaEventRecord(P->ev[7], st));
            MDSIP_CUDA(cudaEventSynchronize(P->ev[7]));
            float a = 0;
            cudaEventElapsedTime(&a, P->ev[5], P->ev[7]);
            P->stats.t_ls_ms += a;
        }
        rec.alpha_max = alpha_max;
        rec.alpha_z = alpha_z;
        rec.n_ls = (int32_t)n_ls;
        rec.gphi = gphi;
        if (!accepted) { status = MDSIP_RESTORATION_NEEDED; P->log.push_back(rec); break; }
        rec.alpha = alpha;
        rec.ftype = (ftype && armijo) ? 1 : 0;
        // A.7 filter augmentation
        if (!(ftype && armijo))
            filt.emplace_back((1 - o.gamma_theta) * th_k, phi_k - o.gamma_phi * th_k);
        // A.6 accept: the trial becomes the iterate
        swap_trial(P);
        P->V.accept(P->I, P->Dir, alpha, alpha_z, mu, o.kappa_sigma);
        if (lin_step) {   // y_g moved by alpha dy_g (k_accept): A^T y_g and A x_d follow
            std::swap(P->ax_cur, P->ax_t);
            P->V.axpby(D.n_d, P->bATy.as<double>(), alpha, P->bdATy.as<double>(), P->bATy.as<double>());
        } else if (carry_products(P)) {   // the accepted trial's constraints were formed from x_t
            P->V.copy(P->V.rowtmp, P->ax_cur, D.m_E);
            P->lin_ax = true;
            P->lin_aty = false;
        }
        f = f_t;
        th = th_t;
        P->log.push_back(rec);
        ++k;
    }
    MDSIP_CUDA(cudaEventRecord(P->ev[7], st));
    MDSIP_CUDA(cudaEventSynchronize(P->ev[7]));
    float tt = 0;
    cudaEventElapsedTime(&tt, P->ev[6], P->ev[7]);
    P->stats.t_total_ms = tt;
    P->stats.status = status;
    P->stats.iters = (int32_t)k;
    P->stats.f = f;
    P->stats.mu = mu;
    if (!P->log.empty()) {
        P->stats.E0 = P->log.back().E0;
        P->stats.inf_pr = P->log.back().inf_pr;
        P->stats.inf_du = P->log.back().inf_du;
    }
    return status;
}

// packed layout offsets
static void packed_offsets(const Dims &D, int64_t off[9]) {
    const int64_t sizes[8] = {D.n, D.m_I, D.m_E, D.m_I, D.n, D.n, D.m_I, D.m_I};
    off[0] = 0;
    for (int i = 0; i < 8; ++i) off[i + 1] = off[i] + sizes[i];
}

static void copy_packed(Problem *P, double *const dst_or_src[8], const double *packed, double *out,
                        int mem, bool to_device) {
    int64_t off[9];
    packed_offsets(P->D, off);
    const bool dev = mem == MDSIP_MEM_DEVICE;
    for (int i = 0; i < 8; ++i) {
        const int64_t cnt = off[i + 1] - off[i];
        if (cnt <= 0) continue;
        if (to_device)
            MDSIP_CUDA(cudaMemcpyAsync(dst_or_src[i], packed + off[i], cnt * sizeof(double),
                                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                       P->ctx->stream));
        else
            MDSIP_CUDA(cudaMemcpyAsync(out + off[i], dst_or_src[i], cnt * sizeof(double),
                                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                       P->ctx->stream));
    }
    MDSIP_CUDA(cudaStreamSynchronize(P->ctx->stream));
}

static void iterate_ptrs(Problem *P, double *p[8]) {
    p[0] = P->I.x; p[1] = P->I.d; p[2] = P->I.yg; p[3] = P->I.yh;
    p[4] = P->I.zl; p[5] = P->I.zu; p[6] = P->I.vl; p[7] = P->I.vu;
}

static void debug_direction(Problem *P, const double *packed, double mu, double dw, double dc,
                            int32_t refine, double *dir_out, int32_t inertia_out[3], int mem) {
    prepare_path(P);
    prepare_tc(P);
    double *ptr[8];
    iterate_ptrs(P, ptr);
    copy_packed(P, ptr, packed, nullptr, mem, true);
    double *sc = P->scal();
    MDSIP_REQUIRE(P->bounds_set, MDSIP_ERR_INVALID_ARG, "bounds not set (mdsip_set_bounds)");
    model_f(P, P->I.x, P->grad, sc + SC_F);
    model_cons(P, P->I.x, P->I.d, P->cg, P->ch, sc + SC_THETA);
    P->lin_ax = P->lin_aty = P->dir_prod = false;   // the carried products belong to a solve
    eval_derivatives(P);
    Inertia in = factor_attempt(P, dw, dc);
    const int64_t saved = P->opt.refine_max;
    if (refine > 0) P->opt.refine_max = refine;
    try {
        direction_step(P, mu, dw, dc, false, &in);   // `in`: the factor the direction came from
    } catch (...) {
        P->opt.refine_max = saved;
        throw;
    }
    P->opt.refine_max = saved;
    double *dp[8] = {P->Dir.dx, P->Dir.dd, P->Dir.dyg, P->Dir.dyh,
                     P->Dir.dzl, P->Dir.dzu, P->Dir.dvl, P->Dir.dvu};
    copy_packed(P, dp, nullptr, dir_out, mem, false);
    if (inertia_out) {
        inertia_out[0] = (int32_t)in.pos;
        inertia_out[1] = (int32_t)in.neg;
        inertia_out[2] = (int32_t)in.zero;
    }
}

static bool set_option(Options &o, const std::string &name, double v, bool is_int) {
    struct D { const char *n; double *p; };
    struct I { const char *n; int64_t *p; };
    const D dopts[] = {{"tol", &o.tol}, {"mu0", &o.mu0}, {"kappa_eps", &o.kappa_eps},
                       {"kappa_mu", &o.kappa_mu}, {"theta_mu", &o.theta_mu}, {"tau_min", &o.tau_min},
                       {"s_max", &o.s_max}, {"kappa_1", &o.kappa_1}, {"kappa_2", &o.kappa_2},
                       {"kappa_sigma", &o.kappa_sigma}, {"gamma_theta", &o.gamma_theta},
                       {"gamma_phi", &o.gamma_phi}, {"delta", &o.delta}, {"s_theta", &o.s_theta},
                       {"s_phi", &o.s_phi}, {"eta_phi", &o.eta_phi}, {"gamma_alpha", &o.gamma_alpha},
                       {"theta_max_fact", &o.theta_max_fact}, {"theta_min_fact", &o.theta_min_fact},
                       {"dw0", &o.dw0}, {"dw_min", &o.dw_min}, {"dw_max", &o.dw_max},
                       {"kw_minus", &o.kw_minus}, {"kw_plus", &o.kw_plus}, {"kw_plus_bar", &o.kw_plus_bar},
                       {"dc_bar", &o.dc_bar}, {"kappa_c", &o.kappa_c}, {"zero_tol", &o.zero_tol},
                       {"time_limit_s", &o.time_limit_s}, {"refine_tol", &o.refine_tol},
                       {"refine_fallback_tol", &o.refine_fallback_tol}};
    const I iopts[] = {{"max_iter", &o.max_iter}, {"path", &o.path}, {"max_ls", &o.max_ls},
                       {"refine_max", &o.refine_max}, {"precision", &o.precision}, {"graphs", &o.graphs},
                       {"autotune", &o.autotune}, {"ldlt_spec", &o.ldlt_spec},
                       {"direction_check", &o.direction_check}};
    if (is_int) {
        for (auto &e : iopts)
            if (name == e.n) { *e.p = (int64_t)v; return true; }
    } else {
        for (auto &e : dopts)
            if (name == e.n) { *e.p = v; return true; }
    }
    return false;
}

}  // namespace mdsip

// ===========================================================================
// C ABI
// ===========================================================================
using namespace mdsip;

// Opaque handles are the internal objects themselves.
static inline Ctx *C_(mdsip_ctx *c) { return reinterpret_cast<Ctx *>(c); }
static inline const Ctx *C_(const mdsip_ctx *c) { return reinterpret_cast<const Ctx *>(c); }
static inline Problem *P_(mdsip_problem *p) { return reinterpret_cast<Problem *>(p); }
static inline const Problem *P_(const mdsip_problem *p) { return reinterpret_cast<const Problem *>(p); }


extern "C" {

const char *mdsip_status_str(mdsip_status s) {
    switch (s) {
        case MDSIP_OK: return "OK";
        case MDSIP_ERR_INVALID_ARG: return "INVALID_ARG";
        case MDSIP_ERR_CUDA: return "CUDA";
        case MDSIP_ERR_OOM: return "OOM";
        case MDSIP_ERR_CALLBACK: return "CALLBACK";
        case MDSIP_ERR_NONFINITE: return "NONFINITE";
        case MDSIP_ERR_INERTIA: return "INERTIA";
        case MDSIP_RESTORATION_NEEDED: return "RESTORATION_NEEDED";
        case MDSIP_MAX_ITER: return "MAX_ITER";
        case MDSIP_TIMEOUT: return "TIMEOUT";
        case MDSIP_ERR_PRECONDITION: return "PRECONDITION";
        case MDSIP_ERR_DEVICE: return "DEVICE";
    }
    return "UNKNOWN";
}

mdsip_status mdsip_ctx_create(int device, void *stream, const mdsip_alloc_hooks *hooks,
                              mdsip_ctx **out) {
    if (!out) return MDSIP_ERR_INVALID_ARG;
    *out = nullptr;
    if (hooks && (!hooks->alloc || !hooks->free)) return MDSIP_ERR_INVALID_ARG;
    auto *c = new Ctx();
    mdsip_status s = guarded(c, [&] {
        int count = 0;
        MDSIP_CUDA(cudaGetDeviceCount(&count));
        MDSIP_REQUIRE(device >= 0 && device < count, MDSIP_ERR_INVALID_ARG, "no such device");
        DeviceGuard g(device);
        c->device = device;
        c->stream = static_cast<cudaStream_t>(stream);
        if (hooks) {
            c->hooks = *hooks;
            c->has_hooks = true;
        }
        MDSIP_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    });
    if (s != MDSIP_OK) {
        delete c;
        return s;
    }
    *out = reinterpret_cast<mdsip_ctx *>(c);
    return MDSIP_OK;
}

void mdsip_ctx_destroy(mdsip_ctx *hctx) {
    if (!hctx) return;
    Ctx *ctx = C_(hctx);
    try {
        DeviceGuard g(ctx->device);
        if (ctx->scratch) {
            cudaStreamSynchronize(ctx->stream);
            ctx->release(ctx->scratch, ctx->scratch_bytes);
        }
    } catch (...) {
    }
    delete ctx;
}

const char *mdsip_ctx_last_error(const mdsip_ctx *ctx) { return ctx ? C_(ctx)->last_error.c_str() : ""; }

mdsip_status mdsip_problem_create_synthetic(mdsip_ctx *hctx, const mdsip_synth_data *data, int mem,
                                            mdsip_problem **out) {
    if (!hctx || !out) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    *out = nullptr;
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        Problem *p = create_synthetic(ctx, data, mem);
        *out = reinterpret_cast<mdsip_problem *>(p);
    });
}

mdsip_status mdsip_problem_create(mdsip_ctx *hctx, const mdsip_dims *dims, const int32_t *Jsg_rows,
                                  const int32_t *Jsg_cols, const mdsip_callbacks *cb, void *user, int mem,
                                  mdsip_problem **out) {
    if (!hctx || !out) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    *out = nullptr;
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        Problem *p = create_callbacks(ctx, dims, Jsg_rows, Jsg_cols, cb, user, mem);
        *out = reinterpret_cast<mdsip_problem *>(p);
    });
}

mdsip_status mdsip_set_bounds(mdsip_problem *hp, const double *xl, const double *xu, const double *hl,
                              const double *hu, const double *gE, const double *x0, int mem) {
    if (!hp) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        DeviceGuard g(p->ctx->device);
        MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
        const Dims &D = p->D;
        auto vxl = fetch(xl, D.n, mem), vxu = fetch(xu, D.n, mem);
        auto vhl = fetch(hl, D.m_I, mem), vhu = fetch(hu, D.m_I, mem);
        auto vgE = fetch(gE, D.m_E, mem);
        std::vector<double> vx0 = x0 ? fetch(x0, D.n, mem) : std::vector<double>(D.n, 0.0);
        set_bounds_host(p, vxl, vxu, vhl, vhu, vgE, vx0);
    });
}

void mdsip_problem_destroy(mdsip_problem *hp) {
    if (!hp) return;
    Problem *p = P_(hp);
    try {
        DeviceGuard g(p->ctx->device);
        cudaStreamSynchronize(p->ctx->stream);
        delete p;
    } catch (...) {
    }
}

mdsip_status mdsip_set_option_int(mdsip_problem *hp, const char *name, int64_t value) {
    if (!hp || !name) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        MDSIP_REQUIRE(set_option(p->opt, name, (double)value, true), MDSIP_ERR_INVALID_ARG,
                      std::string("unknown int option ") + name);
        if (std::string(name) == "ldlt_spec") p->drop_graphs();   // captured factorizations use the old choice
        MDSIP_REQUIRE(p->opt.path >= 0 && p->opt.path <= 2, MDSIP_ERR_INVALID_ARG, "bad path");
        MDSIP_REQUIRE(p->opt.precision >= 0 && p->opt.precision <= 2, MDSIP_ERR_INVALID_ARG, "bad precision");
        MDSIP_REQUIRE(p->opt.ldlt_spec >= 0 && p->opt.ldlt_spec <= 2, MDSIP_ERR_INVALID_ARG, "bad ldlt_spec");
    });
}

mdsip_status mdsip_set_option_double(mdsip_problem *hp, const char *name, double value) {
    if (!hp || !name) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        MDSIP_REQUIRE(set_option(p->opt, name, value, false), MDSIP_ERR_INVALID_ARG,
                      std::string("unknown double option ") + name);
    });
}

mdsip_status mdsip_set_option_str(mdsip_problem *hp, const char *name, const char *value) {
    if (!hp || !name || !value) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        struct W { const char *opt, *word; int64_t v; };
        static const W words[] = {
            {"path", "auto", MDSIP_PATH_AUTO},     {"path", "p1", MDSIP_PATH_P1},
            {"path", "p2", MDSIP_PATH_P2},         {"precision", "fp64", MDSIP_PREC_FP64},
            {"precision", "tf32", MDSIP_PREC_TF32}, {"precision", "bf16", MDSIP_PREC_BF16},
            {"graphs", "yes", 1},   {"graphs", "no", 0},   {"autotune", "yes", 1},
            {"autotune", "no", 0},  {"ldlt_spec", "yes", 1}, {"ldlt_spec", "no", 0},
            {"ldlt_spec", "persistent", 2}};
        const std::string n(name), v(value);
        bool known = false;
        for (const W &w : words) {
            if (n != w.opt) continue;
            known = true;
            if (v != w.word) continue;
            set_option(p->opt, n, (double)w.v, true);
            if (n == "ldlt_spec") p->drop_graphs();
            return;
        }
        MDSIP_REQUIRE(false, MDSIP_ERR_INVALID_ARG,
                      known ? "bad value '" + v + "' for option " + n : "unknown string option " + n);
    });
}

int64_t mdsip_packed_size(const mdsip_problem *hp) {
    if (!hp) return 0;
    const Problem *p = P_(hp);
    return 3 * p->D.n + 4 * p->D.m_I + p->D.m_E;
}

mdsip_status mdsip_set_start(mdsip_problem *hp, const double *packed, double mu0, int mem) {
    if (!hp) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    if (!packed) {
        p->has_start = false;
        p->start_mu0 = -1.0;
        return MDSIP_OK;
    }
    return guarded(p->ctx, [&] {
        DeviceGuard g(p->ctx->device);
        double *ptr[8];
        iterate_ptrs(p, ptr);
        copy_packed(p, ptr, packed, nullptr, mem, true);
        p->has_start = true;
        p->start_mu0 = mu0;
    });
}

mdsip_status mdsip_set_start_predicted(mdsip_problem *hp, const float *pred, double push, int mem) {
    if (!hp) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        MDSIP_REQUIRE(pred != nullptr, MDSIP_ERR_INVALID_ARG, "null prediction");
        MDSIP_REQUIRE(push > 0.0 && push < 0.5, MDSIP_ERR_INVALID_ARG, "push must lie in (0, 0.5)");
        MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
        MDSIP_REQUIRE(p->bounds_set, MDSIP_ERR_INVALID_ARG, "bounds not set (mdsip_set_bounds)");
        DeviceGuard g(p->ctx->device);
        const int64_t np = mdsip_packed_size(hp);
        cudaStream_t st = p->ctx->stream;
        DBuf tmp;
        const float *dpred = pred;
        float logmu = 0.0f;
        if (mem == MDSIP_MEM_HOST) {
            float *d = tmp.get<float>(p->ctx, (size_t)np + 1);
            MDSIP_CUDA(cudaMemcpyAsync(d, pred, ((size_t)np + 1) * sizeof(float), cudaMemcpyHostToDevice, st));
            dpred = d;
            logmu = pred[np];
        } else {
            MDSIP_CUDA(cudaMemcpyAsync(&logmu, pred + np, sizeof(float), cudaMemcpyDeviceToHost, st));
            MDSIP_CUDA(cudaStreamSynchronize(st));
        }
        // mu0 from the predicted log mu0, kept inside [tol / 10, option mu0]
        const double lo = std::log(p->opt.tol / 10.0), hi = std::log(p->opt.mu0);
        const double lm = std::isfinite((double)logmu) ? std::min(hi, std::max(lo, (double)logmu)) : hi;
        const double mu0 = std::exp(lm);
        p->V.start_predicted(dpred, push, mu0, p->I);
        MDSIP_CUDA(cudaStreamSynchronize(st));
        p->has_start = true;
        p->start_mu0 = mu0;
    });
}

mdsip_status mdsip_warmstart_target(mdsip_problem *hp, double e0_level, double *out, int mem) {
    if (!hp || !out) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
        MDSIP_REQUIRE(!p->log.empty(), MDSIP_ERR_INVALID_ARG, "no solve recorded");
        DeviceGuard g(p->ctx->device);
        double mu = p->log.back().mu;
        for (const mdsip_iter_rec &r : p->log)
            if (r.E0 <= e0_level) {
                mu = r.mu;
                break;
            }
        double *ptr[8];
        iterate_ptrs(p, ptr);
        copy_packed(p, ptr, nullptr, out, mem, false);
        const int64_t np = mdsip_packed_size(hp);
        const double lm = std::log(mu);
        if (mem == MDSIP_MEM_HOST) {
            out[np] = lm;
        } else {
            MDSIP_CUDA(cudaMemcpyAsync(out + np, &lm, sizeof(double), cudaMemcpyHostToDevice, p->ctx->stream));
            MDSIP_CUDA(cudaStreamSynchronize(p->ctx->stream));
        }
    });
}

mdsip_status mdsip_solve(mdsip_problem *hp) {
    if (!hp) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    mdsip_status result = MDSIP_OK;
    mdsip_status s = guarded(p->ctx, [&] {
        DeviceGuard g(p->ctx->device);
        result = run_ipm(p);
    });
    if (s != MDSIP_OK) {
        p->stats.status = s;
        return s;
    }
    return result;
}

mdsip_status mdsip_batch_solve(mdsip_problem *const *problems, int32_t count, int32_t max_concurrent,
                               int32_t *statuses) {
    if (count < 0 || (count > 0 && (!problems || !statuses))) return MDSIP_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (!problems[i]) return MDSIP_ERR_INVALID_ARG;
    // one group per stream: a stream (and so each context on it, with its
    // last-error text) is used by one thread at a time.  Contexts created on
    // one stream share it; concurrent use from two threads would, among other
    // things, let one thread's launches enter another thread's stream capture.
    std::map<cudaStream_t, std::vector<int32_t>> by_stream;
    for (int32_t i = 0; i < count; ++i) by_stream[P_(problems[i])->ctx->stream].push_back(i);
    std::vector<std::vector<int32_t>> groups;
    for (auto &kv : by_stream) groups.push_back(kv.second);
    const int ngroups = (int)groups.size();
    int nthreads = max_concurrent > 0 ? std::min<int>(max_concurrent, ngroups) : ngroups;
    nthreads = std::max(1, nthreads);
    std::atomic<int> next{0};
    auto worker = [&] {
        while (true) {
            const int g = next.fetch_add(1);
            if (g >= ngroups) break;
            for (int32_t i : groups[g]) statuses[i] = (int32_t)mdsip_solve(problems[i]);
        }
    };
    std::vector<std::thread> pool;
    try {
        for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    } catch (...) {
        // could not start more threads: the remaining groups run on the calling thread
    }
    worker();
    for (auto &t : pool) t.join();
    return MDSIP_OK;
}

mdsip_status mdsip_get_iterate(mdsip_problem *hp, double *packed, int mem) {
    if (!hp || !packed) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        DeviceGuard g(p->ctx->device);
        double *ptr[8];
        iterate_ptrs(p, ptr);
        copy_packed(p, ptr, nullptr, packed, mem, false);
    });
}

mdsip_status mdsip_get_stats(mdsip_problem *hp, mdsip_stats *out) {
    if (!hp || !out) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    *out = p->stats;
    return MDSIP_OK;
}

mdsip_status mdsip_get_log(mdsip_problem *hp, mdsip_iter_rec *buf, int32_t cap, int32_t *n) {
    if (!hp || !n) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    *n = (int32_t)p->log.size();
    if (buf && cap > 0) std::memcpy(buf, p->log.data(), std::min<size_t>(cap, p->log.size()) * sizeof(mdsip_iter_rec));
    return MDSIP_OK;
}

mdsip_status mdsip_debug_direction(mdsip_problem *hp, const double *packed, double mu, double dw,
                                   double dc, int32_t refine, double *dir_out,
                                   int32_t inertia_out[3], int mem) {
    if (!hp || !packed || !dir_out) return MDSIP_ERR_INVALID_ARG;
    Problem *p = P_(hp);
    return guarded(p->ctx, [&] {
        DeviceGuard g(p->ctx->device);
        debug_direction(p, packed, mu, dw, dc, refine, dir_out, inertia_out, mem);
    });
}

int64_t mdsip_launch_count(void) { return (int64_t)g_launches.load(); }

mdsip_status mdsip_probe_fp64_fma(mdsip_ctx *hctx, int32_t blocks, int64_t iters, double *sink) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(blocks > 0 && iters > 0 && sink, MDSIP_ERR_INVALID_ARG, "probe: bad arguments");
        launch_fp64_fma_probe(ctx->stream, blocks, iters, sink);
    });
}

mdsip_status mdsip_syrk_scaled(mdsip_ctx *hctx, int64_t m, int64_t n, const double *A, int64_t lda,
                               const double *w, double beta, double *C, int64_t ldc) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(m >= 0 && n >= 0 && lda >= n && lda % 2 == 0 && ldc >= n, MDSIP_ERR_INVALID_ARG,
                      "syrk: bad sizes");
        MDSIP_REQUIRE(beta == 0.0 || beta == 1.0, MDSIP_ERR_INVALID_ARG, "syrk: beta must be 0 or 1");
        MDSIP_REQUIRE((reinterpret_cast<uintptr_t>(A) & 15) == 0, MDSIP_ERR_INVALID_ARG,
                      "syrk: A must be 16-byte aligned");
        MDSIP_REQUIRE(n == 0 || (A && w && C) || m == 0, MDSIP_ERR_INVALID_ARG, "syrk: null pointer");
        launch_syrk_fp64(ctx, A, m, n, lda, w, beta, C, ldc);
    });
}

mdsip_status mdsip_syrk_scaled_tc(mdsip_ctx *hctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                  const double *w, double beta, double *C, int64_t ldc,
                                  int precision) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(m >= 0 && n >= 0 && lda >= n && ldc >= n, MDSIP_ERR_INVALID_ARG, "syrk_tc: bad sizes");
        MDSIP_REQUIRE(beta == 0.0 || beta == 1.0, MDSIP_ERR_INVALID_ARG, "syrk_tc: beta must be 0 or 1");
        MDSIP_REQUIRE(precision == MDSIP_PREC_TF32 || precision == MDSIP_PREC_BF16, MDSIP_ERR_INVALID_ARG,
                      "syrk_tc: precision must be TF32 or BF16");
        if (n == 0) return;
        MDSIP_REQUIRE(A && w && C, MDSIP_ERR_INVALID_ARG, "syrk_tc: null pointer");
        const TcPlan pl = syrk_tc_plan(m, n, ctx->num_sms, precision);
        const size_t aft = ((size_t)n * pl.ldt * sizeof(float) + 1023) / 1024 * 1024;
        const size_t wsb = syrk_tc_workspace_bytes(pl, n, precision);
        char *base = static_cast<char *>(ctx->scratch_at_least(aft + wsb + 256));
        float *AfT = reinterpret_cast<float *>(base);
        int *err = reinterpret_cast<int *>(base + aft + wsb);
        MDSIP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
        launch_transpose_f32(ctx->stream, A, m, n, lda, AfT, pl.ldt);
        launch_syrk_tc(ctx->stream, ctx->num_sms, precision, AfT, m, n, w, beta, C, ldc, base + aft, err);
        int herr = 0;
        MDSIP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
        MDSIP_REQUIRE(herr == 0, MDSIP_ERR_DEVICE, "syrk_tc: a bounded device wait expired");
    });
}

// fused: cpre, winv (m) and ATw (n) given (mdsip_gemv_pair_df_next)
static mdsip_status gemv_pair_df_impl(mdsip_ctx *hctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                      const double *x, const double *v, double *Ax, double *ATv, bool fused,
                                      const double *cpre, const double *winv, double *ATw) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(m >= 0 && n >= 0 && lda >= n && lda % 4 == 0 && m <= (1 << 20) && n <= (1 << 20),
                      MDSIP_ERR_INVALID_ARG, "gemv_pair_df: bad sizes");
        if (fused)
            MDSIP_REQUIRE(gemv_both_fusable(n) && (m == 0 || (cpre && winv)) && ATw, MDSIP_ERR_INVALID_ARG,
                          "gemv_pair_df_next: n must be in 1 .. 2048, null operand");
        if (m == 0 && n == 0) return;
        MDSIP_REQUIRE((m == 0 || Ax) && (n == 0 || ATv), MDSIP_ERR_INVALID_ARG, "gemv_pair_df: null output");
        if (m > 0 && n > 0)
            MDSIP_REQUIRE(A && x && v && (reinterpret_cast<uintptr_t>(A) & 15) == 0, MDSIP_ERR_INVALID_ARG,
                          "gemv_pair_df: null or misaligned input");
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };
        const size_t nA = (size_t)m * (size_t)lda;
        const size_t o_lo = up(nA * sizeof(float)), o_xs = o_lo + up(nA * sizeof(float));
        const size_t o_ys = o_xs + up((size_t)n * sizeof(float2)), o_part = o_ys + up((size_t)m * sizeof(float2));
        const size_t o_cw = o_part + up((size_t)kRedBlocks * (size_t)n * sizeof(double));
        const size_t o_wf = o_cw + up((size_t)m * sizeof(float2));
        const size_t o_err = o_wf + up((size_t)m * sizeof(float));
        const size_t total = o_err + 256;
        char *base = static_cast<char *>(ctx->scratch_at_least(total));
        float *hi = reinterpret_cast<float *>(base), *lo = reinterpret_cast<float *>(base + o_lo);
        int *err = reinterpret_cast<int *>(base + o_err);
        MDSIP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
        if (m > 0 && n > 0) launch_split_matrix(ctx->stream, A, m, n, lda, hi, lo);
        BothNextArgs nx{reinterpret_cast<float2 *>(base + o_cw), reinterpret_cast<float *>(base + o_wf), ATw};
        if (fused) {
            launch_split_vector(ctx->stream, cpre, m, reinterpret_cast<float2 *>(base + o_cw));
            launch_round_vector(ctx->stream, winv, m, reinterpret_cast<float *>(base + o_wf));
        }
        launch_gemv_both_df(ctx->stream, hi, lo, m, n, lda, x, v, reinterpret_cast<float2 *>(base + o_xs),
                            reinterpret_cast<float2 *>(base + o_ys), reinterpret_cast<double *>(base + o_part), Ax,
                            ATv, err, fused ? &nx : nullptr);
        int herr = 0;
        MDSIP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
        MDSIP_REQUIRE(herr == 0, MDSIP_ERR_DEVICE, "gemv_pair_df: a bounded device wait expired");
    });
}

mdsip_status mdsip_gemv_pair_df(mdsip_ctx *hctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                const double *x, const double *v, double *Ax, double *ATv) {
    return gemv_pair_df_impl(hctx, m, n, A, lda, x, v, Ax, ATv, false, nullptr, nullptr, nullptr);
}

mdsip_status mdsip_gemv_pair_df_next(mdsip_ctx *hctx, int64_t m, int64_t n, const double *A, int64_t lda,
                                     const double *x, const double *v, const double *cpre, const double *winv,
                                     double *Ax, double *ATv, double *ATw) {
    return gemv_pair_df_impl(hctx, m, n, A, lda, x, v, Ax, ATv, true, cpre, winv, ATw);
}

static mdsip_status ldlt_factor_impl(mdsip_ctx *hctx, int64_t N, double *S, int64_t ld, double zero_tol,
                                     double *L, double *Dd, double *Doff, int32_t *perm, int32_t *kind,
                                     int32_t *inertia, bool fp32_update, int spec = 1);

mdsip_status mdsip_ldlt_factor(mdsip_ctx *hctx, int64_t N, double *S, int64_t ld, double zero_tol,
                               double *L, double *Dd, double *Doff, int32_t *perm, int32_t *kind,
                               int32_t *inertia) {
    return ldlt_factor_impl(hctx, N, S, ld, zero_tol, L, Dd, Doff, perm, kind, inertia, false);
}

mdsip_status mdsip_ldlt_factor_ex(mdsip_ctx *hctx, int64_t N, double *S, int64_t ld, double zero_tol,
                                  int32_t flags, double *L, double *Dd, double *Doff, int32_t *perm,
                                  int32_t *kind, int32_t *inertia) {
    if ((flags & ~(MDSIP_LDLT_FP32_UPDATES | MDSIP_LDLT_NO_SPECULATION | MDSIP_LDLT_PERSISTENT)) ||
        ((flags & MDSIP_LDLT_NO_SPECULATION) && (flags & MDSIP_LDLT_PERSISTENT))) {
        if (hctx) C_(hctx)->last_error = "ldlt: unknown or contradictory flags";
        return MDSIP_ERR_INVALID_ARG;
    }
    const int spec = (flags & MDSIP_LDLT_NO_SPECULATION) ? 0 : ((flags & MDSIP_LDLT_PERSISTENT) ? 2 : 1);
    return ldlt_factor_impl(hctx, N, S, ld, zero_tol, L, Dd, Doff, perm, kind, inertia,
                            (flags & MDSIP_LDLT_FP32_UPDATES) != 0, spec);
}

static mdsip_status ldlt_factor_impl(mdsip_ctx *hctx, int64_t N, double *S, int64_t ld, double zero_tol,
                                     double *L, double *Dd, double *Doff, int32_t *perm, int32_t *kind,
                                     int32_t *inertia, bool fp32_update, int spec) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(N >= 0 && ld == N, MDSIP_ERR_INVALID_ARG, "ldlt: need ld == N");
        MDSIP_REQUIRE(inertia, MDSIP_ERR_INVALID_ARG, "ldlt: null inertia");
        if (N == 0) {
            MDSIP_CUDA(cudaMemsetAsync(inertia, 0, 3 * sizeof(int32_t), ctx->stream));
            return;
        }
        MDSIP_REQUIRE(S && L && Dd && Doff && perm && kind, MDSIP_ERR_INVALID_ARG, "ldlt: null pointer");
        const size_t ws = ldlt_scratch_bytes(N) + 64 + 8 * kRedBlocks + 64;
        char *w = static_cast<char *>(ctx->scratch_at_least(ws));
        double *partial = reinterpret_cast<double *>(w + ldlt_scratch_bytes(N) + 64);
        double *maxabs = partial + kRedBlocks;
        int *err = reinterpret_cast<int *>(w + ldlt_scratch_bytes(N));   // err, then two panel counts
        MDSIP_REQUIRE((reinterpret_cast<uintptr_t>(partial) & 7) == 0, MDSIP_ERR_INVALID_ARG,
                      "ldlt: misaligned scratch layout");
        MDSIP_CUDA(cudaMemsetAsync(err, 0, 3 * sizeof(int), ctx->stream));
        launch_maxabs_lower(ctx->stream, N, S, ld, partial, maxabs);
        LdltOut o{L, Dd, Doff, perm, kind, inertia, err + 1};
        launch_ldlt(ctx->stream, ctx->num_sms, N, S, ld, maxabs, zero_tol, o, w, err, fp32_update, 0, spec);
        int herr[3] = {0, 0, 0};
        MDSIP_CUDA(cudaMemcpyAsync(herr, err, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
        ctx->ldlt_panels[0] = herr[1];
        ctx->ldlt_panels[1] = herr[2];
        MDSIP_REQUIRE(herr[0] == 0, MDSIP_ERR_DEVICE, "ldlt: a bounded device wait expired");
    });
}

mdsip_status mdsip_ldlt_panel_counts(mdsip_ctx *hctx, int32_t *out2) {
    if (!hctx || !out2) return MDSIP_ERR_INVALID_ARG;
    out2[0] = C_(hctx)->ldlt_panels[0];
    out2[1] = C_(hctx)->ldlt_panels[1];
    return MDSIP_OK;
}

mdsip_status mdsip_ldlt_factor_noalloc(mdsip_ctx *hctx, int64_t N, double *S, int64_t ld,
                                       double zero_tol, double *L, double *Dd, double *Doff,
                                       int32_t *perm, int32_t *kind, int32_t *inertia) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        LdltOut o{L, Dd, Doff, perm, kind, inertia};
        ldlt_factor_fixed_scratch(ctx->stream, ctx->device, ctx->num_sms, N, S, ld, zero_tol, o);
    });
}

mdsip_status mdsip_ldlt_solve(mdsip_ctx *hctx, int64_t N, const double *L, const double *Dd,
                              const double *Doff, const int32_t *perm, int64_t nrhs, double *B,
                              int64_t ldb) {
    if (!hctx) return MDSIP_ERR_INVALID_ARG;
    Ctx *ctx = C_(hctx);
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        MDSIP_REQUIRE(N >= 0 && nrhs >= 0 && ldb >= N, MDSIP_ERR_INVALID_ARG, "ldlt_solve: bad sizes");
        if (N == 0 || nrhs == 0) return;
        MDSIP_REQUIRE(L && Dd && Doff && perm && B, MDSIP_ERR_INVALID_ARG, "ldlt_solve: null pointer");
        const size_t ws = ldlt_solve_scratch_bytes(N);
        char *w = static_cast<char *>(ctx->scratch_at_least(ws + 256));
        int *err = reinterpret_cast<int *>(w + ws);
        MDSIP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
        launch_ldlt_solve_prepare(ctx->stream, N, L, w, false);
        launch_ldlt_solve_coop(ctx->stream, ctx->num_sms, N, Dd, Doff, perm, nrhs, B, ldb, w, err, false);
        int herr = 0;
        MDSIP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
        MDSIP_REQUIRE(herr == 0, MDSIP_ERR_DEVICE, "ldlt_solve: a bounded device wait expired");
    });
}

}  // extern "C"
