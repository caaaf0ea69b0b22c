// Warm-start network: a two-hidden-layer ReLU perceptron
//
//     h1 = relu(W1 xn + b1),  h2 = relu(W2 h1 + b2),  yn = W3 h2 + b3
//
// mapping the parameters p of a parametric problem family (xn: p
// standardised per input) to a standardised primal-dual point plus log mu0
// (y = yn * out_std + out_mean).  Training minimises the mean squared error in
// standardised units, L = sum (yn - (y* - out_mean) / out_std)^2 / (B O), with
// Adam.  Every contraction (three forward, five backward) runs on the BF16
// tcgen05 GEMM with FP32 accumulation; parameters, moments and gradients are
// FP32; the bias, ReLU, loss and transposes are fused into the kernels that
// produce the BF16 operands of the next contraction.
//
// BF16 operand points (each value rounded to nearest even once): the
// standardised input, W1, W2, W3, h1, h2, the output gradient dL/dyn, and the
// hidden-layer gradients dL/dz2, dL/dz1.  Bias gradients are column sums of
// the rounded BF16 gradients.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace mdsip {

size_t gemm_bf16_ws_bytes(int64_t M, int64_t N, int64_t K, int num_sms);
void launch_gemm_bf16(cudaStream_t s, int num_sms, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                      int64_t ldb, int64_t M, int64_t N, int64_t K, float *C, int64_t ldc, void *ws, int *err_dev);

namespace {

using bf16 = __nv_bfloat16;

constexpr int TT = 32;  // transpose tile edge

int64_t r8(int64_t v) { return (std::max<int64_t>(v, 1) + 7) / 8 * 8; }

// Xb[b][i] = bf16((X[row(b)][i] - mean_i) / std_i), XbT[i][b] = Xb[b][i]
__global__ void k_gather_x(int64_t B, int64_t I, const double *__restrict__ X, int64_t ldx,
                           const int32_t *__restrict__ idx, const float *__restrict__ mean,
                           const float *__restrict__ sd, bf16 *__restrict__ Xb, int64_t ldI, bf16 *__restrict__ XbT,
                           int64_t ldB) {
    __shared__ bf16 t[TT][TT + 2];
    const int64_t i0 = (int64_t)blockIdx.x * TT, b0 = (int64_t)blockIdx.y * TT;
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t b = b0 + r, i = i0 + threadIdx.x;
        bf16 v = __float2bfloat16_rn(0.0f);
        if (b < B && i < I) {
            const int64_t row = idx ? (int64_t)idx[b] : b;
            v = __float2bfloat16_rn((float)((X[row * ldx + i] - (double)mean[i]) / (double)sd[i]));
            Xb[b * ldI + i] = v;
        }
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    if (!XbT) return;
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t i = i0 + r, b = b0 + threadIdx.x;
        if (i < I && b < B) XbT[i * ldB + b] = t[threadIdx.x][r];
    }
}

// Hh[b][j] = bf16(relu(Z[b][j] + bias[j])), HT[j][b] = Hh[b][j]
__global__ void k_bias_relu(int64_t B, int64_t Hn, const float *__restrict__ Z, int64_t ldz,
                            const float *__restrict__ bias, bf16 *__restrict__ Hh, int64_t ldh, bf16 *__restrict__ HT,
                            int64_t ldB) {
    __shared__ bf16 t[TT][TT + 2];
    const int64_t j0 = (int64_t)blockIdx.x * TT, b0 = (int64_t)blockIdx.y * TT;
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t b = b0 + r, j = j0 + threadIdx.x;
        bf16 v = __float2bfloat16_rn(0.0f);
        if (b < B && j < Hn) {
            v = __float2bfloat16_rn(fmaxf(Z[b * ldz + j] + bias[j], 0.0f));
            Hh[b * ldh + j] = v;
        }
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t j = j0 + r, b = b0 + threadIdx.x;
        if (j < Hn && b < B) HT[j * ldB + b] = t[threadIdx.x][r];
    }
}

// Output layer and loss: yn = Z + b3, target tn = (Y[row(b)][o] - mean_o) /
// std_o, dY = bf16(scale (yn - tn)) in both orientations; per-block partial of
// sum (yn - tn)^2 in FP64.
__global__ void k_out_loss(int64_t B, int64_t O, const float *__restrict__ Z, int64_t ldz,
                           const float *__restrict__ b3, const double *__restrict__ Y, int64_t ldy,
                           const int32_t *__restrict__ idx, const float *__restrict__ mean,
                           const float *__restrict__ sd, float scale, bf16 *__restrict__ dY, int64_t ldO,
                           bf16 *__restrict__ dYT, int64_t ldB, double *__restrict__ part) {
    __shared__ bf16 t[TT][TT + 2];
    __shared__ double red[TT * 8];
    const int64_t o0 = (int64_t)blockIdx.x * TT, b0 = (int64_t)blockIdx.y * TT;
    double acc = 0.0;
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t b = b0 + r, o = o0 + threadIdx.x;
        bf16 g = __float2bfloat16_rn(0.0f);
        if (b < B && o < O) {
            const int64_t row = idx ? (int64_t)idx[b] : b;
            const float yn = Z[b * ldz + o] + b3[o];
            const float tn = (float)((Y[row * ldy + o] - (double)mean[o]) / (double)sd[o]);
            const float d = yn - tn;
            acc += (double)d * (double)d;
            g = __float2bfloat16_rn(scale * d);
            dY[b * ldO + o] = g;
        }
        t[r][threadIdx.x] = g;
    }
    const int tid = threadIdx.y * TT + threadIdx.x;
    red[tid] = acc;
    __syncthreads();
    for (int w = TT * 8 / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t o = o0 + r, b = b0 + threadIdx.x;
        if (o < O && b < B) dYT[o * ldB + b] = t[threadIdx.x][r];
    }
}

// dZ = bf16(dH * [Hact > 0]) in both orientations (dZ optional)
__global__ void k_relu_back(int64_t B, int64_t Hn, const float *__restrict__ dH, int64_t ldd,
                            const bf16 *__restrict__ Hact, int64_t ldh, bf16 *__restrict__ dZ,
                            bf16 *__restrict__ dZT, int64_t ldB) {
    __shared__ bf16 t[TT][TT + 2];
    const int64_t j0 = (int64_t)blockIdx.x * TT, b0 = (int64_t)blockIdx.y * TT;
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t b = b0 + r, j = j0 + threadIdx.x;
        bf16 v = __float2bfloat16_rn(0.0f);
        if (b < B && j < Hn) {
            const float h = __bfloat162float(Hact[b * ldh + j]);
            v = __float2bfloat16_rn(h > 0.0f ? dH[b * ldd + j] : 0.0f);
            if (dZ) dZ[b * ldh + j] = v;
        }
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < TT; r += blockDim.y) {
        const int64_t j = j0 + r, b = b0 + threadIdx.x;
        if (j < Hn && b < B) dZT[j * ldB + b] = t[threadIdx.x][r];
    }
}

// out[r] = sum_{c < cols} T[r][c]  (one warp per row, fixed order)
__global__ void k_rowsum_bf16(int64_t rows, int64_t cols, const bf16 *__restrict__ T, int64_t ld,
                              float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x / 32;
    for (int64_t r = (int64_t)blockIdx.x * wpb + threadIdx.x / 32; r < rows; r += (int64_t)gridDim.x * wpb) {
        float s = 0.0f;
        for (int64_t c = lane; c < cols; c += 32) s += __bfloat162float(T[r * ld + c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[r] = s;
    }
}

// single-block fixed-order sum of n doubles
__global__ void k_sum_partials(int64_t n, const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adam (bias-corrected first and second moments)
__global__ void k_adam(int64_t n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// dst[r][c] = bf16(src[r][c]) and/or dstT[c][r] = bf16(src[r][c])
__global__ void k_cast_bf16(int64_t rows, int64_t cols, const float *__restrict__ src, int64_t lds,
                            bf16 *__restrict__ dst, int64_t ldd, bf16 *__restrict__ dstT, int64_t ldt) {
    __shared__ bf16 t[TT][TT + 2];
    const int64_t c0 = (int64_t)blockIdx.x * TT, r0 = (int64_t)blockIdx.y * TT;
    for (int rr = threadIdx.y; rr < TT; rr += blockDim.y) {
        const int64_t r = r0 + rr, c = c0 + threadIdx.x;
        bf16 v = __float2bfloat16_rn(0.0f);
        if (r < rows && c < cols) {
            v = __float2bfloat16_rn(src[r * lds + c]);
            if (dst) dst[r * ldd + c] = v;
        }
        t[rr][threadIdx.x] = v;
    }
    if (!dstT) return;
    __syncthreads();
    for (int rr = threadIdx.y; rr < TT; rr += blockDim.y) {
        const int64_t c = c0 + rr, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dstT[c * ldt + r] = t[threadIdx.x][rr];
    }
}

// y[b][o] = (Z[b][o] + b3[o]) * std_o + mean_o
__global__ void k_out_denorm(int64_t B, int64_t O, const float *__restrict__ Z, int64_t ldz,
                             const float *__restrict__ b3, const float *__restrict__ mean,
                             const float *__restrict__ sd, float *__restrict__ Yo, int64_t ldy) {
    const int64_t total = B * O;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / O, o = e % O;
        Yo[b * ldy + o] = (Z[b * ldz + o] + b3[o]) * sd[o] + mean[o];
    }
}

// Column mean and standard deviation (two passes, FP64, fixed order); a
// standard deviation below 1e-6 max(1, |mean|) is replaced by that floor.
__global__ void k_col_stats(int64_t rows, int64_t cols, const double *__restrict__ Y, int64_t ldy,
                            float *__restrict__ mean, float *__restrict__ sd) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t r = 0; r < rows; ++r) s += Y[r * ldy + c];
        const double mu = rows > 0 ? s / (double)rows : 0.0;
        double q = 0.0;
        for (int64_t r = 0; r < rows; ++r) {
            const double d = Y[r * ldy + c] - mu;
            q += d * d;
        }
        const double sdev = rows > 0 ? sqrt(q / (double)rows) : 0.0;
        mean[c] = (float)mu;
        sd[c] = (float)fmax(sdev, 1e-6 * fmax(1.0, fabs(mu)));
    }
}

__global__ void k_fill_f32(int64_t n, float *p, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

int grid_for(int64_t n, int num_sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * 16, ceil_div(n, 256)));
}

dim3 tgrid(int64_t cols, int64_t rows) { return dim3((unsigned)ceil_div(cols, TT), (unsigned)ceil_div(rows, TT)); }

}  // namespace

struct Mlp {
    Ctx *ctx = nullptr;
    int64_t I = 0, H = 0, O = 0;
    int64_t ldI = 8, ldH = 8, ldO = 8;
    int64_t off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0, n_params = 0;
    double beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
    int64_t t = 0;  // Adam steps taken
    DBuf params, grads, m1, m2;
    DBuf W1b, W2b, W2bT, W3b, W3bT;
    DBuf in_mean, in_std, out_mean, out_std;
    DBuf err, loss;
    // activations, sized for `cap` rows
    int64_t cap = 0, ldB = 8;
    DBuf Xb, XbT, H1, H1T, H2, H2T, dY, dYT, dZ2, dZ2T, dZ1T, Zbuf, lpart, gws;
    size_t gws_bytes = 0;

    float *P() const { return params.as<float>(); }
    float *G() const { return grads.as<float>(); }

    void ensure(int64_t B) {
        if (B <= cap) return;
        cap = std::max<int64_t>(B, 64);
        ldB = r8(cap);
        Xb.get<bf16>(ctx, cap * ldI);
        XbT.get<bf16>(ctx, I * ldB);
        H1.get<bf16>(ctx, cap * ldH);
        H1T.get<bf16>(ctx, H * ldB);
        H2.get<bf16>(ctx, cap * ldH);
        H2T.get<bf16>(ctx, H * ldB);
        dY.get<bf16>(ctx, cap * ldO);
        dYT.get<bf16>(ctx, O * ldB);
        dZ2.get<bf16>(ctx, cap * ldH);
        dZ2T.get<bf16>(ctx, H * ldB);
        dZ1T.get<bf16>(ctx, H * ldB);
        Zbuf.get<float>(ctx, cap * std::max(ldO, ldH));
        lpart.get<double>(ctx, ceil_div(O, TT) * ceil_div(cap, TT));
        const int sms = ctx->num_sms;
        gws_bytes = std::max({gemm_bf16_ws_bytes(cap, H, I, sms), gemm_bf16_ws_bytes(cap, H, H, sms),
                              gemm_bf16_ws_bytes(cap, O, H, sms), gemm_bf16_ws_bytes(O, H, cap, sms),
                              gemm_bf16_ws_bytes(cap, H, O, sms), gemm_bf16_ws_bytes(H, H, cap, sms),
                              gemm_bf16_ws_bytes(H, I, cap, sms), (size_t)16});
        gws.get<uint8_t>(ctx, gws_bytes);
    }

    void gemm(const bf16 *A, int64_t lda, const bf16 *Bm, int64_t ldb, int64_t M, int64_t N, int64_t K, float *C,
              int64_t ldc) {
        launch_gemm_bf16(ctx->stream, ctx->num_sms, A, lda, Bm, ldb, M, N, K, C, ldc, gws.ptr, err.as<int>());
    }

    // BF16 copies of the weights (W2 and W3 also transposed)
    void cast_weights() {
        cudaStream_t s = ctx->stream;
        const dim3 blk(TT, 8);
        k_cast_bf16<<<tgrid(I, H), blk, 0, s>>>(H, I, P() + off_W1, I, W1b.as<bf16>(), ldI, nullptr, 0);
        MDSIP_LAUNCHED();
        k_cast_bf16<<<tgrid(H, H), blk, 0, s>>>(H, H, P() + off_W2, H, W2b.as<bf16>(), ldH, W2bT.as<bf16>(), ldH);
        MDSIP_LAUNCHED();
        k_cast_bf16<<<tgrid(H, O), blk, 0, s>>>(O, H, P() + off_W3, H, W3b.as<bf16>(), ldH, W3bT.as<bf16>(), ldO);
        MDSIP_LAUNCHED();
    }

    // forward through h2 (kept for the backward pass); Zbuf ends with the
    // output-layer pre-bias values (B x O, row stride ldO)
    void forward(const double *X, int64_t ldx, const int32_t *idx, int64_t B) {
        cudaStream_t s = ctx->stream;
        const dim3 blk(TT, 8);
        float *Z = Zbuf.as<float>();
        k_gather_x<<<tgrid(I, B), blk, 0, s>>>(B, I, X, ldx, idx, in_mean.as<float>(), in_std.as<float>(),
                                               Xb.as<bf16>(), ldI, XbT.as<bf16>(), ldB);
        MDSIP_LAUNCHED();
        gemm(Xb.as<bf16>(), ldI, W1b.as<bf16>(), ldI, B, H, I, Z, ldH);
        k_bias_relu<<<tgrid(H, B), blk, 0, s>>>(B, H, Z, ldH, P() + off_b1, H1.as<bf16>(), ldH, H1T.as<bf16>(), ldB);
        MDSIP_LAUNCHED();
        gemm(H1.as<bf16>(), ldH, W2b.as<bf16>(), ldH, B, H, H, Z, ldH);
        k_bias_relu<<<tgrid(H, B), blk, 0, s>>>(B, H, Z, ldH, P() + off_b2, H2.as<bf16>(), ldH, H2T.as<bf16>(), ldB);
        MDSIP_LAUNCHED();
        gemm(H2.as<bf16>(), ldH, W3b.as<bf16>(), ldH, B, O, H, Z, ldO);
    }

    // loss (device scalar) and gradients into G()
    void backward(const double *Y, int64_t ldy, const int32_t *idx, int64_t B) {
        cudaStream_t s = ctx->stream;
        const dim3 blk(TT, 8);
        float *Z = Zbuf.as<float>();
        float *G_ = G();
        const float scale = (float)(2.0 / ((double)B * (double)O));
        const dim3 lg = tgrid(O, B);
        k_out_loss<<<lg, blk, 0, s>>>(B, O, Z, ldO, P() + off_b3, Y, ldy, idx, out_mean.as<float>(),
                                      out_std.as<float>(), scale, dY.as<bf16>(), ldO, dYT.as<bf16>(), ldB,
                                      lpart.as<double>());
        MDSIP_LAUNCHED();
        k_sum_partials<<<1, 256, 0, s>>>((int64_t)lg.x * lg.y, lpart.as<double>(), loss.as<double>());
        MDSIP_LAUNCHED();
        // output layer: dW3 = dY^T h2, db3 = column sums of dY
        gemm(dYT.as<bf16>(), ldB, H2T.as<bf16>(), ldB, O, H, B, G_ + off_W3, H);
        k_rowsum_bf16<<<grid_for(O * 32, ctx->num_sms), 256, 0, s>>>(O, B, dYT.as<bf16>(), ldB, G_ + off_b3);
        MDSIP_LAUNCHED();
        // second hidden layer: dh2 = dY W3, dz2 = dh2 [h2 > 0]
        gemm(dY.as<bf16>(), ldO, W3bT.as<bf16>(), ldO, B, H, O, Z, ldH);
        k_relu_back<<<tgrid(H, B), blk, 0, s>>>(B, H, Z, ldH, H2.as<bf16>(), ldH, dZ2.as<bf16>(), dZ2T.as<bf16>(),
                                               ldB);
        MDSIP_LAUNCHED();
        gemm(dZ2T.as<bf16>(), ldB, H1T.as<bf16>(), ldB, H, H, B, G_ + off_W2, H);
        k_rowsum_bf16<<<grid_for(H * 32, ctx->num_sms), 256, 0, s>>>(H, B, dZ2T.as<bf16>(), ldB, G_ + off_b2);
        MDSIP_LAUNCHED();
        // first hidden layer: dh1 = dz2 W2, dz1 = dh1 [h1 > 0]
        gemm(dZ2.as<bf16>(), ldH, W2bT.as<bf16>(), ldH, B, H, H, Z, ldH);
        k_relu_back<<<tgrid(H, B), blk, 0, s>>>(B, H, Z, ldH, H1.as<bf16>(), ldH, nullptr, dZ1T.as<bf16>(), ldB);
        MDSIP_LAUNCHED();
        gemm(dZ1T.as<bf16>(), ldB, XbT.as<bf16>(), ldB, H, I, B, G_ + off_W1, I);
        k_rowsum_bf16<<<grid_for(H * 32, ctx->num_sms), 256, 0, s>>>(H, B, dZ1T.as<bf16>(), ldB, G_ + off_b1);
        MDSIP_LAUNCHED();
    }

    void check_err() {
        int e = 0;
        MDSIP_CUDA(cudaMemcpyAsync(&e, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        MDSIP_CUDA(cudaStreamSynchronize(ctx->stream));
        MDSIP_REQUIRE(e == 0, MDSIP_ERR_DEVICE, "tensor-core GEMM pipeline wait expired");
    }
};

}  // namespace mdsip

using mdsip::Ctx;
using mdsip::DeviceGuard;
using mdsip::Mlp;
using mdsip::guarded;

static inline Mlp *M_(mdsip_mlp *m) { return reinterpret_cast<Mlp *>(m); }
static inline const Mlp *M_(const mdsip_mlp *m) { return reinterpret_cast<const Mlp *>(m); }

static void copy_in(void *dst, const void *src, size_t bytes, int mem, cudaStream_t s) {
    MDSIP_REQUIRE(src != nullptr || bytes == 0, MDSIP_ERR_INVALID_ARG, "null data pointer");
    MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
    if (bytes == 0) return;
    MDSIP_CUDA(cudaMemcpyAsync(dst, src, bytes, mem == MDSIP_MEM_HOST ? cudaMemcpyHostToDevice
                                                                      : cudaMemcpyDeviceToDevice, s));
    MDSIP_CUDA(cudaStreamSynchronize(s));
}

static void copy_out(void *dst, const void *src, size_t bytes, int mem, cudaStream_t s) {
    MDSIP_REQUIRE(dst != nullptr || bytes == 0, MDSIP_ERR_INVALID_ARG, "null output pointer");
    MDSIP_REQUIRE(mem == MDSIP_MEM_HOST || mem == MDSIP_MEM_DEVICE, MDSIP_ERR_INVALID_ARG, "bad mem tag");
    if (bytes == 0) return;
    MDSIP_CUDA(cudaMemcpyAsync(dst, src, bytes, mem == MDSIP_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                      : cudaMemcpyDeviceToDevice, s));
    MDSIP_CUDA(cudaStreamSynchronize(s));
}

extern "C" {

mdsip_status mdsip_mlp_create(mdsip_ctx *hctx, int64_t n_in, int64_t n_hidden, int64_t n_out, mdsip_mlp **out) {
    if (!hctx || !out) return MDSIP_ERR_INVALID_ARG;
    *out = nullptr;
    Ctx *ctx = reinterpret_cast<Ctx *>(hctx);
    return guarded(ctx, [&] {
        MDSIP_REQUIRE(n_in > 0 && n_hidden > 0 && n_out > 0 && n_in <= (1 << 20) && n_hidden <= (1 << 16) &&
                          n_out <= (1LL << 30),
                      MDSIP_ERR_INVALID_ARG, "mlp: sizes out of range");
        DeviceGuard g(ctx->device);
        auto *m = new Mlp();
        try {
            m->ctx = ctx;
            m->I = n_in;
            m->H = n_hidden;
            m->O = n_out;
            m->ldI = mdsip::r8(n_in);
            m->ldH = mdsip::r8(n_hidden);
            m->ldO = mdsip::r8(n_out);
            // parameter layout: W1 (H x I) | b1 (H) | W2 (H x H) | b2 (H) | W3 (O x H) | b3 (O),
            // each block starting on a 16-byte boundary
            auto al4 = [](int64_t v) { return (v + 3) / 4 * 4; };
            int64_t o = 0;
            m->off_W1 = o; o = al4(o + n_hidden * n_in);
            m->off_b1 = o; o = al4(o + n_hidden);
            m->off_W2 = o; o = al4(o + n_hidden * n_hidden);
            m->off_b2 = o; o = al4(o + n_hidden);
            m->off_W3 = o; o = al4(o + n_out * n_hidden);
            m->off_b3 = o; o = al4(o + n_out);
            m->n_params = o;
            cudaStream_t s = ctx->stream;
            for (mdsip::DBuf *b : {&m->params, &m->grads, &m->m1, &m->m2}) {
                b->get<float>(ctx, m->n_params);
                MDSIP_CUDA(cudaMemsetAsync(b->ptr, 0, m->n_params * sizeof(float), s));
            }
            m->W1b.get<__nv_bfloat16>(ctx, n_hidden * m->ldI);
            m->W2b.get<__nv_bfloat16>(ctx, n_hidden * m->ldH);
            m->W2bT.get<__nv_bfloat16>(ctx, n_hidden * m->ldH);
            m->W3b.get<__nv_bfloat16>(ctx, n_out * m->ldH);
            m->W3bT.get<__nv_bfloat16>(ctx, n_hidden * m->ldO);
            m->in_mean.get<float>(ctx, n_in);
            m->in_std.get<float>(ctx, n_in);
            m->out_mean.get<float>(ctx, n_out);
            m->out_std.get<float>(ctx, n_out);
            mdsip::k_fill_f32<<<1, 256, 0, s>>>(n_in, m->in_mean.as<float>(), 0.0f);
            MDSIP_LAUNCHED();
            mdsip::k_fill_f32<<<1, 256, 0, s>>>(n_in, m->in_std.as<float>(), 1.0f);
            MDSIP_LAUNCHED();
            mdsip::k_fill_f32<<<mdsip::grid_for(n_out, ctx->num_sms), 256, 0, s>>>(n_out, m->out_mean.as<float>(),
                                                                                     0.0f);
            MDSIP_LAUNCHED();
            mdsip::k_fill_f32<<<mdsip::grid_for(n_out, ctx->num_sms), 256, 0, s>>>(n_out, m->out_std.as<float>(),
                                                                                     1.0f);
            MDSIP_LAUNCHED();
            m->err.get<int>(ctx, 1);
            MDSIP_CUDA(cudaMemsetAsync(m->err.ptr, 0, sizeof(int), s));
            m->loss.get<double>(ctx, 1);
            m->cast_weights();
            MDSIP_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            delete m;
            throw;
        }
        *out = reinterpret_cast<mdsip_mlp *>(m);
    });
}

void mdsip_mlp_destroy(mdsip_mlp *hm) {
    if (!hm) return;
    Mlp *m = M_(hm);
    try {
        DeviceGuard g(m->ctx->device);
        cudaStreamSynchronize(m->ctx->stream);
        delete m;
    } catch (...) {
    }
}

int64_t mdsip_mlp_num_params(const mdsip_mlp *hm) { return hm ? M_(hm)->n_params : 0; }

mdsip_status mdsip_mlp_param_offsets(const mdsip_mlp *hm, int64_t offsets[6]) {
    if (!hm || !offsets) return MDSIP_ERR_INVALID_ARG;
    const Mlp *m = M_(hm);
    offsets[0] = m->off_W1;
    offsets[1] = m->off_b1;
    offsets[2] = m->off_W2;
    offsets[3] = m->off_b2;
    offsets[4] = m->off_W3;
    offsets[5] = m->off_b3;
    return MDSIP_OK;
}

mdsip_status mdsip_mlp_set_params(mdsip_mlp *hm, const float *params, int mem) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        DeviceGuard g(m->ctx->device);
        cudaStream_t s = m->ctx->stream;
        copy_in(m->params.ptr, params, m->n_params * sizeof(float), mem, s);
        MDSIP_CUDA(cudaMemsetAsync(m->m1.ptr, 0, m->n_params * sizeof(float), s));
        MDSIP_CUDA(cudaMemsetAsync(m->m2.ptr, 0, m->n_params * sizeof(float), s));
        m->t = 0;
        m->cast_weights();
        MDSIP_CUDA(cudaStreamSynchronize(s));
    });
}

mdsip_status mdsip_mlp_get_params(mdsip_mlp *hm, float *params, int mem) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        DeviceGuard g(m->ctx->device);
        copy_out(params, m->params.ptr, m->n_params * sizeof(float), mem, m->ctx->stream);
    });
}

mdsip_status mdsip_mlp_set_adam(mdsip_mlp *hm, double beta1, double beta2, double eps) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps > 0.0)) {
        m->ctx->last_error = "mlp: Adam constants out of range";
        return MDSIP_ERR_INVALID_ARG;
    }
    m->beta1 = beta1;
    m->beta2 = beta2;
    m->eps = eps;
    return MDSIP_OK;
}

mdsip_status mdsip_mlp_set_scaling(mdsip_mlp *hm, const float *in_mean, const float *in_std, const float *out_mean,
                                   const float *out_std, int mem) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        DeviceGuard g(m->ctx->device);
        cudaStream_t s = m->ctx->stream;
        if (mem == MDSIP_MEM_HOST) {
            auto pos = [](const float *v, int64_t n) {
                for (int64_t i = 0; i < n; ++i)
                    if (!(v[i] > 0.0f)) return false;
                return true;
            };
            MDSIP_REQUIRE((!in_std || pos(in_std, m->I)) && (!out_std || pos(out_std, m->O)), MDSIP_ERR_INVALID_ARG,
                          "mlp: scaling standard deviations must be positive");
        }
        if (in_mean) copy_in(m->in_mean.ptr, in_mean, m->I * sizeof(float), mem, s);
        if (in_std) copy_in(m->in_std.ptr, in_std, m->I * sizeof(float), mem, s);
        if (out_mean) copy_in(m->out_mean.ptr, out_mean, m->O * sizeof(float), mem, s);
        if (out_std) copy_in(m->out_std.ptr, out_std, m->O * sizeof(float), mem, s);
    });
}

mdsip_status mdsip_mlp_get_scaling(mdsip_mlp *hm, float *in_mean, float *in_std, float *out_mean, float *out_std,
                                   int mem) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        DeviceGuard g(m->ctx->device);
        cudaStream_t s = m->ctx->stream;
        if (in_mean) copy_out(in_mean, m->in_mean.ptr, m->I * sizeof(float), mem, s);
        if (in_std) copy_out(in_std, m->in_std.ptr, m->I * sizeof(float), mem, s);
        if (out_mean) copy_out(out_mean, m->out_mean.ptr, m->O * sizeof(float), mem, s);
        if (out_std) copy_out(out_std, m->out_std.ptr, m->O * sizeof(float), mem, s);
    });
}

mdsip_status mdsip_mlp_fit_scaling(mdsip_mlp *hm, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                                   int64_t count) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        MDSIP_REQUIRE(X && Y && count > 0 && ldx >= m->I && ldy >= m->O, MDSIP_ERR_INVALID_ARG,
                      "mlp: bad training data");
        DeviceGuard g(m->ctx->device);
        cudaStream_t s = m->ctx->stream;
        mdsip::k_col_stats<<<mdsip::grid_for(m->I, m->ctx->num_sms), 256, 0, s>>>(
            count, m->I, X, ldx, m->in_mean.as<float>(), m->in_std.as<float>());
        MDSIP_LAUNCHED();
        mdsip::k_col_stats<<<mdsip::grid_for(m->O, m->ctx->num_sms), 256, 0, s>>>(
            count, m->O, Y, ldy, m->out_mean.as<float>(), m->out_std.as<float>());
        MDSIP_LAUNCHED();
        MDSIP_CUDA(cudaStreamSynchronize(s));
    });
}

mdsip_status mdsip_mlp_forward(mdsip_mlp *hm, const double *X, int64_t ldx, int64_t batch, float *Y, int64_t ldy) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        MDSIP_REQUIRE(batch >= 0 && ldx >= m->I && ldy >= m->O, MDSIP_ERR_INVALID_ARG, "mlp: bad forward arguments");
        if (batch == 0) return;
        MDSIP_REQUIRE(X && Y, MDSIP_ERR_INVALID_ARG, "mlp: null data pointer");
        DeviceGuard g(m->ctx->device);
        m->ensure(batch);
        m->forward(X, ldx, nullptr, batch);
        mdsip::k_out_denorm<<<mdsip::grid_for(batch * m->O, m->ctx->num_sms), 256, 0, m->ctx->stream>>>(
            batch, m->O, m->Zbuf.as<float>(), m->ldO, m->P() + m->off_b3, m->out_mean.as<float>(),
            m->out_std.as<float>(), Y, ldy);
        MDSIP_LAUNCHED();
        m->check_err();
    });
}

static void run_gradient(Mlp *m, const double *X, int64_t ldx, const double *Y, int64_t ldy, const int32_t *idx,
                         int64_t batch) {
    MDSIP_REQUIRE(X && Y && batch > 0 && ldx >= m->I && ldy >= m->O, MDSIP_ERR_INVALID_ARG,
                  "mlp: bad training arguments");
    m->ensure(batch);
    m->forward(X, ldx, idx, batch);
    m->backward(Y, ldy, idx, batch);
}

mdsip_status mdsip_mlp_gradient(mdsip_mlp *hm, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                                const int32_t *idx, int64_t batch, float *grad, double *loss) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        DeviceGuard g(m->ctx->device);
        run_gradient(m, X, ldx, Y, ldy, idx, batch);
        m->check_err();
        if (grad) copy_out(grad, m->grads.ptr, m->n_params * sizeof(float), MDSIP_MEM_DEVICE, m->ctx->stream);
        if (loss) copy_out(loss, m->loss.ptr, sizeof(double), MDSIP_MEM_HOST, m->ctx->stream);
        if (loss) *loss /= (double)batch * (double)m->O;
    });
}

mdsip_status mdsip_mlp_train_step(mdsip_mlp *hm, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                                  const int32_t *idx, int64_t batch, double lr, double *loss) {
    if (!hm) return MDSIP_ERR_INVALID_ARG;
    Mlp *m = M_(hm);
    return guarded(m->ctx, [&] {
        MDSIP_REQUIRE(lr >= 0.0, MDSIP_ERR_INVALID_ARG, "mlp: negative learning rate");
        DeviceGuard g(m->ctx->device);
        run_gradient(m, X, ldx, Y, ldy, idx, batch);
        m->t += 1;
        // the moments decay with the FP32 rates the kernel uses, so the bias
        // corrections 1 - beta^t take those same rates (Kingma-Ba Algorithm 1);
        // with the FP64 rates 1 - 0.999 and 1 - fl32(0.999) differ by 1.3e-5
        const float b1f = (float)m->beta1, b2f = (float)m->beta2;
        const double bc1 = 1.0 - std::pow((double)b1f, (double)m->t), bc2 = 1.0 - std::pow((double)b2f, (double)m->t);
        mdsip::k_adam<<<mdsip::grid_for(m->n_params, m->ctx->num_sms), 256, 0, m->ctx->stream>>>(
            m->n_params, m->P(), m->G(), m->m1.as<float>(), m->m2.as<float>(), (float)lr, b1f, b2f,
            (float)m->eps, (float)bc1, (float)bc2);
        MDSIP_LAUNCHED();
        m->cast_weights();
        if (loss) {
            m->check_err();
            copy_out(loss, m->loss.ptr, sizeof(double), MDSIP_MEM_HOST, m->ctx->stream);
            *loss /= (double)batch * (double)m->O;
        }
    });
}

}  // extern "C"
