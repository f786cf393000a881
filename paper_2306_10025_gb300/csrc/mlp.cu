// Learned assignment (the paper leaves deep-learning assisted clustering to
// future work, end of section 3.2): per-patch features, a d -> h -> h -> m
// ReLU network predicting the database entry of every patch, trained by
// softmax cross-entropy with Adam, all on the GPU.
//
// GEMMs: the tensor-core kernel of gemm_tc.cu (3xTF32 on tcgen05, FP32
// accumulation in TMEM, FP32-level results) with arbitrary operand strides,
// so forward (X W^T), weight gradients (G^T H) and input gradients (G W)
// share it; the forward epilogue adds the bias and writes both Z and relu(Z).
#include "psr_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <random>
#include <vector>

struct psr_mlp {
    int d = 0, h = 0, m = 0;
    int64_t np = 0;               // number of parameters
    float* params = nullptr;      // packed W1 b1 W2 b2 W3 b3
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int64_t step = 0;
    // activations (resized on demand)
    int cap = 0;
    float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *L = nullptr;
    float *G1 = nullptr, *G2 = nullptr, *G3 = nullptr;
    float* loss_part = nullptr;
    int32_t* cnt = nullptr;
    int32_t* tc_err = nullptr;    // set when a tensor-core GEMM wait gave up
};

namespace psr {

struct MlpView {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};

static MlpView view(float* base, int d, int h, int m) {
    MlpView v;
    v.W1 = base;
    v.b1 = v.W1 + (int64_t)h * d;
    v.W2 = v.b1 + h;
    v.b2 = v.W2 + (int64_t)h * h;
    v.W3 = v.b2 + h;
    v.b3 = v.W3 + (int64_t)m * h;
    return v;
}

// C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]); A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj], C row-major with ldc.  relu_out (optional)
// receives max(C, 0).
// C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]); A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj], C row-major with ldc.  relu_out (optional)
// receives max(C, 0).
__global__ void __launch_bounds__(256) k_gemm_f32(int M, int N, int K, const float* __restrict__ A, int64_t sai,
                                                  int64_t sak, const float* __restrict__ B, int64_t sbk, int64_t sbj,
                                                  float* __restrict__ C, int64_t ldc, const float* __restrict__ bias,
                                                  float* __restrict__ relu_out) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, ii = e % 64;
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.f;
            const int gj = j0 + ii;
            Bs[kk][ii] = (gj < N && gk < K) ? B[gk * sbk + gj * sbj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
            for (int qi = 0; qi < 4; ++qi)
#pragma unroll
                for (int qj = 0; qj < 4; ++qj) acc[qi][qj] = fmaf(a[qi], b[qj], acc[qi][qj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int qi = 0; qi < 4; ++qi) {
        const int gi = i0 + ty * 4 + qi;
        if (gi >= M) continue;
#pragma unroll
        for (int qj = 0; qj < 4; ++qj) {
            const int gj = j0 + tx * 4 + qj;
            if (gj >= N) continue;
            float v = acc[qi][qj] + (bias ? bias[gj] : 0.f);
            C[gi * ldc + gj] = v;
            if (relu_out) relu_out[gi * ldc + gj] = fmaxf(v, 0.f);
        }
    }
}

void launch_gemm_tc(int M, int N, int K, const float* A, int64_t sai, int64_t sak, const float* B, int64_t sbk,
                    int64_t sbj, float* C, int64_t ldc, const float* bias, float* relu_out, int32_t* err,
                    cudaStream_t s);
int gemm_tc_prepare();

static int32_t* g_tc_err = nullptr;   // set by the network that launches (one flag per network)

static void gemm(int M, int N, int K, const float* A, int64_t sai, int64_t sak, const float* B, int64_t sbk,
                 int64_t sbj, float* C, int64_t ldc, const float* bias, float* relu_out, cudaStream_t s) {
    launch_gemm_tc(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, relu_out, g_tc_err, s);
}

// softmax cross-entropy: G = (softmax(L) - onehot(y)) / B, loss partials
__global__ void k_softmax_xent(const float* __restrict__ L, const int32_t* __restrict__ y, int Bn, int m,
                               float* __restrict__ G, float* __restrict__ part, int32_t* cnt, float* loss_out) {
    __shared__ float sh[32];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    float lsum = 0.f;
    for (int row = blockIdx.x * nw + wid; row < Bn; row += gridDim.x * nw) {
        const float* l = L + (int64_t)row * m;
        float mx = -3.0e38f;
        for (int j = lane; j < m; j += 32) mx = fmaxf(mx, l[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float se = 0.f;
        for (int j = lane; j < m; j += 32) se += expf(l[j] - mx);
        se = warp_sumf(se);
        const int yy = y[row];
        for (int j = lane; j < m; j += 32) {
            const float pj = expf(l[j] - mx) / se;
            G[(int64_t)row * m + j] = (pj - (j == yy ? 1.f : 0.f)) / (float)Bn;
        }
        if (lane == 0) lsum += -(l[yy] - mx - logf(se));
    }
    if (lane == 0) sh[wid] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += sh[w];
        part[blockIdx.x] = t;
        __threadfence();
        const int ticket = atomicAdd(cnt, 1);
        if (ticket == (int)gridDim.x - 1) {
            __threadfence();
            float tot = 0.f;
            for (int b = 0; b < (int)gridDim.x; ++b) tot += part[b];
            if (loss_out) *loss_out = tot / (float)Bn;
            *cnt = 0;
        }
    }
}

// G *= (Z > 0)
__global__ void k_relu_mask(float* __restrict__ G, const float* __restrict__ Z, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(Z[i] > 0.f)) G[i] = 0.f;
}

// bias gradient: column sums of G (B x n), one thread per column
__global__ void k_colsum(const float* __restrict__ G, int Bn, int n, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f;
    for (int b = 0; b < Bn; ++b) s += G[(int64_t)b * n + j];
    out[j] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_argmax(const float* __restrict__ L, int Bn, int m, int32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= Bn) return;
    const float* l = L + (int64_t)row * m;
    float best = -3.0e38f;
    int bi = m;
    for (int j = lane; j < m; j += 32)
        if (l[j] > best) { best = l[j]; bi = j; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) out[row] = (bi < m) ? bi : 0;
}

// Features: A_k / ||A_k||_F (row-major), log ||A_k||_F, log coef_k (0 without)
__global__ void k_features(const double* __restrict__ A, int npch, int p, const double* __restrict__ coef,
                           float* __restrict__ X) {
    const int lane = threadIdx.x & 31;
    const int pp = p * p;
    const int d = pp + 2;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < npch; k += (gridDim.x * blockDim.x) >> 5) {
        const double* a = A + (int64_t)k * pp;
        double s = 0.0;
        for (int e = lane; e < pp; e += 32) s = fma(a[e], a[e], s);
        s = warp_sum(s);
        const double fro = sqrt(s);
        float* x = X + (int64_t)k * d;
        for (int e = lane; e < pp; e += 32) x[e] = (float)(a[e] / fro);
        if (lane == 0) {
            x[pp] = (float)log(fro);
            x[pp + 1] = coef ? (float)log(coef[k]) : 0.f;
        }
    }
}

static int ensure_cap(psr_mlp* net, int Bn) {
    if (Bn <= net->cap) return PSR_OK;
    psr::AllocPause keep;                  // the network owns these beyond the calling setup
    for (float* p : {net->Z1, net->H1, net->Z2, net->H2, net->L, net->G1, net->G2, net->G3, net->loss_part}) psr::dev_free(p);
    psr::dev_free(net->cnt);
    const size_t bh = (size_t)Bn * net->h, bm = (size_t)Bn * net->m;
    if (psr::dev_alloc(&net->Z1, bh * 4) || psr::dev_alloc(&net->H1, bh * 4) || psr::dev_alloc(&net->Z2, bh * 4) ||
        psr::dev_alloc(&net->H2, bh * 4) || psr::dev_alloc(&net->L, bm * 4) || psr::dev_alloc(&net->G1, bh * 4) ||
        psr::dev_alloc(&net->G2, bh * 4) || psr::dev_alloc(&net->G3, bm * 4) || psr::dev_alloc(&net->loss_part, 1024 * 4) ||
        psr::dev_alloc(&net->cnt, 4)) {
        cudaGetLastError();
        net->cap = 0;
        set_error(nullptr, "MLP activation allocation failed");
        return PSR_ERR_OOM;
    }
    cudaMemset(net->cnt, 0, 4);
    cudaDeviceSynchronize();               // the zero is in place before any stream's kernel reads it
    net->cap = Bn;
    return PSR_OK;
}

static void forward(psr_mlp* net, const float* X, int Bn, cudaStream_t s) {
    const int d = net->d, h = net->h, m = net->m;
    g_tc_err = net->tc_err;
    MlpView P = view(net->params, d, h, m);
    gemm(Bn, h, d, X, d, 1, P.W1, 1, d, net->Z1, h, P.b1, net->H1, s);
    gemm(Bn, h, h, net->H1, h, 1, P.W2, 1, h, net->Z2, h, P.b2, net->H2, s);
    gemm(Bn, m, h, net->H2, h, 1, P.W3, 1, h, net->L, m, P.b3, nullptr, s);
}

static void backward(psr_mlp* net, const float* X, const int32_t* y, int Bn, float* loss_out, cudaStream_t s) {
    const int d = net->d, h = net->h, m = net->m;
    g_tc_err = net->tc_err;
    MlpView P = view(net->params, d, h, m);
    MlpView G = view(net->grads, d, h, m);
    const int nb = std::min(1024, (Bn + 7) / 8);
    count_launch();
    k_softmax_xent<<<nb, 256, 0, s>>>(net->L, y, Bn, m, net->G3, net->loss_part, net->cnt, loss_out);
    gemm(m, h, Bn, net->G3, 1, m, net->H2, h, 1, G.W3, h, nullptr, nullptr, s);        // G3^T H2
    count_launch();
    k_colsum<<<(m + 127) / 128, 128, 0, s>>>(net->G3, Bn, m, G.b3);
    gemm(Bn, h, m, net->G3, m, 1, P.W3, h, 1, net->G2, h, nullptr, nullptr, s);        // G3 W3
    const int64_t bh = (int64_t)Bn * h;
    const int eb = (int)std::min<int64_t>((bh + 255) / 256, 152 * 16);
    count_launch();
    k_relu_mask<<<eb, 256, 0, s>>>(net->G2, net->Z2, bh);
    gemm(h, h, Bn, net->G2, 1, h, net->H1, h, 1, G.W2, h, nullptr, nullptr, s);       // G2^T H1
    count_launch();
    k_colsum<<<(h + 127) / 128, 128, 0, s>>>(net->G2, Bn, h, G.b2);
    gemm(Bn, h, h, net->G2, h, 1, P.W2, h, 1, net->G1, h, nullptr, nullptr, s);        // G2 W2
    count_launch();
    k_relu_mask<<<eb, 256, 0, s>>>(net->G1, net->Z1, bh);
    gemm(h, d, Bn, net->G1, 1, h, X, d, 1, G.W1, d, nullptr, nullptr, s);             // G1^T X
    count_launch();
    k_colsum<<<(h + 127) / 128, 128, 0, s>>>(net->G1, Bn, h, G.b1);
}

}  // namespace psr

using namespace psr;

extern "C" {

int psr_mlp_create(int32_t in_dim, int32_t hidden, int32_t classes, psr_mlp** out) {
    if (!out || in_dim < 1 || hidden < 1 || classes < 1) { set_error(nullptr, "invalid MLP shape"); return PSR_ERR_INVALID_ARG; }
    psr::AllocPause keep;                  // the network outlives any call that creates it
    psr_mlp* net = new psr_mlp();
    net->d = in_dim;
    net->h = hidden;
    net->m = classes;
    net->np = (int64_t)hidden * in_dim + hidden + (int64_t)hidden * hidden + hidden + (int64_t)classes * hidden + classes;
    const size_t b = (size_t)net->np * 4;
    if (psr::dev_alloc(&net->params, b) || psr::dev_alloc(&net->grads, b) || psr::dev_alloc(&net->adam_m, b) ||
        psr::dev_alloc(&net->adam_v, b)) {
        cudaGetLastError();
        psr::dev_free(net->params); psr::dev_free(net->grads); psr::dev_free(net->adam_m); psr::dev_free(net->adam_v);
        delete net;
        set_error(nullptr, "MLP parameter allocation failed");
        return PSR_ERR_OOM;
    }
    cudaMemset(net->params, 0, b);
    cudaMemset(net->adam_m, 0, b);
    cudaMemset(net->adam_v, 0, b);
    if (psr::dev_alloc(&net->tc_err, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        psr_mlp_destroy(net);
        set_error(nullptr, "MLP allocation failed");
        return PSR_ERR_OOM;
    }
    cudaMemset(net->tc_err, 0, sizeof(int32_t));
    cudaDeviceSynchronize();               // the zeros are in place before any stream's kernel reads them
    int rc = gemm_tc_prepare();
    if (rc != PSR_OK) { psr_mlp_destroy(net); return rc; }
    *out = net;
    return PSR_OK;
}

int64_t psr_mlp_num_params(const psr_mlp* net) { return net ? net->np : 0; }

int psr_mlp_set_params(psr_mlp* net, const float* packed, void* stream) {
    if (!net || !packed) { set_error(nullptr, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    PSR_CUDA(nullptr, cudaMemcpyAsync(net->params, packed, (size_t)net->np * 4, cudaMemcpyDeviceToDevice, s));
    PSR_CUDA(nullptr, cudaMemsetAsync(net->adam_m, 0, (size_t)net->np * 4, s));
    PSR_CUDA(nullptr, cudaMemsetAsync(net->adam_v, 0, (size_t)net->np * 4, s));
    net->step = 0;
    return PSR_OK;
}

int psr_mlp_get_params(const psr_mlp* net, float* packed, void* stream) {
    if (!net || !packed) { set_error(nullptr, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    PSR_CUDA(nullptr, cudaMemcpyAsync(packed, net->params, (size_t)net->np * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PSR_OK;
}

int psr_mlp_loss_grad(psr_mlp* net, const float* X, const int32_t* y, int32_t batch, float* loss, float* grads,
                      void* stream) {
    if (!net || !X || !y || batch < 1) { set_error(nullptr, "invalid MLP arguments"); return PSR_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_cap(net, batch);
    if (rc != PSR_OK) return rc;
    forward(net, X, batch, s);
    backward(net, X, y, batch, loss, s);
    if (grads) PSR_CUDA(nullptr, cudaMemcpyAsync(grads, net->grads, (size_t)net->np * 4, cudaMemcpyDeviceToDevice, s));
    PSR_CUDA(nullptr, cudaGetLastError());
    return PSR_OK;
}

int psr_mlp_train_step(psr_mlp* net, const float* X, const int32_t* y, int32_t batch, float lr, float* loss,
                       void* stream) {
    int rc = psr_mlp_loss_grad(net, X, y, batch, loss, nullptr, stream);
    if (rc != PSR_OK) return rc;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
    const int blocks = (int)std::min<int64_t>((net->np + 255) / 256, 152 * 16);
    count_launch();
    k_adam<<<blocks, 256, 0, (cudaStream_t)stream>>>(net->params, net->grads, net->adam_m, net->adam_v, net->np, lr,
                                                     b1, b2, 1e-8f, c1, c2);
    PSR_CUDA(nullptr, cudaGetLastError());
    return PSR_OK;
}

int psr_mlp_predict(psr_mlp* net, const float* X, int32_t batch, int32_t* cls, float* logits, void* stream) {
    if (!net || !X || batch < 1) { set_error(nullptr, "invalid MLP arguments"); return PSR_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_cap(net, batch);
    if (rc != PSR_OK) return rc;
    forward(net, X, batch, s);
    if (cls) {
        count_launch();
        k_argmax<<<(batch * 32 + 255) / 256, 256, 0, s>>>(net->L, batch, net->m, cls);
    }
    if (logits) PSR_CUDA(nullptr, cudaMemcpyAsync(logits, net->L, (size_t)batch * net->m * 4, cudaMemcpyDeviceToDevice, s));
    PSR_CUDA(nullptr, cudaGetLastError());
    return PSR_OK;
}

void psr_mlp_destroy(psr_mlp* net) {
    if (!net) return;
    for (float* p : {net->params, net->grads, net->adam_m, net->adam_v, net->Z1, net->H1, net->Z2, net->H2, net->L,
                     net->G1, net->G2, net->G3, net->loss_part})
        psr::dev_free(p);
    psr::dev_free(net->cnt);
    psr::dev_free(net->tc_err);
    delete net;
}

int psr_features(const double* A, int32_t n_patches, int32_t p, const double* coef, float* X, void* stream) {
    if (!A || !X || n_patches < 0 || p < 1) { set_error(nullptr, "invalid feature arguments"); return PSR_ERR_INVALID_ARG; }
    if (n_patches == 0) return PSR_OK;
    const int blocks = std::min((n_patches * 32 + 255) / 256, 152 * 16);
    count_launch();
    k_features<<<blocks, 256, 0, (cudaStream_t)stream>>>(A, n_patches, p, coef, X);
    PSR_CUDA(nullptr, cudaGetLastError());
    return PSR_OK;
}

void psr_default_train_opts(psr_train_opts* t) {
    if (!t) return;
    t->hidden = 256;
    t->epochs = 300;
    t->lr = 1e-3f;
    t->train_fraction = 1.0f;
    t->seed = 0;
}

psr_mlp* psr_ctx_mlp(psr_ctx* ctx) { return ctx ? ctx->mlp : nullptr; }

int psr_mlp_train(psr_ctx* ctx, const float* features, const psr_train_opts* topts, void* stream,
                  psr_train_info* info) {
    using namespace psr;
    if (!ctx) { set_error(nullptr, "ctx is NULL"); return PSR_ERR_INVALID_ARG; }
    psr_train_opts t;
    if (topts) t = *topts; else psr_default_train_opts(&t);
    if (ctx->groups.size() != 1 || ctx->groups[0].p > 32 || !ctx->groups[0].dbA || ctx->m_p < 1 || t.hidden < 1 ||
        t.epochs < 0 || !(t.lr > 0.f) || !(t.train_fraction > 0.f) || t.train_fraction > 1.f) {
        set_error(ctx, "psr_mlp_train needs a one-size (p <= 32) setup with a database and valid training options");
        return PSR_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const int p = ctx->groups[0].p;
    const int n = ctx->n_patches;
    const int d = p * p + 2;
    const int n_train = std::max(1, std::min(n, (int)std::ceil((double)t.train_fraction * n)));
    float* X = nullptr;
    double* A = nullptr;
    float* loss = nullptr;
    int32_t* pred = nullptr;
    psr_mlp* net = nullptr;
    auto done = [&](int rc) {
        psr::dev_free(X);
        psr::dev_free(A);
        psr::dev_free(loss);
        psr::dev_free(pred);
        if (rc != PSR_OK && net) psr_mlp_destroy(net);
        return rc;
    };
    if (!features) {
        // features from the context's patch matrices (extracted again from its CSR and map copies)
        if (psr::dev_alloc(&A, sizeof(double) * (size_t)n * p * p) != cudaSuccess ||
            psr::dev_alloc(&X, sizeof(float) * (size_t)n * d) != cudaSuccess) {
            cudaGetLastError();
            set_error(ctx, "out of device memory for the training features");
            return done(PSR_ERR_OOM);
        }
        int rc = launch_extract(ctx->rowptr, ctx->colidx, ctx->vals, ctx->offsets, ctx->dofs, ctx->mat_off, n, 0,
                                (int64_t)n * p, A, s);
        if (rc != PSR_OK) return done(rc);
        if ((rc = psr_features(A, n, p, nullptr, X, stream)) != PSR_OK) return done(rc);
        features = X;
    }
    int rc = psr_mlp_create(d, t.hidden, ctx->m_p, &net);
    if (rc != PSR_OK) { net = nullptr; return done(rc); }
    {
        // initial weights N(0, 1/fan_in), biases 0 (host generator from the seed)
        std::vector<float> w((size_t)net->np, 0.f);
        std::mt19937_64 gen(t.seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        MlpView v = view(w.data(), d, t.hidden, ctx->m_p);
        auto fill = [&](float* W, int64_t cnt, int fan_in) {
            const double sc = 1.0 / std::sqrt((double)fan_in);
            for (int64_t i = 0; i < cnt; ++i) W[i] = (float)(nd(gen) * sc);
        };
        fill(v.W1, (int64_t)t.hidden * d, d);
        fill(v.W2, (int64_t)t.hidden * t.hidden, t.hidden);
        fill(v.W3, (int64_t)ctx->m_p * t.hidden, t.hidden);
        PSR_CUDA(ctx, cudaMemcpyAsync(net->grads, w.data(), (size_t)net->np * 4, cudaMemcpyHostToDevice, s));
        if ((rc = psr_mlp_set_params(net, net->grads, stream)) != PSR_OK) return done(rc);
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
    }
    if (psr::dev_alloc(&loss, sizeof(float)) != cudaSuccess || psr::dev_alloc(&pred, sizeof(int32_t) * n_train) != cudaSuccess) {
        cudaGetLastError();
        set_error(ctx, "out of device memory for the training state");
        return done(PSR_ERR_OOM);
    }
    for (int e = 0; e < t.epochs; ++e)
        if ((rc = psr_mlp_train_step(net, features, ctx->phi, n_train, t.lr, loss, stream)) != PSR_OK) return done(rc);
    if ((rc = psr_mlp_predict(net, features, n_train, pred, nullptr, stream)) != PSR_OK) return done(rc);
    std::vector<int32_t> hp(n_train), hy(n_train);
    float hl = 0.f;
    PSR_CUDA(ctx, cudaMemcpyAsync(hp.data(), pred, sizeof(int32_t) * n_train, cudaMemcpyDeviceToHost, s));
    PSR_CUDA(ctx, cudaMemcpyAsync(hy.data(), ctx->phi, sizeof(int32_t) * n_train, cudaMemcpyDeviceToHost, s));
    PSR_CUDA(ctx, cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    int32_t herr = 0;
    PSR_CUDA(ctx, cudaMemcpy(&herr, net->tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (herr) { set_error(ctx, "a tensor-core GEMM wait gave up during training"); return done(PSR_ERR_TIMEOUT); }
    int hits = 0;
    for (int i = 0; i < n_train; ++i) hits += hp[i] == hy[i];
    if (ctx->mlp) psr_mlp_destroy(ctx->mlp);
    ctx->mlp = net;
    ctx->mlp_classes = ctx->m_p;
    if (info) {
        info->n_train = n_train;
        info->classes = ctx->m_p;
        info->final_loss = t.epochs > 0 ? hl : 0.f;
        info->train_accuracy = (float)hits / (float)n_train;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return done(PSR_OK);
}

}  // extern "C"
