// The two-level combination preconditioner of Eq. (2):
//     M_combo^{-1} = M^{-1} + P0 A0^{-1} R0,   R0 = P0^T,   A0 = R0 A P0,
// M^{-1} the patch method (Eq. 3), P0 the interpolation from a low-order
// representation (the caller's n x n0 CSR), and a direct solve with the
// Galerkin operator A0 in place of the first-order AMG (as in Experiment 1).
//
// Setup: R0 = P0^T by a counting transpose, A0 assembled densely on the
// device (one thread per row of A scatters its entries through the at most
// few interpolation weights of the two DOFs), then inverted in place by
// Gauss-Jordan without pivoting (A0 is symmetric positive definite for a
// symmetric positive definite A and a full-rank P0); A0^{-1} is kept dense.
// Apply: rc = R0 r (CSR, warp per row), yc = A0^{-1} rc (dense, warp per
// row), z += P0 yc (CSR), after the patch sweep.
#include "psr_internal.cuh"

#include <vector>

namespace psr {

struct Coarse {
    int n0 = 0;
    int32_t *prow = nullptr, *pcol = nullptr;     // P0 (n x n0)
    double* pval = nullptr;
    int32_t *rrow = nullptr, *rcol = nullptr;     // R0 = P0^T (n0 x n)
    double* rval = nullptr;
    double* Minv = nullptr;                       // A0^{-1}, n0 x n0 row-major
    double* rc = nullptr;                         // R0 r
    double* yc = nullptr;                         // A0^{-1} R0 r
    double* col = nullptr;                        // Gauss-Jordan scratch column
};

// A0 += sum over the entries a_ij of A of P0[i, :]^T a_ij P0[j, :]
__global__ void k_galerkin(const int32_t* __restrict__ arow, const int32_t* __restrict__ acol,
                           const double* __restrict__ aval, int n, const int32_t* __restrict__ prow,
                           const int32_t* __restrict__ pcol, const double* __restrict__ pval, int n0,
                           double* __restrict__ A0) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int q = arow[i]; q < arow[i + 1]; ++q) {
            const int j = acol[q];
            const double a = aval[q];
            for (int u = prow[i]; u < prow[i + 1]; ++u) {
                const double pa = pval[u] * a;
                const int64_t rbase = (int64_t)pcol[u] * n0;
                for (int v = prow[j]; v < prow[j + 1]; ++v) atomicAdd(&A0[rbase + pcol[v]], pa * pval[v]);
            }
        }
    }
}

// Gauss-Jordan step k on M (n0 x n0), in place: row k scaled by 1/M[k][k]
// (M[k][k] := 1/M[k][k]), the old column k saved and zeroed elsewhere.  One
// block: every thread reads the pivot before it is overwritten.
__global__ void k_gj_pivot(double* __restrict__ M, int n0, int k, double* __restrict__ col) {
    const double piv = M[(int64_t)k * n0 + k];
    const double inv = 1.0 / piv;
    for (int t = threadIdx.x; t < n0; t += blockDim.x) {
        if (t != k) {
            col[t] = M[(int64_t)t * n0 + k];
            M[(int64_t)t * n0 + k] = 0.0;
            M[(int64_t)k * n0 + t] *= inv;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        col[k] = 0.0;
        M[(int64_t)k * n0 + k] = inv;
    }
}

// M[i][j] -= col[i] * M[k][j] for every i != k (col[k] = 0)
__global__ void k_gj_update(double* __restrict__ M, int n0, int k, const double* __restrict__ col) {
    const int64_t total = (int64_t)n0 * n0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n0), j = (int)(e - (int64_t)i * n0);
        const double c = col[i];
        if (c != 0.0) M[e] -= c * M[(int64_t)k * n0 + j];
    }
}

// y = M x (CSR, one warp per row), add: y += M x
__global__ void k_csr_mv(const int32_t* __restrict__ row, const int32_t* __restrict__ colx,
                         const double* __restrict__ val, const double* __restrict__ x, int nrows,
                         double* __restrict__ y, int add, const int32_t* __restrict__ stop) {
    if (stop && *stop) return;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nrows; i += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (int q = row[i] + lane; q < row[i + 1]; q += 32) s = fma(val[q], x[colx[q]], s);
        s = warp_sum(s);
        if (lane == 0) y[i] = add ? y[i] + s : s;
    }
}

// y = M x, M dense n0 x n0 row-major (one warp per row, four chains per lane)
__global__ void k_dense_mv(const double* __restrict__ M, const double* __restrict__ x, int n0,
                           double* __restrict__ y, const int32_t* __restrict__ stop) {
    if (stop && *stop) return;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n0; i += (gridDim.x * blockDim.x) >> 5) {
        const double* m = M + (int64_t)i * n0;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = lane;
        for (; j + 96 < n0; j += 128) {
            s0 = fma(m[j], x[j], s0);
            s1 = fma(m[j + 32], x[j + 32], s1);
            s2 = fma(m[j + 64], x[j + 64], s2);
            s3 = fma(m[j + 96], x[j + 96], s3);
        }
        for (; j < n0; j += 32) s0 = fma(m[j], x[j], s0);
        const double s = warp_sum((s0 + s1) + (s2 + s3));
        if (lane == 0) y[i] = s;
    }
}

void coarse_free(psr_ctx* ctx) {
    Coarse* c = ctx->coarse;
    if (!c) return;
    for (void* p : {(void*)c->prow, (void*)c->pcol, (void*)c->pval, (void*)c->rrow, (void*)c->rcol, (void*)c->rval,
                    (void*)c->Minv, (void*)c->rc, (void*)c->yc, (void*)c->col})
        psr::dev_free(p);
    delete c;
    ctx->coarse = nullptr;
}

int coarse_apply(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s) {
    Coarse* c = ctx->coarse;
    if (!c) return PSR_OK;
    const int wpb = 8;
    const int b0 = std::max(1, std::min((c->n0 + wpb - 1) / wpb, 152 * 16));
    const int bn = std::max(1, std::min((ctx->n + wpb - 1) / wpb, 152 * 16));
    count_launch(); k_csr_mv<<<b0, wpb * 32, 0, s>>>(c->rrow, c->rcol, c->rval, r, c->n0, c->rc, 0, stop);
    count_launch(); k_dense_mv<<<b0, wpb * 32, 0, s>>>(c->Minv, c->rc, c->n0, c->yc, stop);
    count_launch(); k_csr_mv<<<bn, wpb * 32, 0, s>>>(c->prow, c->pcol, c->pval, c->yc, ctx->n, z, 1, stop);
    PSR_CHECK_LAUNCH(ctx, "coarse correction");
    return PSR_OK;
}

}  // namespace psr

using namespace psr;

extern "C" int psr_set_coarse(psr_ctx* ctx, const psr_csr_rect* P0, void* stream) {
    if (!ctx || !P0 || !P0->rowptr || (P0->nnz > 0 && (!P0->colidx || !P0->vals))) {
        set_error(ctx, "NULL argument");
        return PSR_ERR_INVALID_ARG;
    }
    const int n = ctx->n, n0 = P0->n_cols;
    if (P0->n_rows != n || n0 < 1 || n0 > PSR_COARSE_MAX || P0->nnz < 0) {
        set_error(ctx, "P0 must have n rows and 1..PSR_COARSE_MAX columns");
        return PSR_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    coarse_free(ctx);
    if (ctx->g_cycle) {                       // the captured cycle does not hold the correction
        cudaGraphExecDestroy(ctx->g_cycle);
        ctx->g_cycle = nullptr;
    }
    Coarse* c = new Coarse();
    ctx->coarse = c;
    c->n0 = n0;
    const int64_t nnz = P0->nnz;
    // host copy of P0: checked, transposed
    std::vector<int32_t> hr((size_t)n + 1), hc((size_t)nnz);
    std::vector<double> hv((size_t)nnz);
    PSR_CUDA(ctx, cudaMemcpy(hr.data(), P0->rowptr, sizeof(int32_t) * hr.size(), cudaMemcpyDeviceToHost));
    if (nnz > 0) {
        PSR_CUDA(ctx, cudaMemcpy(hc.data(), P0->colidx, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost));
        PSR_CUDA(ctx, cudaMemcpy(hv.data(), P0->vals, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost));
    }
    bool ok = hr[0] == 0 && hr[n] == nnz;
    for (int i = 0; ok && i < n; ++i) ok = hr[i + 1] >= hr[i];
    for (int64_t q = 0; ok && q < nnz; ++q) ok = hc[q] >= 0 && hc[q] < n0;
    if (!ok) {
        coarse_free(ctx);
        set_error(ctx, "P0 is not a valid CSR matrix");
        return PSR_ERR_INVALID_ARG;
    }
    std::vector<int32_t> tr((size_t)n0 + 1, 0), tc((size_t)nnz);
    std::vector<double> tv((size_t)nnz);
    for (int64_t q = 0; q < nnz; ++q) ++tr[(size_t)hc[q] + 1];
    for (int a = 0; a < n0; ++a) tr[a + 1] += tr[a];
    {
        std::vector<int32_t> fill(tr.begin(), tr.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int q = hr[i]; q < hr[i + 1]; ++q) {
                const int32_t at = fill[hc[q]]++;
                tc[at] = i;
                tv[at] = hv[q];
            }
    }
    auto up = [&](auto** dst, const auto& src) -> int {
        using T = typename std::remove_reference<decltype(src)>::type::value_type;
        PSR_CUDA(ctx, psr::dev_alloc(dst, sizeof(T) * std::max<size_t>(src.size(), 1)));
        if (!src.empty()) PSR_CUDA(ctx, cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
        return PSR_OK;
    };
    int rc = PSR_OK;
    if ((rc = up(&c->prow, hr)) || (rc = up(&c->pcol, hc)) || (rc = up(&c->pval, hv)) || (rc = up(&c->rrow, tr)) ||
        (rc = up(&c->rcol, tc)) || (rc = up(&c->rval, tv))) {
        coarse_free(ctx);
        return rc;
    }
    const size_t mbytes = sizeof(double) * (size_t)n0 * n0;
    if (psr::dev_alloc(&c->Minv, mbytes) != cudaSuccess) {
        cudaGetLastError();
        coarse_free(ctx);
        set_error(ctx, "out of device memory for the coarse inverse");
        return PSR_ERR_OOM;
    }
    PSR_CUDA(ctx, psr::dev_alloc(&c->rc, sizeof(double) * n0));
    PSR_CUDA(ctx, psr::dev_alloc(&c->yc, sizeof(double) * n0));
    PSR_CUDA(ctx, psr::dev_alloc(&c->col, sizeof(double) * n0));
    PSR_CUDA(ctx, cudaMemsetAsync(c->Minv, 0, mbytes, s));
    count_launch();
    k_galerkin<<<std::max(1, std::min((n + 255) / 256, 152 * 8)), 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, n,
                                                                            c->prow, c->pcol, c->pval, n0, c->Minv);
    const int ub = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n0 * n0 + 255) / 256, 152 * 32));
    for (int k = 0; k < n0; ++k) {
        count_launch(); k_gj_pivot<<<1, 1024, 0, s>>>(c->Minv, n0, k, c->col);
        count_launch(); k_gj_update<<<ub, 256, 0, s>>>(c->Minv, n0, k, c->col);
    }
    PSR_CHECK_LAUNCH(ctx, "coarse operator");
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    return PSR_OK;
}
