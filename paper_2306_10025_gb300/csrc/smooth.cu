// The smoothing iteration of Experiment 3 (section 4): x <- x + omega M^-1 r
// with r = b - A x, repeated a given number of sweeps; M^-1 the patch method
// of Eq. (3) (plus the coarse term of Eq. (2) when one is set).  Each sweep:
// the residual from the SELL copy of A, the preconditioner apply, the update.
#include "psr_internal.cuh"

namespace psr {


// r = b - A x (SELL-32: one thread per row, all rows of a warp in one slice)
__global__ void __launch_bounds__(256) k_residual_sell(const int64_t* __restrict__ sptr,
                                                       const int32_t* __restrict__ scols,
                                                       const double* __restrict__ svals,
                                                       const int32_t* __restrict__ rowmap, const double* __restrict__ x,
                                                       const double* __restrict__ b, double* __restrict__ r, int n,
                                                       int nrows_pad) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows_pad) return;
    const int s = row >> 5, lane = row & 31;
    const int64_t o = sptr[s] + lane;
    const int width = (int)((sptr[s + 1] - sptr[s]) >> 5);
    double sum = 0.0;
    for (int k = 0; k < width; ++k) sum = fma(svals[o + 32 * (int64_t)k], x[scols[o + 32 * (int64_t)k]], sum);
    const int orow = rowmap ? rowmap[row] : (row < n ? row : -1);
    if (orow >= 0) r[orow] = b[orow] - sum;
}

__global__ void k_axpy(double* __restrict__ x, double a, const double* __restrict__ z, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = fma(a, z[i], x[i]);
}

}  // namespace psr

using namespace psr;

extern "C" int psr_smooth(psr_ctx* ctx, const double* b, double* x, double omega, int32_t sweeps, void* stream) {
    if (!ctx || !b || !x) { set_error(ctx, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    if (sweeps < 0 || !(omega == omega)) { set_error(ctx, "sweeps must be >= 0 and omega a number"); return PSR_ERR_INVALID_ARG; }
    KrylovWS& w = ctx->ws;
    if (!w.sell_ptr || !w.r || !w.z) { set_error(ctx, "context has no solve workspace"); return PSR_ERR_INVALID_ARG; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n = ctx->n, nrows_pad = w.nslices * 32;
    const int gb = std::max(1, std::min((n + 255) / 256, 152 * 8));
    for (int it = 0; it < sweeps; ++it) {
        count_launch();
        k_residual_sell<<<(nrows_pad + 255) / 256, 256, 0, s>>>(w.sell_ptr, w.sell_cols, w.sell_vals, w.sell_row, x, b,
                                                                 w.r, n, nrows_pad);
        int rc = sweep_apply_ex(ctx, w.r, w.z, nullptr, s);
        if (rc != PSR_OK) return rc;
        count_launch();
        k_axpy<<<gb, 256, 0, s>>>(x, omega, w.z, n);
    }
    PSR_CHECK_LAUNCH(ctx, "smoothing iteration");
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    return PSR_OK;
}
