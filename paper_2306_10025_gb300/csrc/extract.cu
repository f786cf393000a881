// Step a1 / a1': input validation, patch extraction A_k = V_k A V_k^T and the
// multiplicity weights W = (sum_l V_l^T V_l)^{-1} (section 2 of the paper).
#include "psr_internal.cuh"

namespace psr {

// Rows must have nondecreasing rowptr, strictly increasing columns in [0, n).
__global__ void k_validate_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                               int32_t n, int64_t nnz, int32_t* status) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row = warp; row < n; row += nwarps) {
        int rs = rowptr[row], re = rowptr[row + 1];
        bool bad = (re < rs) || rs < 0 || (int64_t)re > nnz;
        if (!bad) {
            for (int e = rs + lane; e < re; e += 32) {
                int c = colidx[e];
                if (c < 0 || c >= n) bad = true;
                if (e > rs && colidx[e - 1] >= c) bad = true;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_UNSORTED);
    }
}

__global__ void k_validate_map(const int32_t* __restrict__ offsets, int32_t n_patches,
                               const int32_t* __restrict__ dofs, int64_t total, int32_t n,
                               int32_t* status) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < total; i += stride) {
        int d = dofs[i];
        if (d < 0 || d >= n) atomicOr(status, ST_OOB);
    }
    if (offsets) {
        for (int64_t k = tid; k < n_patches; k += stride)
            if (offsets[k + 1] < offsets[k] || offsets[k] < 0) atomicOr(status, ST_OOB);
    }
}

int validate_inputs(psr_ctx* ctx, const psr_csr* A, const int32_t* offsets, const int32_t* dofs,
                    int32_t n_patches, int64_t total_dofs, int32_t* status, cudaStream_t s) {
    int blocks = (int)((A->n + 7) / 8);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    count_launch(); k_validate_csr<<<blocks, 256, 0, s>>>(A->rowptr, A->colidx, A->n, A->nnz, status);
    PSR_CHECK_LAUNCH(ctx, "k_validate_csr");
    int b2 = (int)((total_dofs + 255) / 256);
    if (b2 > 4096) b2 = 4096;
    if (b2 < 1) b2 = 1;
    count_launch(); k_validate_map<<<b2, 256, 0, s>>>(offsets, n_patches, dofs, total_dofs, A->n, status);
    PSR_CHECK_LAUNCH(ctx, "k_validate_map");
    return PSR_OK;
}

// One warp per patch k, its local rows i in turn: A_k[i][j] = A(dofs_k[i],
// dofs_k[j]), found by binary search of the sorted CSR row; an absent entry
// is 0.  offsets == nullptr means every patch has pmax DOFs.  (A warp per
// (patch, row) had to find its patch by a binary search of the offsets, 17
// dependent loads per row on the 3D Stokes 48^3 map.)
__global__ void k_extract(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                          const double* __restrict__ vals, const int32_t* __restrict__ offsets,
                          const int32_t* __restrict__ dofs, const int64_t* __restrict__ mat_off,
                          int32_t n_patches, int32_t pmax, int64_t total, double* __restrict__ out) {
    (void)total;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // a warp per patch (its rows in turn, the lanes over its columns)
    for (int64_t k = warp; k < n_patches; k += nwarps) {
        const int start = offsets ? offsets[k] : (int)(k * pmax);
        const int pk = offsets ? offsets[k + 1] - start : pmax;
        const int64_t base0 = offsets ? mat_off[k] : k * (int64_t)pmax * pmax;
        for (int i = 0; i < pk; ++i) {
            const int row = dofs[start + i];
            const int rs = rowptr[row], re = rowptr[row + 1];
            const int64_t base = base0 + (int64_t)i * pk;
            for (int j = lane; j < pk; j += 32) {
                const int col = dofs[start + j];
                int lo = rs, hi = re;                   // first e with colidx[e] >= col
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (colidx[mid] < col) lo = mid + 1; else hi = mid;
                }
                out[base + j] = (lo < re && colidx[lo] == col) ? vals[lo] : 0.0;
            }
        }
    }
}

int launch_extract(const int32_t* rowptr, const int32_t* colidx, const double* vals,
                   const int32_t* offsets, const int32_t* dofs, const int64_t* mat_off,
                   int32_t n_patches, int32_t pmax, int64_t total, double* A_out, cudaStream_t s) {
    int64_t warps_needed = n_patches;
    int64_t blocks = (warps_needed * 32 + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    count_launch(); k_extract<<<(int)blocks, 256, 0, s>>>(rowptr, colidx, vals, offsets, dofs, mat_off, n_patches,
                                          pmax, total, A_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_extract");
    return PSR_OK;
}

__global__ void k_count(const int32_t* __restrict__ dofs, int64_t total, int32_t* mult) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < total; i += stride) atomicAdd(&mult[dofs[i]], 1);
}

// W_ii = 1 / mult_i (exactly the correctly rounded quotient) and its square
// root for the symmetric weighting.
__global__ void k_weights(const int32_t* __restrict__ mult, int32_t n, double* W, double* sqrtW,
                          int32_t* status) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += stride) {
        int m = mult[i];
        if (m == 0) {
            atomicOr(status, ST_UNCOVERED);
            if (W) W[i] = 0.0;
            if (sqrtW) sqrtW[i] = 0.0;
            continue;
        }
        double w = 1.0 / (double)m;
        if (W) W[i] = w;
        if (sqrtW) sqrtW[i] = sqrt(w);
    }
}

int launch_multiplicity(const int32_t* dofs, int64_t total, int32_t n, int32_t* mult, double* W,
                        double* sqrtW, int32_t* status, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(mult, 0, sizeof(int32_t) * (size_t)n, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "memset mult");
    int b = (int)((total + 255) / 256);
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    count_launch(); k_count<<<b, 256, 0, s>>>(dofs, total, mult);
    int b2 = (n + 255) / 256;
    if (b2 > 8192) b2 = 8192;
    if (b2 < 1) b2 = 1;
    count_launch(); k_weights<<<b2, 256, 0, s>>>(mult, n, W, sqrtW, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_weights");
    return PSR_OK;
}

}  // namespace psr
