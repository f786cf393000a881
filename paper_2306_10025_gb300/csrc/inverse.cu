// Step a2: batched explicit inverses of the stored patches (Eq. 1 needs
// A_k^{-1}; Exp. 3 factors the patches with GETRF).  FP64 always.
//
// One warp inverts one p x p matrix held in shared memory by in-place
// Gauss-Jordan elimination with partial pivoting (pivot = largest |entry| in
// the column, lowest row on ties -- the same pivots LU with partial pivoting
// takes), then undoes the row interchanges on the columns.  This costs p^3
// multiply-adds instead of the 2p^3 of LU + two triangular solves per column.
#include "psr_internal.cuh"
#include "dense.cuh"

namespace psr {

__host__ __device__ inline int inv_warp_bytes(int p) {
    return ((p * (p + 1) + p) * 8 + p * 4 + 15) & ~15;   // keeps every warp's base 16-byte aligned
}

// index == nullptr: matrix b is at A + b*stride_in; else at A + index[b]*stride_in.
__global__ void k_batched_inverse(const double* __restrict__ A, int64_t stride_in,
                                  const int32_t* __restrict__ index, int32_t batch, int32_t p,
                                  double* __restrict__ Ainv, int64_t stride_out,
                                  int32_t* __restrict__ singular) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int ld = p + 1;
    unsigned char* base = smem + (size_t)wid * inv_warp_bytes(p);
    double* S = reinterpret_cast<double*>(base);
    double* colk = S + p * ld;
    int* swaps = reinterpret_cast<int*>(colk + p);
    for (int64_t b = (int64_t)blockIdx.x * wpb + wid; b < batch; b += (int64_t)gridDim.x * wpb) {
        const int64_t src = index ? (int64_t)index[b] : b;
        const double* a = A + src * stride_in;
        for (int e = lane; e < p * p; e += 32) S[(e / p) * ld + (e % p)] = a[e];
        __syncwarp();
        bool sing = gj_invert_warp(S, p, ld, colk, swaps);
        double* out = Ainv + b * stride_out;
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        for (int e = lane; e < p * p; e += 32) out[e] = sing ? nanv : S[(e / p) * ld + (e % p)];
        if (singular && lane == 0) singular[b] = sing ? 1 : 0;
        __syncwarp();
    }
}

int launch_batched_inverse(const double* A, int64_t stride_in, const int32_t* index, int32_t batch,
                           int32_t p, double* Ainv, int64_t stride_out, int32_t* singular,
                           cudaStream_t s) {
    if (batch <= 0) return PSR_OK;
    if (p < 1 || p > 128) return PSR_ERR_INVALID_ARG;
    const int per = inv_warp_bytes(p);
    int wpb = (200 * 1024) / per;
    if (wpb > 8) wpb = 8;
    if (wpb < 1) wpb = 1;
    const size_t smem = (size_t)wpb * per;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_batched_inverse,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "inverse smem attribute");
    }
    int64_t blocks = (batch + wpb - 1) / wpb;
    if (blocks > 152 * 32) blocks = 152 * 32;
    count_launch(); k_batched_inverse<<<(int)blocks, wpb * 32, smem, s>>>(A, stride_in, index, batch, p, Ainv,
                                                         stride_out, singular);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_batched_inverse");
    return PSR_OK;
}

}  // namespace psr
