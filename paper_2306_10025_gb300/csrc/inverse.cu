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

int launch_batched_inverse_block(const double* A, int64_t stride_in, const int32_t* index, int32_t batch, int32_t p,
                                 double* Ainv, int64_t stride_out, int32_t* singular, cudaStream_t s);

int launch_batched_inverse(const double* A, int64_t stride_in, const int32_t* index, int32_t batch,
                           int32_t p, double* Ainv, int64_t stride_out, int32_t* singular,
                           cudaStream_t s) {
    if (batch <= 0) return PSR_OK;
    if (p < 1 || p > 128) return PSR_ERR_INVALID_ARG;
    if (p > 32) return launch_batched_inverse_block(A, stride_in, index, batch, p, Ainv, stride_out, singular, s);
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

namespace psr {

// Larger patches (p > 32): one block of 128 threads per matrix, thread t owns
// column t.  The warp kernel leaves at most three matrices of 89 x 89 per SM
// (65 KB of shared memory each) with one warp apiece, too few warps to keep
// the FP64 pipe busy (27 % of its peak on the 3D Stokes patches); here each
// of those matrices is worked on by four warps.  Same arithmetic as
// gj_invert_warp: partial pivoting (largest |entry|, lowest row on ties), the
// pivot row divided by the pivot, every other row updated with one FMA per
// entry, the interchanges undone on the columns at the end.
constexpr int INV_BT = 128;

__host__ __device__ inline size_t inv_block_bytes(int p) {
    return ((size_t)p * (p + 1) + p + 16) * 8 + (size_t)p * 4 + 64;
}

__global__ void __launch_bounds__(INV_BT) k_batched_inverse_block(const double* __restrict__ A, int64_t stride_in,
                                                                  const int32_t* __restrict__ index, int32_t batch,
                                                                  int32_t p, double* __restrict__ Ainv,
                                                                  int64_t stride_out, int32_t* __restrict__ singular) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    const int t = threadIdx.x;
    const int lane = t & 31, wid = t >> 5;
    double* S = reinterpret_cast<double*>(smem);
    double* colk = S + (size_t)p * ld;
    double* red = colk + p;                       // 4 values + 4 indices (as doubles) + amax
    int* swaps = reinterpret_cast<int*>(red + 16);
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        const int64_t src = index ? (int64_t)index[b] : b;
        const double* a = A + src * stride_in;
        double amax = 0.0;
        for (int e = t; e < p * p; e += INV_BT) {
            const double v = a[e];
            S[(e / p) * ld + (e % p)] = v;
            amax = fmax(amax, fabs(v));
        }
        amax = warp_max(amax);
        if (lane == 0) red[8 + wid] = amax;
        __syncthreads();
        amax = fmax(fmax(red[8], red[9]), fmax(red[10], red[11]));
        const double thresh = (double)p * 0x1p-53 * amax;
        bool sing = !(amax > 0.0);
        for (int k = 0; k < p; ++k) {
            __syncthreads();                      // column k as the previous step left it
            // pivot: largest |S[i][k]|, i >= k, lowest row on ties
            double best = -1.0;
            int bi = p;
            if (t >= k && t < p) { best = fabs(S[t * ld + k]); bi = t; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { red[wid] = best; red[4 + wid] = (double)bi; }
            __syncthreads();
            best = red[0];
            bi = (int)red[4];
            for (int w = 1; w < 4; ++w) {
                const double ob = red[w];
                const int oi = (int)red[4 + w];
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            const int piv = (bi < p) ? bi : k;    // an all-NaN column has no valid pivot
            if (!(best > thresh)) sing = true;
            if (t < p && piv != k) {              // rows k <-> piv in my column
                const double x = S[k * ld + t];
                S[k * ld + t] = S[piv * ld + t];
                S[piv * ld + t] = x;
            }
            if (t == 0) swaps[k] = piv;
            __syncthreads();
            if (t < p) colk[t] = S[t * ld + k];
            __syncthreads();
            double pv = colk[k];
            if (pv == 0.0) pv = 1.0;              // singular: keep going, result discarded
            if (t < p) {
                const double rj = (t == k ? 1.0 : S[k * ld + t]) / pv;
                for (int i = 0; i < p; ++i) {
                    if (i == k) continue;
                    const double x = (t == k) ? 0.0 : S[i * ld + t];
                    S[i * ld + t] = fma(-colk[i], rj, x);
                }
                S[k * ld + t] = rj;
            }
        }
        __syncthreads();
        // X = (P A)^{-1} = A^{-1} P^T  =>  A^{-1} = X P: swap columns back, last first
        for (int k = p - 1; k >= 0; --k) {
            const int piv = swaps[k];
            if (piv != k && t < p) {
                const double x = S[t * ld + k];
                S[t * ld + k] = S[t * ld + piv];
                S[t * ld + piv] = x;
            }
            __syncthreads();
        }
        double* out = Ainv + b * stride_out;
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        for (int e = t; e < p * p; e += INV_BT) out[e] = sing ? nanv : S[(e / p) * ld + (e % p)];
        if (singular && t == 0) singular[b] = sing ? 1 : 0;
        __syncthreads();
    }
}

int launch_batched_inverse_block(const double* A, int64_t stride_in, const int32_t* index, int32_t batch, int32_t p,
                                 double* Ainv, int64_t stride_out, int32_t* singular, cudaStream_t s) {
    const size_t smem = inv_block_bytes(p);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_batched_inverse_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "inverse smem attribute");
    }
    int64_t blocks = batch;
    if (blocks > 152 * 16) blocks = 152 * 16;
    count_launch();
    k_batched_inverse_block<<<(int)blocks, INV_BT, smem, s>>>(A, stride_in, index, batch, p, Ainv, stride_out, singular);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_batched_inverse_block");
    return PSR_OK;
}

}  // namespace psr
