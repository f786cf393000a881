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
#include "pairs.cuh"

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
                                 double* Ainv, int64_t stride_out, int32_t* singular, cudaStream_t s,
                                 float2* pout = nullptr, int32_t* pexp = nullptr);

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

// Larger patches (p > 32): one block per matrix, thread t owns column t,
// 32 * ceil(p / 32) threads.  The warp kernel leaves at most three matrices of
// 89 x 89 per SM (65 KB of shared memory each) with one warp apiece, too few
// warps to keep the FP64 pipe busy (27 % of its peak on the 3D Stokes
// patches); here each of those matrices is worked on by three warps (96 and
// 128 threads per block measured the same).  Same arithmetic as
// gj_invert_warp: partial pivoting (largest |entry|, lowest row on ties), the
// pivot row divided by the pivot, every other row updated with one FMA per
// entry, the interchanges undone on the columns at the end.  Two block
// barriers per step: the warp owning column k+1 finds the next pivot right
// after that column's update (a shuffle reduction, ties to the lowest row),
// and column k itself is never swapped (it is overwritten by the
// step; the swapped copy the update needs is read from it in permuted order).
// 30,000 random 89 x 89 matrices: 49.0 ms, 68 % of the FP64 peak measured
// on this GPU (628 G FMA/s, an FMA-only kernel); the four-barrier form with a
// shuffle pivot search took 71.7 ms (47 %); results bitwise equal.  Three
// 89 x 89 blocks fit an SM, nine warps on its four schedulers, and an
// FMA-only kernel with that many warps reaches 80 % of the peak.
constexpr int INV_BT = 128;   // upper bound of the block size (p <= 128)

__host__ __device__ inline size_t inv_block_bytes(int p) {
    return ((size_t)p * (p + 1) + p + 16) * 8 + (size_t)p * 4 + 64;
}

// Order key of |x| for pivot search: the bits of |x| as an integer (monotone
// for non-negative doubles); NaN ranks below every number.
__device__ __forceinline__ long long abs_key(double x) {
    const long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
    return b > 0x7ff0000000000000LL ? -1LL : b;
}

// pout (may be NULL): instead of Ainv, write each inverse in the streamed
// sweep's FP64-pair layout -- column-major (hi, lo) FP32 pairs of B 2^-e with
// e the frexp exponent of max|B| (0 for a zero or singular matrix, whose
// entries are NaN), e to pexp -- without the FP64 round trip through memory.
// The pairs are split with integer operations (truncated, |error| < 2^-46
// |B|) where the separate conversion rounds (2^-48).
__global__ void __launch_bounds__(INV_BT) k_batched_inverse_block(const double* __restrict__ A, int64_t stride_in,
                                                                  const int32_t* __restrict__ index, int32_t batch,
                                                                  int32_t p, double* __restrict__ Ainv,
                                                                  int64_t stride_out, int32_t* __restrict__ singular,
                                                                  float2* __restrict__ pout,
                                                                  int32_t* __restrict__ pexp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    const int t = threadIdx.x;
    const int nt = blockDim.x;
    const int lane = t & 31, wid = t >> 5, nw = nt >> 5;
    double* S = reinterpret_cast<double*>(smem);
    double* colk = S + (size_t)p * ld;
    double* red = colk + p;                       // per-warp amax; [12] pivot |value|; [13] pivot row
    int* swaps = reinterpret_cast<int*>(red + 16);
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        const int64_t src = index ? (int64_t)index[b] : b;
        const double* a = A + src * stride_in;
        double amax = 0.0;
        for (int e = t; e < p * p; e += nt) {
            const double v = a[e];
            S[(e / p) * ld + (e % p)] = v;
            amax = fmax(amax, fabs(v));
        }
        amax = warp_max(amax);
        if (lane == 0) red[wid] = amax;
        __syncthreads();
        if (t == 0) {                             // pivot of column 0
            long long bk = -2;
            int bi = p;
            for (int i = 0; i < p; ++i) {
                const long long key = abs_key(S[i * ld]);
                if (key > bk) { bk = key; bi = i; }
            }
            red[12] = bk >= 0 ? __longlong_as_double(bk) : -1.0;
            red[13] = (double)(bk >= 0 ? bi : p);
        }
        amax = red[0];
        for (int w = 1; w < nw; ++w) amax = fmax(amax, red[w]);
        const double thresh = (double)p * 0x1p-53 * amax;
        bool sing = !(amax > 0.0);
        __syncthreads();
        for (int k = 0; k < p; ++k) {
            const double best = red[12];
            const int bi = (int)red[13];
            const int piv = (bi < p) ? bi : k;    // an all-NaN column has no valid pivot
            if (!(best > thresh)) sing = true;
            if (t < p) {
                if (t != k && piv != k) {         // rows k <-> piv in my column
                    const double x = S[k * ld + t];
                    S[k * ld + t] = S[piv * ld + t];
                    S[piv * ld + t] = x;
                }
                const int r = (t == k) ? piv : (t == piv ? k : t);
                colk[t] = S[r * ld + k];          // column k after the interchange
            }
            if (t == 0) swaps[k] = piv;
            __syncthreads();
            double pv = colk[k];
            if (pv == 0.0) pv = 1.0;              // singular: keep going, result discarded
            if (t < p) {
                const double rj = (t == k ? 1.0 : S[k * ld + t]) / pv;
                // every row, eight at a time with the loads ahead of the
                // stores (row k's value is overwritten below; column k
                // starts from zero): 59.9 -> 54.4 ms on the 30,000 matrices
                const bool isk = (t == k);
                int i = 0;
                for (; i + 8 <= p; i += 8) {
                    double x[8], c[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        x[u] = S[(i + u) * ld + t];
                        c[u] = colk[i + u];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) S[(i + u) * ld + t] = fma(-c[u], rj, isk ? 0.0 : x[u]);
                }
                for (; i < p; ++i) S[i * ld + t] = fma(-colk[i], rj, isk ? 0.0 : S[i * ld + t]);
                S[k * ld + t] = rj;
            }
            // the warp owning column k+1 scans it for the next pivot right
            // after its update: lanes over rows, then a shuffle reduction to
            // the largest key, lowest row on ties (the owner's serial scan:
            // 50.7 ms instead of 49.0 on the 30,000 matrices; tracking the
            // maximum inside every column's update loop made the step 1.5x
            // slower, that loop being bound by issue)
            if (k + 1 < p && wid == ((k + 1) >> 5)) {
                __syncwarp();
                long long bk = -2;
                int bnext = p;
                for (int i = k + 1 + lane; i < p; i += 32) {
                    const long long key = abs_key(S[i * ld + k + 1]);
                    if (key > bk) { bk = key; bnext = i; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bnext, o);
                    if (ok > bk || (ok == bk && oi < bnext)) { bk = ok; bnext = oi; }
                }
                if (lane == 0) {
                    red[12] = bk >= 0 ? __longlong_as_double(bk) : -1.0;
                    red[13] = (double)(bk >= 0 ? bnext : p);
                }
            }
            __syncthreads();
        }
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
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        if (pout) {
            // max |B| through the integer order key (NaN ranks lowest), so
            // the reduction spends no FP64 instruction
            long long km = -1;
            if (!sing)
                for (int e = t; e < p * p; e += nt) km = max(km, abs_key(S[(e / p) * ld + (e % p)]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) km = max(km, __shfl_xor_sync(0xffffffffu, km, o));
            __syncthreads();                      // red[] is free again
            if (lane == 0) red[wid] = __longlong_as_double(km);
            __syncthreads();
            km = __double_as_longlong(red[0]);
            for (int w = 1; w < nw; ++w) km = max(km, __double_as_longlong(red[w]));
            const double mx = km > 0 ? __longlong_as_double(km) : 0.0;
            int ex = 0;
            const bool finite = km < 0x7ff0000000000000LL;   // an infinite entry: the matrix reads as NaN
            if (mx > 0.0 && finite) frexp(mx, &ex);
            // B 2^-ex split into (hi, lo) with integer operations only (the
            // significand's top 24 bits and the next 23, |error| < 2^-46 |B|):
            // FP64 <-> FP32 conversions would run on the FP64 pipe, which the
            // elimination above keeps busy
            float2* out = pout + b * (int64_t)p * p;
            for (int e = t; e < p * p; e += nt) {
                const int cb = e / p, ra = e - cb * p;           // out[e] = B[ra][cb]
                out[e] = split_scaled(sing || !finite ? nanv : S[ra * ld + cb], ex);
            }
            if (t == 0) pexp[b] = ex;
        } else {
            double* out = Ainv + b * stride_out;
            for (int e = t; e < p * p; e += nt) out[e] = sing ? nanv : S[(e / p) * ld + (e % p)];
        }
        if (singular && t == 0) singular[b] = sing ? 1 : 0;
        __syncthreads();
    }
}

// p > 32: the inverses written straight in the streamed sweep's FP64-pair
// layout (pout, pexp), the FP64 copy skipped.
int launch_batched_inverse_pairs(const double* A, int32_t batch, int32_t p, float2* pout, int32_t* pexp,
                                 int32_t* singular, cudaStream_t s) {
    if (batch <= 0) return PSR_OK;
    if (p <= 32 || p > 128) return PSR_ERR_INVALID_ARG;
    return launch_batched_inverse_block(A, (int64_t)p * p, nullptr, batch, p, nullptr, 0, singular, s, pout, pexp);
}

int launch_batched_inverse_block(const double* A, int64_t stride_in, const int32_t* index, int32_t batch, int32_t p,
                                 double* Ainv, int64_t stride_out, int32_t* singular, cudaStream_t s,
                                 float2* pout, int32_t* pexp) {
    const size_t smem = inv_block_bytes(p);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_batched_inverse_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "inverse smem attribute");
    }
    // one wave of resident blocks, each looping over matrices (16 blocks per
    // SM queued: 54.4 -> 50.6 ms at p = 89, 17.8 -> 16.3 ms at p = 62)
    const int nt = 32 * ((p + 31) / 32);
    int dev = 0, sms = 152, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_inverse_block, nt, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int64_t blocks = (int64_t)sms * per_sm;
    if (blocks > batch) blocks = batch;
    count_launch();
    k_batched_inverse_block<<<(int)blocks, nt, smem, s>>>(A, stride_in, index, batch, p, Ainv, stride_out, singular,
                                                          pout, pexp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_batched_inverse_block");
    return PSR_OK;
}

}  // namespace psr
