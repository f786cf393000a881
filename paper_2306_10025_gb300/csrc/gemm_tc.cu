// FP32 GEMM on the 5th-generation tensor cores for the learned-assignment
// network: C = A B (+ bias, optional ReLU copy), A and B FP32 in global
// memory with arbitrary strides, FP32 accumulation in TMEM.
//
// Precision: every operand element a is split a = hi + lo with hi = a
// rounded to TF32 (11 significant bits) and lo = a - hi (exact in FP32);
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi (kind::tf32).  The dropped lo*lo
// term is below 2^-22 |a||b| per product and lo enters the MMA truncated to
// TF32 (relative 2^-11 of lo), so the result carries FP32-level error.
//
// Tiles: one CTA of 4 warps per 128 x 128 output tile, K in slices of 32,
// two shared-memory stages.  Each slice is converted by the CTA into the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes = 8 x 4 FP32 per
// core matrix) while the tensor cores work on the previous one; one elected
// thread issues 4 K-steps x 3 MMAs (M = 128, N = 128, K = 8) and commits to
// the stage's mbarrier; all waits are bounded.  The epilogue reads each
// warp's 32 TMEM lanes (one output row per thread).
#include "psr_internal.cuh"
#include "tcgen05.cuh"

namespace psr {

namespace {

constexpr int GM = 128, GN = 128, GK = 32;
constexpr int TILE_BYTES = GM * GK * 4;               // one operand slice (A or B), FP32
constexpr uint32_t GSBO = (GK / 4) * 128;             // row-group stride of the core layout

// Instruction descriptor, kind::tf32: D F32 (bit 4), A TF32 (bits 7-9 = 2),
// B TF32 (bits 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

// a rounded to TF32 (nearest, ties away), low 13 mantissa bits zero
__device__ __forceinline__ float to_tf32(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return __uint_as_float(r);
}

// byte offset of (row, k) in a 128 x 32 FP32 slice, core-matrix layout
__device__ __forceinline__ int core_off32(int row, int k) {
    return ((row >> 3) * (GK / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// One 128 x 32 slice of a strided operand into hi / lo shared buffers:
// op(r, k) = X[r * srow + k * sk], zero outside rows < nrow, k < nk.  The
// element order follows the unit stride so the global loads coalesce; each
// thread requests 16 elements before converting and storing any of them.
__device__ __forceinline__ void load_slice(const float* __restrict__ X, int64_t srow, int64_t sk, int r0, int nrow,
                                           int k0, int nk, unsigned char* hi, unsigned char* lo) {
    const bool kfast = (sk == 1);
    constexpr int PER = GM * GK / 128;                   // elements per thread (128 threads)
#pragma unroll
    for (int g = 0; g < PER; g += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = threadIdx.x + 128 * (g + u);
            const int r = kfast ? e / GK : e % GM;
            const int k = kfast ? e % GK : e / GM;
            const int gr = r0 + r, gk = k0 + k;
            v[u] = (gr < nrow && gk < nk) ? __ldg(X + (int64_t)gr * srow + (int64_t)gk * sk) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = threadIdx.x + 128 * (g + u);
            const int r = kfast ? e / GK : e % GM;
            const int k = kfast ? e % GK : e / GM;
            const float h = to_tf32(v[u]);
            const int off = core_off32(r, k);
            *reinterpret_cast<float*>(hi + off) = h;
            *reinterpret_cast<float*>(lo + off) = v[u] - h;
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const float* __restrict__ A, int64_t sai,
                                                 int64_t sak, const float* __restrict__ B, int64_t sbk, int64_t sbj,
                                                 float* __restrict__ C, int64_t ldc, const float* __restrict__ bias,
                                                 float* __restrict__ relu_out, int32_t* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // two stages of four operand slices: A hi, A lo, B hi, B lo
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int i0 = blockIdx.y * GM, j0 = blockIdx.x * GN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(GN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_tf32(GM, GN);
    uint32_t issued[2] = {0u, 0u}, waited[2] = {0u, 0u};   // commits per stage buffer
    bool failed = false;
    const int nslices = (K + GK - 1) / GK;
    // Software pipeline: while the tensor cores work on slice t, the CTA
    // converts slice t+1 into the other stage; a stage is refilled only after
    // the MMAs that read it have committed.
    for (int t = 0; t < nslices; ++t) {
        const int b = t & 1;
        unsigned char* st = smem + (size_t)b * 4 * TILE_BYTES;
        if (issued[b] > waited[b]) {
            const bool ok = mbar_wait_bounded(smem_u32(&mbar[b]), waited[b] & 1u);
            ++waited[b];
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        const int k0 = t * GK;
        load_slice(A, sai, sak, i0, M, k0, K, st, st + TILE_BYTES);
        load_slice(B, sbj, sbk, j0, N, k0, K, st + 2 * TILE_BYTES, st + 3 * TILE_BYTES);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t ah = smem_u32(st), al = ah + TILE_BYTES, bh = ah + 2 * TILE_BYTES, bl = ah + 3 * TILE_BYTES;
#pragma unroll
            for (int s = 0; s < GK / 8; ++s) {
                const uint32_t o = s * 256;                   // two core matrices along K
                mma_tf32(tmem, make_desc(ah + o, 128, GSBO), make_desc(bh + o, 128, GSBO), idesc,
                         (t > 0 || s > 0) ? 1u : 0u);
                mma_tf32(tmem, make_desc(ah + o, 128, GSBO), make_desc(bl + o, 128, GSBO), idesc, 1u);
                mma_tf32(tmem, make_desc(al + o, 128, GSBO), make_desc(bh + o, 128, GSBO), idesc, 1u);
            }
            mma_commit(smem_u32(&mbar[b]));
        }
        ++issued[b];
    }
    // wait for every outstanding commit (the last one covers all MMAs)
    for (int b = 0; b < 2 && !failed; ++b) {
        while (issued[b] > waited[b]) {
            const bool ok = mbar_wait_bounded(smem_u32(&mbar[b]), waited[b] & 1u);
            ++waited[b];
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!failed) {
        const int row = i0 + tid;                           // TMEM lane = row of the tile
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < GN; c0 += 16) {
            float y[16];
            if (K > 0) {
                tmem_ld16(trow + c0, y);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) y[q] = 0.f;
            }
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = j0 + c0 + q;
                    if (col < N) {
                        const float v = y[q] + (bias ? bias[col] : 0.f);
                        C[(int64_t)row * ldc + col] = v;
                        if (relu_out) relu_out[(int64_t)row * ldc + col] = fmaxf(v, 0.f);
                    }
                }
            }
        }
    }
    if (failed) {
        if (tid == 0 && err) atomicOr(err, 1);
        // the tile's outputs become NaN so that the failure shows in the loss
        const int row = i0 + tid;
        if (row < M)
            for (int col = j0; col < min(N, j0 + GN); ++col) C[(int64_t)row * ldc + col] = __int_as_float(0x7fc00000);
        for (int b = 0; b < 2; ++b)                   // let MMAs still in flight finish (bounded)
            while (issued[b] > waited[b]) {
                mbar_wait_bounded(smem_u32(&mbar[b]), waited[b] & 1u);
                ++waited[b];
            }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)GN) : "memory");
}

size_t gemm_tc_smem() { return (size_t)2 * 4 * TILE_BYTES; }

int gemm_tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem());
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tensor-core GEMM smem attribute");
    return PSR_OK;
}

void launch_gemm_tc(int M, int N, int K, const float* A, int64_t sai, int64_t sak, const float* B, int64_t sbk,
                    int64_t sbj, float* C, int64_t ldc, const float* bias, float* relu_out, int32_t* err,
                    cudaStream_t s) {
    dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
    count_launch();
    k_gemm_tc<<<grid, 128, gemm_tc_smem(), s>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, relu_out, err);
}

}  // namespace psr
