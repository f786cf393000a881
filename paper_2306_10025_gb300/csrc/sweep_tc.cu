// Step a4 with representative inverses stored in BF16 and applied on the
// 5th-generation tensor cores (tcgen05.mma, FP32 accumulation in TMEM).
//
// A tile is up to 128 patches that share one database entry B_c^{-1}.  The
// gathered residuals form the M = 128 operand (one patch per row, K = patch
// DOFs padded to P), B_c^{-1} the N = P operand, both K-major in shared
// memory; D[m][n] = sum_k r_m[k] B_c^{-1}[n][k] = (B_c^{-1} r_m)[n] lands in
// TMEM, each of the 4 warps reads back its 32 rows and scatter-adds them.
// The residual is split r = hi + lo into two BF16 operands accumulated into
// the same TMEM tile (effective 16-bit mantissa for r); the stored inverse
// is BF16, so the applied operator is the fixed, rounded (symmetrised) one.
// Every rounding to BF16 goes FP64 -> FP32 -> BF16, round to nearest even.
//
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core
// matrices, core (g, c) of a matrix with P columns at byte (g*(P/8) + c)*128;
// leading (K) core stride 128 B, stride (row-group) core stride P*16 B.  The
// database is stored in global memory already in this layout, so staging an
// entry is a straight 16-byte-vector copy.
#include "psr_internal.cuh"
#include "tcgen05.cuh"

#include <algorithm>

namespace psr {

// byte offset of element (row, k) in the core-matrix layout with P columns
__host__ __device__ __forceinline__ int core_off(int row, int k, int P) {
    return ((row >> 3) * (P >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

template <int P>
__global__ void __launch_bounds__(128) k_sweep_tc(const int32_t* __restrict__ tiles, int ntiles, int p,
                                                  const __nv_bfloat16* __restrict__ rinv,
                                                  const int32_t* __restrict__ sdofs,
                                                  const double* __restrict__ r, const double* __restrict__ wg,
                                                  const double* __restrict__ wsc, double* __restrict__ z,
                                                  const int32_t* __restrict__ stop, int32_t* __restrict__ err) {
    constexpr int ABYTES = 128 * P * 2;
    constexpr int BBYTES = P * P * 2;
    constexpr uint32_t TCOLS = (P <= 32) ? 32 : (P <= 64 ? 64 : 128);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sAh = smem;
    unsigned char* sAl = smem + ABYTES;
    unsigned char* sB = smem + 2 * ABYTES;
    int32_t* sD = reinterpret_cast<int32_t*>(smem + 2 * ABYTES + BBYTES);     // 128 x p DOFs
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    if (stop && *stop) return;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t mbar_a = smem_u32(&mbar);
    constexpr uint32_t idesc = make_idesc(128, P);
    const uint32_t sbo = (P / 8) * 128;
    uint32_t phase = 0;
    int prev_c = -1;
    bool failed = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int c = tiles[3 * t], start = tiles[3 * t + 1], cnt = tiles[3 * t + 2];
        if (c != prev_c) {
            const uint4* src = reinterpret_cast<const uint4*>(rinv + (int64_t)c * P * P);
            for (int i = tid; i < BBYTES / 16; i += 128) reinterpret_cast<uint4*>(sB)[i] = src[i];
            prev_c = c;
        }
        // tile DOFs: coalesced copy of the contiguous cnt x p block
        const int32_t* dsrc = sdofs + (int64_t)start * p;
        for (int i = tid; i < cnt * p; i += 128) sD[i] = dsrc[i];
        __syncthreads();
        // gather row m = tid, split into hi + lo, write 16-byte chunks
        const bool live = tid < cnt;
#pragma unroll
        for (int k0 = 0; k0 < P; k0 += 8) {
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int a = k0 + q;
                double v = 0.0;
                if (live && a < p) {
                    const int d = sD[tid * p + a];
                    v = r[d];
                    if (wg) v *= wg[d];
                }
                const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                hi[q] = h;
                lo[q] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
            }
            const int off = core_off(tid, k0, P);
            *reinterpret_cast<uint4*>(sAh + off) = *reinterpret_cast<const uint4*>(hi);
            *reinterpret_cast<uint4*>(sAl + off) = *reinterpret_cast<const uint4*>(lo);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bb = smem_u32(sB);
#pragma unroll
            for (int s = 0; s < P / 16; ++s)
                mma_bf16(tmem, make_desc(ah + s * 256, 128, sbo), make_desc(bb + s * 256, 128, sbo), idesc, s > 0);
#pragma unroll
            for (int s = 0; s < P / 16; ++s)
                mma_bf16(tmem, make_desc(al + s * 256, 128, sbo), make_desc(bb + s * 256, 128, sbo), idesc, 1);
            mma_commit(mbar_a);
        }
        const bool ok = mbar_wait_bounded(mbar_a, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) { failed = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < P; c0 += 16) {
            float y[16];
            tmem_ld16(trow + c0, y);
            if (live) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int a = c0 + q;
                    if (a < p) {
                        const int d = sD[tid * p + a];
                        atomicAdd(&z[d], (double)y[q] * wsc[d]);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicOr(err, ST_NAN);
        mbar_wait_bounded(mbar_a, phase ^ 1u);      // let an MMA still in flight finish (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS) : "memory");
}

// FP64 database (m x p x p, row-major) -> BF16 in the core-matrix layout with
// P x P padding (zeros), symmetrised first when sym != 0.
__global__ void k_convert_tc(const double* __restrict__ src, int m, int p, int P, int sym,
                             __nv_bfloat16* __restrict__ dst) {
    const int64_t total = (int64_t)m * P * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / ((int64_t)P * P);
        const int nk = (int)(e - c * P * P);
        const int n = nk / P, k = nk % P;
        double v = 0.0;
        if (n < p && k < p) {
            v = src[c * p * p + (int64_t)n * p + k];
            if (sym) v = 0.5 * (v + src[c * p * p + (int64_t)k * p + n]);
        }
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(dst + c * P * P) + core_off(n, k, P)) =
            __float2bfloat16_rn((float)v);
    }
}

int tc_pad(int p) {
    if (p <= 16) return 16;
    if (p <= 32) return 32;
    if (p <= 64) return 64;
    if (p <= 96) return 96;
    return 128;
}

static size_t tc_smem(int P, int p) { return (size_t)2 * 128 * P * 2 + (size_t)P * P * 2 + (size_t)128 * p * 4; }

int convert_tc(const double* src, int m, int p, int sym, __nv_bfloat16** out, cudaStream_t s) {
    const int P = tc_pad(p);
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)std::max(m, 1) * P * P;
    cudaError_t e = psr::dev_alloc(out, bytes);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bf16 database");
    const int64_t total = (int64_t)m * P * P;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
    count_launch();
    k_convert_tc<<<blocks, 256, 0, s>>>(src, m, p, P, sym, *out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_convert_tc");
    return PSR_OK;
}

int tc_prepare() {
    const int bytes = 200 * 1024;
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(k_sweep_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_tc<96>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tensor-core sweep smem attribute");
    return PSR_OK;
}

int launch_sweep_tc(const int32_t* tiles, int ntiles, int p, const __nv_bfloat16* rinv, const int32_t* sdofs,
                    const double* r, const double* wg, const double* wsc, double* z, const int32_t* stop,
                    int32_t* err, cudaStream_t s) {
    const int P = tc_pad(p);
    const size_t sm = tc_smem(P, p);
    const int blocks = std::max(1, std::min(ntiles, 152 * 4));
    count_launch();
    switch (P) {
        case 16: k_sweep_tc<16><<<blocks, 128, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, wg, wsc, z, stop, err); break;
        case 32: k_sweep_tc<32><<<blocks, 128, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, wg, wsc, z, stop, err); break;
        case 64: k_sweep_tc<64><<<blocks, 128, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, wg, wsc, z, stop, err); break;
        case 96: k_sweep_tc<96><<<blocks, 128, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, wg, wsc, z, stop, err); break;
        default: k_sweep_tc<128><<<blocks, 128, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, wg, wsc, z, stop, err); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_sweep_tc");
    return PSR_OK;
}

}  // namespace psr
