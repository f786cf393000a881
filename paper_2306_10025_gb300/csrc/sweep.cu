// Step a4: the additive Schwarz / Vanka sweep of Eq. (3),
//     z = W sum_k V_k^T B_phi(k)^{-1} V_k r        (LEFT weighting)
//     z = W^1/2 sum_k V_k^T B_phi(k)^{-1} V_k W^1/2 r  (SYM weighting)
//
// Layout built at setup.  Inside each size group the patches are sorted by
// database entry (stable), their DOF lists are stored in that order, and the
// sorted range of every entry is cut into tiles of at most T patches.  A CTA
// takes a tile, stages that entry's inverse in shared memory once, and its
// warps stream the tile's patches: gather r at the patch DOFs, multiply by
// the staged inverse, scatter-add the weighted result into z.  Reusing one
// staged inverse for a whole tile is what makes the compressed sweep bound by
// the residual gather / scatter instead of by factor bytes (the paper's
// remark on solving all patches of a cluster together, Exp. 3).
//
// Precision: FP64 storage computes in FP64; FP32 storage gathers r in FP64,
// rounds it to FP32, multiplies in FP32 and scatters in FP64.
#include "psr_internal.cuh"
#include "pairs.cuh"

#include <algorithm>
#include <numeric>
#include <type_traits>

namespace psr {

struct GroupDesc {          // device copy for the grouped persistent kernel
    const int32_t* sdofs;
    const void* rinv;
    int p;
    int pad;
};

// Storage type T -> compute type: FP64 and FP32 compute in their own
// precision, BF16 storage is widened to FP32.
template <typename T> struct Comp { using type = T; };
template <> struct Comp<__nv_bfloat16> { using type = float; };

template <typename C> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T> __device__ __forceinline__ T to_store(double v) { return (T)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

// Read-only loads kept in the order written and never moved into a
// conditional block (volatile asm), so that a batch of them is in flight
// together before the first use.
__device__ __forceinline__ double ldg_nc(const double* p) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ldg_nc_i(const int32_t* p) {
    int v;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Asynchronous global -> shared copies of one element (4 or 8 bytes): the
// whole staged inverse is requested before the first wait instead of one
// load latency per loop trip.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    if (BYTES == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(sa), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Stage one inverse (pp entries of T) into shared memory as compute type C
// by the whole block; the caller synchronises the block afterwards.
template <typename T, typename C>
__device__ __forceinline__ void stage_inverse(C* sR, const T* __restrict__ src, int pp) {
    if constexpr (sizeof(T) == sizeof(C) && (sizeof(T) == 4 || sizeof(T) == 8)) {
        for (int e = threadIdx.x; e < pp; e += blockDim.x) cp_async_elem<sizeof(T)>(sR + e, src + e);
        cp_async_wait_all();
    } else {
        for (int e = threadIdx.x; e < pp; e += blockDim.x) sR[e] = (C)src[e];
    }
}

// The patches of one tile (all sharing the staged inverse sR, p <= 128) as
// work items (patch, chunk of 32 rows) dealt to the block's warps, so that a
// tile of fewer patches than warps (full storage: one) still keeps several
// warps busy.  The warp gathers the patch's residual into its slot sr, then
// lane l forms row 32 q + l and scatter-adds it.
template <typename C>
__device__ __forceinline__ void sweep_tile_items(const C* sR, C* sr, int p, const int32_t* __restrict__ sdofs,
                                                 int start, int cnt, const double* __restrict__ r,
                                                 const double* __restrict__ wg, const double* __restrict__ wsc,
                                                 double* __restrict__ z) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int nrc = (p + 31) >> 5;
    for (int it = wid; it < cnt * nrc; it += wpb) {
        const int k = start + it / nrc, q = it % nrc;
        const int32_t* dk = sdofs + (int64_t)k * p;
        // map and residual loads unconditional (index clamped to p-1), so the
        // chunks' loads are in flight together
        int dof[4] = {0, 0, 0, 0};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < nrc) dof[u] = ldg_nc_i(dk + min(lane + 32 * u, p - 1));
        double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < nrc) v[u] = ldg_nc(r + dof[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = lane + 32 * u;
            if (a < p) sr[a] = (C)(wg ? v[u] * wg[dof[u]] : v[u]);
        }
        __syncwarp();
        const int a = lane + 32 * q;
        if (a < p) {
            C y = (C)0;
            const C* row = sR + a * p;
            for (int b = 0; b < p; ++b) y = fma(row[b], sr[b], y);
            const int d = (q == 0) ? dof[0] : (q == 1) ? dof[1] : (q == 2) ? dof[2] : dof[3];
            atomicAdd(&z[d], (double)y * wsc[d]);
        }
        __syncwarp();
    }
}


// ------------------------------------------------------------ kernels
// Generic, p <= 128: (patch, 32-row chunk) work items over the block's warps,
// lane l of an item forms row 32 q + l of B^-1 r_k.
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_warp(const int32_t* __restrict__ tiles, int ntiles, int p,
                                                    const T* __restrict__ rinv, const int32_t* __restrict__ sdofs,
                                                    const double* __restrict__ r, const double* __restrict__ wg,
                                                    const double* __restrict__ wsc, double* __restrict__ z,
                                                    const int32_t* __restrict__ stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = typename Comp<T>::type;
    if (stop && *stop) return;
    C* sR = reinterpret_cast<C*>(smem);
    const int wid = threadIdx.x >> 5;
    const int pp = p * p;
    C* sr = reinterpret_cast<C*>(smem + (((size_t)pp * sizeof(C) + 15) & ~(size_t)15)) + wid * 128;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int c = tiles[3 * t], start = tiles[3 * t + 1], cnt = tiles[3 * t + 2];
        const T* src = rinv + (int64_t)c * pp;
        __syncthreads();
        stage_inverse<T, C>(sR, src, pp);
        __syncthreads();
        sweep_tile_items<C>(sR, sr, p, sdofs, start, cnt, r, wg, wsc, z);
    }
}

// Generic, p <= 128, staged: per tile the inverse and the DOF lists of up to
// `sub` patches at a time are copied into shared memory (cp.async), then r,
// the output weight and (SYM) the input weight at those DOFs are gathered
// into shared memory the same way, so a tile costs two memory round trips
// instead of two per patch and warp; the weighted residual is rounded to the
// compute type once per entry, and every thread forms one (patch, row) of
// B^-1 r_k (two accumulation chains) and scatter-adds it.
__host__ __device__ inline size_t staged_align(size_t b) { return (b + 15) & ~(size_t)15; }
template <typename C>
__host__ __device__ inline size_t staged_smem(int p, int sub, bool sym) {
    const size_t ne = (size_t)sub * p;
    return staged_align((size_t)p * p * sizeof(C)) + staged_align(ne * 4) + 2 * staged_align(ne * 8) +
           (sym ? staged_align(ne * 8) : 0) + staged_align(ne * sizeof(C));
}

template <typename T>
__global__ void __launch_bounds__(256) k_sweep_staged(const int32_t* __restrict__ tiles, int ntiles, int p, int sub,
                                                      const T* __restrict__ rinv, const int32_t* __restrict__ sdofs,
                                                      const double* __restrict__ r, const double* __restrict__ wg,
                                                      const double* __restrict__ wsc, double* __restrict__ z,
                                                      const int32_t* __restrict__ stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = typename Comp<T>::type;
    if (stop && *stop) return;
    const int pp = p * p;
    const size_t ne_max = (size_t)sub * p;
    size_t off = staged_align((size_t)pp * sizeof(C));
    C* sR = reinterpret_cast<C*>(smem);
    int32_t* sd = reinterpret_cast<int32_t*>(smem + off);
    off += staged_align(ne_max * 4);
    double* sx = reinterpret_cast<double*>(smem + off);
    off += staged_align(ne_max * 8);
    double* sw = reinterpret_cast<double*>(smem + off);
    off += staged_align(ne_max * 8);
    double* sg = nullptr;
    if (wg) {
        sg = reinterpret_cast<double*>(smem + off);
        off += staged_align(ne_max * 8);
    }
    C* sc = reinterpret_cast<C*>(smem + off);
    const int nt = blockDim.x;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int c = tiles[3 * t], start = tiles[3 * t + 1], cnt = tiles[3 * t + 2];
        const T* src = rinv + (int64_t)c * pp;
        for (int k0 = 0; k0 < cnt; k0 += sub) {
            const int kc = min(sub, cnt - k0);
            const int ne = kc * p;
            const int32_t* dk = sdofs + (int64_t)(start + k0) * p;
            __syncthreads();                          // the previous sub-tile's readers are done
            // round trip 1: the inverse (first sub-tile only) and the DOF lists
            if (k0 == 0) {
                if constexpr (sizeof(T) == sizeof(C)) {
                    for (int e = threadIdx.x; e < pp; e += nt) cp_async_elem<sizeof(T)>(sR + e, src + e);
                } else {
                    for (int e = threadIdx.x; e < pp; e += nt) sR[e] = (C)src[e];
                }
            }
            for (int e = threadIdx.x; e < ne; e += nt) cp_async_elem<4>(sd + e, dk + e);
            cp_async_wait_all();
            __syncthreads();
            // round trip 2: gathers at the DOFs
            for (int e = threadIdx.x; e < ne; e += nt) {
                const int d = sd[e];
                cp_async_elem<8>(sx + e, r + d);
                cp_async_elem<8>(sw + e, wsc + d);
                if (wg) cp_async_elem<8>(sg + e, wg + d);
            }
            cp_async_wait_all();
            __syncthreads();
            for (int e = threadIdx.x; e < ne; e += nt) sc[e] = (C)(wg ? sx[e] * sg[e] : sx[e]);
            __syncthreads();
            for (int it = threadIdx.x; it < ne; it += nt) {
                const int k = it / p, a = it - k * p;
                const C* row = sR + a * p;
                const C* x = sc + k * p;
                C y0 = (C)0, y1 = (C)0;
                if ((p & 1) == 0) {
                    // even p: rows and residual slots start on 2-element
                    // boundaries, so both are read as element pairs
                    using V2 = typename Vec2<C>::type;
                    const V2* r2 = reinterpret_cast<const V2*>(row);
                    const V2* x2 = reinterpret_cast<const V2*>(x);
                    for (int b2 = 0; b2 < (p >> 1); ++b2) {
                        const V2 rv = r2[b2], xv = x2[b2];
                        y0 = fma(rv.x, xv.x, y0);
                        y1 = fma(rv.y, xv.y, y1);
                    }
                } else {
                    int b = 0;
                    for (; b + 1 < p; b += 2) {
                        y0 = fma(row[b], x[b], y0);
                        y1 = fma(row[b + 1], x[b + 1], y1);
                    }
                    y0 = fma(row[b], x[b], y0);
                }
                atomicAdd(&z[sd[it]], (double)(y0 + y1) * sw[it]);
            }
        }
    }
}

// Shared memory of the staged kernel on pairs: that of the FP64 form plus
// one exponent per patch of the sub-tile.
__host__ __device__ inline size_t staged_pair_smem(int p, int sub, bool sym) {
    return staged_smem<double>(p, sub, sym) + staged_align((size_t)sub * 4);
}

// The staged kernel for FP64 entries on FP32 pair arithmetic: the entry's
// inverse staged as scaled pairs (column-major, so the threads of a patch read
// consecutive elements), every patch's weighted residual split into pairs
// after a power-of-two shift that brings its largest entry into [1, 2), each
// (patch, row) summed with compensated products and unshifted in FP64.
__global__ void __launch_bounds__(256) k_sweep_staged_pair(const int32_t* __restrict__ tiles, int ntiles, int p,
                                                           int sub, const float2* __restrict__ Bt,
                                                           const int32_t* __restrict__ bexp,
                                                           const int32_t* __restrict__ sdofs,
                                                           const double* __restrict__ r, const double* __restrict__ wg,
                                                           const double* __restrict__ wsc, double* __restrict__ z,
                                                           const int32_t* __restrict__ stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (stop && *stop) return;
    const int pp = p * p;
    const size_t ne_max = (size_t)sub * p;
    size_t off = staged_align((size_t)pp * 8);
    float2* sR = reinterpret_cast<float2*>(smem);
    int32_t* sd = reinterpret_cast<int32_t*>(smem + off);
    off += staged_align(ne_max * 4);
    double* sx = reinterpret_cast<double*>(smem + off);
    off += staged_align(ne_max * 8);
    double* sw = reinterpret_cast<double*>(smem + off);
    off += staged_align(ne_max * 8);
    double* sg = nullptr;
    if (wg) {
        sg = reinterpret_cast<double*>(smem + off);
        off += staged_align(ne_max * 8);
    }
    float2* sc = reinterpret_cast<float2*>(smem + off);
    off += staged_align(ne_max * 8);
    int* sex = reinterpret_cast<int*>(smem + off);
    const int nt = blockDim.x;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int c = tiles[3 * t], start = tiles[3 * t + 1], cnt = tiles[3 * t + 2];
        const float2* src = Bt + (int64_t)c * pp;
        const int bx = __ldg(bexp + c);
        for (int k0 = 0; k0 < cnt; k0 += sub) {
            const int kc = min(sub, cnt - k0);
            const int ne = kc * p;
            const int32_t* dk = sdofs + (int64_t)(start + k0) * p;
            __syncthreads();                          // the previous sub-tile's readers are done
            if (k0 == 0)
                for (int e = threadIdx.x; e < pp; e += nt) cp_async_elem<8>(sR + e, src + e);
            for (int e = threadIdx.x; e < ne; e += nt) cp_async_elem<4>(sd + e, dk + e);
            for (int k = threadIdx.x; k < kc; k += nt) sex[k] = 0;
            cp_async_wait_all();
            __syncthreads();
            for (int e = threadIdx.x; e < ne; e += nt) {
                const int d = sd[e];
                cp_async_elem<8>(sx + e, r + d);
                cp_async_elem<8>(sw + e, wsc + d);
                if (wg) cp_async_elem<8>(sg + e, wg + d);
            }
            cp_async_wait_all();
            __syncthreads();
            for (int e = threadIdx.x; e < ne; e += nt) {
                const double v = wg ? sx[e] * sg[e] : sx[e];
                sx[e] = v;
                const int ex = (int)((unsigned)(__double2hiint(v) >> 20) & 0x7ffu);
                if (ex != 0x7ff) atomicMax(&sex[e / p], ex);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < ne; e += nt) sc[e] = split_scaled(sx[e], sex[e / p] - 1023);
            __syncthreads();
            for (int it = threadIdx.x; it < ne; it += nt) {
                const int k = it / p, a = it - k * p;
                const float2* x = sc + k * p;
                float sh = 0.f, sl = 0.f;
                for (int b = 0; b < p; ++b) {
                    const float2 bv = sR[b * p + a];
                    const float2 xv = x[b];
                    pair_fma(sh, sl, bv.x, bv.y, xv.x, xv.y);
                }
                atomicAdd(&z[sd[it]], ldexp((double)sh + (double)sl, sex[k] - 1023 + bx) * sw[it]);
            }
        }
    }
}

// Small patches (p <= 16): two patches per warp, one per half-warp, r values
// exchanged with width-16 shuffles.
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_half(const int32_t* __restrict__ tiles, int ntiles, int p,
                                                    const T* __restrict__ rinv, const int32_t* __restrict__ sdofs,
                                                    const double* __restrict__ r, const double* __restrict__ wg,
                                                    const double* __restrict__ wsc, double* __restrict__ z,
                                                    const int32_t* __restrict__ stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = typename Comp<T>::type;
    if (stop && *stop) return;
    C* sR = reinterpret_cast<C*>(smem);
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4;
    const int a = lane & 15;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int pp = p * p;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int c = tiles[3 * t], start = tiles[3 * t + 1], cnt = tiles[3 * t + 2];
        const T* src = rinv + (int64_t)c * pp;
        __syncthreads();
        for (int e = threadIdx.x; e < pp; e += blockDim.x) sR[e] = (C)src[e];
        __syncthreads();
        for (int k0 = start + 2 * wid; k0 < start + cnt; k0 += 2 * wpb) {
            const int k = k0 + half;
            const bool live = (k < start + cnt) && (a < p);
            int dof = 0;
            C rv = (C)0;
            if (live) {
                dof = sdofs[(int64_t)k * p + a];
                double v = r[dof];
                if (wg) v *= wg[dof];
                rv = (C)v;
            }
            C y = (C)0;
            for (int b = 0; b < p; ++b) {
                const C rb = __shfl_sync(0xffffffffu, rv, b, 16);
                y = fma(sR[a * p + b < pp ? a * p + b : 0], rb, y);
            }
            if (live) atomicAdd(&z[dof], (double)y * wsc[dof]);
        }
    }
}

// Clustered, p <= 32: one patch per THREAD.  A warp tile is up to 32
// consecutive sorted patches that share one entry, so every lane reads the
// same inverse element at the same time (one broadcast load from L1); each
// lane keeps its patch's p residual values in registers, which puts p
// independent gathers in flight per thread.  DOFs come from the transposed
// map (local DOF major), so lane k's load of DOF a is coalesced across the warp.
template <typename T, int PM>
__global__ void __launch_bounds__(256) k_sweep_tpp(const int32_t* __restrict__ wtiles, int nwt, int p, int count,
                                                   const T* __restrict__ rinv, const int32_t* __restrict__ sdofs_t,
                                                   const double* __restrict__ r, const double* __restrict__ wg,
                                                   const double* __restrict__ wsc, double* __restrict__ z,
                                                   const int32_t* __restrict__ stop) {
    using C = typename Comp<T>::type;
    if (stop && *stop) return;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nwt; t += nw) {
        const int c = wtiles[3 * t], start = wtiles[3 * t + 1], cnt = wtiles[3 * t + 2];
        const bool live = lane < cnt;
        const int k = start + (live ? lane : 0);
        // Unconditional loads (local DOF index clamped to p-1, idle lanes on
        // the tile's first patch): the p map loads, then the p gathers of r,
        // are each in flight together instead of one dependent pair per DOF.
        int dof[PM];
        C x[PM];
#pragma unroll
        for (int a = 0; a < PM; ++a) dof[a] = ldg_nc_i(sdofs_t + (int64_t)min(a, p - 1) * count + k);
        double rv[PM];
#pragma unroll
        for (int a = 0; a < PM; ++a) rv[a] = ldg_nc(r + dof[a]);
        if (wg) {
#pragma unroll
            for (int a = 0; a < PM; ++a) rv[a] *= ldg_nc(wg + dof[a]);
        }
#pragma unroll
        for (int a = 0; a < PM; ++a) x[a] = (live && a < p) ? (C)rv[a] : (C)0;
        const T* B = rinv + (int64_t)c * p * p;
#pragma unroll
        for (int a = 0; a < PM; ++a) {
            if (a >= p) break;
            C y = (C)0;
            const T* row = B + a * p;
#pragma unroll
            for (int b = 0; b < PM; ++b)
                if (b < p) y = fma((C)__ldg(row + b), x[b], y);
            if (live) atomicAdd(&z[dof[a]], (double)y * wsc[dof[a]]);
        }
    }
}

// Full storage (every patch its own inverse, Eq. 1), p <= 32: one patch per
// warp; the warp streams its inverse into its own shared-memory slot with
// coalesced loads, then lane a forms row a of B^-1 r_k.
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_full(int count, int p, const T* __restrict__ rinv,
                                                    const int32_t* __restrict__ sphi,
                                                    const int32_t* __restrict__ sdofs,
                                                    const double* __restrict__ r, const double* __restrict__ wg,
                                                    const double* __restrict__ wsc, double* __restrict__ z,
                                                    const int32_t* __restrict__ stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = typename Comp<T>::type;
    if (stop && *stop) return;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int pp = p * p;
    const size_t slot = (((size_t)pp + 32) * sizeof(C) + 15) & ~(size_t)15;
    C* sB = reinterpret_cast<C*>(smem + wid * slot);
    C* sr = sB + pp;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < count; k += nw) {
        const T* B = rinv + (int64_t)sphi[k] * pp;
        for (int e = lane; e < pp; e += 32) sB[e] = (C)B[e];
        int dof = 0;
        if (lane < p) {
            dof = sdofs[(int64_t)k * p + lane];
            double v = r[dof];
            if (wg) v *= wg[dof];
            sr[lane] = (C)v;
        }
        __syncwarp();
        if (lane < p) {
            C y = (C)0;
            const C* row = sB + lane * p;
            for (int b = 0; b < p; ++b) y = fma(row[b], sr[b], y);
            atomicAdd(&z[dof], (double)y * wsc[dof]);
        }
        __syncwarp();
    }
}

// Grouped persistent kernel (one launch for all size groups): CTAs pull
// tiles (group, entry, start, count) from a global counter.  Generic warp
// mapping as k_sweep_warp; the staged inverse is sized for the largest group.
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_grouped(const int32_t* __restrict__ tiles, int ntiles,
                                                       const GroupDesc* __restrict__ groups,
                                                       const double* __restrict__ r, const double* __restrict__ wg,
                                                       const double* __restrict__ wsc, double* __restrict__ z,
                                                       int32_t* __restrict__ counter, int pmax,
                                                       const int32_t* __restrict__ stop) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = typename Comp<T>::type;
    __shared__ int s_tile;
    if (stop && *stop) return;
    C* sR = reinterpret_cast<C*>(smem);
    const int wid = threadIdx.x >> 5;
    C* sr = reinterpret_cast<C*>(smem + (((size_t)pmax * pmax * sizeof(C) + 15) & ~(size_t)15)) + wid * 128;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const int g = tiles[4 * t], c = tiles[4 * t + 1], start = tiles[4 * t + 2], cnt = tiles[4 * t + 3];
        const GroupDesc gd = groups[g];
        const int p = gd.p, pp = p * p;
        const T* src = reinterpret_cast<const T*>(gd.rinv) + (int64_t)c * pp;
        stage_inverse<T, C>(sR, src, pp);
        __syncthreads();
        sweep_tile_items<C>(sR, sr, p, gd.sdofs, start, cnt, r, wg, wsc, z);
    }
    // the last CTA to leave resets the counter for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        const int finished = atomicAdd(counter + 1, 1);
        if (finished == (int)gridDim.x - 1) {
            counter[0] = 0;
            counter[1] = 0;
            __threadfence();
        }
    }
}

// FP64 database -> storage precision, optionally symmetrised first.
template <typename T>
__global__ void k_convert(const double* __restrict__ src, int m, int p, int sym, T* __restrict__ dst) {
    const int64_t total = (int64_t)m * p * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / ((int64_t)p * p);
        const int ij = (int)(e - c * p * p);
        const int i = ij / p, j = ij % p;
        double v = src[e];
        if (sym) v = 0.5 * (v + src[c * p * p + (int64_t)j * p + i]);
        dst[e] = to_store<T>(v);
    }
}

// ------------------------------------------------------------ host side
static size_t sweep_smem(int p, int prec, int warps) {
    const size_t es = (prec == PSR_PREC_FP64) ? 8 : 4;
    return ((p * p * es + 15) & ~(size_t)15) + (size_t)warps * 128 * es;
}

static int cuda_fail_if(psr_ctx* ctx, cudaError_t e, const char* what) {
    return e == cudaSuccess ? PSR_OK : cuda_fail(ctx, e, what);
}

// Tiles (entry, first sorted patch, count <= T) of a group's sweep order.
// keep: 0 = every entry, 1 = entries not flagged in `hi`, 2 = flagged ones only.
static std::vector<int32_t> tiles_host(const std::vector<int32_t>& sorted_phi, int count, int T,
                                       const std::vector<char>* hi = nullptr, int keep = 0) {
    std::vector<int32_t> t;
    int i = 0;
    while (i < count) {
        const int c = sorted_phi[i];
        int j = i;
        while (j < count && sorted_phi[j] == c) ++j;
        const bool flagged = hi && !hi->empty() && (*hi)[c];
        if (keep != 0 && flagged != (keep == 2)) { i = j; continue; }
        for (int s = i; s < j; s += T) {
            t.push_back(c);
            t.push_back(s);
            t.push_back(std::min(T, j - s));
        }
        i = j;
    }
    return t;
}

static int make_tiles(psr_ctx* ctx, Group& G, const std::vector<int32_t>& sorted_phi, int T) {
    const bool split = !G.h_hi.empty();
    const std::vector<int32_t> t = tiles_host(sorted_phi, G.count, T, &G.h_hi, split ? 1 : 0);
    if (G.tiles) psr::dev_free(G.tiles);
    G.tiles = nullptr;
    G.ntiles = (int)(t.size() / 3);
    PSR_CUDA(ctx, psr::dev_alloc(&G.tiles, sizeof(int32_t) * std::max<size_t>(t.size(), 3)));
    PSR_CUDA(ctx, cudaMemcpy(G.tiles, t.data(), sizeof(int32_t) * t.size(), cudaMemcpyHostToDevice));
    G.tile_patches = T;
    if (split) {
        const std::vector<int32_t> th = tiles_host(sorted_phi, G.count, 32, &G.h_hi, 2);
        if (G.tiles_hi) psr::dev_free(G.tiles_hi);
        G.tiles_hi = nullptr;
        G.ntiles_hi = (int)(th.size() / 3);
        PSR_CUDA(ctx, psr::dev_alloc(&G.tiles_hi, sizeof(int32_t) * std::max<size_t>(th.size(), 3)));
        PSR_CUDA(ctx, cudaMemcpy(G.tiles_hi, th.data(), sizeof(int32_t) * th.size(), cudaMemcpyHostToDevice));
    }
    return PSR_OK;
}

// Precision check of a rounded database (psr_opts.prec_check), one block per
// entry: B~ = the stored value of (B + B^T)/2 (sym) or B rounded to FP32 /
// BF16 exactly as the conversion kernels round it, then rho = ||B~ A_c - I||_F
// in FP64 (column j of the product by thread j), and, when spd, an FP64
// Cholesky of B~ (global scratch, one p x p slice per block).  flag[e] = 1
// when rho > theta or B~ is not positive definite.
__device__ __forceinline__ double rounded_entry(const double* B, int p, int i, int k, int sym, int prec) {
    double v = B[i * p + k];
    if (sym) v = 0.5 * (v + B[k * p + i]);
    const float f = __double2float_rn(v);
    if (prec == PSR_PREC_BF16) return (double)__bfloat162float(__float2bfloat16_rn(f));
    return (double)f;
}

__global__ void __launch_bounds__(128) k_prec_check(const double* __restrict__ Binv, const double* __restrict__ Adb,
                                                    int m, int p, int sym, int prec, int spd, double theta,
                                                    double* __restrict__ scratch, int32_t* __restrict__ flag) {
    __shared__ double red[4];
    __shared__ int s_bad;
    const int t = threadIdx.x;
    const int64_t pp = (int64_t)p * p;
    double* H = scratch + (int64_t)blockIdx.x * pp;
    for (int e = blockIdx.x; e < m; e += gridDim.x) {
        const double* B = Binv + e * pp;
        const double* A = Adb + e * pp;
        double r2 = 0.0;
        for (int j = t; j < p; j += blockDim.x) {
            for (int i = 0; i < p; ++i) {
                double sacc = 0.0;
                for (int k = 0; k < p; ++k) sacc = fma(rounded_entry(B, p, i, k, sym, prec), A[k * p + j], sacc);
                const double d = sacc - (i == j ? 1.0 : 0.0);
                r2 = fma(d, d, r2);
            }
        }
        r2 = warp_sum(r2);
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = r2;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        bool bad = !(sqrt(tot) <= theta);                // NaN fails too
        if (spd && !bad) {
            for (int q = t; q < (int)pp; q += blockDim.x) H[q] = rounded_entry(B, p, q / p, q % p, 1, prec);
            if (t == 0) s_bad = 0;
            __syncthreads();
            for (int k = 0; k < p; ++k) {
                const double akk = *((volatile double*)&H[k * p + k]);
                if (!(akk > 0.0)) { if (t == 0) s_bad = 1; break; }
                const double lkk = sqrt(akk);
                __syncthreads();
                for (int r = k + 1 + t; r < p; r += blockDim.x) H[r * p + k] /= lkk;
                __syncthreads();
                for (int r = k + 1 + t; r < p; r += blockDim.x) {
                    const double lrk = H[r * p + k];
                    for (int j = k + 1; j <= r; ++j) H[r * p + j] = fma(-lrk, H[j * p + k], H[r * p + j]);
                }
                __syncthreads();
            }
            __syncthreads();
            bad = s_bad != 0;
        }
        if (t == 0) flag[e] = bad ? 1 : 0;
        __syncthreads();
    }
}

// Runs the check on a group's FP64 database (before its conversion) and, when
// an entry fails, keeps an FP64 copy for the flagged entries' tiles.
static int check_precision(psr_ctx* ctx, Group& G, const double* db64, int prec, cudaStream_t s, int* n_bad) {
    *n_bad = 0;
    G.h_hi.clear();
    if (ctx->opts.prec_check <= 0.0 || prec == PSR_PREC_FP64 || !G.dbA || G.m >= G.count || G.m < 1) return PSR_OK;
    const int64_t pp = (int64_t)G.p * G.p;
    const int blocks = std::max(1, std::min(G.m, 152 * 4));
    double* scratch = nullptr;
    int32_t* flag = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&scratch, sizeof(double) * (size_t)blocks * pp));
    PSR_CUDA(ctx, psr::dev_alloc(&flag, sizeof(int32_t) * (size_t)G.m));
    const int spd = (ctx->opts.krylov == PSR_KRYLOV_CG) ? 1 : 0;
    count_launch();
    k_prec_check<<<blocks, 128, 0, s>>>(db64, G.dbA, G.m, G.p, ctx->opts.symmetrize, prec, spd, ctx->opts.prec_check,
                                        scratch, flag);
    PSR_CHECK_LAUNCH(ctx, "k_prec_check");
    std::vector<int32_t> hf(G.m);
    PSR_CUDA(ctx, cudaMemcpyAsync(hf.data(), flag, sizeof(int32_t) * G.m, cudaMemcpyDeviceToHost, s));
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    psr::dev_free(scratch);
    psr::dev_free(flag);
    int bad = 0;
    for (int32_t f : hf) bad += f ? 1 : 0;
    if (bad == 0) return PSR_OK;
    G.h_hi.assign(hf.begin(), hf.end());
    PSR_CUDA(ctx, psr::dev_alloc(&G.rinv_hi, sizeof(double) * (size_t)G.m * pp));
    PSR_CUDA(ctx, cudaMemcpyAsync(G.rinv_hi, db64, sizeof(double) * (size_t)G.m * pp, cudaMemcpyDeviceToDevice, s));
    *n_bad = bad;
    return PSR_OK;
}

// Sweep-order DOF list of a group, gathered from the flat DOF map: sorted
// patch i is patch[i], its DOFs go to sdofs[i * p .. i * p + p).
__global__ void k_gather_sdofs(const int32_t* __restrict__ patch, int count, int p,
                               const int32_t* __restrict__ offsets, const int32_t* __restrict__ dofs,
                               int32_t* __restrict__ sdofs) {
    const int64_t total = (int64_t)count * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / p);
        sdofs[e] = dofs[offsets[patch[i]] + (int)(e - (int64_t)i * p)];
    }
}

// Local-DOF-major copy for the thread-per-patch kernel: sdofs_t[a * count + i].
__global__ void k_transpose_sdofs(const int32_t* __restrict__ sdofs, int count, int p, int32_t* __restrict__ sdofs_t) {
    const int64_t total = (int64_t)count * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / count);
        const int i = (int)(e - (int64_t)a * count);
        sdofs_t[e] = sdofs[(int64_t)i * p + a];
    }
}

static int gather_grid(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8)); }

// Build the sweep layout from the Alg. 1 output left in every group
// (G.sphi = local phi in original order, G.rinv = FP64 database), and the
// global phi / rep_ids.  The DOF lists in sweep order are gathered on the
// device from the flat DOF map (ctx->offsets, ctx->dofs).
int build_sweep_layout(psr_ctx* ctx, const std::vector<std::vector<int32_t>>& gidx, cudaStream_t s) {
    const int prec = ctx->opts.store_prec;
    std::vector<int32_t> phi_global(ctx->n_patches, -1);
    std::vector<int32_t> rep_global;
    int entry_base = 0;
    int n_fallback = 0;
    int64_t factor_bytes = 0, index_bytes = 0;
    for (size_t g = 0; g < ctx->groups.size(); ++g) {
        Group& G = ctx->groups[g];
        const int p = G.p, count = G.count;
        std::vector<int32_t> lphi(count);
        PSR_CUDA(ctx, cudaMemcpy(lphi.data(), G.sphi, sizeof(int32_t) * count, cudaMemcpyDeviceToHost));
        std::vector<int32_t> order(count);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lphi[a] < lphi[b]; });
        std::vector<int32_t> hp(count), hs(count);
        for (int i = 0; i < count; ++i) {
            const int l = order[i];
            const int k = gidx[g][l];
            hp[i] = k;
            hs[i] = lphi[l];
            phi_global[k] = entry_base + lphi[l];
        }
        for (int j = 0; j < G.m; ++j) rep_global.push_back(G.h_rep[j] >= 0 ? gidx[g][G.h_rep[j]] : -1);
        psr::dev_free(G.sphi);
        G.sphi = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&G.patch, sizeof(int32_t) * count));
        PSR_CUDA(ctx, psr::dev_alloc(&G.sphi, sizeof(int32_t) * count));
        PSR_CUDA(ctx, psr::dev_alloc(&G.sdofs, sizeof(int32_t) * (size_t)count * p));
        // on the stream of the gather below (a pageable source is staged
        // before the call returns)
        PSR_CUDA(ctx, cudaMemcpyAsync(G.patch, hp.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
        PSR_CUDA(ctx, cudaMemcpyAsync(G.sphi, hs.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
        count_launch();
        k_gather_sdofs<<<gather_grid((int64_t)count * p), 256, 0, s>>>(G.patch, count, p, ctx->offsets, ctx->dofs, G.sdofs);
        PSR_CHECK_LAUNCH(ctx, "k_gather_sdofs");
        // storage precision
        double* db64 = reinterpret_cast<double*>(G.rinv);
        const int64_t ne = (int64_t)G.m * p * p;
        const bool in_place = (db64 == ctx->A_ext + G.mat_off);
        int n_bad = 0;
        // weakly clustered (more than a quarter of the patches are entries):
        // tiles would hold one or two patches each, so the group is applied
        // like full storage, every patch's entry inverse streamed -- unless the
        // tensor cores are forced or an entry needs its FP64 fallback tiles
        bool expand = G.m < G.count && (int64_t)G.m * 4 > G.count && ctx->opts.sweep_kernel != PSR_SWEEP_TENSOR;
        if (G.m < G.count) {
            int rc = check_precision(ctx, G, db64, prec, s, &n_bad);
            if (rc != PSR_OK) return rc;
            if (n_bad > 0) expand = false;
            if (!expand) n_fallback += n_bad;
        }
        if (G.stream) {
            // inverses already written in the stream layout by the setup
            factor_bytes += (int64_t)G.count * p * p * (int64_t)sizeof(float2);
        } else if (G.m == G.count || expand) {
            // every patch its own entry (or expanded to it): column-major stream (sweep_stream.cu)
            int64_t fb = 0;
            int rc = stream_convert(ctx, G, db64, s, &fb, expand ? G.sphi : nullptr);
            if (rc != PSR_OK) return rc;
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            if (!in_place) psr::dev_free(db64);
            factor_bytes += fb;
        } else if (prec == PSR_PREC_FP64) {
            if (in_place) {
                G.rinv = db64;              // full storage: inverses live where the patches were
            } else {                        // shrink the round buffer to m entries
                double* keep = nullptr;
                PSR_CUDA(ctx, psr::dev_alloc(&keep, sizeof(double) * std::max<int64_t>(ne, 1)));
                PSR_CUDA(ctx, cudaMemcpyAsync(keep, db64, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
                PSR_CUDA(ctx, cudaStreamSynchronize(s));
                psr::dev_free(db64);
                G.rinv = keep;
            }
            factor_bytes += ne * 8;
        } else if (prec == PSR_PREC_FP32) {
            float* f = nullptr;
            PSR_CUDA(ctx, psr::dev_alloc(&f, sizeof(float) * std::max<int64_t>(ne, 1)));
            int blocks = (int)std::min<int64_t>((ne + 255) / 256, 152 * 16);
            count_launch(); k_convert<float><<<std::max(blocks, 1), 256, 0, s>>>(db64, G.m, p, ctx->opts.symmetrize, f);
            PSR_CHECK_LAUNCH(ctx, "k_convert fp32");
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            if (!in_place) psr::dev_free(db64);
            G.rinv = f;
            factor_bytes += ne * 4;
        } else {
            // BF16: clustered groups go to the tensor cores (entries stored in
            // the MMA operand layout) when their 128-patch tiles are at least
            // a quarter full on average: a tile costs the same MMA work
            // whatever its fill.  Full storage and weakly clustered groups
            // stay on the SIMT path.
            int64_t tc_tiles = 0;
            for (int i = 0; i < count;) {
                int j = i;
                while (j < count && hs[j] == hs[i]) ++j;
                tc_tiles += (j - i + 127) / 128;
                i = j;
            }
            G.tc = (G.m < G.count) &&
                   ((int64_t)count * 4 >= tc_tiles * 128 || ctx->opts.sweep_kernel == PSR_SWEEP_TENSOR);
            if (G.tc) {
                __nv_bfloat16* bt = nullptr;
                int rc = convert_tc(db64, G.m, p, ctx->opts.symmetrize, &bt, s);
                if (rc != PSR_OK) { set_error(ctx, "BF16 conversion failed"); return rc; }
                const int P = tc_pad(p);
                factor_bytes += (int64_t)G.m * P * P * 2;
                G.rinv = bt;
            } else {
                __nv_bfloat16* bt = nullptr;
                PSR_CUDA(ctx, psr::dev_alloc(&bt, sizeof(__nv_bfloat16) * std::max<int64_t>(ne, 1)));
                int blocks = (int)std::min<int64_t>((ne + 255) / 256, 152 * 16);
                count_launch(); k_convert<__nv_bfloat16><<<std::max(blocks, 1), 256, 0, s>>>(db64, G.m, p, ctx->opts.symmetrize, bt);
                PSR_CHECK_LAUNCH(ctx, "k_convert bf16");
                factor_bytes += ne * 2;
                G.rinv = bt;
            }
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            if (!in_place) psr::dev_free(db64);
        }
        G.h_sorted_phi = hs;
        if (!G.tc && !G.stream && G.m < G.count && p <= 32) {
            std::vector<int32_t> wt;
            PSR_CUDA(ctx, psr::dev_alloc(&G.sdofs_t, sizeof(int32_t) * (size_t)count * p));
            count_launch();
            k_transpose_sdofs<<<gather_grid((int64_t)count * p), 256, 0, s>>>(G.sdofs, count, p, G.sdofs_t);
            PSR_CHECK_LAUNCH(ctx, "k_transpose_sdofs");
            int i = 0;
            while (i < count) {
                int j = i;
                while (j < count && hs[j] == hs[i]) ++j;
                if (!G.h_hi.empty() && G.h_hi[hs[i]]) { i = j; continue; }   // applied in FP64
                for (int s0 = i; s0 < j; s0 += 32) {
                    wt.push_back(hs[i]);
                    wt.push_back(s0);
                    wt.push_back(std::min(32, j - s0));
                }
                i = j;
            }
            G.nwt = (int)(wt.size() / 3);
            PSR_CUDA(ctx, psr::dev_alloc(&G.wtiles, sizeof(int32_t) * wt.size()));
            PSR_CUDA(ctx, cudaMemcpy(G.wtiles, wt.data(), sizeof(int32_t) * wt.size(), cudaMemcpyHostToDevice));
            G.tpp = true;
        }
        // clustered FP64 entries on pair arithmetic: the thread-per-patch and
        // staged kernels read a pair copy (the FP64 copy stays for the kernels
        // without a pair form: half-warp patches, the grouped launch)
        if (prec == PSR_PREC_FP64 && ctx->opts.fp64_arith == PSR_FP64_PAIRS && G.m < G.count && !G.stream) {
            int rc = pair_db_convert(ctx, G, reinterpret_cast<const double*>(G.rinv), s);
            if (rc != PSR_OK) return rc;
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
        }
        if (!G.stream) {
            int T = G.tc ? 128 : ((p <= 16) ? 64 : 32);
            int rc = make_tiles(ctx, G, G.h_sorted_phi, T);
            if (rc != PSR_OK) return rc;
        }
        index_bytes += (int64_t)count * p * 4 + (int64_t)count * 4;
        entry_base += G.m;
    }
    ctx->m_p = entry_base;
    ctx->h_rep_ids = rep_global;
    PSR_CUDA(ctx, cudaMemcpy(ctx->phi, phi_global.data(), sizeof(int32_t) * ctx->n_patches, cudaMemcpyHostToDevice));
    if (!rep_global.empty())
        PSR_CUDA(ctx, cudaMemcpy(ctx->rep_ids, rep_global.data(), sizeof(int32_t) * rep_global.size(), cudaMemcpyHostToDevice));
    ctx->stats.factor_bytes = factor_bytes;
    ctx->stats.index_bytes = index_bytes;
    ctx->stats.prec_fallback = n_fallback;
    ctx->stats.tc_groups = 0;
    for (const Group& G : ctx->groups) ctx->stats.tc_groups += G.tc ? 1 : 0;
    ctx->stats.m_p = ctx->m_p;
    int rc = build_grouped_tables(ctx);
    if (rc != PSR_OK) return rc;
    rc = stream_build_table(ctx);
    if (rc != PSR_OK) return rc;
    PSR_CUDA(ctx, psr::dev_alloc(&ctx->gcounter, sizeof(int32_t) * 2));
    PSR_CUDA(ctx, cudaMemset(ctx->gcounter, 0, sizeof(int32_t) * 2));
    ctx->grouped_blocks = 152 * 2;
    int mode = ctx->opts.sweep_kernel;
    if (mode == PSR_SWEEP_AUTO) mode = (ctx->groups.size() > 1) ? PSR_SWEEP_GROUPED : PSR_SWEEP_PERGROUP;
    if (mode == PSR_SWEEP_TENSOR) mode = PSR_SWEEP_PERGROUP;
    if (n_fallback > 0) mode = PSR_SWEEP_PERGROUP;         // FP64 tiles of flagged entries run per group
    ctx->sweep_mode = mode;
    return PSR_OK;
}

// Tile table of the grouped persistent kernel: every group's tiles as
// (group, entry, first, count), larger groups first (their heavier tiles are
// dealt out early), plus one descriptor per group.
int build_grouped_tables(psr_ctx* ctx) {
    std::vector<int32_t> gt;
    std::vector<GroupDesc> gd(ctx->groups.size());
    for (size_t g = 0; g < ctx->groups.size(); ++g) {
        Group& G = ctx->groups[g];
        gd[g] = GroupDesc{G.sdofs, G.rinv, G.p, 0};
        if (G.stream) continue;             // streamed by k_sweep_stream
        std::vector<int32_t> ht((size_t)G.ntiles * 3);
        PSR_CUDA(ctx, cudaMemcpy(ht.data(), G.tiles, sizeof(int32_t) * ht.size(), cudaMemcpyDeviceToHost));
        for (int t = 0; t < G.ntiles; ++t) {
            gt.push_back((int)g);
            gt.push_back(ht[3 * t]);
            gt.push_back(ht[3 * t + 1]);
            gt.push_back(ht[3 * t + 2]);
        }
    }
    psr::dev_free(ctx->gtiles);
    psr::dev_free(ctx->gdesc);
    ctx->gntiles = (int)(gt.size() / 4);
    PSR_CUDA(ctx, psr::dev_alloc(&ctx->gtiles, sizeof(int32_t) * std::max<size_t>(gt.size(), 4)));
    PSR_CUDA(ctx, cudaMemcpy(ctx->gtiles, gt.data(), sizeof(int32_t) * gt.size(), cudaMemcpyHostToDevice));
    PSR_CUDA(ctx, psr::dev_alloc(&ctx->gdesc, sizeof(GroupDesc) * std::max<size_t>(gd.size(), 1)));
    PSR_CUDA(ctx, cudaMemcpy(ctx->gdesc, gd.data(), sizeof(GroupDesc) * gd.size(), cudaMemcpyHostToDevice));
    return PSR_OK;
}

// Grid of the streaming sweep (blocks of 8 warps): one warm-up apply, then
// two timed applies per candidate grid, the faster of the two kept.  Streamed
// groups are large (every inverse is read once per apply: 1 ms on the 3D
// Stokes 48^3 workload), so two samples decide, and more would lengthen the
// setup (seven applies here against 21 with the tile tuner's timer).
static int tune_stream_grid(psr_ctx* ctx, double* r, double* z, cudaStream_t s, cudaEvent_t* ev) {
    if (ctx->n_stream == 0) return PSR_OK;
    int rc = sweep_apply_ex(ctx, r, z, nullptr, s);
    if (rc != PSR_OK) return rc;
    const int Bs[] = {152 * 4, 152 * 8, 152 * 16};
    float best = 1e30f;
    int bB = ctx->stream_blocks;
    for (int B : Bs) {
        ctx->stream_blocks = B;
        PSR_CUDA(ctx, cudaEventRecord(ev[0], s));
        if ((rc = sweep_apply_ex(ctx, r, z, nullptr, s)) != PSR_OK) return rc;
        PSR_CUDA(ctx, cudaEventRecord(ev[1], s));
        if ((rc = sweep_apply_ex(ctx, r, z, nullptr, s)) != PSR_OK) return rc;
        PSR_CUDA(ctx, cudaEventRecord(ev[2], s));
        PSR_CUDA(ctx, cudaEventSynchronize(ev[2]));
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        const float ms = std::min(a, b);
        if (ms < best) { best = ms; bB = B; }
    }
    ctx->stream_blocks = bB;
    return PSR_OK;
}

// Project-written autotuner: times candidate tile shapes of the sweep on the
// caller's stream (CUDA events) and keeps the fastest.  Per size group for
// the per-group kernels (patches per tile x warps per CTA, and the
// thread-per-patch kernel where it applies): every candidate's tiles go to
// the device in one copy, all candidates run back to back (one warm-up and
// three timed applies each, median kept) and the host waits once per group.
// Tiles per group x persistent grid size for the grouped kernel.
// Tensor-core tiles are fixed at 128 patches (M = 128).
int autotune_sweep(psr_ctx* ctx, cudaStream_t s) {
    if (!ctx->opts.autotune) return PSR_OK;
    double* r = ctx->ws.r;
    double* z = ctx->ws.z;
    if (!r || !z) return PSR_OK;
    PSR_CUDA(ctx, cudaMemsetAsync(r, 0, sizeof(double) * (size_t)ctx->n, s));
    int rc = PSR_OK;
    if (ctx->sweep_mode == PSR_SWEEP_GROUPED && ctx->opts.store_prec != PSR_PREC_BF16) {
        constexpr int NT = 5;
        cudaEvent_t ev[NT + 1];
        for (auto& e : ev) PSR_CUDA(ctx, cudaEventCreate(&e));
        auto time_apply = [&](float* out_ms) -> int {
            for (int w = 0; w < 2; ++w) {
                int rc2 = sweep_apply_ex(ctx, r, z, nullptr, s);
                if (rc2 != PSR_OK) return rc2;
            }
            cudaEventRecord(ev[0], s);
            for (int it = 0; it < NT; ++it) {
                int rc2 = sweep_apply_ex(ctx, r, z, nullptr, s);
                if (rc2 != PSR_OK) return rc2;
                cudaEventRecord(ev[it + 1], s);
            }
            cudaEventSynchronize(ev[NT]);
            std::vector<float> ts;
            for (int it = 0; it < NT; ++it) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[it], ev[it + 1]);
                ts.push_back(ms);
            }
            std::sort(ts.begin(), ts.end());
            *out_ms = ts[ts.size() / 2];
            return PSR_OK;
        };
        const int Ts[] = {16, 32, 64, 128};
        const int Bs[] = {152 * 2, 152 * 4, 152 * 8};
        float best = 1e30f;
        int bT = 32, bB = 152 * 2;
        for (int T : Ts) {
            if (ctx->gntiles == 0) break;   // every group streamed
            for (auto& G : ctx->groups)
                if (!G.stream && (rc = make_tiles(ctx, G, G.h_sorted_phi, T)) != PSR_OK) break;
            if (rc != PSR_OK || (rc = build_grouped_tables(ctx)) != PSR_OK) break;
            for (int B : Bs) {
                ctx->grouped_blocks = B;
                float ms;
                if ((rc = time_apply(&ms)) != PSR_OK) break;
                if (ms < best) { best = ms; bT = T; bB = B; }
            }
            if (rc != PSR_OK) break;
        }
        if (rc == PSR_OK && ctx->gntiles > 0) {
            for (auto& G : ctx->groups)
                if (!G.stream && (rc = make_tiles(ctx, G, G.h_sorted_phi, bT)) != PSR_OK) break;
            if (rc == PSR_OK) rc = build_grouped_tables(ctx);
            ctx->grouped_blocks = bB;
        }
        if (rc == PSR_OK) rc = tune_stream_grid(ctx, r, z, s, ev);
        for (auto& e : ev) cudaEventDestroy(e);
        return rc;
    }
    constexpr int NT = 3;
    struct Cand { int T, W; bool tpp; size_t off, len; };
    for (auto& G : ctx->groups) {
        if (G.tc || G.stream || (G.m == G.count && G.p <= 32)) continue;   // fixed shapes
        const int shapes[][2] = {{8, 8}, {16, 8}, {16, 4}, {32, 4}, {64, 4}, {32, 8}, {64, 8}, {128, 8}};
        std::vector<Cand> cand;
        std::vector<int32_t> all;
        if (G.tpp) cand.push_back(Cand{G.tile_patches, G.warps, true, 0, 0});
        for (auto& sh : shapes) {
            const std::vector<int32_t> t = tiles_host(G.h_sorted_phi, G.count, sh[0], &G.h_hi, G.h_hi.empty() ? 0 : 1);
            cand.push_back(Cand{sh[0], sh[1], false, all.size(), t.size()});
            all.insert(all.end(), t.begin(), t.end());
        }
        int32_t* d_all = nullptr;
        std::vector<cudaEvent_t> ev(cand.size() * (NT + 1), nullptr);
        PSR_CUDA(ctx, psr::dev_alloc(&d_all, sizeof(int32_t) * std::max<size_t>(all.size(), 3)));
        rc = cuda_fail_if(ctx, cudaMemcpyAsync(d_all, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice, s),
                          "autotune tiles");
        for (size_t e = 0; rc == PSR_OK && e < ev.size(); ++e)
            rc = cuda_fail_if(ctx, cudaEventCreate(&ev[e]), "autotune events");
        // the group's own tiles stay owned by G; candidates point into d_all
        int32_t* own = G.tiles;
        const int own_n = G.ntiles, own_T = G.tile_patches, own_W = G.warps;
        for (size_t c = 0; rc == PSR_OK && c < cand.size(); ++c) {
            G.tpp = cand[c].tpp;
            if (!cand[c].tpp) {
                G.tiles = d_all + cand[c].off;
                G.ntiles = (int)(cand[c].len / 3);
                G.tile_patches = cand[c].T;
                G.warps = cand[c].W;
            }
            cudaEvent_t* e = &ev[c * (NT + 1)];
            if ((rc = sweep_apply_ex(ctx, r, z, nullptr, s)) != PSR_OK) break;
            cudaEventRecord(e[0], s);
            for (int it = 0; it < NT && rc == PSR_OK; ++it) {
                rc = sweep_apply_ex(ctx, r, z, nullptr, s);
                cudaEventRecord(e[it + 1], s);
            }
            G.tiles = own;
            G.ntiles = own_n;
            G.tile_patches = own_T;
            G.warps = own_W;
        }
        if (rc == PSR_OK) rc = cuda_fail_if(ctx, cudaEventSynchronize(ev.back()), "autotune wait");
        float best = 1e30f;
        size_t bc = 0;
        for (size_t c = 0; rc == PSR_OK && c < cand.size(); ++c) {
            float ts[NT];
            for (int it = 0; it < NT; ++it) cudaEventElapsedTime(&ts[it], ev[c * (NT + 1) + it], ev[c * (NT + 1) + it + 1]);
            std::sort(ts, ts + NT);
            if (ts[NT / 2] < best) { best = ts[NT / 2]; bc = c; }
        }
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        if (rc != PSR_OK) { cudaStreamSynchronize(s); psr::dev_free(d_all); break; }
        psr::dev_free(d_all);
        G.tpp = cand[bc].tpp;
        if (!cand[bc].tpp) {
            G.warps = cand[bc].W;
            if ((rc = make_tiles(ctx, G, G.h_sorted_phi, cand[bc].T)) != PSR_OK) break;
        }
    }
    if (rc == PSR_OK) rc = build_grouped_tables(ctx);
    if (rc == PSR_OK && ctx->n_stream > 0) {
        cudaEvent_t ev[3];
        for (auto& e : ev) PSR_CUDA(ctx, cudaEventCreate(&e));
        rc = tune_stream_grid(ctx, r, z, s, ev);
        for (auto& e : ev) cudaEventDestroy(e);
    }
    return rc;
}

// Shared memory of one staged sweep block (two blocks per SM fit).
constexpr size_t STAGED_SMEM_MAX = 96 * 1024;

template <typename T>
static int launch_group_lo(psr_ctx* ctx, const Group& G, const double* r, double* z, const int32_t* stop,
                           cudaStream_t s);

// Tiles (entry, first, count) of one group with inverses of type T: half
// warps per patch for p <= 16, else the staged kernel (the warp kernel when
// a staging does not fit).
template <typename T>
static int launch_tiles(psr_ctx* ctx, int p, const int32_t* tiles, int ntiles, int tile_patches, int warps,
                        const void* rinv_v, const int32_t* sdofs, const double* r, double* z, const int32_t* stop,
                        cudaStream_t s, const void* pair_db = nullptr, const int32_t* pair_exp = nullptr) {
    const int blocks = std::min(ntiles, 152 * 8);
    if (blocks < 1) return PSR_OK;
    const T* rinv = reinterpret_cast<const T*>(rinv_v);
    const int prec = std::is_same<T, double>::value ? PSR_PREC_FP64 : PSR_PREC_FP32;
    const size_t sm = sweep_smem(p, prec, warps);
    if (pair_db && p > 16) {                      // FP64 entries on pair arithmetic, staged
        const bool sym = ctx->Wg != nullptr;
        int sub = tile_patches;
        while (sub > 1 && staged_pair_smem(p, sub, sym) > STAGED_SMEM_MAX) sub >>= 1;
        const size_t ssm = staged_pair_smem(p, sub, sym);
        if (ssm <= STAGED_SMEM_MAX) {
            count_launch();
            k_sweep_staged_pair<<<blocks, warps * 32, ssm, s>>>(tiles, ntiles, p, sub,
                                                                reinterpret_cast<const float2*>(pair_db), pair_exp,
                                                                sdofs, r, ctx->Wg, ctx->W, z, stop);
            PSR_CHECK_LAUNCH(ctx, "sweep kernel (staged, FP64 pairs)");
            return PSR_OK;
        }
    }
    if (p <= 16) {
        count_launch(); k_sweep_half<T><<<blocks, warps * 32, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, ctx->Wg, ctx->W, z, stop);
    } else {
        using C = typename Comp<T>::type;
        const bool sym = ctx->Wg != nullptr;
        int sub = tile_patches;
        while (sub > 1 && staged_smem<C>(p, sub, sym) > STAGED_SMEM_MAX) sub >>= 1;
        const size_t ssm = staged_smem<C>(p, sub, sym);
        if (ssm <= STAGED_SMEM_MAX) {
            count_launch(); k_sweep_staged<T><<<blocks, warps * 32, ssm, s>>>(tiles, ntiles, p, sub, rinv, sdofs, r, ctx->Wg, ctx->W, z, stop);
        } else {
            count_launch(); k_sweep_warp<T><<<blocks, warps * 32, sm, s>>>(tiles, ntiles, p, rinv, sdofs, r, ctx->Wg, ctx->W, z, stop);
        }
    }
    PSR_CHECK_LAUNCH(ctx, "sweep kernel");
    return PSR_OK;
}

// A group's sweep: its tiles in the storage precision, then the tiles of the
// entries that failed the precision check on the FP64 copy.
template <typename T>
static int launch_group(psr_ctx* ctx, const Group& G, const double* r, double* z, const int32_t* stop,
                        cudaStream_t s) {
    int rc = launch_group_lo<T>(ctx, G, r, z, stop, s);
    if (rc != PSR_OK || G.ntiles_hi == 0) return rc;
    return launch_tiles<double>(ctx, G.p, G.tiles_hi, G.ntiles_hi, 32, 4, G.rinv_hi, G.sdofs, r, z, stop, s);
}

template <typename T>
static int launch_group_lo(psr_ctx* ctx, const Group& G, const double* r, double* z, const int32_t* stop,
                           cudaStream_t s) {
    const int warps = G.warps;
    const int prec = ctx->opts.store_prec;
    const size_t sm = sweep_smem(G.p, prec, warps);
    int blocks = std::min(G.ntiles, 152 * 8);
    if (blocks < 1) return PSR_OK;
    const T* rinv = reinterpret_cast<const T*>(G.rinv);
    if (G.tc) {
        int rc = launch_sweep_tc(G.tiles, G.ntiles, G.p, reinterpret_cast<const __nv_bfloat16*>(G.rinv), G.sdofs,
                                 r, ctx->Wg, ctx->W, z, stop, ctx->status, s);
        if (rc != PSR_OK) set_error(ctx, "tensor-core sweep launch failed");
        return rc;
    }
    if (G.tpp && G.rinv_pair && std::is_same<T, double>::value) return launch_sweep_tpp_pair(ctx, G, r, z, stop, s);
    if (G.tpp) {
        const int tb = std::max(1, std::min((G.nwt + 7) / 8, 152 * 16));
        if (G.p <= 16) {
            count_launch(); k_sweep_tpp<T, 16><<<tb, 256, 0, s>>>(G.wtiles, G.nwt, G.p, G.count, rinv, G.sdofs_t, r, ctx->Wg, ctx->W, z, stop);
        } else {
            count_launch(); k_sweep_tpp<T, 32><<<tb, 256, 0, s>>>(G.wtiles, G.nwt, G.p, G.count, rinv, G.sdofs_t, r, ctx->Wg, ctx->W, z, stop);
        }
        PSR_CHECK_LAUNCH(ctx, "sweep kernel (thread per patch)");
        return PSR_OK;
    }
    if (G.m == G.count && G.p <= 32) {
        const int wpb = 8;
        using C = typename Comp<T>::type;
        const size_t slot = (((size_t)G.p * G.p + 32) * sizeof(C) + 15) & ~(size_t)15;
        const int fb = std::min((G.count + wpb - 1) / wpb, 152 * 16);
        count_launch(); k_sweep_full<T><<<fb, wpb * 32, wpb * slot, s>>>(G.count, G.p, rinv, G.sphi, G.sdofs, r, ctx->Wg,
                                                          ctx->W, z, stop);
    } else {
        const bool pairs = std::is_same<T, double>::value && G.rinv_pair != nullptr;
        return launch_tiles<T>(ctx, G.p, G.tiles, G.ntiles, G.tile_patches, warps, G.rinv, G.sdofs, r, z, stop, s,
                               pairs ? G.rinv_pair : nullptr, pairs ? G.bexp : nullptr);
    }
    PSR_CHECK_LAUNCH(ctx, "sweep kernel");
    return PSR_OK;
}

// z = M^-1 r (Eq. 3), plus P0 A0^-1 R0 r when a coarse space is set (Eq. 2)
static int sweep_patches(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s, bool z_zeroed);

int sweep_apply_ex(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s, bool z_zeroed) {
    const int rc = sweep_patches(ctx, r, z, stop, s, z_zeroed);
    if (rc != PSR_OK) return rc;
    return coarse_apply(ctx, r, z, stop, s);
}

static int sweep_patches(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s,
                         bool z_zeroed) {
    if (!z_zeroed) PSR_CUDA(ctx, cudaMemsetAsync(z, 0, sizeof(double) * (size_t)ctx->n, s));
    const int prec = ctx->opts.store_prec;
    if (ctx->n_stream > 0) {
        const int rc = launch_sweep_stream(ctx, r, z, stop, s);
        if (rc != PSR_OK) return rc;
    }
    if (ctx->sweep_mode == PSR_SWEEP_GROUPED && prec != PSR_PREC_BF16) {
        if (ctx->gntiles == 0) return PSR_OK;
        int pmax = 0;
        for (auto& G : ctx->groups) pmax = std::max(pmax, G.p);
        const int warps = 8;
        const size_t sm = sweep_smem(pmax, prec, warps);
        const GroupDesc* gd = reinterpret_cast<const GroupDesc*>(ctx->gdesc);
        if (prec == PSR_PREC_FP64) {
            count_launch(); k_sweep_grouped<double><<<ctx->grouped_blocks, warps * 32, sm, s>>>(ctx->gtiles, ctx->gntiles, gd, r, ctx->Wg, ctx->W, z, ctx->gcounter, pmax, stop);
        } else {
            count_launch(); k_sweep_grouped<float><<<ctx->grouped_blocks, warps * 32, sm, s>>>(ctx->gtiles, ctx->gntiles, gd, r, ctx->Wg, ctx->W, z, ctx->gcounter, pmax, stop);
        }
        PSR_CHECK_LAUNCH(ctx, "grouped sweep");
        return PSR_OK;
    }
    for (auto& G : ctx->groups) {
        if (G.stream) continue;
        int rc = (prec == PSR_PREC_FP64)   ? launch_group<double>(ctx, G, r, z, stop, s)
                 : (prec == PSR_PREC_FP32) ? launch_group<float>(ctx, G, r, z, stop, s)
                                           : launch_group<__nv_bfloat16>(ctx, G, r, z, stop, s);
        if (rc != PSR_OK) return rc;
    }
    return PSR_OK;
}

// Raise the dynamic shared-memory limit of every sweep kernel once, outside
// any stream capture.
int sweep_prepare(psr_ctx* ctx) {
    const int bytes = 200 * 1024;
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_grouped<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_grouped<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_warp<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_staged<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_staged<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_staged<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_staged_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_full<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    {
        int rc = tc_prepare();
        if (rc != PSR_OK) return rc;
    }
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_full<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    PSR_CUDA(ctx, cudaFuncSetAttribute(k_sweep_full<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return PSR_OK;
}

int sweep_apply(psr_ctx* ctx, const double* r, double* z, cudaStream_t s) {
    return sweep_apply_ex(ctx, r, z, nullptr, s);
}

void free_sweep(psr_ctx* ctx) {
    for (auto& G : ctx->groups) {
        psr::dev_free(G.patch);
        psr::dev_free(G.sdofs);
        psr::dev_free(G.sphi);
        psr::dev_free(G.tiles);
        psr::dev_free(G.sdofs_t);
        psr::dev_free(G.wtiles);
        psr::dev_free(G.dbA);
        psr::dev_free(G.bexp);
        psr::dev_free(G.rinv_pair);
        psr::dev_free(G.rinv_hi);
        psr::dev_free(G.tiles_hi);
        if (G.rinv && !(ctx->A_ext && reinterpret_cast<double*>(G.rinv) >= ctx->A_ext &&
                         reinterpret_cast<double*>(G.rinv) < ctx->A_ext + ctx->A_ext_len))
            psr::dev_free(G.rinv);
        G = Group{};
    }
    psr::dev_free(ctx->gtiles);
    psr::dev_free(ctx->gdesc);
    psr::dev_free(ctx->gcounter);
    stream_free(ctx);
    ctx->gtiles = nullptr;
    ctx->gdesc = nullptr;
    ctx->gcounter = nullptr;
}

}  // namespace psr
