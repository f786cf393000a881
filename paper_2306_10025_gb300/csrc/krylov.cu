// Step a5: the outer Krylov solve of A x = b preconditioned on the right by
// the patch sweep (section 4: GMRES with x0 = 0 until the initial residual is
// reduced by 1e-8).  PCG for symmetric positive definite problems with the
// symmetric weighting; flexible GMRES(m) otherwise.
//
// Everything stays on the device: scalars (alpha, beta, Hessenberg matrix,
// Givens rotations, residual estimates) live in device memory and every
// kernel checks a device stop flag, so a whole CG block or FGMRES cycle is
// enqueued (and captured into one CUDA graph) without host decisions; the
// host reads the stop flag once per block / cycle.
//
// Reductions are deterministic: a fixed grid writes per-block partial sums,
// the last block to finish (ticket counter) adds them in a fixed order.
// FGMRES orthogonalises with classical Gram-Schmidt applied twice (two
// batched passes instead of j+1 dependent ones); residual history entries are
// |g_{j+1}| / ||r_0|| as in the FP64 reference formulation.
#include "psr_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <vector>

namespace psr {


enum { S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RN, S_R0, S_RTOL, S_H = 16 };
enum { I_STOP = 0, I_CONV, I_IT, I_K, I_MAXIT, I_M, I_REORTH, I_ERR, I_CNT = 8, I_NCNT = 8 };

struct KDims {
    int n, m, nb;
    double* scal;
    int32_t* ictl;
    double* part;
    double* hist;
    int32_t* rflag;        // [m] second Gram-Schmidt pass taken at step j of the cycle
};

__device__ __forceinline__ double* Hm(double* sc, int m) { return sc + S_H; }
__device__ __forceinline__ double* CSv(double* sc, int m) { return sc + S_H + (m + 1) * m; }
__device__ __forceinline__ double* SNv(double* sc, int m) { return CSv(sc, m) + m; }
__device__ __forceinline__ double* Gv(double* sc, int m) { return SNv(sc, m) + m; }
__device__ __forceinline__ double* Yv(double* sc, int m) { return Gv(sc, m) + m + 1; }
__device__ __forceinline__ double* Hv(double* sc, int m) { return Yv(sc, m) + m; }   // pass vector (<=64)
static inline int scal_count(int m) { return S_H + (m + 1) * m + m + m + (m + 1) + m + 64 + 8; }

// Block-wide sum, result valid in thread 0.  sh: 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < nw) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Last-block ticket: returns true in exactly one block, after every block has
// published its partials.
__device__ __forceinline__ bool last_block(int32_t* cnt) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int t = atomicAdd(cnt, 1);
        s_last = (t == (int)gridDim.x - 1);
        if (s_last) *cnt = 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// part[start], part[start + step], ... below end, with four independent
// accumulators so the loads overlap instead of forming one dependent chain.
__device__ __forceinline__ double sum_strided(const double* part, int start, int end, int step) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = start;
    for (; b + 3 * step < end; b += 4 * step) {
        a0 += part[b];
        a1 += part[b + step];
        a2 += part[b + 2 * step];
        a3 += part[b + 3 * step];
    }
    for (; b < end; b += step) a0 += part[b];
    return (a0 + a1) + (a2 + a3);
}

// Sum of nb partials in a fixed order by the whole block; valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* part, int nb) {
    __shared__ double sp[32];
    return block_sum(sum_strided(part, threadIdx.x, nb, blockDim.x), sp);
}

// Read-only load that the compiler neither sinks into a conditional block nor
// reorders with the other loads of its batch (volatile asm), so that a batch
// of basis loads is in flight together before the first use.
__device__ __forceinline__ double ldnc(const double* p) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ldnc_i(const int32_t* p) {
    int v;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Entries e of basis vectors i0 .. i0+CH-1 (row index clamped to nv-1, so
// every address is valid; the clamped copies are never used).
template <int CH>
__device__ __forceinline__ void load_basis(const double* __restrict__ V, int n, int e, int i0, int nv,
                                           double (&v)[CH]) {
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = ldnc(V + (int64_t)min(i0 + c, nv - 1) * n + e);
}

// ---------------------------------------------------------------- SpMV
// Last block of a reducing SpMV (thread 0): fin 1 = CG pq and alpha;
// fin 2 = FGMRES restart, beta = ||b - A x||.
__device__ void spmv_finish(KDims kd, int fin, double tot) {
    double* sc = kd.scal;
    int32_t* ic = kd.ictl;
    if (fin == 1) {
        sc[S_PQ] = tot;
        sc[S_ALPHA] = sc[S_RZ] / tot;
    } else if (fin == 2) {
        const double beta = sqrt(tot);
        sc[S_RN] = beta;
        double* g = Gv(sc, ic[I_M]);
        g[0] = beta;
        if (beta == 0.0) { ic[I_STOP] = 1; ic[I_CONV] = 1; }
    }
}

// mode 0: y = A x;  mode 1: y = b - A x and ||y||^2;  mode 2: y = A x and (x . y)
template <int TPR>
__global__ void __launch_bounds__(256) k_spmv(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                              const double* __restrict__ vals, const double* __restrict__ x,
                                              double* __restrict__ y, const double* __restrict__ b, int n, int mode,
                                              KDims kd, int stop_check, int fin) {
    __shared__ double sh[32];
    if (stop_check && kd.ictl[I_STOP]) return;
    const int sub = threadIdx.x % TPR;
    const int rows_per_block = blockDim.x / TPR;
    double acc = 0.0;
    // The loop bound is uniform across the warp (rows of one warp move
    // together), so every lane reaches the width-TPR shuffles.
    for (int base = blockIdx.x * rows_per_block; base < n; base += gridDim.x * rows_per_block) {
        const int row = base + threadIdx.x / TPR;
        const bool valid = row < n;
        double s = 0.0;
        if (valid) {
            const int rs = rowptr[row], re = rowptr[row + 1];
            // Four entries per lane per pass.  The loads are unconditional
            // (positions past the row end are clamped to its last entry and
            // their products zeroed), so all twelve of a pass are in flight
            // together instead of each waiting for the multiply before it.
            // The per-lane summation order (e, e + TPR, ...) is unchanged.
            for (int e = rs + sub; e < re; e += 4 * TPR) {
                const bool b1 = e + TPR < re, b2 = e + 2 * TPR < re, b3 = e + 3 * TPR < re;
                const int e1 = b1 ? e + TPR : e, e2 = b2 ? e + 2 * TPR : e, e3 = b3 ? e + 3 * TPR : e;
                const int c0 = ldnc_i(colidx + e), c1 = ldnc_i(colidx + e1);
                const int c2 = ldnc_i(colidx + e2), c3 = ldnc_i(colidx + e3);
                const double a0 = ldnc(vals + e), a1 = ldnc(vals + e1), a2 = ldnc(vals + e2), a3 = ldnc(vals + e3);
                const double x0 = ldnc(x + c0), x1 = ldnc(x + c1), x2 = ldnc(x + c2), x3 = ldnc(x + c3);
                s = fma(a0, x0, s);
                s = fma(b1 ? a1 : 0.0, x1, s);
                s = fma(b2 ? a2 : 0.0, x2, s);
                s = fma(b3 ? a3 : 0.0, x3, s);
            }
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
        if (valid && sub == 0) {
            if (mode == 1) {
                const double v = b[row] - s;
                y[row] = v;
                acc = fma(v, v, acc);
            } else {
                y[row] = s;
                if (mode == 2) acc = fma(x[row], s, acc);
            }
        }
    }
    if (mode == 0) return;
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
    if (!last_block(kd.ictl + I_CNT + 0)) return;
    const double tot = sum_partials(kd.part, gridDim.x);
    if (threadIdx.x != 0) return;
    spmv_finish(kd, fin, tot);
}

// ---------------------------------------------------------------- SpMV (SELL-32)
// Sliced ELL copy of A built at setup: slices of 32 consecutive rows, each
// padded to its longest row and stored column-major (entry k of the slice's
// lane l at slice_ptr[s] + 32 k + l), padding with value 0 and the row's own
// column.  One thread per row: the loads of a warp are contiguous, the
// entries of a row are summed in CSR order by one thread (no cross-lane
// reduction, no FP64 instruction spent on another row's tail: all rows of a
// warp share the slice width).  Four independent accumulation chains per row
// were measured slower on the 2D Stokes workload (27.4 against 24.9 us).
__global__ void k_sell_width(const int32_t* __restrict__ rowptr, int n, int nslices, int32_t* __restrict__ width) {
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nslices) return;
    const int r = s * 32 + lane;
    int len = (r < n) ? rowptr[r + 1] - rowptr[r] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) width[s] = len;
}

__global__ void k_sell_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                            const double* __restrict__ vals, int n, int nslices, const int64_t* __restrict__ sptr,
                            int32_t* __restrict__ scols, double* __restrict__ svals) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = r >> 5, lane = r & 31;
    if (s >= nslices) return;
    const int64_t base = sptr[s] + lane;
    const int width = (int)((sptr[s + 1] - sptr[s]) >> 5);
    const int rs = (r < n) ? rowptr[r] : 0;
    const int len = (r < n) ? rowptr[r + 1] - rs : 0;
    const int self = (r < n) ? r : 0;
    for (int k = 0; k < width; ++k) {
        const bool in = k < len;
        scols[base + 32 * (int64_t)k] = in ? colidx[rs + k] : self;
        svals[base + 32 * (int64_t)k] = in ? vals[rs + k] : 0.0;
    }
}

// Length-sorted slices (SELL-C-sigma): when rows of very different lengths
// alternate (the 3D Stokes velocity rows of vertex, edge, face and cell
// nodes: 43 % padding in slices of consecutive rows), the rows of every
// window of SELL_SIGMA consecutive rows are ordered by decreasing length
// before being cut into slices, and rowmap gives each slice row its row of A.
constexpr int SELL_SIGMA = 1024;

// The row map of the sorted slices: within each window of SELL_SIGMA rows
// (a block each) the rows in decreasing order of length, ties in row order (a
// stable sort), by ranking every row against the window's others in shared
// memory.  Positions past the last row keep -1.
__global__ void __launch_bounds__(SELL_SIGMA) k_sell_sort_windows(const int32_t* __restrict__ rowptr, int n,
                                                                  int32_t* __restrict__ rowmap) {
    __shared__ int32_t slen[SELL_SIGMA];
    const int w0 = blockIdx.x * SELL_SIGMA;
    const int cnt = min(SELL_SIGMA, n - w0);
    const int i = threadIdx.x;
    if (i < cnt) slen[i] = rowptr[w0 + i + 1] - rowptr[w0 + i];
    __syncthreads();
    if (i < cnt) {
        const int li = slen[i];
        int rank = 0;
        for (int j = 0; j < cnt; ++j) {
            const int lj = slen[j];
            rank += (lj > li) || (lj == li && j < i);
        }
        rowmap[w0 + rank] = w0 + i;
    }
}

// Slice widths of the sorted slices: the longest mapped row of each slice.
__global__ void k_sell_width_map(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ rowmap,
                                 int nslices, int32_t* __restrict__ width) {
    const int lane = threadIdx.x & 31;
    const int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslices) return;
    const int r = rowmap[sl * 32 + lane];
    int len = (r >= 0) ? rowptr[r + 1] - rowptr[r] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) width[sl] = len;
}

__global__ void k_sell_fill_map(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                const double* __restrict__ vals, const int32_t* __restrict__ rowmap, int nslices,
                                const int64_t* __restrict__ sptr, int32_t* __restrict__ scols,
                                double* __restrict__ svals) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = r >> 5, lane = r & 31;
    if (s >= nslices) return;
    const int64_t base = sptr[s] + lane;
    const int width = (int)((sptr[s + 1] - sptr[s]) >> 5);
    const int orig = rowmap[r];
    const int rs = (orig >= 0) ? rowptr[orig] : 0;
    const int len = (orig >= 0) ? rowptr[orig + 1] - rs : 0;
    const int self = (orig >= 0) ? orig : 0;
    for (int k = 0; k < width; ++k) {
        const bool in = k < len;
        scols[base + 32 * (int64_t)k] = in ? colidx[rs + k] : self;
        svals[base + 32 * (int64_t)k] = in ? vals[rs + k] : 0.0;
    }
}

// mode 0: y = A x;  mode 1: y = b - A x and ||y||^2;  mode 2: y = A x and (x . y)
// rowmap (or null): the row of A of every padded slice row (-1 for none).
__global__ void __launch_bounds__(256) k_spmv_sell(const int64_t* __restrict__ sptr, const int32_t* __restrict__ scols,
                                                   const double* __restrict__ svals, const int32_t* __restrict__ rowmap,
                                                   const double* __restrict__ x,
                                                   double* __restrict__ y, const double* __restrict__ b, int n,
                                                   int nrows_pad, int mode, KDims kd, int stop_check, int fin) {
    __shared__ double sh[32];
    if (stop_check && kd.ictl[I_STOP]) return;
    double acc = 0.0;
    // block-uniform loop bound: every thread reaches the block reduction
    for (int base = blockIdx.x * blockDim.x; base < nrows_pad; base += gridDim.x * blockDim.x) {
        const int row = base + threadIdx.x;
        const int s = row >> 5, lane = row & 31;
        const bool live = row < nrows_pad;               // whole warps: slices are 32 rows
        const int64_t o = live ? sptr[s] + lane : 0;
        const int width = live ? (int)((sptr[s + 1] - sptr[s]) >> 5) : 0;
        double sum = 0.0;
        // Software pipeline over groups of four entries: the indices and
        // values of group g+1 are requested before the x gathers of group g
        // are consumed, so each group costs about one gather latency.
        const int ng = width >> 2;
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (ng > 0) {
            c0 = ldnc_i(scols + o); c1 = ldnc_i(scols + o + 32); c2 = ldnc_i(scols + o + 64); c3 = ldnc_i(scols + o + 96);
            a0 = ldnc(svals + o); a1 = ldnc(svals + o + 32); a2 = ldnc(svals + o + 64); a3 = ldnc(svals + o + 96);
        }
        for (int g = 0; g < ng; ++g) {
            const double x0 = ldnc(x + c0), x1 = ldnc(x + c1), x2 = ldnc(x + c2), x3 = ldnc(x + c3);
            const double b0 = a0, b1 = a1, b2 = a2, b3 = a3;
            if (g + 1 < ng) {                              // warp-uniform (one slice per warp)
                const int64_t q = o + 128 * (int64_t)(g + 1);
                c0 = ldnc_i(scols + q); c1 = ldnc_i(scols + q + 32); c2 = ldnc_i(scols + q + 64); c3 = ldnc_i(scols + q + 96);
                a0 = ldnc(svals + q); a1 = ldnc(svals + q + 32); a2 = ldnc(svals + q + 64); a3 = ldnc(svals + q + 96);
            }
            sum = fma(b0, x0, sum);
            sum = fma(b1, x1, sum);
            sum = fma(b2, x2, sum);
            sum = fma(b3, x3, sum);
        }
        for (int k = 4 * ng; k < width; ++k)
            sum = fma(ldnc(svals + o + 32 * (int64_t)k), ldnc(x + ldnc_i(scols + o + 32 * (int64_t)k)), sum);
        const int orow = rowmap ? (live ? rowmap[row] : -1) : (row < n ? row : -1);
        if (orow >= 0) {
            if (mode == 1) {
                const double v = b[orow] - sum;
                y[orow] = v;
                acc = fma(v, v, acc);
            } else {
                y[orow] = sum;
                if (mode == 2) acc = fma(x[orow], sum, acc);
            }
        }
    }
    if (mode == 0) return;
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
    if (!last_block(kd.ictl + I_CNT + 0)) return;
    const double tot = sum_partials(kd.part, gridDim.x);
    if (threadIdx.x != 0) return;
    spmv_finish(kd, fin, tot);
}

// ---------------------------------------------------------------- vectors
// ||v||^2 -> initial residual (fin 0) ; also copies v into out (if non-null)
__global__ void k_init_norm(const double* __restrict__ v, double* __restrict__ out1, double* __restrict__ out2,
                            int n, KDims kd, int zero_x, double* __restrict__ x) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double a = v[i];
        if (out1) out1[i] = a;
        if (out2) out2[i] = a;
        if (zero_x) x[i] = 0.0;
        acc = fma(a, a, acc);
    }
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
    if (!last_block(kd.ictl + I_CNT + 1)) return;
    const double tot = sum_partials(kd.part, gridDim.x);
    if (threadIdx.x != 0) return;
    double* sc = kd.scal;
    int32_t* ic = kd.ictl;
    const double r0 = sqrt(tot);
    sc[S_R0] = r0;
    sc[S_RN] = r0;
    kd.hist[0] = 1.0;
    ic[I_IT] = 0;
    ic[I_K] = 0;
    ic[I_CONV] = (r0 == 0.0);
    ic[I_STOP] = (r0 == 0.0);
    if (ic[I_M] > 0) Gv(sc, ic[I_M])[0] = r0;
}

// dot(a, b) with a finalisation: fin 1 = CG rz initial; fin 2 = CG beta update
__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int n, KDims kd, int fin) {
    __shared__ double sh[32];
    if (kd.ictl[I_STOP]) return;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc = fma(a[i], b[i], acc);
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
    if (!last_block(kd.ictl + I_CNT + 2)) return;
    const double tot = sum_partials(kd.part, gridDim.x);
    if (threadIdx.x != 0) return;
    double* sc = kd.scal;
    if (fin == 1) {
        sc[S_RZ] = tot;
    } else {
        sc[S_BETA] = tot / sc[S_RZ];
        sc[S_RZ] = tot;
    }
}

__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, int n, KDims kd) {
    if (kd.ictl[I_STOP]) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// CG: x += alpha p; r -= alpha q; ||r|| -> history, convergence
__global__ void k_cg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                        const double* __restrict__ q, int n, KDims kd) {
    __shared__ double sh[32];
    if (kd.ictl[I_STOP]) return;
    const double alpha = kd.scal[S_ALPHA];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
    if (!last_block(kd.ictl + I_CNT + 3)) return;
    const double tot = sum_partials(kd.part, gridDim.x);
    if (threadIdx.x != 0) return;
    double* sc = kd.scal;
    int32_t* ic = kd.ictl;
    const double rn = sqrt(tot);
    sc[S_RN] = rn;
    const int it = ic[I_IT] + 1;
    ic[I_IT] = it;
    kd.hist[it] = rn / sc[S_R0];
    if (rn <= sc[S_RTOL] * sc[S_R0]) { ic[I_CONV] = 1; ic[I_STOP] = 1; }
    else if (it >= ic[I_MAXIT]) ic[I_STOP] = 1;
}

__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z, int n, KDims kd) {
    if (kd.ictl[I_STOP]) return;
    const double beta = kd.scal[S_BETA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = fma(beta, p[i], z[i]);
}

// ---------------------------------------------------------------- pair arithmetic
// A value carried as an unevaluated pair of FP32 numbers hi + lo (about 48
// significant bits).  On this GPU FP64 instructions, conversions between FP64
// and FP32 included, issue at 2 per clock per SM and FP32 ones at 128, so the
// fused Arnoldi step does its dot products and updates on pairs.  The error-free
// transformations are Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based
// TwoProduct; the _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// exact when |a| >= |b| or a == 0
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (ah, al) += (xh + xl)(yh + yl), the xl*yl term dropped (below 2^-46 of the product)
__device__ __forceinline__ void df_fma(float& ah, float& al, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    const float pe = __fmaf_rn(xh, yh, -p);
    const float c = __fmaf_rn(xh, yl, __fmul_rn(xl, yh));
    float t, e;
    two_sum(ah, p, t, e);
    ah = t;
    al = __fadd_rn(al, __fadd_rn(e, __fadd_rn(pe, c)));
}

__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
    float t, e;
    two_sum(ah, bh, t, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(t, e, ah, al);
}

// x = hi + lo: hi = x truncated to 24 significant bits (built from the bit
// fields, no conversion instruction), lo = x - hi rounded to FP32 (relative
// error 2^-47 of x).  Outside the FP32 normal range hi = 0 and lo = fl32(x).
__device__ __forceinline__ float2 split_f64(double x) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    const bool normal = ex > 896 && ex < 1151;
    const double t = normal ? __longlong_as_double(b & (long long)0xFFFFFFFFE0000000ull) : 0.0;
    const unsigned int hb = ((unsigned int)((unsigned long long)b >> 32) & 0x80000000u) |
                            ((unsigned int)(ex - 896) << 23) | (unsigned int)((b >> 29) & 0x7fffff);
    return make_float2(normal ? __uint_as_float(hb) : 0.f, __double2float_rn(x - t));
}

// ---------------------------------------------------------------- FGMRES
// cycle start: V_0 = r / beta, g = (beta, 0, ...), K = 0
// (with Vs0: the pair copy of V_0 for the fused Arnoldi step, and V_0 the
// exact FP64 value of the pair)
// Z0 (may be null): cleared for the first sweep of the cycle, which adds
// into it.
__global__ void k_fg_start(const double* __restrict__ r, double* __restrict__ V0, float2* __restrict__ Vs0, int n,
                           KDims kd, double* __restrict__ Z0) {
    if (kd.ictl[I_STOP]) return;
    const double beta = kd.scal[S_RN];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (Z0) Z0[i] = 0.0;
        const double v = r[i] / beta;
        if (Vs0) {
            const float2 q = split_f64(v);
            Vs0[i] = q;
            V0[i] = (double)q.x + (double)q.y;
        } else {
            V0[i] = v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int m = kd.m;
        double* g = Gv(kd.scal, m);
        g[0] = beta;
        for (int i = 1; i <= m; ++i) g[i] = 0.0;
        kd.ictl[I_K] = 0;
    }
}

// ---- classical Gram-Schmidt, applied twice (CGS2)
// The nv = j + 1 basis vectors V_0..V_j are rows of V (stride n).  Kernels are
// templated on NV >= nv (8, 16 or 32 per-thread accumulators / basis values),
// run 256-thread blocks on a single-wave grid (kgrid) and reduce per vector
// deterministically: warp -> block partial -> last block in fixed order.
constexpr int KT = 256;                 // threads per block of the CGS2 kernels

// FP64 operations that depend on each other take about 64 clocks each on this
// GPU (FP32: about 5), so the sums on the critical path of a step are trees in
// a fixed order (the same in every block), never running chains.
static_assert(KT / 32 == 8, "tree8 sums one value per warp of a block");
__device__ __forceinline__ double tree8(const double* x) {
    return ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
}

// Sum over a KT-thread block, the total in every thread (fixed order).
// sh: at least KT / 32 doubles of shared memory.
__device__ __forceinline__ double block_sum_kt(double v, double* sh) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    return tree8(sh);
}

// Total of G block partials part[0..G) in every thread.
__device__ __forceinline__ double norm_total(const double* __restrict__ part, int G, double* sh) {
    double u = 0.0;
    for (int k = threadIdx.x; k < G; k += KT) u += part[k];
    return block_sum_kt(u, sh);
}

// acc[i] of every thread -> part[i * gridDim.x + blockIdx.x] (i < nv): the
// warp sums NV accumulators by recursive halving (at step h a lane keeps the
// half of the indices picked by its lane bit h and adds its partner's copy,
// so lane L ends with vector L mod NV), then lanes that differ above bit
// log2(NV) are added, then the warps of the block in order.
template <int NV>
__device__ __forceinline__ void block_partials(double (&acc)[NV], int nv, double* __restrict__ part,
                                               double (*sh)[KT / 32 + 1]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int h = NV / 2; h >= 1; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = upper ? acc[i] : acc[i + h];
            const double keep = upper ? acc[i + h] : acc[i];
            acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
#pragma unroll
    for (int o = NV; o < 32; o <<= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
    if (lane < NV) sh[lane][wid] = acc[0];
    __syncthreads();
    if (threadIdx.x < nv) part[threadIdx.x * gridDim.x + blockIdx.x] = tree8(sh[threadIdx.x]);
}

// Last block: total of vector i = threadIdx.x / (KT / NV) over the G block
// partials, in a fixed order; valid where threadIdx.x % (KT / NV) == 0.
template <int NV>
__device__ __forceinline__ double final_partials(const double* __restrict__ part, int nv, int G) {
    constexpr int T = KT / NV;           // threads per vector, <= 32
    const int i = threadIdx.x / T, q = threadIdx.x % T;
    double v = 0.0;
    if (i < nv) {
        if (G <= KT) {
            // every load of the thread in flight at once (G / T <= NV of them)
            double x[NV];
#pragma unroll
            for (int u = 0; u < NV; ++u) x[u] = (q + u * T < G) ? part[(int64_t)i * G + q + u * T] : 0.0;
#pragma unroll
            for (int h = NV / 2; h >= 1; h >>= 1)     // pairwise tree
#pragma unroll
                for (int u = 0; u < h; ++u) x[u] = x[u] + x[u + h];
            v = x[0];
        } else {
            v = sum_strided(part + (int64_t)i * G, q, G, T);
        }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, T);
    return v;
}

// The vector totals of final_partials and, valid in thread 0, the total of
// the G norm partials stored after them (part[NV * G ...]); the norm
// partials are requested before the vector partials so that both are in
// flight together.
template <int NV>
__device__ __forceinline__ double final_partials_w2(const double* __restrict__ part, int nv, int G, double* shw,
                                                    double& w2) {
    double u = 0.0;
    for (int k = threadIdx.x; k < G; k += KT) u += part[(int64_t)NV * G + k];
    const double v = final_partials<NV>(part, nv, G);
    w2 = block_sum_kt(u, shw);
    return v;
}

// Arnoldi finish of step j (thread 0 of the last block): H[j+1][j] = ||w||,
// the previous Givens rotations applied to column j, the new rotation, the
// residual estimate |g_{j+1}| and the stopping tests.
__device__ void arnoldi_finish(KDims kd, int j, double wn2) {
    double* sc = kd.scal;
    int32_t* ic = kd.ictl;
    const int m = kd.m;
    double* H = Hm(sc, m);
    double* cs = CSv(sc, m);
    double* sn = SNv(sc, m);
    double* g = Gv(sc, m);
    const double hn = sqrt(wn2);
    H[(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
    }
    const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
    cs[j] = H[j * m + j] / den;
    sn[j] = H[(j + 1) * m + j] / den;
    H[j * m + j] = den;
    sc[S_BETA] = hn;                    // keep ||w|| for the normalisation
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const int it = ic[I_IT] + 1;
    ic[I_IT] = it;
    ic[I_K] = j + 1;
    const double res = fabs(g[j + 1]);
    kd.hist[it] = res / sc[S_R0];
    sc[S_RN] = res;
    if (res <= sc[S_RTOL] * sc[S_R0]) { ic[I_CONV] = 1; ic[I_STOP] = 1; }
    else if (it >= ic[I_MAXIT] || den == 0.0) ic[I_STOP] = 1;
}

// Arnoldi finish of step j in the fused step, by warp 0 of block 0 on shared
// copies loaded at the start of the launch: col = H[0..j][j] before the
// rotations, rot = the previous cosines (rot[0..j-1]) and sines
// (rot[NV..NV+j-1]), sg = {g[j], r0, rtol}, si = {iteration count, cap};
// hn = ||w||.  The previous rotations applied in order leave entry i as
// cs_i d_i + sn_i c_{i+1} with d_0 = c_0 and d_i = cs_{i-1} c_i - sn_{i-1} d_{i-1},
// a first-order linear recurrence: lanes compose the affine maps
// d -> a d + b in an inclusive scan (5 dependent steps instead of j).
__device__ void arnoldi_finish_warp(KDims kd, int j, double hn, const double* col, const double* rot, int NV,
                                    const double* sg, const int* si) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    double* sc = kd.scal;
    int32_t* ic = kd.ictl;
    const int m = kd.m;
    double* H = Hm(sc, m);
    const double ci = lane <= j ? col[lane] : 0.0;
    const bool mid = lane >= 1 && lane <= j;
    double a = mid ? -rot[NV + lane - 1] : 0.0;
    double b = mid ? rot[lane - 1] * ci : (lane == 0 ? ci : 0.0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double ap = __shfl_up_sync(full, a, off);
        const double bp = __shfl_up_sync(full, b, off);
        if (lane >= off) {
            b = fma(a, bp, b);
            a = a * ap;
        }
    }
    const double cnext = __shfl_down_sync(full, ci, 1);     // c_{i+1}
    const double dj = __shfl_sync(full, b, j);
    const double den = hypot(dj, hn);
    const double cj = dj / den, sj = hn / den;
    if (lane < j) H[lane * m + j] = rot[lane] * b + rot[NV + lane] * cnext;
    if (lane == j) H[j * m + j] = den;
    if (lane != 0) return;
    H[(j + 1) * m + j] = 0.0;
    CSv(sc, m)[j] = cj;
    SNv(sc, m)[j] = sj;
    sc[S_BETA] = hn;
    double* g = Gv(sc, m);
    const double gj = sg[0];
    const double g1 = -sj * gj;
    g[j + 1] = g1;
    g[j] = cj * gj;
    const int it = si[0] + 1;
    ic[I_IT] = it;
    ic[I_K] = j + 1;
    const double res = fabs(g1);
    kd.hist[it] = res / sg[1];
    sc[S_RN] = res;
    if (res <= sg[2] * sg[1]) { ic[I_CONV] = 1; ic[I_STOP] = 1; }
    else if (it >= si[1] || den == 0.0) ic[I_STOP] = 1;
}

// h = V^T w and ||w||^2 (first pass): H[:, j] = h, h kept for the update.
// The last block also decides whether the step needs a second pass: by the
// Kahan-Parlett criterion ("twice is enough"), when the projected vector
// keeps less than half of the squared norm, ||w||^2 - ||h||^2 < ||w||^2 / 2.
template <int NV>
__global__ void __launch_bounds__(KT) k_mdot(const double* __restrict__ V, const double* __restrict__ w, int n,
                                             int j, KDims kd) {
    __shared__ double sh[NV][KT / 32 + 1];
    __shared__ double shw[32];
    if (kd.ictl[I_STOP]) return;
    const int nv = j + 1;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    double accw = 0.0;
    constexpr int CH = NV < 16 ? NV : 16;
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
        const double we = w[e];
        accw = fma(we, we, accw);
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < nv) {
                double v[CH];
                load_basis<CH>(V, n, e, c0, nv, v);
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < nv) acc[c0 + c] = fma(v[c], we, acc[c0 + c]);
            }
        }
    }
    block_partials<NV>(acc, nv, kd.part, sh);
    const double bw = block_sum(accw, shw);
    if (threadIdx.x == 0) kd.part[(int64_t)NV * gridDim.x + blockIdx.x] = bw;
    if (!last_block(kd.ictl + I_CNT + 4)) return;
    const double v = final_partials<NV>(kd.part, nv, gridDim.x);
    const double wn2 = sum_partials(kd.part + (int64_t)NV * gridDim.x, gridDim.x);
    const int m = kd.m;
    const int i = threadIdx.x / (KT / NV);
    if (i < nv && threadIdx.x % (KT / NV) == 0) {
        Hv(kd.scal, m)[i] = v;
        Hm(kd.scal, m)[i * m + j] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double* hv = Hv(kd.scal, m);
        double h2 = 0.0;
        for (int q = 0; q < nv; ++q) h2 = fma(hv[q], hv[q], h2);
        const int rf = (wn2 - h2 < 0.5 * wn2) ? 1 : 0;
        kd.ictl[I_REORTH] = rf;
        kd.rflag[j] = rf;
    }
}

// Update w <- w - V h.  Without a second pass it also accumulates ||w||^2
// and its last block finishes the Arnoldi step; with one, it accumulates the
// second projection h2 = V^T w on the same loads of V (H[:, j] += h2, h2 kept
// for the second update).
template <int NV>
__global__ void __launch_bounds__(KT) k_maxpy_mdot(const double* __restrict__ V, double* __restrict__ w, int n,
                                                   int j, KDims kd) {
    __shared__ double sh[NV][KT / 32 + 1];
    __shared__ double sh_h[NV];
    __shared__ double shw[32];
    if (kd.ictl[I_STOP]) return;
    const bool reorth = kd.ictl[I_REORTH] != 0;
    const int nv = j + 1;
    const int m = kd.m;
    if (threadIdx.x < NV) sh_h[threadIdx.x] = (threadIdx.x < nv) ? Hv(kd.scal, m)[threadIdx.x] : 0.0;
    __syncthreads();
    if (!reorth) {
        double accw = 0.0;
        constexpr int CH = NV < 16 ? NV : 16;
        for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
            double we = w[e];
#pragma unroll
            for (int c0 = 0; c0 < NV; c0 += CH) {
                if (c0 < nv) {
                    double v[CH];
                    load_basis<CH>(V, n, e, c0, nv, v);
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (c0 + c < nv) we = fma(-sh_h[c0 + c], v[c], we);
                }
            }
            w[e] = we;
            accw = fma(we, we, accw);
        }
        const double bs = block_sum(accw, shw);
        if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
        if (!last_block(kd.ictl + I_CNT + 5)) return;
        const double tot = sum_partials(kd.part, gridDim.x);
        if (threadIdx.x == 0) arnoldi_finish(kd, j, tot);
        return;
    }
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    constexpr int CH = NV < 16 ? NV : 16;
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
        double we = w[e];
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < nv) {
                double v[CH];
                load_basis<CH>(V, n, e, c0, nv, v);
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < nv) we = fma(-sh_h[c0 + c], v[c], we);
            }
        }
        w[e] = we;
        // second projection: the chunks are read again (L1 hits)
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < nv) {
                double v[CH];
                load_basis<CH>(V, n, e, c0, nv, v);
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < nv) acc[c0 + c] = fma(v[c], we, acc[c0 + c]);
            }
        }
    }
    block_partials<NV>(acc, nv, kd.part, sh);
    if (!last_block(kd.ictl + I_CNT + 4)) return;
    const double v = final_partials<NV>(kd.part, nv, gridDim.x);
    const int i = threadIdx.x / (KT / NV);
    if (i < nv && threadIdx.x % (KT / NV) == 0) {
        Hv(kd.scal, m)[i] = v;
        Hm(kd.scal, m)[i * m + j] += v;
    }
}

// Second update w <- w - V h2 with ||w||^2 and the Arnoldi finish; returns at
// once when the step needed no second pass.
template <int NV>
__global__ void __launch_bounds__(KT) k_maxpy(const double* __restrict__ V, double* __restrict__ w, int n, int j,
                                              KDims kd) {
    __shared__ double sh[32];
    __shared__ double sh_h[NV];
    if (kd.ictl[I_STOP] || !kd.ictl[I_REORTH]) return;
    const int nv = j + 1;
    const int m = kd.m;
    if (threadIdx.x < NV) sh_h[threadIdx.x] = (threadIdx.x < nv) ? Hv(kd.scal, m)[threadIdx.x] : 0.0;
    __syncthreads();
    double acc = 0.0;
    constexpr int CH = NV < 16 ? NV : 16;
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
        double we = w[e];
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < nv) {
                double v[CH];
                load_basis<CH>(V, n, e, c0, nv, v);
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < nv) we = fma(-sh_h[c0 + c], v[c], we);
            }
        }
        w[e] = we;
        acc = fma(we, we, acc);
    }
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) kd.part[blockIdx.x] = bs;
    if (!last_block(kd.ictl + I_CNT + 5)) return;
    const double tot = sum_partials(kd.part, gridDim.x);
    if (threadIdx.x == 0) arnoldi_finish(kd, j, tot);
}

// ---------------------------------------------------------------- fused Arnoldi step
// Grid barrier of a cooperatively launched kernel (all blocks co-resident, so
// every wait ends); the spin is bounded all the same: past the limit the
// error flag is set, the stop flag raised and the barrier left, so a fault
// surfaces as PSR_ERR_TIMEOUT on the host instead of a hang.
__device__ __forceinline__ void grid_barrier(unsigned int* bar, int32_t* ictl) {
    __threadfence();                                  // every thread's writes before arriving
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = bar + 1;
        const unsigned int g = *vgen;
        const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g) {
                if (++spins > (1ll << 24)) {
                    atomicExch(ictl + I_ERR, 1);
                    atomicExch(ictl + I_STOP, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// w <- w - V h over the thread's elements (h in shared memory, nv entries);
// PROJ: also acc[i] += V_i[e] w[e] (second projection), else accw += w[e]^2.
template <int NV, bool PROJ>
__device__ __forceinline__ void update_pass(const double* __restrict__ V, double* __restrict__ w, int n, int nv,
                                            const double* sh_h, double (&acc)[NV], double& accw) {
    constexpr int CH = NV < 16 ? NV : 16;
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
        double we = w[e];
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < nv) {
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < nv) we = fma(-sh_h[c0 + c], V[(int64_t)(c0 + c) * n + e], we);
            }
        }
        w[e] = we;
        if (PROJ) {
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i < nv) acc[i] = fma(V[(int64_t)i * n + e], we, acc[i]);
        } else {
            accw = fma(we, we, accw);
        }
    }
}

// Pair form of block_partials: the same recursive halving on (hi, lo)
// accumulators, one conversion to FP64 per lane, then the warps in order.
template <int NV>
__device__ __forceinline__ void block_partials_df(float (&ah)[NV], float (&al)[NV], int nv, double* __restrict__ part,
                                                  double (*sh)[KT / 32 + 1]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int h = NV / 2; h >= 1; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send_h = upper ? ah[i] : ah[i + h];
            const float send_l = upper ? al[i] : al[i + h];
            const float keep_h = upper ? ah[i + h] : ah[i];
            const float keep_l = upper ? al[i + h] : al[i];
            const float rh = __shfl_xor_sync(0xffffffffu, send_h, h);
            const float rl = __shfl_xor_sync(0xffffffffu, send_l, h);
            ah[i] = keep_h;
            al[i] = keep_l;
            df_add(ah[i], al[i], rh, rl);
        }
    }
#pragma unroll
    for (int o = NV; o < 32; o <<= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, ah[0], o);
        const float rl = __shfl_xor_sync(0xffffffffu, al[0], o);
        df_add(ah[0], al[0], rh, rl);
    }
    if (lane < NV) sh[lane][wid] = (double)ah[0] + (double)al[0];
    __syncthreads();
    if (threadIdx.x < nv) part[threadIdx.x * gridDim.x + blockIdx.x] = tree8(sh[threadIdx.x]);
}

// Pair update of the scaled vector w' (pair copy Ws, multiplied on load by
// the power of two scf): w' <- scf w' - V hs with hs the pair coefficients in
// shared memory; PROJ: also (ah, al)_i += V_i[e] w'[e] (second projection),
// else accw += w'[e]^2 in FP64.
template <int NV, bool PROJ>
__device__ __forceinline__ void pair_update(const float2* __restrict__ Vs, float2* __restrict__ Ws, int n, int nv,
                                            const float2* hs, float scf, float (&ah)[NV], float (&al)[NV],
                                            double& accw, float* nh2 = nullptr) {
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
        // all loads first (rows past nv read as zero, their coefficients are
        // zero), then the arithmetic without branches
        float2 vv[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) vv[c] = (c < nv) ? Vs[(int64_t)c * n + e] : make_float2(0.f, 0.f);
        float2 q = Ws[e];
        q.x *= scf;
        q.y *= scf;
        // V hs in four independent chains (c mod 4), joined at the end
        float ch[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < NV; ++c) df_fma(ch[c & 3], cl[c & 3], hs[c].x, hs[c].y, vv[c].x, vv[c].y);
        df_add(ch[0], cl[0], ch[1], cl[1]);
        df_add(ch[2], cl[2], ch[3], cl[3]);
        df_add(ch[0], cl[0], ch[2], cl[2]);
        const float sh_ = ch[0], sl_ = cl[0];
        float t, d, nh, nl;
        two_sum(q.x, -sh_, t, d);
        d = __fadd_rn(d, __fsub_rn(q.y, sl_));
        fast_two_sum(t, d, nh, nl);
        Ws[e] = make_float2(nh, nl);
        if (PROJ) {
#pragma unroll
            for (int i = 0; i < NV; ++i) df_fma(ah[i], al[i], vv[i].x, vv[i].y, nh, nl);
            if (nh2) df_fma(nh2[0], nh2[1], nh, nl, nh, nl);     // ||w'||^2 on pairs
        } else {
            const double wd = (double)nh + (double)nl;
            accw = fma(wd, wd, accw);
        }
    }
}

// The last update fused with the normalisation when ||w'|| is known before it:
// w' <- (scf w' - V hs) * inv, written as the pair Ws and the FP64 w.  The
// product by inv on pairs when pair_scale, else in FP64.
template <int NV, bool PAIR_SCALE>
__device__ __forceinline__ void pair_update_normalize(const float2* __restrict__ Vs, float2* __restrict__ Ws,
                                                      double* __restrict__ w, int n, int nv, const float2* hs,
                                                      float scf, double inv) {
    const float2 is = split_f64(PAIR_SCALE ? inv : 1.0);
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
        float2 vv[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) vv[c] = (c < nv) ? Vs[(int64_t)c * n + e] : make_float2(0.f, 0.f);
        float2 q = Ws[e];
        q.x *= scf;
        q.y *= scf;
        float ch[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < NV; ++c) df_fma(ch[c & 3], cl[c & 3], hs[c].x, hs[c].y, vv[c].x, vv[c].y);
        df_add(ch[0], cl[0], ch[1], cl[1]);
        df_add(ch[2], cl[2], ch[3], cl[3]);
        df_add(ch[0], cl[0], ch[2], cl[2]);
        float t, d, nh, nl;
        two_sum(q.x, -ch[0], t, d);
        d = __fadd_rn(d, __fsub_rn(q.y, cl[0]));
        fast_two_sum(t, d, nh, nl);
        float2 v;
        if (PAIR_SCALE) {
            const float p = __fmul_rn(nh, is.x);
            const float pe = __fmaf_rn(nh, is.x, -p);
            const float c2 = __fmaf_rn(nh, is.y, __fmul_rn(nl, is.x));
            fast_two_sum(p, __fadd_rn(pe, c2), v.x, v.y);
        } else {
            v = split_f64(((double)nh + (double)nl) * inv);
        }
        Ws[e] = v;
        w[e] = (double)v.x + (double)v.y;
    }
}

// Rare forms of the pair path, out of line like the FP64 form below: the
// last update with the product by inv in FP64 (inv beyond the FP32 range)...
template <int NV>
__device__ __noinline__ void pair_update_normalize_wide(const float2* __restrict__ Vs, float2* __restrict__ Ws,
                                                        double* __restrict__ w, int n, int nv, const float2* hs,
                                                        float scf, double inv) {
    pair_update_normalize<NV, false>(Vs, Ws, w, n, nv, hs, scf, inv);
}

// ... the second update with an explicit norm (when ||x||^2 - ||h2||^2 may
// cancel), returning ||w'||^2 ...
template <int NV>
__device__ __noinline__ double pair_pass3_norm(const float2* __restrict__ Vs, float2* __restrict__ Ws, int n, int nv,
                                               const float2* hs, double* shw, double* __restrict__ P3,
                                               unsigned int* bar, int32_t* ictl) {
    float ah[NV], al[NV];
    double accw = 0.0;
    pair_update<NV, false>(Vs, Ws, n, nv, hs, 1.f, ah, al, accw);
    const double bs = block_sum_kt(accw, shw);
    if (threadIdx.x == 0) P3[(int64_t)NV * gridDim.x + blockIdx.x] = bs;
    grid_barrier(bar, ictl);
    return norm_total(P3 + (int64_t)NV * gridDim.x, gridDim.x, shw);
}

// ... and the normalisation after it.
__device__ __noinline__ void pair_normalize(float2* __restrict__ Ws, double* __restrict__ w, int n, double inv) {
    if (inv <= 0x1p100) {
        const float2 is = split_f64(inv);
        for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
            const float2 q = Ws[e];
            const float p = __fmul_rn(q.x, is.x);
            const float pe = __fmaf_rn(q.x, is.x, -p);
            const float c = __fmaf_rn(q.x, is.y, __fmul_rn(q.y, is.x));
            float vh, vl;
            fast_two_sum(p, __fadd_rn(pe, c), vh, vl);
            Ws[e] = make_float2(vh, vl);
            w[e] = (double)vh + (double)vl;
        }
    } else {
        for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += gridDim.x * KT) {
            const float2 q = Ws[e];
            const float2 v = split_f64(((double)q.x + (double)q.y) * inv);
            Ws[e] = v;
            w[e] = (double)v.x + (double)v.y;
        }
    }
}

// The FP64 form of the step (PSR_ORTHO_FP64, or w outside the pair range),
// kept out of line so that the pair path's code stays contiguous.  All
// threads of the block call them; sh, shw, s_w2, sh_h and s_col are the
// kernel's shared arrays.
// Pass 1 in FP64: h = V^T w (returned where the vector's lane group holds
// it) and ||w||^2 into *s_w2.
template <int NV>
__device__ __noinline__ double fp64_pass1(const double* __restrict__ V, const double* __restrict__ w, int n, int nv,
                                          double* __restrict__ P4, double (*sh)[KT / 32 + 1], double* shw,
                                          double* s_w2, unsigned int* bar, int32_t* ictl) {
    const int G = gridDim.x;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    double accw = 0.0;
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += G * KT) {
        const double we = w[e];
        accw = fma(we, we, accw);
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (i < nv) acc[i] = fma(V[(int64_t)i * n + e], we, acc[i]);
    }
    block_partials<NV>(acc, nv, P4, sh);
    const double bs = block_sum_kt(accw, shw);
    if (threadIdx.x == 0) P4[(int64_t)NV * G + blockIdx.x] = bs;
    grid_barrier(bar, ictl);
    double t;
    const double hv = final_partials_w2<NV>(P4, nv, G, shw, t);
    if (threadIdx.x == 0) *s_w2 = t;
    __syncthreads();
    return hv;
}

// The FP64 updates (the second projection when reorth), the norm and the
// normalisation (with the pair copy); returns ||w||.
template <int NV>
__device__ __noinline__ double fp64_rest(const double* __restrict__ V, double* __restrict__ w,
                                         float2* __restrict__ Ws, int n, int nv, bool reorth, double* sh_h,
                                         double (*sh)[KT / 32 + 1], double* shw, double* s_col, double* s_w2,
                                         double* __restrict__ P2, double* __restrict__ P3, unsigned int* bar,
                                         int32_t* ictl) {
    const int G = gridDim.x;
    constexpr int T = KT / NV;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    double accw = 0.0;
    if (reorth) {
        update_pass<NV, true>(V, w, n, nv, sh_h, acc, accw);
        block_partials<NV>(acc, nv, P2, sh);
        grid_barrier(bar, ictl);
        const double v2 = final_partials<NV>(P2, nv, G);
        __syncthreads();
        if (threadIdx.x / T < nv && threadIdx.x % T == 0) sh_h[threadIdx.x / T] = v2;
        __syncthreads();
        if (blockIdx.x == 0 && threadIdx.x < nv) s_col[threadIdx.x] += sh_h[threadIdx.x];
        update_pass<NV, false>(V, w, n, nv, sh_h, acc, accw);
        const double bs = block_sum_kt(accw, shw);
        if (threadIdx.x == 0) P3[(int64_t)NV * G + blockIdx.x] = bs;
        grid_barrier(bar, ictl);
        const double t = norm_total(P3 + (int64_t)NV * G, G, shw);
        if (threadIdx.x == 0) *s_w2 = t;
    } else {
        update_pass<NV, false>(V, w, n, nv, sh_h, acc, accw);
        const double bs = block_sum_kt(accw, shw);
        if (threadIdx.x == 0) P2[(int64_t)NV * G + blockIdx.x] = bs;
        grid_barrier(bar, ictl);
        const double t = norm_total(P2 + (int64_t)NV * G, G, shw);
        if (threadIdx.x == 0) *s_w2 = t;
    }
    __syncthreads();
    const double hn = sqrt(*s_w2);
    const double inv = hn != 0.0 ? 1.0 / hn : 1.0;
    for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += G * KT) {
        const float2 v = split_f64(w[e] * inv);
        Ws[e] = v;
        w[e] = (double)v.x + (double)v.y;
    }
    return hn;
}

// The whole orthogonalisation of step j in one cooperative launch: w = V_{j+1}
// (on entry A z_j) is projected (h = V^T w, ||w||^2), updated, projected and
// updated again when the Kahan-Parlett test asks for it, normalised, and the
// Arnoldi step finished.  Grid barriers replace the kernel boundaries; every
// block sums the block partials of a pass itself (same order everywhere, so
// all blocks hold bitwise the same h and norms), and each pass has its own
// partial region.
//
// Arithmetic: the basis is read from its pair copy Vs (Vs_i = V_i exactly,
// V_i being written as the FP64 value of its pair); w is split into a pair
// once, dots and updates run on pairs, ||w||^2 and the partial sums in FP64.
// After the first pass w is scaled by the power of two 2^k that brings ||w||
// near 1 (exact), so cancellation in the updates stays far from the FP32
// range limits; the coefficients are scaled alike and unscaled exactly.  When
// ||w||^2 lies outside [2^-160, 2^120], or with fp64 set, the step is computed
// in FP64 instead (the same passes on V), so the pair path never meets
// overflow or underflow of the incoming vector.
template <int NV>
__global__ void __launch_bounds__(KT, 1) k_arnoldi(const double* __restrict__ V, double* __restrict__ w,
                                               float2* __restrict__ Vs, int n, int j, KDims kd,
                                               double* __restrict__ part, unsigned int* bar, int fp64,
                                               double* __restrict__ zn) {
    __shared__ double sh[NV][KT / 32 + 1];
    __shared__ double sh_h[NV];
    __shared__ float2 sh_hs[NV];
    __shared__ double shw[32];
    __shared__ double s_w2;
    __shared__ double s_h2;
    __shared__ int s_reorth;
    __shared__ double s_col[NV + 1];                  // block 0: column j of H
    __shared__ double s_rot[2 * NV];                  // block 0: previous rotations
    __shared__ double s_g[3];
    __shared__ int s_it[2];
    if (kd.ictl[I_STOP]) return;                      // same value in every block
    const int nv = j + 1;
    const int m = kd.m;
    const int G = gridDim.x;
    // the next sweep's output (it adds into a cleared vector); plain stores
    // that no pass of this step waits for
    if (zn)
        for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += G * KT) zn[e] = 0.0;
    const int T = KT / NV;
    if (blockIdx.x == 0) {                            // used by the finish at the end
        if (threadIdx.x < j) {
            s_rot[threadIdx.x] = CSv(kd.scal, m)[threadIdx.x];
            s_rot[NV + threadIdx.x] = SNv(kd.scal, m)[threadIdx.x];
        }
        if (threadIdx.x == 0) {
            s_g[0] = Gv(kd.scal, m)[j];
            s_g[1] = kd.scal[S_R0];
            s_g[2] = kd.scal[S_RTOL];
            s_it[0] = kd.ictl[I_IT];
            s_it[1] = kd.ictl[I_MAXIT];
        }
    }
    double* P1 = part;
    double* P2 = part + (int64_t)(NV + 1) * G;
    double* P3 = part + (int64_t)2 * (NV + 1) * G;
    double* P4 = part + (int64_t)3 * (NV + 1) * G;
    float2* Ws = Vs + (int64_t)nv * n;                // pair copy of w (row j+1)
    double hv = 0.0;
    bool pairs = false;
    // pass 1 on pairs: h = V^T w, ||w||^2 in FP64, Ws = split(w)
    if (!fp64) {
        float ah[NV], al[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) ah[i] = al[i] = 0.f;
        double accw = 0.0;
        for (int e = blockIdx.x * KT + threadIdx.x; e < n; e += G * KT) {
            const double we = w[e];
            float2 vv[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) vv[i] = (i < nv) ? Vs[(int64_t)i * n + e] : make_float2(0.f, 0.f);
            accw = fma(we, we, accw);
            const float2 q = split_f64(we);
            Ws[e] = q;
#pragma unroll
            for (int i = 0; i < NV; ++i) df_fma(ah[i], al[i], vv[i].x, vv[i].y, q.x, q.y);
        }
        block_partials_df<NV>(ah, al, nv, P1, sh);
        const double bs = block_sum_kt(accw, shw);
        if (threadIdx.x == 0) P1[(int64_t)NV * G + blockIdx.x] = bs;
        grid_barrier(bar, kd.ictl);
        double t;
        hv = final_partials_w2<NV>(P1, nv, G, shw, t);
        if (threadIdx.x == 0) s_w2 = t;
        __syncthreads();
        pairs = s_w2 >= 0x1p-160 && s_w2 <= 0x1p120;  // same in every block
    }
    if (!pairs) hv = fp64_pass1<NV>(V, w, n, nv, P4, sh, shw, &s_w2, bar, kd.ictl);
    // scale 2^k of the pair path: ||2^k w|| in [1, 2)
    const int k = pairs ? -(ilogb(s_w2) >> 1) : 0;
    if (threadIdx.x % T == 0) {                       // every slot i < NV (zero past nv)
        sh_h[threadIdx.x / T] = hv;
        sh_hs[threadIdx.x / T] = split_f64(ldexp(hv, k));
    }
    __syncthreads();
    if (threadIdx.x < 32) {                           // ||h||^2 by warp 0 (sh_h is zero past nv)
        const double hq = threadIdx.x < NV ? sh_h[threadIdx.x] : 0.0;
        const double h2 = warp_sum(hq * hq);
        if (threadIdx.x == 0) {
            s_reorth = (s_w2 - h2 < 0.5 * s_w2) ? 1 : 0;
            s_h2 = h2;
        }
    }
    __syncthreads();
    const bool reorth = s_reorth != 0;
    if (blockIdx.x == 0) {
        if (threadIdx.x < nv) s_col[threadIdx.x] = sh_h[threadIdx.x];
        if (threadIdx.x == 0) kd.rflag[j] = reorth ? 1 : 0;
    }
    double hn_w;                                      // ||w|| for H[j+1][j]
    if (pairs) {
        const float scf = ldexpf(1.f, k);             // exact: k in [-60, 80]; w' = 2^k w on the first update
        float ah[NV], al[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) ah[i] = al[i] = 0.f;
        double accw = 0.0;
        // ||w'||^2 of the vector left by the last update.  It is known before
        // that update from ||x||^2 - ||V^T x||^2 (x the vector it starts
        // from, V orthonormal): without a second pass because the
        // Kahan-Parlett test kept more than half of ||w||^2, with one when
        // the second coefficients are below a tenth of ||x|| (the usual
        // case: twice is enough).  Then the last update and the
        // normalisation are one pass and the step saves a grid barrier.
        double ws2 = 0.0;
        bool known = false;
        float last_scf = scf;
        if (reorth) {
            float n2[2] = {0.f, 0.f};
            pair_update<NV, true>(Vs, Ws, n, nv, sh_hs, scf, ah, al, accw, n2);
            block_partials_df<NV>(ah, al, nv, P2, sh);
            {
                const double bs = block_sum_kt((double)n2[0] + (double)n2[1], shw);
                if (threadIdx.x == 0) P2[(int64_t)NV * G + blockIdx.x] = bs;
            }
            grid_barrier(bar, kd.ictl);
            double x2;                                            // ||w1'||^2
            const double v2 = final_partials_w2<NV>(P2, nv, G, shw, x2);      // 2^k h2
            __syncthreads();                                      // sh_hs of pass 2 fully read
            if (threadIdx.x % T == 0) {
                sh_h[threadIdx.x / T] = ldexp(v2, -k);
                sh_hs[threadIdx.x / T] = split_f64(v2);
            }
            __syncthreads();
            if (blockIdx.x == 0 && threadIdx.x < nv) s_col[threadIdx.x] += sh_h[threadIdx.x];
            if (threadIdx.x < 32) {                               // ||2^k h2||^2 by warp 0
                const double hq = threadIdx.x < NV ? sh_h[threadIdx.x] : 0.0;
                const double q2 = warp_sum(hq * hq);
                if (threadIdx.x == 0) s_h2 = ldexp(q2, 2 * k);
            }
            __syncthreads();
            last_scf = 1.f;
            // pairs carry ||w1'||^2 accurately only well inside the FP32 range
            if (x2 >= 0x1p-60 && s_h2 <= 0.01 * x2) {
                ws2 = x2 - s_h2;
                known = true;
            } else {
                ws2 = pair_pass3_norm<NV>(Vs, Ws, n, nv, sh_hs, shw, P3, bar, kd.ictl);
            }
        } else {
            ws2 = ldexp(s_w2 - s_h2, 2 * k);              // > ||w'||^2 / 2 by the test
            known = true;
        }
        // normalise: v = w' / ||w'|| on pairs (inverse within FP32 range), else in FP64
        const double hn = sqrt(ws2);
        hn_w = ldexp(hn, -k);                         // exact: sqrt(2^2k x) = 2^k sqrt(x)
        const double inv = hn != 0.0 ? 1.0 / hn : 1.0;
        if (known && inv <= 0x1p100) {
            pair_update_normalize<NV, true>(Vs, Ws, w, n, nv, sh_hs, last_scf, inv);
        } else if (known) {
            pair_update_normalize_wide<NV>(Vs, Ws, w, n, nv, sh_hs, last_scf, inv);
        } else {
            pair_normalize(Ws, w, n, inv);
        }
    } else {
        hn_w = fp64_rest<NV>(V, w, Ws, n, nv, reorth, sh_h, sh, shw, s_col, &s_w2, P2, P3, bar, kd.ictl);
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) arnoldi_finish_warp(kd, j, hn_w, s_col, s_rot, NV, s_g, s_it);
}

__global__ void k_fg_scale(double* __restrict__ w, int n, KDims kd) {
    if (kd.ictl[I_STOP]) return;
    const double hn = kd.scal[S_BETA];
    if (hn == 0.0) return;
    const double inv = 1.0 / hn;       // one division per thread, FP64 multiplies per element
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = w[i] * inv;
}

// Cycle end: y = H(1:K,1:K)^{-1} g(1:K) by back substitution (one thread).
// End of an FGMRES cycle: y = R^-1 g with R the K x K upper triangle left in
// H by the Givens rotations (K <= 32), then x += sum_{i<K} y_i Z_i; every
// block solves the small system itself.  The block stages R in shared
// memory; warp 0 takes the reciprocals of the diagonal at once, then y_i
// for i = K-1 .. 0, each followed by the update of the remaining right-hand
// sides below it (lane l subtracts R[l][i] y_i), so a step costs a
// multiply, a shuffle and an FMA instead of a division and a row dot.
__global__ void k_fg_update(double* __restrict__ x, const double* __restrict__ Z, int n, KDims kd) {
    __shared__ double sy[32];
    __shared__ double sR[32][33];
    const int K = kd.ictl[I_K];
    if (K == 0) return;
    const int m = kd.m;
    const double* H = Hm(kd.scal, m);
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) sR[e / K][e % K] = H[(e / K) * m + e % K];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        double sl = l < K ? Gv(kd.scal, m)[l] : 0.0;
        const double rinv = l < K ? 1.0 / sR[l][l] : 0.0;
        double yl = 0.0;
        for (int i = K - 1; i >= 0; --i) {
            const double yi = __shfl_sync(0xffffffffu, sl * rinv, i);
            if (l == i) yl = yi;
            if (l < i) sl = fma(-sR[l][i], yi, sl);
        }
        sy[l] = yl;
    }
    __syncthreads();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double xe = x[e];
        for (int i = 0; i < K; ++i) xe = fma(sy[i], Z[(int64_t)i * n + e], xe);
        x[e] = xe;
    }
}

// ---------------------------------------------------------------- host
static int spmv_tpr(psr_ctx* ctx) {
    const double avg = ctx->n ? (double)ctx->nnz / ctx->n : 1.0;
    // each lane loads up to four entries per pass; few lanes per row keep the
    // FP64 reduction across the row's lanes (TPR log2 TPR adds) small
    if (avg <= 64) return 4;
    if (avg <= 128) return 8;
    return 16;
}

static void launch_spmv(psr_ctx* ctx, const double* x, double* y, const double* b, int mode, int fin,
                        KDims kd, int stop_check, int nb_max, cudaStream_t s) {
    const KrylovWS& w = ctx->ws;
    if (w.sell_ptr) {
        const int nrows_pad = w.nslices * 32;
        const int need = (nrows_pad + 255) / 256;
        const int nb = std::max(1, mode == 0 ? need : std::min(need, nb_max));
        count_launch();
        k_spmv_sell<<<nb, 256, 0, s>>>(w.sell_ptr, w.sell_cols, w.sell_vals, w.sell_row, x, y, b, ctx->n, nrows_pad,
                                       mode, kd, stop_check, fin);
        return;
    }
    const int tpr = spmv_tpr(ctx);
    const int n = ctx->n;
    // one row per TPR-thread group; mode 0 (no reduction) covers all rows in
    // one pass, the reducing modes keep the grid within the partial slots
    const int rows_per_block = 256 / tpr;
    const int need = (n + rows_per_block - 1) / rows_per_block;
    const int nb = std::max(1, mode == 0 ? need : std::min(need, nb_max));
    switch (tpr) {
        case 4: count_launch(); k_spmv<4><<<nb, 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, x, y, b, n, mode, kd, stop_check, fin); break;
        case 8: count_launch(); k_spmv<8><<<nb, 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, x, y, b, n, mode, kd, stop_check, fin); break;
        case 16: count_launch(); k_spmv<16><<<nb, 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, x, y, b, n, mode, kd, stop_check, fin); break;
        default: count_launch(); k_spmv<32><<<nb, 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, x, y, b, n, mode, kd, stop_check, fin); break;
    }
}

// ---------------------------------------------------------------- timing
// Per-kernel event marks (psr_set_kernel_timing).  Marks are recorded while a
// block is enqueued (or captured: the event records become graph nodes) and
// read back after the host's per-block synchronisation.
static double sweep_bytes(const psr_ctx* ctx) {
    const double tot = ctx->h_offsets.empty() ? 0.0 : (double)ctx->h_offsets.back();
    return 24.0 * ctx->n + 4.0 * tot + 4.0 * ctx->n_patches + (double)ctx->stats.factor_bytes;
}
static double spmv_bytes(const psr_ctx* ctx) {
    return 12.0 * (double)ctx->nnz + 4.0 * (ctx->n + 1.0) + 16.0 * ctx->n;
}
// FP64 flops of the sweep: the patch products when they run on FP64 units
// (FP64 inverses, except streamed groups applied in FP32 pair arithmetic),
// the weighted scatter-add of every patch DOF
static double sweep_flops(const psr_ctx* ctx) {
    double sp = 0.0, sp2 = 0.0;
    const bool fp64 = ctx->opts.store_prec == PSR_PREC_FP64;
    for (const Group& G : ctx->groups) {
        sp += (double)G.count * G.p;
        // pair arithmetic: streamed groups, and clustered groups with a pair copy
        // in the thread-per-patch or staged kernel (the half-warp kernel of
        // p <= 16 and the grouped launch stay FP64)
        const bool pairs = (G.stream || (G.rinv_pair && (G.tpp || G.p > 16) &&
                                         ctx->sweep_mode != PSR_SWEEP_GROUPED)) &&
                           ctx->opts.fp64_arith != PSR_FP64_NATIVE;
        if (fp64 && !pairs) sp2 += (double)G.count * G.p * G.p;
    }
    return 2.0 * sp2 + 2.0 * sp;
}

// While the stream is captured the record becomes an event-record node of
// the graph (external flag); otherwise it is a plain record.
static cudaError_t kt_record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &st);
    if (ce != cudaSuccess) return ce;
    return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

static int kt_begin(psr_ctx* ctx, int kind, int j, double bytes, double flops, cudaStream_t s) {
    if (!ctx->kt_on) return PSR_OK;
    const size_t i = ctx->kt_marks.size();
    while (ctx->kt_ev.size() < 2 * i + 2) {
        cudaEvent_t e;
        PSR_CUDA(ctx, cudaEventCreate(&e));
        ctx->kt_ev.push_back(e);
    }
    ctx->kt_marks.push_back(KtMark{kind, j, bytes, 0.0, flops, 0.0});
    PSR_CUDA(ctx, kt_record(ctx->kt_ev[2 * i], s));
    return PSR_OK;
}

static int kt_end(psr_ctx* ctx, cudaStream_t s) {
    if (!ctx->kt_on) return PSR_OK;
    const size_t i = ctx->kt_marks.size() - 1;
    PSR_CUDA(ctx, kt_record(ctx->kt_ev[2 * i + 1], s));
    return PSR_OK;
}

// After a block ran `done` iterations (all its events have completed);
// rflag[j] (host copy, FGMRES only) tells whether step j took the second
// Gram-Schmidt pass, whose bytes a mark carries separately.
static int kt_collect(psr_ctx* ctx, int done, const int32_t* rflag) {
    if (!ctx->kt_on) return PSR_OK;
    for (size_t i = 0; i < ctx->kt_marks.size(); ++i) {
        const KtMark& mk = ctx->kt_marks[i];
        if (mk.j >= done) continue;
        float ms = 0.f;
        PSR_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->kt_ev[2 * i], ctx->kt_ev[2 * i + 1]));
        ctx->kt_ms[mk.kind] += ms;
        ctx->kt_n[mk.kind] += 1;
        const bool ro = rflag && rflag[mk.j];
        ctx->kt_bytes[mk.kind] += mk.bytes + (ro ? mk.bytes_reorth : 0.0);
        ctx->kt_flops[mk.kind] += mk.flops + (ro ? mk.flops_reorth : 0.0);
    }
    return PSR_OK;
}

#define KT_BEGIN(kind, j, bytes, flops)                            \
    do {                                                           \
        int rk_ = kt_begin(ctx, (kind), (j), (bytes), (flops), s); \
        if (rk_ != PSR_OK) return rk_;                             \
    } while (0)
// extra bytes / FP64 flops of the mark just opened when its step reorthogonalises
#define KT_REORTH(bytes, flops)                                    \
    do {                                                           \
        if (ctx->kt_on && !ctx->kt_marks.empty()) {                \
            ctx->kt_marks.back().bytes_reorth = (bytes);           \
            ctx->kt_marks.back().flops_reorth = (flops);           \
        }                                                          \
    } while (0)
#define KT_END()                                                   \
    do {                                                           \
        int rk_ = kt_end(ctx, s);                                  \
        if (rk_ != PSR_OK) return rk_;                             \
    } while (0)

int krylov_alloc(psr_ctx* ctx, cudaStream_t s) {
    KrylovWS& w = ctx->ws;
    const size_t n = (size_t)ctx->n;
    int m = ctx->opts.restart;
    if (m < 1) m = 1;
    if (m > 32) m = 32;
    ctx->opts.restart = m;
    w.nblk = (int)std::min<size_t>(std::max<size_t>((n + 255) / 256, 1), 152 * 4);
    PSR_CUDA(ctx, psr::dev_alloc(&w.x, n * 8));
    PSR_CUDA(ctx, psr::dev_alloc(&w.b, n * 8));
    PSR_CUDA(ctx, psr::dev_alloc(&w.r, n * 8));
    PSR_CUDA(ctx, psr::dev_alloc(&w.z, n * 8));
    if (ctx->opts.krylov == PSR_KRYLOV_CG) {
        PSR_CUDA(ctx, psr::dev_alloc(&w.p, n * 8));
        PSR_CUDA(ctx, psr::dev_alloc(&w.q, n * 8));
    } else {
        PSR_CUDA(ctx, psr::dev_alloc(&w.V, (size_t)(m + 1) * n * 8));
        PSR_CUDA(ctx, psr::dev_alloc(&w.Z, (size_t)m * n * 8));
    }
    // SELL-32 copy of A for the SpMV
    {
        w.nslices = (ctx->n + 31) / 32;
        int32_t* widths = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&widths, sizeof(int32_t) * (size_t)w.nslices));
        count_launch();
        k_sell_width<<<(w.nslices + 7) / 8, 256, 0, s>>>(ctx->rowptr, ctx->n, w.nslices, widths);
        std::vector<int32_t> hw((size_t)w.nslices);
        PSR_CUDA(ctx, cudaMemcpyAsync(hw.data(), widths, sizeof(int32_t) * hw.size(), cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        psr::dev_free(widths);
        int64_t natural = 0;
        for (int q = 0; q < w.nslices; ++q) natural += 32 * (int64_t)hw[q];
        // more than 15 % padding on a large matrix: length-sorted windows
        // more than 15 % padding on a large matrix: length-sorted windows,
        // their row map built on the device
        const bool sorted = ctx->nnz > 0 && (double)natural > 1.15 * (double)ctx->nnz && ctx->n >= 4 * SELL_SIGMA;
        if (sorted) {
            PSR_CUDA(ctx, psr::dev_alloc(&w.sell_row, sizeof(int32_t) * (size_t)w.nslices * 32));
            PSR_CUDA(ctx, cudaMemsetAsync(w.sell_row, 0xff, sizeof(int32_t) * (size_t)w.nslices * 32, s));
            count_launch();
            k_sell_sort_windows<<<(ctx->n + SELL_SIGMA - 1) / SELL_SIGMA, SELL_SIGMA, 0, s>>>(ctx->rowptr, ctx->n, w.sell_row);
            int32_t* widths2 = nullptr;
            PSR_CUDA(ctx, psr::dev_alloc(&widths2, sizeof(int32_t) * (size_t)w.nslices));
            count_launch();
            k_sell_width_map<<<(w.nslices + 7) / 8, 256, 0, s>>>(ctx->rowptr, w.sell_row, w.nslices, widths2);
            PSR_CHECK_LAUNCH(ctx, "SELL row map");
            PSR_CUDA(ctx, cudaMemcpyAsync(hw.data(), widths2, sizeof(int32_t) * hw.size(), cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            psr::dev_free(widths2);
        }
        std::vector<int64_t> hp((size_t)w.nslices + 1, 0);
        for (int q = 0; q < w.nslices; ++q) hp[q + 1] = hp[q] + 32 * (int64_t)hw[q];
        const int64_t total = std::max<int64_t>(hp.back(), 1);
        PSR_CUDA(ctx, psr::dev_alloc(&w.sell_ptr, sizeof(int64_t) * hp.size()));
        PSR_CUDA(ctx, cudaMemcpyAsync(w.sell_ptr, hp.data(), sizeof(int64_t) * hp.size(), cudaMemcpyHostToDevice, s));
        PSR_CUDA(ctx, psr::dev_alloc(&w.sell_cols, sizeof(int32_t) * (size_t)total));
        PSR_CUDA(ctx, psr::dev_alloc(&w.sell_vals, sizeof(double) * (size_t)total));
        count_launch();
        if (!sorted) {
            k_sell_fill<<<(w.nslices * 32 + 255) / 256, 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, ctx->n, w.nslices,
                                                                w.sell_ptr, w.sell_cols, w.sell_vals);
        } else {
            k_sell_fill_map<<<(w.nslices * 32 + 255) / 256, 256, 0, s>>>(ctx->rowptr, ctx->colidx, ctx->vals, w.sell_row,
                                                                    w.nslices, w.sell_ptr, w.sell_cols, w.sell_vals);
        }
        PSR_CHECK_LAUNCH(ctx, "SELL build");
        PSR_CUDA(ctx, cudaStreamSynchronize(s));   // hp (host) is read by the copy above
    }
    w.nspmv = 152 * 16;                     // partial slots available to the SpMV reductions
    PSR_CUDA(ctx, cudaDeviceGetAttribute(&w.sms, cudaDevAttrMultiProcessorCount, ctx->device));
    PSR_CUDA(ctx, psr::dev_alloc(&w.partial, (size_t)std::max(w.nblk * 34, w.nspmv) * 8));
    PSR_CUDA(ctx, psr::dev_alloc(&w.scal, (size_t)scal_count(m) * 8));
    PSR_CUDA(ctx, cudaMemsetAsync(w.scal, 0, (size_t)scal_count(m) * 8, s));
    PSR_CUDA(ctx, psr::dev_alloc(&w.hist, (size_t)(ctx->opts.maxit + 2) * 8));
    PSR_CUDA(ctx, psr::dev_alloc(&w.ictl, 32 * sizeof(int32_t)));
    PSR_CUDA(ctx, psr::dev_alloc(&w.rflag, 64 * sizeof(int32_t)));
    PSR_CUDA(ctx, cudaMemsetAsync(w.rflag, 0, 64 * sizeof(int32_t), s));
    // fused Arnoldi step: cooperative launches of one block per SM
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    w.coop = false;
    if (coop && ctx->opts.krylov == PSR_KRYLOV_FGMRES) {
        int b8 = 0, b16 = 0, b32 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b8, (const void*)k_arnoldi<8>, KT, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b16, (const void*)k_arnoldi<16>, KT, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, (const void*)k_arnoldi<32>, KT, 0);
        cudaGetLastError();
        w.coop = b8 >= 1 && b16 >= 1 && b32 >= 1;
    }
    if (w.coop) PSR_CUDA(ctx, psr::dev_alloc(&w.Vs, (size_t)(m + 1) * n * sizeof(float2)));
    PSR_CUDA(ctx, psr::dev_alloc(&w.part_arn, (size_t)4 * 33 * w.sms * sizeof(double)));
    PSR_CUDA(ctx, psr::dev_alloc(&w.bar, 2 * sizeof(unsigned int)));
    PSR_CUDA(ctx, cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned int), s));
    PSR_CUDA(ctx, cudaMemsetAsync(w.ictl, 0, 32 * sizeof(int32_t), s));
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    return PSR_OK;
}

void krylov_free(psr_ctx* ctx) {
    KrylovWS& w = ctx->ws;
    for (double* p : {w.x, w.b, w.r, w.z, w.p, w.q, w.V, w.Z, w.partial, w.scal, w.hist}) psr::dev_free(p);
    psr::dev_free(w.ictl);
    psr::dev_free(w.rflag);
    psr::dev_free(w.part_arn);
    psr::dev_free(w.Vs);
    psr::dev_free(w.bar);
    psr::dev_free(w.sell_ptr);
    psr::dev_free(w.sell_cols);
    psr::dev_free(w.sell_row);
    w.sell_row = nullptr;
    psr::dev_free(w.sell_vals);
    w = KrylovWS{};
    if (ctx->g_cycle) cudaGraphExecDestroy(ctx->g_cycle);
    ctx->g_cycle = nullptr;
    for (cudaEvent_t e : ctx->kt_ev) cudaEventDestroy(e);
    ctx->kt_ev.clear();
    ctx->kt_marks.clear();
}

int kernel_timing_enable(psr_ctx* ctx, bool on) {
    if (ctx->g_cycle) cudaGraphExecDestroy(ctx->g_cycle);
    ctx->g_cycle = nullptr;
    ctx->kt_marks.clear();
    ctx->kt_on = on;
    if (on) {
        for (int k = 0; k < PSR_KT_COUNT; ++k) {
            ctx->kt_ms[k] = 0.0;
            ctx->kt_n[k] = 0;
            ctx->kt_bytes[k] = 0.0;
            ctx->kt_flops[k] = 0.0;
        }
    }
    return PSR_OK;
}

// One enqueued block of work that the host repeats until the stop flag is set.
static int enqueue_cg_block(psr_ctx* ctx, KDims kd, int iters, cudaStream_t s) {
    KrylovWS& w = ctx->ws;
    const int n = ctx->n, nb = w.nblk;
    const double vb = 8.0 * n;
    for (int t = 0; t < iters; ++t) {
        KT_BEGIN(PSR_KT_SPMV, t, spmv_bytes(ctx), 2.0 * ctx->nnz + 2.0 * n);
        launch_spmv(ctx, w.p, w.q, nullptr, 2, 1, kd, 1, w.nspmv, s);
        KT_END();
        KT_BEGIN(PSR_KT_VEC, t, 6 * vb, 6.0 * n);
        count_launch(); k_cg_xr<<<nb, 256, 0, s>>>(w.x, w.r, w.p, w.q, n, kd);
        KT_END();
        KT_BEGIN(PSR_KT_SWEEP, t, sweep_bytes(ctx), sweep_flops(ctx));
        int rc = sweep_apply_ex(ctx, w.r, w.z, kd.ictl + I_STOP, s);
        if (rc != PSR_OK) return rc;
        KT_END();
        KT_BEGIN(PSR_KT_VEC, t, 2 * vb, 2.0 * n);
        count_launch(); k_dot<<<nb, 256, 0, s>>>(w.r, w.z, n, kd, 2);
        KT_END();
        KT_BEGIN(PSR_KT_VEC, t, 3 * vb, 2.0 * n);
        count_launch(); k_cg_p<<<nb, 256, 0, s>>>(w.p, w.z, n, kd);
        KT_END();
    }
    PSR_CHECK_LAUNCH(ctx, "CG block");
    return PSR_OK;
}

// Resident blocks per SM of a CGS2 kernel (one architecture per process).
static int blocks_per_sm(const void* f) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, KT, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}

// Grid of a CGS2 kernel: one resident block per SM, so that each thread
// accumulates several elements before the block reduction.  GB300 retires two
// FP64 FMAs per clock per SM, so FP64 instructions, not bytes, bound these
// kernels: the per-element dot products cost nv FMAs, the warp reduction
// about NV adds per thread, and fewer threads amortise the latter.  Capped
// by the elements and by the partial slots (nblk blocks of 34 vectors).
static int cgs_grid(psr_ctx* ctx, int per_sm) {
    const int need = (ctx->n + KT - 1) / KT;
    return std::max(1, std::min(std::min(need, std::min(per_sm, 1) * ctx->ws.sms), ctx->ws.nblk));
}

// One CGS2 orthogonalisation of w = V_{j+1} against V_0..V_j: projection,
// update fused with the second projection, second update with the norm.
template <int NV>
static int enqueue_cgs2(psr_ctx* ctx, KDims kd, int j, double* Vn, cudaStream_t s) {
    KrylovWS& w = ctx->ws;
    const int n = ctx->n;
    const double vb = 8.0 * n;
    static const int o1 = blocks_per_sm((const void*)k_mdot<NV>);
    static const int o2 = blocks_per_sm((const void*)k_maxpy_mdot<NV>);
    static const int o3 = blocks_per_sm((const void*)k_maxpy<NV>);
    const int g1 = cgs_grid(ctx, o1), g2 = cgs_grid(ctx, o2), g3 = cgs_grid(ctx, o3);
    KT_BEGIN(PSR_KT_MDOT, j, (j + 2) * vb, 2.0 * n * (j + 2));
    count_launch(); k_mdot<NV><<<g1, KT, 0, s>>>(w.V, Vn, n, j, kd);
    KT_END();
    KT_BEGIN(PSR_KT_MAXPY, j, (j + 3) * vb, 2.0 * n * (j + 2));
    KT_REORTH(0.0, 2.0 * n * j);
    count_launch(); k_maxpy_mdot<NV><<<g2, KT, 0, s>>>(w.V, Vn, n, j, kd);
    KT_END();
    KT_BEGIN(PSR_KT_MAXPY, j, 0.0, 0.0);
    KT_REORTH((j + 3) * vb, 2.0 * n * (j + 2));
    count_launch(); k_maxpy<NV><<<g3, KT, 0, s>>>(w.V, Vn, n, j, kd);
    KT_END();
    return PSR_OK;
}

// The fused Arnoldi step: one cooperative launch of one block per SM.
template <int NV>
static int enqueue_arnoldi(psr_ctx* ctx, KDims kd, int j, double* Vn, cudaStream_t s) {
    KrylovWS& w = ctx->ws;
    const int n = ctx->n;
    const double vb = 8.0 * n;
    // one block per SM: every block sums all block partials after a barrier,
    // so more blocks lengthen the serial part (measured: two per SM slower)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)w.sms);
    cfg.blockDim = dim3(KT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // bytes: pass 1 reads w and j+1 pair rows and writes the pair of w; the
    // second pass (when taken) reads and writes that pair and reads j+1 rows;
    // the last update, fused with the normalisation, reads the pair and j+1
    // rows and writes the pair and V_{j+1}.  FP64 flops of the pair path (the
    // dots and updates run on FP32 pairs): ||w||^2 and the split in pass 1,
    // the FP64 value of the normalised pair.
    // In FP64 (PSR_ORTHO_FP64): the projection reads w and j+1 rows, each
    // update j+1 rows and w twice, the normalisation writes w and its pair.
    // Not counted: the clearing of Z_{j+1} for the next sweep (zn), which an
    // ideal sweep would not need.
    const int fp64 = ctx->opts.ortho == PSR_ORTHO_FP64 ? 1 : 0;
    if (fp64) {
        KT_BEGIN(PSR_KT_MDOT, j, ((j + 2) + (j + 3) + 3) * vb, 4.0 * n * (j + 2) + 3.0 * n);
        KT_REORTH((j + 3) * vb, 4.0 * n * (j + 1));
    } else {
        KT_BEGIN(PSR_KT_MDOT, j, ((j + 3) + (j + 4)) * vb, 4.0 * n);
        KT_REORTH((j + 3) * vb, 0.0);
    }
    count_launch();
    double* zn = (j + 1 < kd.m) ? w.Z + (size_t)(j + 1) * n : nullptr;
    PSR_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_arnoldi<NV>, (const double*)w.V, Vn, w.Vs, n, j, kd, w.part_arn, w.bar,
                                     fp64, zn));
    KT_END();
    return PSR_OK;
}

static int enqueue_fg_cycle(psr_ctx* ctx, KDims kd, cudaStream_t s) {
    KrylovWS& w = ctx->ws;
    const int n = ctx->n, nb = w.nblk, m = kd.m;
    // The fused step clears the next sweep's output Z_{j+1} (k_fg_start
    // clears Z_0), so the sweeps of the cycle skip their own memset.
    const bool fused = w.coop && ctx->opts.ortho != PSR_ORTHO_SPLIT;
    float2* Vs0 = fused ? w.Vs : nullptr;
    count_launch(); k_fg_start<<<nb, 256, 0, s>>>(w.r, w.V, Vs0, n, kd, fused ? w.Z : nullptr);
    for (int j = 0; j < m; ++j) {
        double* Vj = w.V + (size_t)j * n;
        double* Vn = w.V + (size_t)(j + 1) * n;
        double* Zj = w.Z + (size_t)j * n;
        const double vb = 8.0 * n;
        KT_BEGIN(PSR_KT_SWEEP, j, sweep_bytes(ctx), sweep_flops(ctx));
        int rc = sweep_apply_ex(ctx, Vj, Zj, kd.ictl + I_STOP, s, fused);
        if (rc != PSR_OK) return rc;
        KT_END();
        KT_BEGIN(PSR_KT_SPMV, j, spmv_bytes(ctx), 2.0 * ctx->nnz);
        launch_spmv(ctx, Zj, Vn, nullptr, 0, 0, kd, 1, w.nspmv, s);
        KT_END();
        int rc2 = PSR_OK;
        if (fused) {
            if (j < 8) rc2 = enqueue_arnoldi<8>(ctx, kd, j, Vn, s);
            else if (j < 16) rc2 = enqueue_arnoldi<16>(ctx, kd, j, Vn, s);
            else rc2 = enqueue_arnoldi<32>(ctx, kd, j, Vn, s);
            if (rc2 != PSR_OK) return rc2;
            continue;
        }
        if (j < 8) rc2 = enqueue_cgs2<8>(ctx, kd, j, Vn, s);
        else if (j < 16) rc2 = enqueue_cgs2<16>(ctx, kd, j, Vn, s);
        else rc2 = enqueue_cgs2<32>(ctx, kd, j, Vn, s);
        if (rc2 != PSR_OK) return rc2;
        KT_BEGIN(PSR_KT_VEC, j, 2 * vb, (double)n);
        count_launch(); k_fg_scale<<<nb, 256, 0, s>>>(Vn, n, kd);
        KT_END();
    }
    count_launch(); k_fg_update<<<nb, 256, 0, s>>>(w.x, w.Z, n, kd);
    // restart residual r = b - A x (skipped once stopped)
    launch_spmv(ctx, w.x, w.r, w.b, 1, 2, kd, 1, w.nspmv, s);
    PSR_CHECK_LAUNCH(ctx, "FGMRES cycle");
    return PSR_OK;
}

static int krylov_solve_impl(psr_ctx* ctx, const double* b, double* x, cudaStream_t s, psr_solve_info* info);

// The outer solve inside one NVTX range (visible in a profiler timeline).
int krylov_solve(psr_ctx* ctx, const double* b, double* x, cudaStream_t s, psr_solve_info* info) {
    nvtxRangePushA("psr_solve");
    const int rc = krylov_solve_impl(ctx, b, x, s, info);
    nvtxRangePop();
    return rc;
}

static int krylov_solve_impl(psr_ctx* ctx, const double* b, double* x, cudaStream_t s, psr_solve_info* info) {
    KrylovWS& w = ctx->ws;
    const int n = ctx->n, nb = w.nblk;
    const bool cg = ctx->opts.krylov == PSR_KRYLOV_CG;
    const int m = cg ? 0 : ctx->opts.restart;
    KDims kd{n, cg ? 1 : m, nb, w.scal, w.ictl, w.partial, w.hist, w.rflag};
    cudaEvent_t e0, e1;
    PSR_CUDA(ctx, cudaEventCreate(&e0));
    PSR_CUDA(ctx, cudaEventCreate(&e1));
    PSR_CUDA(ctx, cudaEventRecord(e0, s));
    // control block
    int32_t hctl[32] = {0};
    hctl[I_MAXIT] = ctx->opts.maxit;
    hctl[I_M] = m;
    double rtol = ctx->opts.rtol;
    PSR_CUDA(ctx, cudaMemcpyAsync(w.ictl, hctl, sizeof(hctl), cudaMemcpyHostToDevice, s));
    PSR_CUDA(ctx, cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned int), s));
    PSR_CUDA(ctx, cudaMemcpyAsync(w.scal + S_RTOL, &rtol, sizeof(double), cudaMemcpyHostToDevice, s));
    // r = b, keep a copy of b, x = 0, r0 = ||b||
    count_launch(); k_init_norm<<<nb, 256, 0, s>>>(b, w.b, w.r, n, kd, 1, w.x);
    PSR_CHECK_LAUNCH(ctx, "k_init_norm");
    if (cg) {
        int rc = sweep_apply_ex(ctx, w.r, w.z, w.ictl + I_STOP, s);
        if (rc != PSR_OK) return rc;
        count_launch(); k_dot<<<nb, 256, 0, s>>>(w.r, w.z, n, kd, 1);
        count_launch(); k_copy<<<nb, 256, 0, s>>>(w.z, w.p, n, kd);
    }
    const int block = cg ? 8 : 1;
    int32_t* hstop = nullptr;                     // control ints, then the step flags
    PSR_CUDA(ctx, psr::host_alloc(&hstop, (8 + 64) * sizeof(int32_t)));
    // capture one block / cycle into a graph (the pointers are the context's own)
    auto capture_graph = [&]() -> int {
        cudaStream_t cs;
        PSR_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(ctx, ce, "graph capture"); }
        ctx->kt_marks.clear();
        set_capturing(true);
        int rc2 = cg ? enqueue_cg_block(ctx, kd, block, cs) : enqueue_fg_cycle(ctx, kd, cs);
        set_capturing(false);
        ce = cudaStreamEndCapture(cs, &g);
        if (ce == cudaSuccess && rc2 == PSR_OK) {
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(g, nodes.data(), &nn);
            int kn = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kn;
            }
            ctx->graph_block = kn;
        }
        if (rc2 != PSR_OK) { if (ce == cudaSuccess) cudaGraphDestroy(g); cudaStreamDestroy(cs); return rc2; }
        if (ce != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(ctx, ce, "graph capture"); }
        ce = cudaGraphInstantiate(&ctx->g_cycle, g, 0);
        cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) { ctx->g_cycle = nullptr; return cuda_fail(ctx, ce, "graph instantiate"); }
        return PSR_OK;
    };
    // Without per-kernel timing the first block / cycle is enqueued directly
    // and the graph is captured and instantiated while the device runs it;
    // with timing the graph comes first (the marks of a block are those of
    // the graph).
    const bool capture_behind = ctx->opts.use_graph && !ctx->g_cycle && !ctx->kt_on;
    if (ctx->opts.use_graph && !ctx->g_cycle && !capture_behind) {
        int rc0 = capture_graph();
        if (rc0 != PSR_OK) { psr::host_free(hstop); return rc0; }
    }
    const int max_blocks = cg ? (ctx->opts.maxit + block - 1) / block + 2 : ctx->opts.maxit + 2;
    int rc = PSR_OK;
    int it_before = 0;
    for (int it = 0; it < max_blocks; ++it) {
        if (ctx->g_cycle) {
            PSR_CUDA(ctx, cudaGraphLaunch(ctx->g_cycle, s));
            count_launch(ctx->graph_block);
        } else {
            ctx->kt_marks.clear();
            rc = cg ? enqueue_cg_block(ctx, kd, block, s) : enqueue_fg_cycle(ctx, kd, s);
            if (rc != PSR_OK) break;
            if (it == 0 && capture_behind && (rc = capture_graph()) != PSR_OK) break;
        }
        PSR_CUDA(ctx, cudaMemcpyAsync(hstop, w.ictl, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (ctx->kt_on && !cg)
            PSR_CUDA(ctx, cudaMemcpyAsync(hstop + 8, w.rflag, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        if (hstop[I_ERR]) {
            set_error(ctx, "a grid barrier of the Arnoldi kernel gave up waiting");
            rc = PSR_ERR_TIMEOUT;
            break;
        }
        rc = kt_collect(ctx, hstop[I_IT] - it_before, cg ? nullptr : hstop + 8);
        if (rc != PSR_OK) break;
        it_before = hstop[I_IT];
        if (hstop[I_STOP]) break;
    }
    if (rc != PSR_OK) { psr::host_free(hstop); return rc; }
    PSR_CUDA(ctx, cudaMemcpyAsync(x, w.x, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    PSR_CUDA(ctx, cudaEventRecord(e1, s));
    PSR_CUDA(ctx, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int iters = hstop[I_IT];
    const int conv = hstop[I_CONV];
    psr::host_free(hstop);
    ctx->last_iters = iters;
    ctx->h_hist.assign((size_t)iters + 1, 0.0);
    PSR_CUDA(ctx, cudaMemcpy(ctx->h_hist.data(), w.hist, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost));
    if (info) {
        info->iterations = iters;
        info->converged = conv;
        info->relres = ctx->h_hist.empty() ? 0.0 : ctx->h_hist.back();
        info->seconds = ms * 1e-3;
    }
    if (!conv) {
        set_error(ctx, "outer solve reached maxit before rtol");
        return PSR_ERR_NOT_CONVERGED;
    }
    return PSR_OK;
}

}  // namespace psr
