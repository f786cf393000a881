// Warp-level dense FP64 kernels on small matrices held in shared memory,
// shared by the inverse and criterion translation units.
#pragma once
#include "psr_internal.cuh"

namespace psr {

// Inverts the p x p matrix in S (row stride ld) in place.  colk (p doubles) and
// swaps (p ints) are per-warp scratch in shared memory.  Returns true when some
// pivot satisfied |pivot| <= p * 2^-53 * max|A| (the matrix is then left with
// garbage; the caller writes NaN).  Must be called by all 32 lanes.
__device__ __forceinline__ bool gj_invert_warp(double* S, int p, int ld, double* colk, int* swaps) {
    const int lane = threadIdx.x & 31;
    double amax = 0.0;
    for (int e = lane; e < p * p; e += 32) amax = fmax(amax, fabs(S[(e / p) * ld + (e % p)]));
    amax = warp_max(amax);
    const double thresh = (double)p * 0x1p-53 * amax;
    bool singular = !(amax > 0.0);
    for (int k = 0; k < p; ++k) {
        double best = -1.0;
        int bi = p;
        for (int i = k + lane; i < p; i += 32) {
            double v = fabs(S[i * ld + k]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const int piv = (bi < p) ? bi : k;     // all-NaN column: no valid pivot
        if (!(best > thresh)) singular = true;
        if (piv != k) {
            for (int j = lane; j < p; j += 32) {
                double t = S[k * ld + j];
                S[k * ld + j] = S[piv * ld + j];
                S[piv * ld + j] = t;
            }
        }
        if (lane == 0) swaps[k] = piv;
        __syncwarp();
        for (int i = lane; i < p; i += 32) colk[i] = S[i * ld + k];
        __syncwarp();
        double pv = colk[k];
        if (pv == 0.0) pv = 1.0;                 // singular: keep going, result discarded
        for (int j = lane; j < p; j += 32) {
            const double rj = (j == k ? 1.0 : S[k * ld + j]) / pv;
            // every row, eight at a time with the loads ahead of the stores
            // (row k's value is overwritten below; column k starts from zero)
            const bool isk = (j == k);
            int i = 0;
            for (; i + 8 <= p; i += 8) {
                double x[8], c[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    x[u] = S[(i + u) * ld + j];
                    c[u] = colk[i + u];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) S[(i + u) * ld + j] = fma(-c[u], rj, isk ? 0.0 : x[u]);
            }
            for (; i < p; ++i) S[i * ld + j] = fma(-colk[i], rj, isk ? 0.0 : S[i * ld + j]);
            S[k * ld + j] = rj;
        }
        __syncwarp();
    }
    // X = (P A)^{-1} = A^{-1} P^T  =>  A^{-1} = X P: swap columns back, last first
    for (int k = p - 1; k >= 0; --k) {
        const int piv = swaps[k];
        if (piv != k) {
            for (int i = lane; i < p; i += 32) {
                double t = S[i * ld + k];
                S[i * ld + k] = S[i * ld + piv];
                S[i * ld + piv] = t;
            }
        }
        __syncwarp();
    }
    return singular;
}


// Largest eigenvalue of the symmetric p x p matrix G (shared memory, row
// stride ld) by cyclic two-sided Jacobi rotations; G is overwritten.  Used for
// sigma_max(E) = sqrt(lambda_max(E^T E)), the exact ("small SVD") path of the
// criterion.  All 32 lanes call it; p <= 32 (lane k owns row/column k).
__device__ __forceinline__ double jacobi_lambda_max_warp(double* G, int p, int ld) {
    const int lane = threadIdx.x & 31;
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, dia = 0.0;
        if (lane < p) {
            for (int j = 0; j < p; ++j) {
                double g = G[lane * ld + j];
                if (j == lane) dia += g * g; else off += g * g;
            }
        }
        off = warp_sum(off);
        dia = warp_sum(dia);
        if (!(off > 1e-30 * dia)) break;      // also stops on NaN
        for (int i = 0; i < p - 1; ++i) {
            for (int j = i + 1; j < p; ++j) {
                const double gij = G[i * ld + j];
                const double gii = G[i * ld + i];
                const double gjj = G[j * ld + j];
                if (fabs(gij) <= 1e-300 || fabs(gij) <= 0x1p-60 * sqrt(fabs(gii * gjj))) continue;
                const double theta = (gjj - gii) / (2.0 * gij);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
                const double c = 1.0 / sqrt(fma(t, t, 1.0));
                const double s = t * c;
                __syncwarp();
                if (lane < p) {                   // columns i, j
                    const double a = G[lane * ld + i], b = G[lane * ld + j];
                    G[lane * ld + i] = c * a - s * b;
                    G[lane * ld + j] = s * a + c * b;
                }
                __syncwarp();
                if (lane < p) {                   // rows i, j
                    const double a = G[i * ld + lane], b = G[j * ld + lane];
                    G[i * ld + lane] = c * a - s * b;
                    G[j * ld + lane] = s * a + c * b;
                }
                __syncwarp();
            }
        }
    }
    double lm = -1.0;
    if (lane < p) lm = G[lane * ld + lane];
    return warp_max(lm);
}

// Cholesky A = L L^T of the symmetric p x p matrix in A (row stride ld; the
// lower triangle is read and overwritten by L).  One warp, p <= 32; lane r
// updates row r.  Returns p when every pivot is positive; otherwise the index
// k of the first pivot that is not (uniform over the warp), with columns
// 0..k-1 of L in place, so that A[k][0..k-1] holds row k of L.
__device__ __forceinline__ int cholesky_warp(double* A, int p, int ld) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < p; ++k) {
        __syncwarp();
        const double akk = A[k * ld + k];
        if (!(akk > 0.0)) return k;                    // also stops on NaN
        const double lkk = sqrt(akk);
        __syncwarp();
        if (lane == k) A[k * ld + k] = lkk;
        if (lane > k && lane < p) A[lane * ld + k] /= lkk;
        __syncwarp();
        if (lane > k && lane < p) {
            const double lrk = A[lane * ld + k];
            for (int j = k + 1; j <= lane; ++j) A[lane * ld + j] = fma(-lrk, A[j * ld + k], A[lane * ld + j]);
        }
    }
    __syncwarp();
    return p;
}

// FP32 Cholesky of the symmetric p x p matrix in A (row stride ld, lower
// triangle read and overwritten), one warp, p <= 32; lane r updates row r.
// Returns p when every pivot is positive, else the first index that is not.
__device__ __forceinline__ int cholesky_warp_f(float* A, int p, int ld) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < p; ++k) {
        __syncwarp();
        const float akk = A[k * ld + k];
        if (!(akk > 0.f)) return k;                    // also stops on NaN
        const float lkk = sqrtf(akk);
        __syncwarp();
        if (lane == k) A[k * ld + k] = lkk;
        if (lane > k && lane < p) A[lane * ld + k] = __fdiv_rn(A[lane * ld + k], lkk);
        __syncwarp();
        if (lane > k && lane < p) {
            const float lrk = A[lane * ld + k];
            for (int j = k + 1; j <= lane; ++j) A[lane * ld + j] = fmaf(-lrk, A[j * ld + k], A[lane * ld + j]);
        }
    }
    __syncwarp();
    return p;
}

}  // namespace psr
