// Step a3 for patches of 33..128 DOFs: the criterion d(A_i, B_c) =
// ||(A_c - A_i) B_c^-1||_2 < tol of Alg. 1 (difference form, Eq. 4 / Eq. 5)
// and the round form of Alg. 1 for such size groups (the 3D Stokes Vanka
// patches of 89 / 62 / 44 DOFs, the Q5 cells of Experiment 1).
//
// The warp-per-candidate kernels of criterion.cu keep one row of E per lane
// in registers, which stops at p = 32.  Here a block of 128 threads owns one
// candidate, thread r row r; E lives in shared memory (FP32 for the screening
// stage, then FP64), the entry's FP32 inverse is staged once per block.  The
// certified cascade is the one of criterion.cu, with block reductions in a
// fixed order:
//   D == 0 (bitwise) -> accept; ||D||_F ||B||_F -> accept; ||D w_k|| with the
//   entry's probe vectors -> reject; E in FP32 with its rounding bound
//   (Frobenius / sqrt(||E||_1 ||E||_inf) accept, row norms and power steps
//   reject); the same in FP64; Cholesky certificates on X I - G, G = fl(E^T E)
//   (G in a per-block global scratch).
// A near tie that none of these settles (|sigma - tol| within the rounding of
// the certificates, ~1e-14 relative) is decided by one Cholesky of
// tol^2 I - G without margin (lambda_max(G) < tol^2 as computed) in place of
// the Jacobi eigenvalues of the small-patch path.
//
// The round kernels: a warp per candidate screens it against the entry's
// sketches (the lower bound of criterion.cu, lanes over the sketch entries);
// survivors go to a global list; a block per survivor decides it; the last
// block records the entry and the next one (the smallest rejected index).
#include "psr_internal.cuh"

#include <algorithm>

namespace psr {

namespace {

constexpr double U64 = 0x1p-53;
constexpr int BT = 128;            // threads per block: one per row, p <= 128
constexpr int PBW = 128;           // probe w_2 offset
constexpr int PBS = 256;           // probe stride per entry
constexpr int SKB = 2;             // sketch directions (as criterion.cu)
constexpr int SKD = 128;           // stride of a direction

__device__ __forceinline__ double gamma_u(int k) { return (double)k * U64 / (1.0 - (double)k * U64); }

// Block reductions over BT threads, summed in a fixed order so every thread
// gets bitwise the same value.  red: 4 doubles of shared memory.
__device__ __forceinline__ double bsum(double v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return ((red[0] + red[1]) + red[2]) + red[3];
}
__device__ __forceinline__ double bmax(double v, double* red) {
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
}
__device__ __forceinline__ float bsumf(float v, double* red) {
    v = warp_sumf(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    return (float)(((red[0] + red[1]) + red[2]) + red[3]);
}
// (value, index) of the largest value, lowest index on ties
__device__ __forceinline__ void bargmax(double v, int i, double* red, int* redi, double* out_v, int* out_i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = v; redi[threadIdx.x >> 5] = i; }
    __syncthreads();
    double bv = red[0];
    int bi = redi[0];
    for (int w = 1; w < 4; ++w)
        if (red[w] > bv || (red[w] == bv && redi[w] < bi)) { bv = red[w]; bi = redi[w]; }
    *out_v = bv;
    *out_i = bi;
}

// Cholesky of the symmetric p x p matrix H (global scratch, row stride p,
// lower triangle read and overwritten by L) by the block.  Returns p when
// every pivot is positive, else the index of the first that is not, with
// columns 0..k-1 of L in place.
__device__ int cholesky_block(double* H, int p) {
    const int r = threadIdx.x;
    for (int k = 0; k < p; ++k) {
        __syncthreads();
        const double akk = *((volatile double*)&H[k * p + k]);
        if (!(akk > 0.0)) { __syncthreads(); return k; }
        const double lkk = sqrt(akk);
        __syncthreads();
        if (r == k) H[k * p + k] = lkk;
        if (r > k && r < p) H[r * p + k] /= lkk;
        __syncthreads();
        if (r > k && r < p) {
            const double lrk = H[r * p + k];
            for (int j = k + 1; j <= r; ++j) H[r * p + j] = fma(-lrk, H[j * p + k], H[r * p + j]);
        }
    }
    __syncthreads();
    return p;
}

// Entry-side operands of one decision.
struct BigEntry {
    const double* Ac;      // p x p, global
    const double* B;       // p x p inverse, global
    const float* sB32;     // p x (p+1) FP32 copy, shared
    const double* probe;   // w_1 at [0, p), w_2 at [PBW, PBW + p), global
    double bfro;           // ||B||_F
};

// Shared-memory plan of a deciding block: E (p x (p+1) FP64, which holds
// [E32 | D32] as FP32 during the screening stage), the entry's FP32 inverse,
// two vectors and the reduction slots.
__host__ __device__ inline size_t big_smem(int p) {
    const size_t ld = (size_t)p + 1;
    return ld * p * 8 + ((ld * p * 4 + 15) & ~(size_t)15) + 2 * BT * 8 + 8 * 8 + 8 * 4;
}

struct BigSmem {
    double* E;
    float* B32;
    double* v;
    double* w;
    double* red;
    int* redi;
};

__device__ __forceinline__ BigSmem big_layout(unsigned char* smem, int p) {
    const size_t ld = (size_t)p + 1;
    BigSmem s;
    s.E = reinterpret_cast<double*>(smem);
    s.B32 = reinterpret_cast<float*>(smem + ld * p * 8);
    s.v = reinterpret_cast<double*>(smem + ld * p * 8 + ((ld * p * 4 + 15) & ~(size_t)15));
    s.w = s.v + BT;
    s.red = s.w + BT;
    s.redi = reinterpret_cast<int*>(s.red + 8);
    return s;
}

// Stages the FP32 copy of the entry's inverse (all threads).
__device__ __forceinline__ void stage_b32(const double* __restrict__ B, int p, float* sB32) {
    const int ld = p + 1;
    for (int t = threadIdx.x; t < p * p; t += blockDim.x) sB32[(t / p) * ld + (t % p)] = __double2float_rn(B[t]);
}

// The decision for candidate Ai (global, p x p): 1 accept, 0 reject; *dv the
// deciding value (as criterion.cu).  Gs, Hs: p x p global scratch of this
// block.  All BT threads call it.
__device__ int decide_big(const double* __restrict__ Ai, const BigEntry& en, int p, double tol, BigSmem sm,
                          double* Gs, double* Hs, double* dv, bool* exact) {
    *exact = false;
    const int r = threadIdx.x;
    const bool act = r < p;
    const int ld = p + 1;
    const double* Ac = en.Ac;
    const double* B = en.B;
    // 1. bitwise equal patches: integer compares only
    {
        bool same = true;
        if (act)
            for (int j = 0; j < p; ++j)
                same &= __double_as_longlong(Ac[r * p + j]) == __double_as_longlong(Ai[r * p + j]);
        if (__syncthreads_and(same)) { *dv = 0.0; return 1; }
    }
    // 2. ||D||_F, D w_1, D w_2
    double dn2 = 0.0, dw = 0.0, dw2 = 0.0;
    if (act) {
        for (int j = 0; j < p; ++j) {
            const double d = Ac[r * p + j] - Ai[r * p + j];
            dn2 = fma(d, d, dn2);
            dw = fma(d, en.probe[j], dw);
            dw2 = fma(d, en.probe[PBW + j], dw2);
        }
    }
    dn2 = bsum(dn2, sm.red);
    if (dn2 == 0.0) { *dv = 0.0; return 1; }
    const double dF = sqrt(dn2);
    const double err = 1.01 * (double)(p + 2) * U64 * dF * en.bfro;
    const double shrink = 1.0 - 4.0 * (double)(p + 2) * U64;
    {
        const double ub0 = dF * en.bfro * (1.0 + 4.0 * (double)(p + 2) * U64);
        if (ub0 < tol) { *dv = ub0; return 1; }
    }
    {
        const double a1 = bsum(dw * dw, sm.red);
        const double a2 = bsum(dw2 * dw2, sm.red);
        const double lb1 = fmax(sqrt(a1), sqrt(a2));
        if (lb1 * shrink - 2.0 * err >= tol) { *dv = lb1; return 0; }
    }
    // 3. FP32 screening: E32 = fl32(D) fl32(B^-1), |E32 - D B^-1| <= (p+3) 2^-24 |D||B^-1|
    {
        float* E32 = reinterpret_cast<float*>(sm.E);
        float* D32 = E32 + (size_t)p * ld;
        if (act)
            for (int k = 0; k < p; ++k) D32[r * ld + k] = __double2float_rn(Ac[r * p + k] - Ai[r * p + k]);
        __syncthreads();
        float ra = 0.f, fr = 0.f;
        if (act) {
            for (int jc = 0; jc < p; jc += 32) {
                float f[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) f[j] = 0.f;
                for (int k = 0; k < p; ++k) {
                    const float dk = D32[r * ld + k];
                    const float* brow = sm.B32 + k * ld + jc;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (jc + j < p) f[j] = fmaf(dk, brow[j], f[j]);
                }
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (jc + j < p) {
                        E32[r * ld + jc + j] = f[j];
                        fr = fmaf(f[j], f[j], fr);
                        ra += fabsf(f[j]);
                    }
            }
        }
        const double u32 = 0x1p-24;
        const double err32 = 1.01 * (double)(p + 3) * u32 * dF * en.bfro;
        const float up = 1.0f + 4.0f * (float)(p + 2) * 0x1p-24f;
        const float dn = 1.0f - 4.0f * (float)(p + 2) * 0x1p-24f;
        const float fr2 = bsumf(fr, sm.red);
        const float ni = (float)bmax(act ? (double)ra : 0.0, sm.red);
        float ca = 0.f;
        if (act)
            for (int i = 0; i < p; ++i) ca += fabsf(E32[i * ld + r]);
        const float na = (float)bmax(act ? (double)ca : 0.0, sm.red);
        const double ub32 = (double)(fminf(sqrtf(fr2), sqrtf(na * ni)) * up);
        if (ub32 + err32 < tol) { *dv = ub32 + err32; return 1; }
        double bst;
        int bri;
        bargmax(act ? (double)sqrtf(fr) : -1.0, r, sm.red, sm.redi, &bst, &bri);
        double lb32 = bst * (double)dn;
        if (lb32 - err32 >= tol) { *dv = lb32 - err32; return 0; }
        if (bst > 0.0) {
            float* v32 = reinterpret_cast<float*>(sm.v);
            float* w32 = reinterpret_cast<float*>(sm.w);
            if (act) v32[r] = E32[bri * ld + r] / (float)bst;
            __syncthreads();
            for (int it = 0; it < 12; ++it) {
                float wr = 0.f;
                if (act)
                    for (int j = 0; j < p; ++j) wr = fmaf(E32[r * ld + j], v32[j], wr);
                const float nw = sqrtf(bsumf(wr * wr, sm.red));
                lb32 = fmax(lb32, (double)(nw * dn));
                if (lb32 - err32 >= tol) { *dv = lb32 - err32; return 0; }
                if (!(nw > 0.f)) break;
                if (act) w32[r] = wr;
                __syncthreads();
                float uj = 0.f;
                if (act)
                    for (int i = 0; i < p; ++i) uj = fmaf(E32[i * ld + r], w32[i], uj);
                const float nu = sqrtf(bsumf(uj * uj, sm.red));
                lb32 = fmax(lb32, (double)(nu / nw * dn));
                if (lb32 - err32 >= tol) { *dv = lb32 - err32; return 0; }
                if (!(nu > 0.f)) break;
                __syncthreads();
                if (act) v32[r] = uj / nu;
                __syncthreads();
            }
        }
        __syncthreads();
    }
    // 4. FP64 E (row r by thread r; B^-1 rows read by every thread at once)
    double rown2 = 0.0, rabs = 0.0;
    if (act) {
        for (int jc = 0; jc < p; jc += 32) {
            double e[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) e[j] = 0.0;
            for (int k = 0; k < p; ++k) {
                const double dk = Ac[r * p + k] - Ai[r * p + k];
                const double* brow = B + k * p + jc;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (jc + j < p) e[j] = fma(dk, brow[j], e[j]);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (jc + j < p) {
                    sm.E[r * ld + jc + j] = e[j];
                    rown2 = fma(e[j], e[j], rown2);
                    rabs += fabs(e[j]);
                }
        }
    }
    const double fro2 = bsum(rown2, sm.red);
    const double ninf = bmax(act ? rabs : 0.0, sm.red);
    double cabs = 0.0;
    if (act)
        for (int i = 0; i < p; ++i) cabs += fabs(sm.E[i * ld + r]);
    const double none = bmax(act ? cabs : 0.0, sm.red);
    const double slack = 1.0 + 4.0 * (double)(p + 2) * U64;
    const double ub = fmin(sqrt(fro2), sqrt(none * ninf)) * slack;
    if (ub + err < tol) { *dv = ub; return 1; }
    double best;
    int br;
    bargmax(act ? sqrt(rown2) : -1.0, r, sm.red, sm.redi, &best, &br);
    double lb = best;
    if (lb * shrink - err >= tol) { *dv = lb; return 0; }
    if (!(best > 0.0)) { *dv = 0.0; return 1; }
    if (act) sm.v[r] = sm.E[br * ld + r] / best;
    __syncthreads();
    for (int it = 0; it < 16; ++it) {
        double wr = 0.0;
        if (act)
            for (int j = 0; j < p; ++j) wr = fma(sm.E[r * ld + j], sm.v[j], wr);
        const double nw = sqrt(bsum(wr * wr, sm.red));
        lb = fmax(lb, nw);
        if (lb * shrink - err >= tol) { *dv = lb; return 0; }
        if (!(nw > 0.0)) break;
        if (act) sm.w[r] = wr;
        __syncthreads();
        double uj = 0.0;
        if (act)
            for (int i = 0; i < p; ++i) uj = fma(sm.E[i * ld + r], sm.w[i], uj);
        const double nu = sqrt(bsum(uj * uj, sm.red));
        lb = fmax(lb, nu / nw);
        if (lb * shrink - err >= tol) { *dv = lb; return 0; }
        if (!(nu > 0.0)) break;
        if (act) sm.v[r] = uj / nu;
        __syncthreads();
    }
    // 5. certificates on X I - G, G = fl(E^T E) (column r of G by thread r)
    *exact = true;
    if (act) {
        for (int i = 0; i < p; ++i) {
            double g = 0.0;
            for (int q = 0; q < p; ++q) g = fma(sm.E[q * ld + i], sm.E[q * ld + r], g);
            Gs[i * p + r] = g;
        }
    }
    __syncthreads();
    auto load_shifted = [&](double X) {          // Hs <- X I - G
        __syncthreads();
        for (int t = r; t < p * p; t += blockDim.x) {
            const int i = t / p, j = t % p;
            Hs[t] = (i == j ? X : 0.0) - Gs[t];
        }
        __syncthreads();
    };
    const double eg = 1.01 * gamma_u(p) * fro2;
    const double tl = (tol - err) * shrink;
    if (tl > 0.0) {
        const double X = tl * tl * (1.0 - 4.0 * U64) - eg;
        if (X > 0.0) {
            load_shifted(X);
            const double trA = bsum(act ? Hs[r * p + r] : 0.0, sm.red);
            if (trA > 0.0) {
                const double c = 2.0 * gamma_u(p + 1) * trA;
                if (act) Hs[r * p + r] -= c;
                if (cholesky_block(Hs, p) == p) {
                    *dv = (sqrt(X + eg) + err) * (1.0 + 8.0 * U64);
                    return 1;
                }
            }
        }
    }
    {
        const double th = (tol + err) / shrink;
        load_shifted(th * th * (1.0 + 4.0 * U64) + eg);
        const int k = cholesky_block(Hs, p);
        if (k < p) {
            // L11^T y = l (row k of L) by back substitution; z = [-y; 1; 0]
            if (r == 0)
                for (int i = k - 1; i >= 0; --i) {
                    double s = Hs[k * p + i];
                    for (int q = i + 1; q < k; ++q) s -= Hs[q * p + i] * sm.w[q];
                    sm.w[i] = s / Hs[i * p + i];
                }
            __syncthreads();
            if (act) sm.v[r] = (r < k) ? -sm.w[r] : (r == k ? 1.0 : 0.0);
            __syncthreads();
            double t = 0.0;
            if (act)
                for (int j = 0; j < p; ++j) t = fma(sm.E[r * ld + j], sm.v[j], t);
            const double nez = sqrt(bsum(t * t, sm.red));
            const double nz = sqrt(bsum(act ? sm.v[r] * sm.v[r] : 0.0, sm.red));
            const double lbz = (nez * (1.0 - (double)(p + 4) * U64) - 1.01 * gamma_u(p) * sqrt(fro2) * nz) /
                               (nz * (1.0 + (double)(p + 2) * U64)) - err;
            if (lbz * (1.0 - 8.0 * U64) >= tol) { *dv = lbz; return 0; }
        }
    }
    // 6. near tie: lambda_max(G) < tol^2 as decided by one plain factorisation
    load_shifted(tol * tol);
    const int kk = cholesky_block(Hs, p);
    *dv = lb;
    return kk == p ? 1 : 0;
}

// ---------------------------------------------------------------- entry quantities
// Dominant right singular vector of the FP32 matrix M (shared, row stride ld)
// by power iteration on M^T M from the all-ones vector: v (shared, p doubles)
// receives the unit direction (the last finite one).  t: p doubles of scratch.
__device__ void dominant_sv_block(const float* M, int p, int ld, int iters, double* v, double* t, double* red) {
    const int r = threadIdx.x;
    const bool act = r < p;
    float* vf = reinterpret_cast<float*>(t);         // t holds BT doubles: room for two float vectors
    float* tf = vf + BT;
    if (act) vf[r] = 1.f;
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        float tr = 0.f;
        if (act)
            for (int k = 0; k < p; ++k) tr = fmaf(M[r * ld + k], vf[k], tr);
        if (act) tf[r] = tr;
        __syncthreads();
        float u = 0.f;
        if (act)
            for (int q = 0; q < p; ++q) u = fmaf(M[q * ld + r], tf[q], u);
        const float nu = sqrtf(bsumf(u * u, red));
        if (!(nu > 0.f) || !(nu < 3.0e38f)) break;
        if (act) vf[r] = u / nu;
        __syncthreads();
    }
    __syncthreads();
    if (act) v[r] = (double)vf[r];
    __syncthreads();
}

// Per patch (block each): ||B||_F, the probe vectors w_1, w_2 (as
// criterion.cu, stride PBS), the sketches y_k = fl(A x_k) (FP32 copies),
// their widened norms den_k, ||A||_F and rho >= ||B^ A - I||_2.
__global__ void __launch_bounds__(BT) k_entry_big(const double* __restrict__ A, const double* __restrict__ Binv,
                                                  int count, int p, const double* __restrict__ X,
                                                  double* __restrict__ fro, double* __restrict__ wout,
                                                  double* __restrict__ den, float* __restrict__ Y32,
                                                  double* __restrict__ fa, double* __restrict__ rho) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    float* M32 = reinterpret_cast<float*>(smem);
    double* v = reinterpret_cast<double*>(smem + (((size_t)p * ld * 4 + 15) & ~(size_t)15));
    double* t = v + BT;
    double* red = t + BT;
    const int r = threadIdx.x;
    const bool act = r < p;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const double* Ai = A + (int64_t)i * p * p;
        const double* Bi = Binv + (int64_t)i * p * p;
        // ||A||_F, ||B||_F, sketches
        double a2 = 0.0, b2 = 0.0;
        if (act)
            for (int j = 0; j < p; ++j) {
                a2 = fma(Ai[r * p + j], Ai[r * p + j], a2);
                b2 = fma(Bi[r * p + j], Bi[r * p + j], b2);
            }
        const double fA = sqrt(bsum(a2, red));
        const double fB = sqrt(bsum(b2, red));
        for (int k = 0; k < SKB; ++k) {
            double y = 0.0;
            if (act)
                for (int j = 0; j < p; ++j) y = fma(Ai[r * p + j], X[k * SKD + j], y);
            if (act) Y32[((int64_t)i * SKB + k) * p + r] = __double2float_rn(y);
            const double yn2 = bsum(act ? y * y : 0.0, red);
            if (r == 0) den[(int64_t)i * SKB + k] = sqrt(yn2) * (1.0 + (double)(p + 2) * U64) + 1.01 * gamma_u(p) * fA;
        }
        // rho: column r of B^ A - I by thread r
        double res2 = 0.0;
        if (act)
            for (int q = 0; q < p; ++q) {
                double s = 0.0;
                for (int k = 0; k < p; ++k) s = fma(Bi[q * p + k], Ai[k * p + r], s);
                const double d = s - (q == r ? 1.0 : 0.0);
                res2 = fma(d, d, res2);
            }
        res2 = bsum(res2, red);
        if (r == 0) {
            fro[i] = fB;
            fa[i] = fA;
            rho[i] = 1.01 * sqrt(res2) + 1.01 * gamma_u(p + 1) * fB * fA;
        }
        // w_1 = B v / ||v||, v the dominant right singular vector of B
        __syncthreads();
        for (int e = r; e < p * p; e += blockDim.x) M32[(e / p) * ld + (e % p)] = __double2float_rn(Bi[e]);
        __syncthreads();
        dominant_sv_block(M32, p, ld, 10, v, t, red);
        {
            const double nv = sqrt(bsum(act ? v[r] * v[r] : 0.0, red));
            double bv = 0.0;
            if (act)
                for (int k = 0; k < p; ++k) bv = fma(Bi[r * p + k], v[k], bv);
            wout[(int64_t)i * PBS + r] = (act && nv > 0.0) ? bv / nv : 0.0;
        }
        // w_2 = B (A x / ||A x||) with x the dominant right singular vector of A
        __syncthreads();
        for (int e = r; e < p * p; e += blockDim.x) M32[(e / p) * ld + (e % p)] = __double2float_rn(Ai[e]);
        __syncthreads();
        dominant_sv_block(M32, p, ld, 10, v, t, red);
        {
            double ax = 0.0;
            if (act)
                for (int k = 0; k < p; ++k) ax = fma(Ai[r * p + k], v[k], ax);
            const double nax = sqrt(bsum(act ? ax * ax : 0.0, red));
            if (act) t[r] = nax > 0.0 ? ax / nax : 0.0;
            __syncthreads();
            const double nv = sqrt(bsum(act ? t[r] * t[r] : 0.0, red));
            double bt = 0.0;
            if (act)
                for (int k = 0; k < p; ++k) bt = fma(Bi[r * p + k], t[k], bt);
            wout[(int64_t)i * PBS + PBW + r] = (act && nv > 0.0) ? bt / nv : 0.0;
            if (r >= p && r < PBW) {                      // zero the unused probe slots
                wout[(int64_t)i * PBS + r] = 0.0;
                wout[(int64_t)i * PBS + PBW + r] = 0.0;
            }
        }
        __syncthreads();
    }
}

// Sketch directions of a size group: x_0 = dominant right singular vector of
// the group's middle patch, x_1 = a fixed alternating vector; both unit.
__global__ void __launch_bounds__(BT) k_sketch_dirs_big(const double* __restrict__ Ag, int count, int p,
                                                        double* __restrict__ X) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    float* M32 = reinterpret_cast<float*>(smem);
    double* v = reinterpret_cast<double*>(smem + (((size_t)p * ld * 4 + 15) & ~(size_t)15));
    double* t = v + BT;
    double* red = t + BT;
    const int r = threadIdx.x;
    const bool act = r < p;
    const double* Am = Ag + (int64_t)(count / 2) * p * p;
    for (int e = r; e < p * p; e += blockDim.x) M32[(e / p) * ld + (e % p)] = __double2float_rn(Am[e]);
    __syncthreads();
    dominant_sv_block(M32, p, ld, 20, v, t, red);
    for (int k = 0; k < SKB; ++k) {
        double x = (k == 0) ? (act ? v[r] : 0.0) : (act ? ((r & 1) ? -1.0 : 1.0) * (1.0 + (double)(r % 3)) : 0.0);
        double nx = sqrt(bsum(x * x, red));
        if (!(nx > 0.0)) {
            x = (r == 0) ? 1.0 : 0.0;
            nx = 1.0;
        }
        X[k * SKD + r] = act ? x / nx : 0.0;
    }
}

// Brackets [nlo, nhi] of ||A_i||_2 for the norm-window search and each
// patch's window [wlo, whi] (the keys and windows of criterion.cu's warp path,
// for p > 32): a block per patch, thread r row r of
// A in shared memory.  Power iteration on G = A^T A from A's largest row
// until the Rayleigh quotient lambda stalls (three steps gaining < 2^-50, at
// most 300); nlo = sqrt(lambda)(1 - 2^-40), nhi from the first
// X = lambda (1 + 2^-s), s = 40, 36, 32, 26, 20, 12, 4, -4, -12, for which the Cholesky
// factorisation of X I - G - c I (c = 2 gamma_{p+1} tr, its backward error)
// runs to completion, proving lambda_max(G) < X (infinite when none does).
// scratch: 2 p^2 doubles per block (G, then the factorised copy).
__global__ void __launch_bounds__(BT) k_patch_norms_big(const double* __restrict__ Ag, int count, int p,
                                                        double tol, double* __restrict__ nlo,
                                                        double* __restrict__ nhi, double* __restrict__ wlo,
                                                        double* __restrict__ whi, double* __restrict__ scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    double* E = reinterpret_cast<double*>(smem);
    double* v = E + (size_t)p * ld;
    double* w = v + BT;
    double* red = w + BT;
    int* redi = reinterpret_cast<int*>(red + 4);
    const int r = threadIdx.x;
    const bool act = r < p;
    const int64_t pp = (int64_t)p * p;
    double* Gs = scratch + (int64_t)blockIdx.x * 2 * pp;
    double* Hs = Gs + pp;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        __syncthreads();
        for (int e = r; e < p * p; e += BT) E[(e / p) * ld + (e % p)] = Ag[(int64_t)i * pp + e];
        __syncthreads();
        double rn = 0.0;
        if (act)
            for (int j = 0; j < p; ++j) rn = fma(E[r * ld + j], E[r * ld + j], rn);
        double best;
        int br;
        bargmax(act ? rn : -1.0, r, red, redi, &best, &br);
        double lo = 0.0, hi = 0.0;
        if (best != best) lo = best;                // a NaN patch: widened to [0, inf] below
        if (best > 0.0) {
            v[r] = act ? E[br * ld + r] / sqrt(best) : 0.0;
            double lam = 0.0;
            int quiet = 0;
            for (int it = 0; it < 300 && quiet < 3; ++it) {
                __syncthreads();
                double wr = 0.0;
                if (act)
                    for (int j = 0; j < p; ++j) wr = fma(E[r * ld + j], v[j], wr);
                const double l2 = bsum(wr * wr, red);
                quiet = (l2 - lam <= 0x1p-50 * l2) ? quiet + 1 : 0;
                lam = fmax(lam, l2);
                w[r] = wr;
                __syncthreads();
                double uj = 0.0;
                if (act)
                    for (int q = 0; q < p; ++q) uj = fma(E[q * ld + r], w[q], uj);
                const double nu = sqrt(bsum(uj * uj, red));
                if (!(nu > 0.0)) break;
                v[r] = act ? uj / nu : 0.0;
            }
            // G = A^T A, thread r column r
            __syncthreads();
            if (act)
                for (int k = 0; k < p; ++k) {
                    double g = 0.0;
                    for (int q = 0; q < p; ++q) g = fma(E[q * ld + k], E[q * ld + r], g);
                    Gs[k * p + r] = g;
                }
            lo = sqrt(lam) * (1.0 - 0x1p-40);
            hi = __longlong_as_double(0x7ff0000000000000ll);
            const int shifts[9] = {-40, -36, -32, -26, -20, -12, -4, 4, 12};
#pragma unroll 1
            for (int k = 0; k < 9; ++k) {
                const double X = lam * (1.0 + __longlong_as_double((long long)(1023 + shifts[k]) << 52));
                __syncthreads();
                if (act)
                    for (int q = 0; q < p; ++q) Hs[q * p + r] = (q == r ? X : 0.0) - Gs[q * p + r];
                __syncthreads();
                const double tr = bsum(act ? Hs[r * p + r] : 0.0, red);
                if (!(tr > 0.0)) continue;
                if (act) Hs[r * p + r] -= 2.0 * gamma_u(p + 1) * tr;
                if (cholesky_block(Hs, p) == p) {
                    hi = sqrt(X) * (1.0 + 0x1p-50);
                    break;
                }
            }
        }
        if (r == 0) {
            sanitize_bracket(&lo, &hi);
            const NormWin w = norm_window(lo, hi, tol);
            nlo[i] = lo;
            nhi[i] = hi;
            wlo[i] = w.lo;
            whi[i] = w.hi;
        }
    }
}

size_t norms_big_smem(int p) { return ((size_t)p * (p + 1) + 2 * BT + 4) * 8 + 4 * 4; }

// Screen of one candidate by one warp (lanes over the sketch entries): true
// when the certified sketch lower bound reaches tol (see criterion.cu for the
// bound and its rounding terms).
__device__ __forceinline__ bool screen_big(const float* __restrict__ yi, double fi, const float* sy, const double* sden,
                                           double fc, double rhoc, int p, double tol) {
    const int lane = threadIdx.x & 31;
    const double slack = 1.01 * (fc + fi) * (gamma_u(p) + rhoc) + 1.01 * 0x1p-24 * (fc + fi);
    bool rej = false;
#pragma unroll
    for (int k = 0; k < SKB; ++k) {
        float d2 = 0.f;
        for (int q = lane; q < p; q += 32) {
            const float d = sy[k * SKD + q] - __ldg(yi + k * p + q);
            d2 = fmaf(d, d, d2);
        }
        d2 = warp_sumf(d2);
        const double num = (double)sqrtf(d2) * (1.0 - (double)(p + 9 + 5) * 0x1p-24) - slack * (1.0 + 8.0 * U64);
        if (sden[k] > 0.0 && num * (1.0 - 8.0 * U64) >= tol * sden[k] * (1.0 + 4.0 * U64)) rej = true;
    }
    return rej;
}

// sigma_max(E), E = (A_c - A_i) B (A_c, A_i, B global, row stride p), for the
// closest-match pass, all BT threads: D into sm.E, E = D B into Gs and back
// into sm.E (row stride p + 1), lambda_max(E^T E) by power iteration from E's
// largest row (the Rayleigh quotients rise to it; three steps gaining < 2^-50
// or 300 steps), certified by a Cholesky factorisation of X I - G - c I with
// G = fl(E^T E) (in Hs), X = lambda (1 + 2^-40) and c = 2 gamma_{p+1} tr
// covering its backward error: lambda_max(G) < X, so sqrt(lambda) is within
// 2^-41 of sigma_max.  Where the certificate fails, [lambda, tr G] is halved
// with the same test (at most 60 times, to 2^-42 relative) and its midpoint
// taken.  Returns 0 for E = 0, NaN when E holds a NaN.
__device__ double sigma_big(const double* __restrict__ Ai, const double* __restrict__ Ac,
                            const double* __restrict__ B, int p, BigSmem sm, double* Gs, double* Hs) {
    const int r = threadIdx.x;
    const bool act = r < p;
    const int ld = p + 1;
    double* E = sm.E;
    __syncthreads();
    if (act)
        for (int k = 0; k < p; ++k) E[r * ld + k] = Ac[r * p + k] - Ai[r * p + k];
    __syncthreads();
    if (act)
        for (int j = 0; j < p; ++j) {
            double e = 0.0;
            for (int k = 0; k < p; ++k) e = fma(E[r * ld + k], B[k * p + j], e);
            Gs[r * p + j] = e;
        }
    __syncthreads();
    if (act)
        for (int j = 0; j < p; ++j) E[r * ld + j] = Gs[r * p + j];
    __syncthreads();
    double rn = 0.0;
    if (act)
        for (int j = 0; j < p; ++j) rn = fma(E[r * ld + j], E[r * ld + j], rn);
    double best;
    int br;
    bargmax(act ? rn : -1.0, r, sm.red, sm.redi, &best, &br);
    if (best != best) return best;                  // NaN (block-uniform)
    if (!(best > 0.0)) return 0.0;
    double* v = sm.v;
    double* w = sm.w;
    v[r] = act ? E[br * ld + r] / sqrt(best) : 0.0;
    double lam = 0.0;
    int quiet = 0;
    for (int it = 0; it < 300 && quiet < 3; ++it) {
        __syncthreads();
        double wr = 0.0;
        if (act)
            for (int j = 0; j < p; ++j) wr = fma(E[r * ld + j], v[j], wr);
        const double l2 = bsum(wr * wr, sm.red);
        quiet = (l2 - lam <= 0x1p-50 * l2) ? quiet + 1 : 0;
        lam = fmax(lam, l2);
        w[r] = wr;
        __syncthreads();
        double uj = 0.0;
        if (act)
            for (int q = 0; q < p; ++q) uj = fma(E[q * ld + r], w[q], uj);
        const double nu = sqrt(bsum(uj * uj, sm.red));
        if (!(nu > 0.0)) break;
        v[r] = act ? uj / nu : 0.0;
    }
    // G = E^T E into Hs, thread r column r
    __syncthreads();
    if (act)
        for (int k = 0; k < p; ++k) {
            double g = 0.0;
            for (int q = 0; q < p; ++q) g = fma(E[q * ld + k], E[q * ld + r], g);
            Hs[k * p + r] = g;
        }
    // lambda_max(G) < X proved when X I - G - c I factors (into Gs)
    auto below = [&](double X) -> bool {
        __syncthreads();
        if (act)
            for (int q = 0; q < p; ++q) Gs[q * p + r] = (q == r ? X : 0.0) - Hs[q * p + r];
        __syncthreads();
        const double tr = bsum(act ? Gs[r * p + r] : 0.0, sm.red);
        if (!(tr > 0.0)) return false;
        if (act) Gs[r * p + r] -= 2.0 * gamma_u(p + 1) * tr;
        return cholesky_block(Gs, p) == p;
    };
    if (below(lam * (1.0 + 0x1p-40))) return sqrt(lam);
    double lo = lam;
    double hi = bsum(act ? Hs[r * p + r] : 0.0, sm.red) * (1.0 + 0x1p-40);
    for (int it = 0; it < 60 && hi - lo > 0x1p-42 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid)) hi = mid;
        else lo = mid;
    }
    return sqrt(0.5 * (lo + hi));
}

// Closest match (section 3.1, the variant after Alg. 1) for patches of
// 33..128 DOFs, after the first-match rounds: a block per patch compares its
// first match j0 with the later entries whose representative precedes it, in
// entry order: the certified sketch screen (one warp), then the block's
// certified decision against the best distance so far (tol until the first
// match's own distance is needed), and sigma_max (sigma_big) for the first
// match when a later entry passes and for the entries that pass.  A zero
// distance ends the search; every entry after j0 up to the last one looked
// at counts as an evaluation.  scratch: 2 p^2 doubles per block.
__global__ void __launch_bounds__(BT) k_closest_pass_big(int count, int p, const double* __restrict__ Ag,
                                                         const double* __restrict__ Ball,
                                                         const double* __restrict__ fro_all,
                                                         const double* __restrict__ w_all,
                                                         const float* __restrict__ Y32, const double* __restrict__ den,
                                                         const double* __restrict__ fa, const double* __restrict__ rho,
                                                         const int32_t* __restrict__ rep_l, int m, double tol,
                                                         int32_t* __restrict__ phi, double* __restrict__ scratch,
                                                         unsigned long long* __restrict__ evals) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float sy[SKB * SKD];
    __shared__ double sden[SKB];
    __shared__ int s_rej;
    BigSmem sm = big_layout(smem, p);
    const int64_t pp = (int64_t)p * p;
    double* Gs = scratch + (int64_t)blockIdx.x * 2 * pp;
    double* Hs = Gs + pp;
    unsigned long long ev = 0;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int j0 = phi[i];
        if (rep_l[j0] == i) continue;               // an entry keeps its own patch
        const double* Ai = Ag + (int64_t)i * pp;
        const int r0 = rep_l[j0];
        bool same = true;
        for (int e = threadIdx.x; e < pp; e += blockDim.x)
            same &= __double_as_longlong(Ag[(int64_t)r0 * pp + e]) == __double_as_longlong(Ai[e]);
        double bs = __syncthreads_and(same) ? 0.0 : -1.0;   // -1: the first match's distance not known yet
        int best = j0;
        int lo = j0 + 1, hi = m;                   // entries j0 < j < jend: representative before i
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rep_l[mid] > i) hi = mid;
            else lo = mid + 1;
        }
        const int jend = lo;
        int last = j0;
        for (int jj = j0 + 1; jj < jend && bs != 0.0; ++jj) {
            last = jj;
            const int rj = rep_l[jj];
            const double t = bs >= 0.0 ? bs : tol;
            __syncthreads();
            for (int q = threadIdx.x; q < SKB * SKD; q += blockDim.x) {
                const int k = q / SKD, c = q % SKD;
                sy[q] = (c < p) ? Y32[((int64_t)rj * SKB + k) * p + c] : 0.f;
            }
            if (threadIdx.x < SKB) sden[threadIdx.x] = den[(int64_t)rj * SKB + threadIdx.x];
            __syncthreads();
            if (threadIdx.x < 32) {
                const bool rej = screen_big(Y32 + (int64_t)i * SKB * p, fa[i], sy, sden, fa[rj], rho[rj], p, t);
                if (threadIdx.x == 0) s_rej = rej ? 1 : 0;
            }
            __syncthreads();
            if (s_rej) continue;
            stage_b32(Ball + (int64_t)rj * pp, p, sm.B32);
            __syncthreads();
            const BigEntry en{Ag + (int64_t)rj * pp, Ball + (int64_t)rj * pp, sm.B32, w_all + (int64_t)rj * PBS,
                              fro_all[rj]};
            double dv;
            bool ex;
            int dec = decide_big(Ai, en, p, t, sm, Gs, Hs, &dv, &ex);
            if (dec == 1 && bs < 0.0) {             // passes: the first match's distance is needed now
                bs = sigma_big(Ai, Ag + (int64_t)r0 * pp, Ball + (int64_t)r0 * pp, p, sm, Gs, Hs);
                if (bs == 0.0) break;
                dec = decide_big(Ai, en, p, bs, sm, Gs, Hs, &dv, &ex);
            }
            if (dec == 1) {
                const double sj = sigma_big(Ai, Ag + (int64_t)rj * pp, Ball + (int64_t)rj * pp, p, sm, Gs, Hs);
                if (sj < bs) {
                    bs = sj;
                    best = jj;
                }
            }
        }
        ev += (unsigned long long)(last - j0);
        if (threadIdx.x == 0) phi[i] = best;
        __syncthreads();
    }
    if (threadIdx.x == 0 && ev) atomicAdd(evals, ev);
}

struct RoundBig {
    int next, m, done, first_singular;
    int ticket, next_new, nsurv, pad;
    unsigned long long evals, exact, screened;
};

// One round's screen: a warp per unassigned candidate after the entry.
__global__ void __launch_bounds__(256) k_round_screen_big(RoundBig* st, const int32_t* __restrict__ phi, int count,
                                                          int p, const float* __restrict__ Y32,
                                                          const double* __restrict__ den, const double* __restrict__ fa,
                                                          const double* __restrict__ rho, double tol,
                                                          int32_t* __restrict__ surv_list,
                                                          const double* __restrict__ nlo,
                                                          const double* __restrict__ nhi,
                                                          const double* __restrict__ wlo,
                                                          const double* __restrict__ whi) {
    __shared__ float sy[SKB * SKD];
    __shared__ double sden[SKB];
    if (st->done) return;
    const int i0 = st->next;
    for (int t = threadIdx.x; t < SKB * SKD; t += blockDim.x) {
        const int k = t / SKD, q = t % SKD;
        sy[t] = (q < p) ? Y32[((int64_t)i0 * SKB + k) * p + q] : 0.f;
    }
    if (threadIdx.x < SKB) sden[threadIdx.x] = den[(int64_t)i0 * SKB + threadIdx.x];
    __syncthreads();
    const double fc = fa[i0], rhoc = rho[i0];
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ev = 0, scr = 0;
    int my_min = count;
    for (int c = i0 + 1 + gw; c < count; c += nw) {
        if (phi[c] != -1) continue;                 // warp-uniform
        if (nlo && outside_window(NormWin{wlo[c], whi[c]}, nlo[i0], nhi[i0])) {
            my_min = min(my_min, c);                // outside the norm window: not a test
            continue;
        }
        ++ev;
        const bool rej = screen_big(Y32 + (int64_t)c * SKB * p, fa[c], sy, sden, fc, rhoc, p, tol);
        if (rej) {
            ++scr;
            my_min = min(my_min, c);
        } else if (lane == 0) {
            surv_list[atomicAdd(&st->nsurv, 1)] = c;
        }
    }
    if (lane == 0) {
        if (ev) atomicAdd(&st->evals, ev);
        if (scr) atomicAdd(&st->screened, scr);
        if (my_min < count) atomicMin(&st->next_new, my_min);
    }
}

__device__ __forceinline__ bool last_block(int* ticket) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int t = atomicAdd(ticket, 1);
        s_last = (t == (int)gridDim.x - 1);
        if (s_last) *ticket = 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// One round's decisions: a block per survivor; the last block records the
// entry (patch i0 as entry m) and the next entry.
__global__ void __launch_bounds__(BT) k_round_decide_big(RoundBig* st, int32_t* __restrict__ phi, int count,
                                                         const double* __restrict__ Ag, int p,
                                                         const double* __restrict__ Ball,
                                                         const double* __restrict__ fro_all,
                                                         const double* __restrict__ w_all,
                                                         const int32_t* __restrict__ sing_all, double tol,
                                                         const int32_t* __restrict__ surv_list,
                                                         int32_t* __restrict__ rep_local, double* __restrict__ scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (st->done) return;
    const int i0 = st->next;
    const int m = st->m;
    const int ns = st->nsurv;
    const int64_t pp = (int64_t)p * p;
    BigSmem sm = big_layout(smem, p);
    double* Gs = scratch + (int64_t)blockIdx.x * 2 * pp;
    double* Hs = Gs + pp;
    unsigned long long my_exact = 0;
    int my_min = count;
    if ((int)blockIdx.x < ns) {
        stage_b32(Ball + (int64_t)i0 * pp, p, sm.B32);
        __syncthreads();
        const BigEntry en{Ag + (int64_t)i0 * pp, Ball + (int64_t)i0 * pp, sm.B32, w_all + (int64_t)i0 * PBS,
                          fro_all[i0]};
        for (int q = blockIdx.x; q < ns; q += gridDim.x) {
            const int c = surv_list[q];
            double dv;
            bool ex;
            const int dec = decide_big(Ag + (int64_t)c * pp, en, p, tol, sm, Gs, Hs, &dv, &ex);
            if (threadIdx.x == 0) {
                if (dec == 1) phi[c] = m;
                else my_min = min(my_min, c);
                my_exact += ex ? 1 : 0;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && my_exact) atomicAdd(&st->exact, my_exact);
    if (threadIdx.x == 0 && my_min < count) atomicMin(&st->next_new, my_min);
    if (!last_block(&st->ticket)) return;
    if (threadIdx.x == 0) {
        phi[i0] = m;
        rep_local[m] = i0;
        if (sing_all[i0] && st->first_singular < 0) st->first_singular = i0;
        st->m = m + 1;
        const int nx = st->next_new;
        st->next_new = count;
        st->next = nx;
        st->nsurv = 0;
        if (nx >= count) st->done = 1;
    }
}

// Stateless batch (psr_criterion for p > 32): a block per candidate.
__global__ void __launch_bounds__(BT) k_criterion_big(const double* __restrict__ A_i, int batch, int p,
                                                      const double* __restrict__ A_c,
                                                      const double* __restrict__ Binv_c,
                                                      const double* __restrict__ probe, double bfro, double tol,
                                                      int32_t* __restrict__ accept, double* __restrict__ dval,
                                                      double* __restrict__ scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t pp = (int64_t)p * p;
    BigSmem sm = big_layout(smem, p);
    double* Gs = scratch + (int64_t)blockIdx.x * 2 * pp;
    double* Hs = Gs + pp;
    stage_b32(Binv_c, p, sm.B32);
    __syncthreads();
    const BigEntry en{A_c, Binv_c, sm.B32, probe, bfro};
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        double dv;
        bool ex;
        const int dec = decide_big(A_i + (int64_t)b * pp, en, p, tol, sm, Gs, Hs, &dv, &ex);
        if (threadIdx.x == 0) {
            accept[b] = dec;
            if (dval) dval[b] = dv;
        }
        __syncthreads();
    }
}

__global__ void k_gather_entries(const double* __restrict__ Ball, const int32_t* __restrict__ rep_local, int m, int p,
                                 double* __restrict__ out) {
    const int64_t pp = (int64_t)p * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * pp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / pp);
        out[e] = Ball[(int64_t)rep_local[j] * pp + (e - (int64_t)j * pp)];
    }
}

// Set whatever the size: the default dynamic limit is 48 KB minus the
// kernel's static shared memory.
int set_big_smem(const void* f, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "criterion (p > 32) smem attribute");
    return PSR_OK;
}

size_t entry_smem(int p) { return (((size_t)p * (p + 1) * 4 + 15) & ~(size_t)15) + 2 * BT * 8 + 8 * 8; }

}  // namespace

// Alg. 1 (round form) for one size group of p in 33..128.  Ag: the group's
// patches (count x p x p).  Leaves G.m, G.sphi (local phi), G.rinv (FP64
// inverses of the entries, m x p x p), G.h_rep and G.dbA, and adds the
// criterion counts.  Rounds run in batches of launches between host checks.
int run_alg1_big(psr_ctx* ctx, Group& G, const double* Ag, cudaStream_t s, int64_t* evals, int64_t* exact,
                 int64_t* screened, int* first_singular_local) {
    const int p = G.p, count = G.count;
    const double tol = ctx->opts.tol;
    const int64_t pp = (int64_t)p * p;
    int32_t *phi_l = nullptr, *rep_l = nullptr, *sing_all = nullptr, *surv = nullptr;
    double *Ball = nullptr, *fro_all = nullptr, *w_all = nullptr, *X = nullptr, *den = nullptr, *fa = nullptr,
           *rho = nullptr, *scratch = nullptr, *nrm = nullptr;
    const bool window = ctx->opts.search == PSR_SEARCH_NORM_WINDOW;
    float* Y32 = nullptr;
    RoundBig* st = nullptr;
    RoundBig* h_st = nullptr;
    int rc = PSR_OK;
    const int decide_blocks = 152 * 2;
    auto cleanup = [&]() {
        for (void* q : {(void*)rep_l, (void*)sing_all, (void*)surv, (void*)Ball, (void*)fro_all, (void*)w_all,
                        (void*)X, (void*)den, (void*)fa, (void*)rho, (void*)scratch, (void*)Y32, (void*)st,
                        (void*)nrm})
            psr::dev_free(q);
        psr::host_free(h_st);
    };
#define BIG_CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { rc = cuda_fail(ctx, e_, #call); cleanup(); psr::dev_free(phi_l); return rc; } } while (0)
    BIG_CK(psr::dev_alloc(&phi_l, sizeof(int32_t) * count));
    BIG_CK(psr::dev_alloc(&rep_l, sizeof(int32_t) * count));
    BIG_CK(psr::dev_alloc(&sing_all, sizeof(int32_t) * count));
    BIG_CK(psr::dev_alloc(&surv, sizeof(int32_t) * count));
    BIG_CK(psr::dev_alloc(&Ball, sizeof(double) * (size_t)count * pp));
    BIG_CK(psr::dev_alloc(&fro_all, sizeof(double) * count));
    BIG_CK(psr::dev_alloc(&w_all, sizeof(double) * (size_t)count * PBS));
    BIG_CK(psr::dev_alloc(&X, sizeof(double) * SKB * SKD));
    BIG_CK(psr::dev_alloc(&den, sizeof(double) * (size_t)count * SKB));
    BIG_CK(psr::dev_alloc(&fa, sizeof(double) * count));
    BIG_CK(psr::dev_alloc(&rho, sizeof(double) * count));
    BIG_CK(psr::dev_alloc(&Y32, sizeof(float) * (size_t)count * SKB * p));
    BIG_CK(psr::dev_alloc(&scratch, sizeof(double) * (size_t)decide_blocks * 2 * pp));
    BIG_CK(psr::dev_alloc(&st, sizeof(RoundBig)));
    BIG_CK(psr::host_alloc(&h_st, sizeof(RoundBig)));
    BIG_CK(cudaMemsetAsync(phi_l, 0xff, sizeof(int32_t) * count, s));
    GpuSpan span;                                  // the inverses' GPU time (stats.t_invert)
    span.begin(s);
    rc = launch_batched_inverse(Ag, pp, nullptr, count, p, Ball, pp, sing_all, s);
    span.end(s);
    if (rc != PSR_OK) { cleanup(); psr::dev_free(phi_l); return rc; }
    const size_t esm = entry_smem(p);
    if ((rc = set_big_smem((const void*)k_entry_big, esm)) != PSR_OK ||
        (rc = set_big_smem((const void*)k_sketch_dirs_big, esm)) != PSR_OK ||
        (rc = set_big_smem((const void*)k_round_decide_big, big_smem(p))) != PSR_OK) {
        cleanup();
        psr::dev_free(phi_l);
        return rc;
    }
    count_launch();
    k_sketch_dirs_big<<<1, BT, esm, s>>>(Ag, count, p, X);
    count_launch();
    k_entry_big<<<std::max(1, std::min(count, 152 * 8)), BT, esm, s>>>(Ag, Ball, count, p, X, fro_all, w_all, den, Y32,
                                                                       fa, rho);
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "k_entry_big"); cleanup(); psr::dev_free(phi_l); return rc; }
    }
    if (window) {
        // ||A_i||_2 brackets of the norm-window search (scratch reused: the
        // decide blocks outnumber these)
        const int nb = std::max(1, std::min(count, decide_blocks));
        BIG_CK(psr::dev_alloc(&nrm, sizeof(double) * 4 * (size_t)count));
        if ((rc = set_big_smem((const void*)k_patch_norms_big, norms_big_smem(p))) != PSR_OK) {
            cleanup();
            psr::dev_free(phi_l);
            return rc;
        }
        count_launch();
        k_patch_norms_big<<<nb, BT, norms_big_smem(p), s>>>(Ag, count, p, tol, nrm, nrm + count,
                                                            nrm + 2 * (size_t)count, nrm + 3 * (size_t)count,
                                                            scratch);
        BIG_CK(cudaGetLastError());
    }
    RoundBig init{};
    init.first_singular = -1;
    init.next = 0;
    init.next_new = count;
    BIG_CK(cudaMemcpyAsync(st, &init, sizeof(RoundBig), cudaMemcpyHostToDevice, s));
    const int screen_blocks = std::max(1, std::min((count + 7) / 8, 152 * 4));
    int batch = 4, issued = 0;
    bool inv_read = false;
    for (;;) {
        for (int q = 0; q < batch; ++q) {
            count_launch();
            k_round_screen_big<<<screen_blocks, 256, 0, s>>>(
                st, phi_l, count, p, Y32, den, fa, rho, tol, surv, nrm, window ? nrm + count : nullptr,
                window ? nrm + 2 * (size_t)count : nullptr, window ? nrm + 3 * (size_t)count : nullptr);
            count_launch();
            k_round_decide_big<<<decide_blocks, BT, big_smem(p), s>>>(st, phi_l, count, Ag, p, Ball, fro_all, w_all,
                                                                     sing_all, tol, surv, rep_l, scratch);
        }
        {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "Alg. 1 round kernels (p > 32)"); break; }
        }
        issued += batch;
        BIG_CK(cudaMemcpyAsync(h_st, st, sizeof(RoundBig), cudaMemcpyDeviceToHost, s));
        BIG_CK(cudaStreamSynchronize(s));
        if (!inv_read) {                           // the first synchronisation after the inverses
            ctx->stats.t_invert += span.seconds();
            inv_read = true;
        }
        if (h_st->done) break;
        if (issued > count + 8) { set_error(ctx, "Alg. 1 rounds did not terminate"); rc = PSR_ERR_TIMEOUT; break; }
        if (batch < 256) batch *= 2;
    }
    if (rc != PSR_OK) { cleanup(); psr::dev_free(phi_l); return rc; }
    G.m = h_st->m;
    *evals += (int64_t)h_st->evals;
    *exact += (int64_t)h_st->exact;
    *screened += (int64_t)h_st->screened;
    *first_singular_local = h_st->first_singular;
    if (ctx->opts.match == PSR_MATCH_CLOSEST && G.m > 1) {
        // closest match: the entries stay, each patch moves to its closest
        // passing entry (a block per patch)
        unsigned long long* cev = nullptr;
        BIG_CK(psr::dev_alloc(&cev, sizeof(unsigned long long)));
        BIG_CK(cudaMemsetAsync(cev, 0, sizeof(unsigned long long), s));
        if ((rc = set_big_smem((const void*)k_closest_pass_big, big_smem(p))) != PSR_OK) {
            psr::dev_free(cev);
            cleanup();
            psr::dev_free(phi_l);
            return rc;
        }
        count_launch();
        k_closest_pass_big<<<std::max(1, std::min(count, decide_blocks)), BT, big_smem(p), s>>>(
            count, p, Ag, Ball, fro_all, w_all, Y32, den, fa, rho, rep_l, G.m, tol, phi_l, scratch, cev);
        {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                psr::dev_free(cev);
                rc = cuda_fail(ctx, e, "closest-match pass (p > 32)");
                cleanup();
                psr::dev_free(phi_l);
                return rc;
            }
        }
        unsigned long long h_cev = 0;
        BIG_CK(cudaMemcpyAsync(&h_cev, cev, sizeof(h_cev), cudaMemcpyDeviceToHost, s));
        BIG_CK(cudaStreamSynchronize(s));
        psr::dev_free(cev);
        *evals += (int64_t)h_cev;
    }
    std::vector<int32_t> hrep(G.m);
    BIG_CK(cudaMemcpyAsync(hrep.data(), rep_l, sizeof(int32_t) * G.m, cudaMemcpyDeviceToHost, s));
    double* Bdb = nullptr;
    BIG_CK(psr::dev_alloc(&Bdb, sizeof(double) * (size_t)std::max(G.m, 1) * pp));
    BIG_CK(psr::dev_alloc(&G.dbA, sizeof(double) * (size_t)std::max(G.m, 1) * pp));
    {
        const int64_t tot = (int64_t)G.m * pp;
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 16));
        count_launch();
        k_gather_entries<<<gb, 256, 0, s>>>(Ball, rep_l, G.m, p, Bdb);
        count_launch();
        k_gather_entries<<<gb, 256, 0, s>>>(Ag, rep_l, G.m, p, G.dbA);
    }
    BIG_CK(cudaStreamSynchronize(s));
    G.h_rep.assign(hrep.begin(), hrep.end());
    G.sphi = phi_l;
    G.rinv = Bdb;
    cleanup();
    return PSR_OK;
#undef BIG_CK
}

// psr_criterion for 33 <= p <= 128: entry quantities (||B||_F, probe vectors)
// then a block per candidate.
int launch_criterion_big(const double* A_i, int32_t batch, int32_t p, const double* A_c, const double* Binv_c,
                         double tol, int32_t* accept, double* dval, cudaStream_t s) {
    const int64_t pp = (int64_t)p * p;
    const int blocks = std::max(1, std::min(batch, 152 * 2));
    double *w = nullptr, *scratch = nullptr, *misc = nullptr;
    float* Y = nullptr;
    auto done = [&](int rc) {
        psr::dev_free(w);
        psr::dev_free(scratch);
        psr::dev_free(misc);
        psr::dev_free(Y);
        return rc;
    };
    cudaError_t e;
    if ((e = psr::dev_alloc(&w, sizeof(double) * PBS)) != cudaSuccess ||
        (e = psr::dev_alloc(&scratch, sizeof(double) * (size_t)blocks * 2 * pp)) != cudaSuccess ||
        (e = psr::dev_alloc(&misc, sizeof(double) * (SKB * SKD + 8))) != cudaSuccess ||
        (e = psr::dev_alloc(&Y, sizeof(float) * SKB * p)) != cudaSuccess)
        return done(cuda_fail(nullptr, e, "criterion (p > 32) scratch"));
    const size_t esm = entry_smem(p);
    int rc;
    if ((rc = set_big_smem((const void*)k_entry_big, esm)) != PSR_OK) return done(rc);
    if ((rc = set_big_smem((const void*)k_criterion_big, big_smem(p))) != PSR_OK) return done(rc);
    // entry quantities of A_c: the sketch outputs are not used here
    double* X = misc;
    double* fro = misc + SKB * SKD;
    double* den = fro + 1;
    double* fa = den + SKB;
    double* rho = fa + 1;
    if ((e = cudaMemsetAsync(X, 0, sizeof(double) * SKB * SKD, s)) != cudaSuccess)
        return done(cuda_fail(nullptr, e, "criterion (p > 32) directions"));
    count_launch();
    k_entry_big<<<1, BT, esm, s>>>(A_c, Binv_c, 1, p, X, fro, w, den, Y, fa, rho);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(cuda_fail(nullptr, e, "k_entry_big"));
    double h_fro = 0.0;
    if ((e = cudaMemcpyAsync(&h_fro, fro, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return done(cuda_fail(nullptr, e, "criterion (p > 32) entry norm"));
    count_launch();
    k_criterion_big<<<blocks, BT, big_smem(p), s>>>(A_i, batch, p, A_c, Binv_c, w, h_fro, tol, accept, dval, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(cuda_fail(nullptr, e, "k_criterion_big"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return done(cuda_fail(nullptr, e, "k_criterion_big"));
    return done(PSR_OK);
}

}  // namespace psr
