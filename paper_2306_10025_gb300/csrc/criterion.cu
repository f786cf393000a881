// Step a3: the patch-similarity criterion d(A_i, B_c) = ||I - A_i B_c^{-1}||_2
// (Alg. 1, Eq. 4, Eq. 5) and Alg. 1 itself (Patch Tolerance Construction).
//
// Criterion form.  With B_c the stored patch A_c, I - A_i A_c^{-1} equals
// (A_c - A_i) A_c^{-1} in real arithmetic; the library evaluates
// E = D B_c^{-1}, D = A_c - A_i, which is exactly 0 for identical patches.
//
// Certified decision.  Alg. 1 only needs "d < tol".  Per candidate one warp
// runs a cascade and stops at the first conclusive test:
//   1. D == 0                                       -> accept (d = 0)
//   2. ||D||_F ||B^-1||_F (1 + margin) < tol         -> accept (d <= that)
//   3. form E (p^3 FMAs); ub = min(||E||_F, sqrt(||E||_1 ||E||_inf))
//      ub + err < tol                                -> accept
//   4. power iteration on E^T E from the largest row of E; every ||E v|| and
//      ||E^T w|| / ||w|| is a lower bound; lb - err >= tol -> reject
//      (steps 3-4 first with E in FP32 and its rounding bound, an FP32
//      Cholesky certificate on X I - G32 among them, then in FP64)
//   5. Cholesky certificates on X I - G, G = fl(E^T E): a factorisation of
//      X I - G - c I that succeeds proves lambda_max(G) < X -> accept; the
//      first non-positive pivot of another gives a vector z with a lower
//      bound ||E z|| / ||z|| -> reject
//   6. the near ties left: sigma_max(E) = sqrt(lambda_max(E^T E)) by cyclic
//      Jacobi.
// err bounds the GEMM rounding, ||E_computed - E||_F <= p u ||D||_F ||B||_F,
// so tests 2-5 decide "sigma_max(E_computed) < tol" exactly like step 6.
//
// Alg. 1 in rounds.  Sequential Alg. 1 compares patch i with the entries in
// creation order and takes the first with d < tol.  Every entry j was created
// by a patch r_j < i, and every patch below the newest entry's patch is
// already assigned.  Hence, round by round: (a) the smallest unassigned patch
// i0 becomes a new entry; (b) every unassigned patch i > i0 is compared with
// that entry only, and assigned to it if d < tol.  A patch meets the entries
// in creation order and stops at its first match, so phi is identical to the
// sequential loop and so is the number of evaluations; each round is one
// batched pass over the unassigned patches, with no host decision in it.
#include "psr_internal.cuh"
#include "dense.cuh"
#include <atomic>

namespace psr {

static constexpr double U64 = 0x1p-53;
// gamma_k = k u / (1 - k u), the usual bound of k accumulated FP64 roundings.
__device__ __forceinline__ double gamma_u(int k) { return (double)k * U64 / (1.0 - (double)k * U64); }
// Probe storage per entry: w_1 at [0, 32), w_2 at [PROBE_W2, PROBE_W2 + 32).
static constexpr int PROBE_W2 = 32;
static constexpr int PROBE_STRIDE = 64;
// Threads per block of the round kernels (one candidate per thread in the screen).
static constexpr int EVAL_THREADS = 128;

struct RoundDev {
    int next;          // patch that becomes the next entry (smallest unassigned)
    int m;             // entries created so far in this group
    int done;
    int first_singular;
    int ticket;        // last-block counter of the round kernel
    int next_new;      // smallest candidate the current round rejected
    int nsurv;         // survivors of the current round's screen
    int ns2[2], nn2[2];  // persistent rounds: survivors / smallest rejected, by round parity
    int nrounds;       // passes of the multi-entry round kernel
    unsigned long long evals, exact, screened;
    unsigned long long decided;   // pairs the warp cascade decided, counted by Alg. 1 or not
};

struct WarpScratch {  // per-warp shared memory layout for p <= 32
    double* E;         // p x (p+1)
    double* v;         // 32
    double* w;         // 32
};

// Decides d(A_i, B_c) < tol for one candidate.  sAc, sB: shared p x ld.
// PM >= p bounds the unrolled per-lane loops (FP64 instructions of
// predicated-off iterations would still occupy the pipe).
// probe (may be NULL): two vectors w_k = B_c^{-1} v_k / ||v_k|| (at probe and
// probe + 32), so that ||D w_k|| = ||E v_k|| / ||v_k|| <= sigma_max(E) are
// O(p^2) lower bounds.
// Returns 1 accept, 0 reject, -1 undecided (needs the exact path).  *dv gets
// the deciding value.  All lanes call; lane r handles row r.
// DIFF: sAc already holds D = A_c - A_i (formed by the caller with the same
// FP64 subtraction, after its own bitwise-equality test); Ai is not read.
template <int PM = 32, bool DIFF = false>
__device__ int decide_pair(const double* __restrict__ Ai, const double* sAc, const double* sB,
                           int p, int ld, double binv_fro, double tol, WarpScratch ws, double* dv,
                           bool allow_exact_here, const double* probe = nullptr,
                           const float* sB32 = nullptr) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < p;
    auto dval = [&](int r, int j) -> double {
        return DIFF ? sAc[r * ld + j] : sAc[r * ld + j] - Ai[r * p + j];
    };
    // D = 0 when the patches are bitwise equal: integer compares, no FP64
    // instruction (the common accept of uniform meshes)
    if (!DIFF) {
        bool same = true;
        if (act)
            for (int j = 0; j < p; ++j)
                same &= __double_as_longlong(sAc[lane * ld + j]) == __double_as_longlong(Ai[lane * p + j]);
        if (__all_sync(0xffffffffu, same)) { *dv = 0.0; return 1; }
    }
    // pass 1: D = A_c - A_i, ||D||_F and (D w)_lane
    double dn2 = 0.0, dw = 0.0, dw2 = 0.0;
    if (act) {
        for (int j = 0; j < p; ++j) {
            const double d = dval(lane, j);
            dn2 = fma(d, d, dn2);
            if (probe) {
                dw = fma(d, probe[j], dw);
                dw2 = fma(d, probe[PROBE_W2 + j], dw2);
            }
        }
    }
    dn2 = warp_sum(dn2);
    if (dn2 == 0.0) { *dv = 0.0; return 1; }
    const double dF = sqrt(dn2);
    const double err = 1.01 * (double)(p + 2) * U64 * dF * binv_fro;   // GEMM + norm rounding
    const double shrink = 1.0 - 4.0 * (double)(p + 2) * U64;
    {
        const double ub0 = dF * binv_fro * (1.0 + 4.0 * (double)(p + 2) * U64);
        if (ub0 < tol) { *dv = ub0; return 1; }
    }
    if (probe) {
        // w carries its own rounding (B^-1 v computed in FP64): widen by 2 err
        const double lb1 = fmax(sqrt(warp_sum(dw * dw)), sqrt(warp_sum(dw2 * dw2)));
        if (lb1 * shrink - 2.0 * err >= tol) { *dv = lb1; return 0; }
    }
    if (sB32) {
        // FP32 screening: E32 = fl32(D) fl32(B^-1) accumulated in FP32.  With
        // u = 2^-24, |E32 - D B^-1| <= (p+3) u |D| |B^-1| entrywise, so
        // ||E32 - E||_2 <= err32 below; FP32 norms are widened for their own
        // rounding.  Conclusive tests here give the same decision as the FP64
        // path; the rest fall through.
        const double u32 = 0x1p-24;
        const double err32 = 1.01 * (double)(p + 3) * u32 * dF * binv_fro;
        const float up = 1.0f + 4.0f * (float)(p + 2) * 0x1p-24f;
        const float dn = 1.0f - 4.0f * (float)(p + 2) * 0x1p-24f;
        float* E32 = reinterpret_cast<float*>(ws.E);
        float* v32 = reinterpret_cast<float*>(ws.v);
        float* w32 = reinterpret_cast<float*>(ws.w);
        float f[PM];
#pragma unroll
        for (int j = 0; j < PM; ++j) f[j] = 0.f;
        if (act) {
            for (int k = 0; k < p; ++k) {
                const float dk = (float)dval(lane, k);
#pragma unroll
                for (int j = 0; j < PM; ++j)
                    if (j < p) f[j] = fmaf(dk, sB32[k * ld + j], f[j]);
            }
        }
        float fr2 = 0.f, ra = 0.f;
#pragma unroll
        for (int j = 0; j < PM; ++j)
            if (j < p) { fr2 = fmaf(f[j], f[j], fr2); ra += fabsf(f[j]); }
        const float rn = sqrtf(fr2);
        fr2 = warp_sumf(fr2);
        float ni = act ? ra : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ni = fmaxf(ni, __shfl_xor_sync(0xffffffffu, ni, o));
        if (act) {
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) E32[lane * ld + j] = f[j];
        }
        __syncwarp();
        float ca = 0.f;
        if (act)
            for (int r = 0; r < p; ++r) ca += fabsf(E32[r * ld + lane]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ca = fmaxf(ca, __shfl_xor_sync(0xffffffffu, ca, o));
        const double ub32 = (double)(fminf(sqrtf(fr2), sqrtf(ca * ni)) * up);
        if (ub32 + err32 < tol) { *dv = ub32 + err32; return 1; }
        float bst = act ? rn : -1.f;
        int bri = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, bst, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bri, o);
            if (ob > bst || (ob == bst && oi < bri)) { bst = ob; bri = oi; }
        }
        double lb32 = (double)(bst * dn);
        if (lb32 - err32 >= tol) { *dv = lb32 - err32; return 0; }
        if (bst > 0.f) {
            if (act) v32[lane] = E32[bri * ld + lane] / bst;
            __syncwarp();
            for (int it = 0; it < 20; ++it) {
                float wr = 0.f;
                if (act) {
#pragma unroll
                    for (int j = 0; j < PM; ++j)
                        if (j < p) wr = fmaf(f[j], v32[j], wr);
                }
                const float nw = sqrtf(warp_sumf(wr * wr));
                lb32 = fmax(lb32, (double)(nw * dn));
                if (lb32 - err32 >= tol) { *dv = lb32 - err32; return 0; }
                if (!(nw > 0.f)) break;
                if (act) w32[lane] = wr;
                __syncwarp();
                float uj = 0.f;
                if (act)
                    for (int r = 0; r < p; ++r) uj = fmaf(E32[r * ld + lane], w32[r], uj);
                const float nu = sqrtf(warp_sumf(uj * uj));
                lb32 = fmax(lb32, (double)(nu / nw * dn));
                if (lb32 - err32 >= tol) { *dv = lb32 - err32; return 0; }
                if (!(nu > 0.f)) break;
                __syncwarp();
                if (act) v32[lane] = uj / nu;
                __syncwarp();
            }
        }
        __syncwarp();
        // FP32 certificate (accept): G32 = fl32(E32^T E32) next to E32 in the
        // scratch; ||G32 - E32^T E32||_2 <= eg32 = gamma32_p ||E32||_F^2.  A
        // successful FP32 factorisation of X I - G32 - c I (c covering its
        // backward error gamma32_{p+1} tr) proves lambda_max(G32) <= X, so
        // sigma(E) <= sigma(E32) + err32 <= sqrt(X + eg32) + err32 < tol: the
        // same argument as the FP64 certificate below, with u = 2^-24.
        {
            const double u = 0x1p-24;
            auto g32 = [&](int k) { return (double)k * u / (1.0 - (double)k * u); };
            const double f2 = (double)fr2 * (1.0 + (double)(p + 2) * 0x1p-23);
            const double eg = 1.01 * g32(p) * f2;
            const double tl = (tol - err32) * (1.0 - 4.0 * (double)(p + 2) * u);
            const double X = tl > 0.0 ? tl * tl * (1.0 - 8.0 * u) - eg : -1.0;
            if (X > 0.0) {
                float* G32 = E32 + (size_t)p * ld;
                const float Xf = __double2float_rd(X);
                for (int kc = 0; kc < p; kc += 8) {
                    float acc[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
                    if (act) {
                        for (int r = 0; r < p; ++r) {
                            const float a = E32[r * ld + lane];
                            const float* row = E32 + r * ld;
#pragma unroll
                            for (int q = 0; q < 8; ++q) acc[q] = fmaf(a, row[min(kc + q, p - 1)], acc[q]);
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int k = kc + q;
                            // off the diagonal 0 - g is exact; on it X - g rounds
                            // down, so the factored matrix is below X I - G32
                            if (k < p) G32[lane * ld + k] = (k == lane) ? __fsub_rd(Xf, acc[q]) : -acc[q];
                        }
                    }
                }
                __syncwarp();
                float trf = act ? G32[lane * ld + lane] : 0.f;
                trf = warp_sumf(trf);
                const double tr = (double)trf * (1.0 + (double)(p + 2) * 0x1p-23);
                if (tr > 0.0) {
                    const float c = __double2float_ru(2.0 * g32(p + 1) * tr);
                    if (act) G32[lane * ld + lane] = __fsub_rd(G32[lane * ld + lane], c);
                    __syncwarp();
                    if (cholesky_warp_f(G32, p, ld) == p) {
                        *dv = (sqrt((double)Xf + eg) + err32) * (1.0 + 8.0 * U64);
                        return 1;
                    }
                }
            }
        }
        __syncwarp();
    }
    // pass 2: E row = D row * B^-1
    double e[PM];
#pragma unroll
    for (int j = 0; j < PM; ++j) e[j] = 0.0;
    if (act) {
        for (int k = 0; k < p; ++k) {
            const double dk = dval(lane, k);
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) e[j] = fma(dk, sB[k * ld + j], e[j]);
        }
    }
    double fro2 = 0.0, rabs = 0.0;
#pragma unroll
    for (int j = 0; j < PM; ++j) {
        if (j < p) { fro2 = fma(e[j], e[j], fro2); rabs += fabs(e[j]); }
    }
    const double rown = sqrt(fro2);
    fro2 = warp_sum(fro2);
    const double ninf = warp_max(act ? rabs : 0.0);
    if (act) {
#pragma unroll
        for (int j = 0; j < PM; ++j)
            if (j < p) ws.E[lane * ld + j] = e[j];
    }
    __syncwarp();
    double cabs = 0.0;
    if (act)
        for (int r = 0; r < p; ++r) cabs += fabs(ws.E[r * ld + lane]);
    const double none = warp_max(cabs);
    const double slack = 1.0 + 4.0 * (double)(p + 2) * U64;
    const double ub = fmin(sqrt(fro2), sqrt(none * ninf)) * slack;
    if (ub + err < tol) { *dv = ub; return 1; }
    // lower bound: the largest row norm (||E^T e_r||), then power steps
    double best = act ? rown : -1.0;
    int br = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && oi < br)) { best = ob; br = oi; }
    }
    double lb = best;
    if (lb * shrink - err >= tol) { *dv = lb; return 0; }
    if (!(best > 0.0)) { *dv = 0.0; return 1; }   // E == 0 after rounding
    if (act) ws.v[lane] = ws.E[br * ld + lane] / best;
    __syncwarp();
    for (int it = 0; it < 16; ++it) {
        double wr = 0.0;
        if (act) {
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) wr = fma(e[j], ws.v[j], wr);
        }
        const double nw = sqrt(warp_sum(wr * wr));
        lb = fmax(lb, nw);
        if (lb * shrink - err >= tol) { *dv = lb; return 0; }
        if (!(nw > 0.0)) break;
        if (act) ws.w[lane] = wr;
        __syncwarp();
        double uj = 0.0;
        if (act)
            for (int r = 0; r < p; ++r) uj = fma(ws.E[r * ld + lane], ws.w[r], uj);
        const double nu = sqrt(warp_sum(uj * uj));
        lb = fmax(lb, nu / nw);
        if (lb * shrink - err >= tol) { *dv = lb; return 0; }
        if (!(nu > 0.0)) break;
        __syncwarp();
        if (act) ws.v[lane] = uj / nu;
        __syncwarp();
    }
    if (!allow_exact_here) { *dv = lb; return -1; }
    // Certified tests on X I - G with G = fl(E^T E) (E here the computed
    // product, within err of the exact one; ||E^T E - G||_2 <= gamma_p
    // ||E||_F^2 =: eg):
    //   accept: the Cholesky factorisation of X I - G - c I succeeds, c
    //     covering its own rounding (backward error <= gamma_{p+1} tr), so
    //     lambda_max(G) < X, sigma(E) < sqrt(X + eg) + err <= tol;
    //   reject: the factorisation of X' I - G meets a pivot <= 0 at k; then
    //     z = [-L11^-T l; 1; 0] has z^T G z >= X' z^T z, and ||E z|| / ||z||
    //     with its rounding and err removed is a lower bound >= tol.
    // A near tie that neither settles goes to the Jacobi eigenvalues of G.
    __syncwarp();
    // column j of E lives in lane j after a transpose read
    double ecol[PM];
#pragma unroll
    for (int r = 0; r < PM; ++r) ecol[r] = (act && r < p) ? ws.E[r * ld + lane] : 0.0;
    __syncwarp();
    // ws.E <- X I - G (neg) or G; G[lane][k] = sum_r E[r][lane] E[r][k] (r in
    // increasing order).  E goes back to shared memory from the rows held in
    // registers, then G is formed eight columns at a time: eight independent
    // FMA chains per lane, each chunk written over its own columns of E only
    // after every lane has read them (later chunks read other columns, and
    // column `lane` is held in ecol).
    auto build = [&](double X, bool neg) {
        __syncwarp();
        if (act) {
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) ws.E[lane * ld + j] = e[j];
        }
        __syncwarp();
        for (int kc = 0; kc < p; kc += 8) {
            double acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = 0.0;
            for (int r = 0; r < p; ++r) {
                const double a = ecol[r];
                const double* row = ws.E + r * ld;
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = fma(a, row[min(kc + u, p - 1)], acc[u]);
            }
            __syncwarp();
            if (act) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = kc + u;
                    if (k < p) ws.E[lane * ld + k] = neg ? ((k == lane ? X : 0.0) - acc[u]) : acc[u];
                }
            }
            __syncwarp();
        }
    };
    const double eg = 1.01 * gamma_u(p) * fro2;
    const double tl = (tol - err) * shrink;
    if (tl > 0.0) {
        const double X = tl * tl * (1.0 - 4.0 * U64) - eg;
        if (X > 0.0) {
            build(X, true);
            const double trA = warp_sum(act ? ws.E[lane * ld + lane] : 0.0);
            if (trA > 0.0) {
                const double c = 2.0 * gamma_u(p + 1) * trA;
                if (act) ws.E[lane * ld + lane] -= c;
                __syncwarp();
                if (cholesky_warp(ws.E, p, ld) == p) {
                    *dv = (sqrt(X + eg) + err) * (1.0 + 8.0 * U64);
                    return 1;
                }
            }
        }
    }
    {
        const double th = (tol + err) / shrink;
        build(th * th * (1.0 + 4.0 * U64) + eg, true);
        const int k = cholesky_warp(ws.E, p, ld);
        if (k < p) {
            // L11^T y = l (row k of L), back substitution; lane i keeps y_i
            double yl = 0.0;
            for (int i = k - 1; i >= 0; --i) {
                const double part = (lane > i && lane < k) ? ws.E[lane * ld + i] * yl : 0.0;
                const double sum = warp_sum(part);
                const double yi = (ws.E[k * ld + i] - sum) / ws.E[i * ld + i];
                if (lane == i) yl = yi;
            }
            const double z = (lane < k) ? -yl : (lane == k ? 1.0 : 0.0);
            double t = 0.0;
#pragma unroll
            for (int j = 0; j < PM; ++j) t = fma(e[j], __shfl_sync(0xffffffffu, z, j), t);
            const double nez = sqrt(warp_sum(t * t));
            const double nz = sqrt(warp_sum(z * z));
            const double lbz = (nez * (1.0 - (double)(p + 4) * U64) - 1.01 * gamma_u(p) * sqrt(fro2) * nz) /
                               (nz * (1.0 + (double)(p + 2) * U64)) - err;
            if (lbz * (1.0 - 8.0 * U64) >= tol) { *dv = lbz; return 0; }
        }
    }
    build(0.0, false);
    const double lam = jacobi_lambda_max_warp(ws.E, p, ld);
    const double sig = sqrt(fmax(lam, 0.0));
    *dv = sig;
    return sig < tol ? 1 : 0;
}

// ---------------------------------------------------------------- rounds
// block part: A_c, B^-1 (FP64), probes (64), entry sketch (SK 32 + 8),
// B^-1 in FP32; then per warp E + v + w
__host__ __device__ inline int eval_block_doubles(int p) {
    const int ld = p + 1;
    return 2 * p * ld + PROBE_STRIDE + 2 * 32 + 8 + (p * ld + 1) / 2;
}
// decide kernel block part: A_c, B^-1 (FP64), probes (64), B^-1 in FP32
__host__ __device__ inline int decide_block_doubles(int p) {
    const int ld = p + 1;
    return 2 * p * ld + PROBE_STRIDE + (p * ld + 1) / 2;
}
__host__ __device__ inline size_t decide_smem_bytes(int p, int wpb) {
    const int ld = p + 1;
    return (size_t)decide_block_doubles(p) * 8 + (size_t)wpb * ((size_t)p * ld + 64) * 8;
}
__host__ __device__ inline size_t eval_smem_bytes(int p, int wpb) {
    const int ld = p + 1;
    return (size_t)eval_block_doubles(p) * 8 + (size_t)wpb * ((size_t)p * ld + 64) * 8;
}

// Entry database of one size group: patch matrices A_c, inverses B_c^{-1},
// ||B_c^{-1}||_F and the probe vector w_c (32 doubles) of every entry, in
// creation order.
struct EntryDB {
    double* A;
    double* Binv;
    double* fro;
    double* w;
};

// Dominant right singular vector of a p x p matrix M (row stride ld) by power
// iteration on M^T M from the all-ones vector; lane k returns v_k (unit, or 0
// when M v vanishes).  One warp, p <= 32: lane r keeps row r of M, the
// transposed products read M directly, so each step is p fused multiply-adds
// per lane and no warp reductions besides the normalisation.
__device__ double dominant_right_sv_warp(const double* M, int p, int ld, int iters) {
    // FP32: only a direction is sought (any direction gives a valid bound,
    // the bounds themselves are formed in FP64 from it), and FP32 runs at 64x
    // the FP64 rate on this GPU
    const int lane = threadIdx.x & 31;
    const bool act = lane < p;
    float row[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) row[k] = (act && k < p) ? (float)M[lane * ld + k] : 0.f;
    float col[32];                                     // column `lane` of M
#pragma unroll
    for (int r = 0; r < 32; ++r) col[r] = (act && r < p) ? (float)M[r * ld + lane] : 0.f;
    float v = act ? 1.f : 0.f;
    for (int it = 0; it < iters; ++it) {
        float t = 0.f;                                 // t_lane = (M v)_lane
#pragma unroll
        for (int k = 0; k < 32; ++k) t = fmaf(row[k], __shfl_sync(0xffffffffu, v, k), t);
        float u = 0.f;                                 // u_lane = (M^T t)_lane
#pragma unroll
        for (int r = 0; r < 32; ++r) u = fmaf(col[r], __shfl_sync(0xffffffffu, t, r), u);
        const float nu = sqrtf(warp_sumf(u * u));
        if (!(nu > 0.f) || !(nu < 3.0e38f)) return (double)v;   // keep the last finite direction
        v = u / nu;
    }
    return (double)v;
}

// y_lane = (M x)_lane for a lane-held x (row stride ld); all lanes call.
__device__ __forceinline__ double matvec_warp(const double* M, int p, int ld, double x) {
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int k = 0; k < p; ++k) {
        const double xk = __shfl_sync(0xffffffffu, x, k);
        if (lane < p) t = fma(M[lane * ld + k], xk, t);
    }
    return t;
}

// Probe vectors of an entry, both of the form w = B^{-1} v / ||v||, so that
// ||D w|| = ||E v|| / ||v|| <= sigma_max(E) for any v:
//   w_1: v = the dominant right singular vector of B^{-1} (tight where B^{-1}
//        amplifies most);
//   w_2: v = A x / ||A x|| with x the dominant right singular vector of A, so
//        w_2 ~ x / sigma_max(A) and ||D w_2|| ~ ||D x|| / ||A x|| (tight where
//        D acts like a multiple of A away from A's near-kernel, e.g. a scaled
//        coefficient, which w_1 misses when that near-kernel is D's kernel).
__device__ void probe_vectors_warp(const double* A, const double* B, int p, int ld, double* w_out) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < p;
    double v = dominant_right_sv_warp(B, p, ld, 10);
    double nv = sqrt(warp_sum(v * v));
    double t = matvec_warp(B, p, ld, v);
    w_out[lane] = (act && nv > 0.0) ? t / nv : 0.0;
    const double x = dominant_right_sv_warp(A, p, ld, 10);
    const double ax = matvec_warp(A, p, ld, x);
    nv = sqrt(warp_sum(ax * ax));
    t = matvec_warp(B, p, ld, nv > 0.0 ? ax / nv : 0.0);
    v = nv > 0.0 ? ax / nv : 0.0;
    nv = sqrt(warp_sum(v * v));
    w_out[PROBE_W2 + lane] = (act && nv > 0.0) ? t / nv : 0.0;
}

// ||B^{-1}||_F and the probe vectors of every matrix of a batch (patch
// matrices A, inverses Binv; one warp each); flags (any_bad, may be NULL)
// when a singular one is among them.
__global__ void k_entry_fro(const double* __restrict__ A, const double* __restrict__ Binv, int m, int p,
                            double* __restrict__ fro, double* __restrict__ w, const int32_t* __restrict__ sflags,
                            int32_t* __restrict__ any_bad) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= m) return;
    double s = 0.0;
    for (int e = lane; e < p * p; e += 32) s = fma(Binv[(int64_t)j * p * p + e], Binv[(int64_t)j * p * p + e], s);
    s = warp_sum(s);
    probe_vectors_warp(A + (int64_t)j * p * p, Binv + (int64_t)j * p * p, p, p, w + (int64_t)j * PROBE_STRIDE);
    if (lane == 0) {
        fro[j] = sqrt(s);
        if (any_bad && sflags[j]) atomicOr(any_bad, 1);
    }
}

// ---------------------------------------------------------------- sketches
// Certified thread-level screen.  For any x and v = A_c x:
//   ||E||_2 >= ||E v|| / ||v||,   E v = D B^ A_c x = D x + D (B^ A_c - I) x,
// so ||E||_2 >= (||D x|| - ||D||_2 rho_c ||x||) / ||A_c x|| with rho_c an
// upper bound of ||B^ A_c - I||_2 (B^ the computed inverse).  D x = A_c x -
// A_i x comes from sketches y_i = fl(A_i x_k) kept for every patch and a few
// fixed unit directions x_k per size group; ||D||_2 <= ||A_c||_F + ||A_i||_F.
// The rounding of the sketches (|fl(A x) - A x| <= gamma_p |A||x|), of the
// norms and of the residual is added to the slack.  Rejecting a pair this way
// reads SK p values of the candidate instead of its p^2 entries.
constexpr int SK = 2;              // sketch directions per size group
struct SketchDB {
    const double* X;               // [SK][32] unit directions (zero beyond p)
    const double* den;             // [count][SK] den_k >= ||A_i x_k|| (norm of the FP64 sketch, widened)
    const double* fa;              // [count] ||A_i||_F
    const double* rho;             // [count] bound of ||B_i^ A_i - I||_2
    const float* Y32;              // [count][SK][p] y_i rounded to FP32 (the screen's operand)
    const double* nlo;             // [count] brackets of ||A_i||_2 for the norm-window
    const double* nhi;             //   search; null when the search is in creation order
    const double* wlo;             // [count] each patch's norm window (norm_window of
    const double* whi;             //   its bracket)
};

__device__ __forceinline__ NormWin norm_window(const SketchDB& sk, int i) { return NormWin{sk.wlo[i], sk.whi[i]}; }


// Directions of a size group: x_0 = the dominant right singular vector of
// the group's middle patch, x_1 = a fixed alternating vector; both unit.
__global__ void k_sketch_dirs(const double* __restrict__ Ag, int count, int p, double* __restrict__ X) {
    const int lane = threadIdx.x & 31;
    const int k = threadIdx.x >> 5;
    const bool act = lane < p;
    double v;
    if (k == 0) {
        v = dominant_right_sv_warp(Ag + (int64_t)(count / 2) * p * p, p, p, 20);
    } else {
        v = act ? ((lane & 1) ? -1.0 : 1.0) * (1.0 + (double)(lane % 3)) : 0.0;
    }
    double nv = sqrt(warp_sum(v * v));
    if (!(nv > 0.0)) {                 // degenerate: fall back to e_0
        v = (lane == 0) ? 1.0 : 0.0;
        nv = 1.0;
    }
    X[k * 32 + lane] = act ? v / nv : 0.0;
}

// Per matrix of a batch (one warp each): y_k = fl(A x_k), ||A||_F and the
// residual bound rho >= ||B^ A - I||_2 with B^ = Binv.
// (PM >= p: the unrolled loops stop at PM, FP64 instructions past p are not
// issued; predicated-off lanes would still cost the FP64 pipe.)
template <int PM>
__global__ void __launch_bounds__(256) k_sketch(const double* __restrict__ A, const double* __restrict__ Binv,
                                                int count, int p, const double* __restrict__ X,
                                                double* __restrict__ den, float* __restrict__ Y32,
                                                double* __restrict__ fa, double* __restrict__ rho) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= count) return;                            // warp-uniform
    const bool act = lane < p;
    const double* Ai = A + (int64_t)i * p * p;
    const double* Bi = Binv + (int64_t)i * p * p;
    double a[PM], b[PM];
#pragma unroll
    for (int j = 0; j < PM; ++j) {
        a[j] = (act && j < p) ? Ai[lane * p + j] : 0.0;
        b[j] = (act && j < p) ? Bi[lane * p + j] : 0.0;
    }
    double fa2 = 0.0, fb2 = 0.0;
#pragma unroll
    for (int j = 0; j < PM; ++j) {
        fa2 = fma(a[j], a[j], fa2);
        fb2 = fma(b[j], b[j], fb2);
    }
    double yn2[SK];
#pragma unroll
    for (int k = 0; k < SK; ++k) {
        double y = 0.0;
#pragma unroll
        for (int j = 0; j < PM; ++j) y = fma(a[j], X[k * 32 + j], y);
        if (act) Y32[((int64_t)i * SK + k) * p + lane] = (float)y;
        yn2[k] = act ? y * y : 0.0;
    }
    // column j of B^ A: lane r sums b[r][k] A[k][j], A[k][j] from lane k
    double res2 = 0.0;
#pragma unroll
    for (int j = 0; j < PM; ++j) {
        if (j < p) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < PM; ++k) t = fma(b[k], __shfl_sync(0xffffffffu, a[j], k), t);
            const double r = t - ((lane == j) ? 1.0 : 0.0);
            if (act) res2 = fma(r, r, res2);
        }
    }
    fa2 = warp_sum(fa2);
    fb2 = warp_sum(fb2);
    res2 = warp_sum(res2);
#pragma unroll
    for (int k = 0; k < SK; ++k) yn2[k] = warp_sum(yn2[k]);
    if (lane == 0) {
        const double fA = sqrt(fa2), fB = sqrt(fb2);
        fa[i] = fA;
        // computed residual entries carry at most gamma_{p+1} |B^||A| error
        rho[i] = 1.01 * sqrt(res2) + 1.01 * gamma_u(p + 1) * fB * fA;
        // den_k >= ||A x_k||: the computed sketch norm widened for its own
        // rounding and for that of the sketch (gamma_p |A||x_k|)
#pragma unroll
        for (int k = 0; k < SK; ++k)
            den[(int64_t)i * SK + k] = sqrt(yn2[k]) * (1.0 + (double)(p + 2) * U64) + 1.01 * gamma_u(p) * fA;
    }
}

// Entry side of the screen, staged in shared memory: y_c in FP32 (SK x 32,
// zero beyond p) and the denominators den_k >= ||A_c x_k|| (precomputed with
// the sketches).
__device__ __forceinline__ void stage_sketch(const double* __restrict__ denc, const float* __restrict__ Yc32, int p,
                                             float* sy32, double* sden) {
    for (int t = threadIdx.x; t < SK * 32; t += blockDim.x) {
        const int k = t >> 5, r = t & 31;
        sy32[t] = (r < p) ? Yc32[k * p + r] : 0.f;
    }
    if (threadIdx.x < SK) sden[threadIdx.x] = denc[threadIdx.x];
}

__device__ __forceinline__ float ldg_nc_f(const float* q) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(q));
    return v;
}

// Thread-level decision for candidate i against the staged entry: true when
// the certified lower bound reaches tol (reject).  The distance of the
// sketches is formed in FP32 from the FP32 copies: their rounding
// (||y - fl32(y)|| <= 2^-24 ||y||, ||y|| <= 1.01 ||A||_F) and that of the FP32
// norm and of its correctly rounded FP32 square root ((p + 9) 2^-24
// relative) are taken off the bound, and the test num_k >= tol den_k is made
// without a division.  sketch_load issues all SK x PM loads of the candidate
// (indices clamped to p - 1) so that they are in flight with the caller's
// other loads of that candidate.
template <int PM>
__device__ __forceinline__ void sketch_load(const float* __restrict__ yi, int p, float (&v)[SK * PM]) {
#pragma unroll
    for (int k = 0; k < SK; ++k)
#pragma unroll
        for (int r = 0; r < PM; ++r) v[k * PM + r] = ldg_nc_f(yi + k * p + min(r, p - 1));
}

template <int PM>
__device__ __forceinline__ bool sketch_bound_rejects(const float (&v)[SK * PM], double fi, const float* sy32,
                                                     const double* sden, double fc, double rhoc, int p, double tol) {
    const double slack = 1.01 * (fc + fi) * (gamma_u(p) + rhoc) + 1.01 * 0x1p-24 * (fc + fi);
    bool rej = false;
#pragma unroll
    for (int k = 0; k < SK; ++k) {
        float d2 = 0.f;
#pragma unroll
        for (int r = 0; r < PM; ++r) {
            const float d = (r < p) ? sy32[k * 32 + r] - v[k * PM + r] : 0.f;
            d2 = fmaf(d, d, d2);
        }
        const double num = (double)sqrtf(d2) * (1.0 - (double)(p + 9) * 0x1p-24) - slack * (1.0 + 8.0 * U64);
        if (sden[k] > 0.0 && num * (1.0 - 8.0 * U64) >= tol * sden[k] * (1.0 + 4.0 * U64)) rej = true;
    }
    return rej;
}

__device__ __forceinline__ bool round_last_block(int* ticket) {
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

// One round of Alg. 1 in two kernels.  Every patch's inverse, probes, sketch
// and ||A^-1||_F were computed up front in batched launches, so the new entry
// (patch st->next) is ready to stage.
//   k_round_screen: one thread per unassigned candidate after the entry runs
//     the sketch screen; a rejected candidate stays unassigned and bids for
//     being the next entry (atomicMin); the others are appended to a global
//     survivor list.
//   k_round_decide: the warps of the whole grid share the survivor list
//     (accepted ones come in runs of neighbouring patches, so a per-block
//     queue would leave most SMs idle); rejected survivors bid as well.  The
//     last block records the entry and the smallest rejected index, which is
//     exactly the smallest unassigned patch after the round.
template <int PM>
__global__ void __launch_bounds__(EVAL_THREADS) k_round_screen(RoundDev* st, const int32_t* __restrict__ phi,
                                                               int count, int p, SketchDB sk, double tol,
                                                               int32_t* __restrict__ surv_list) {
    __shared__ float sy[SK * 32];
    __shared__ double sden[SK];
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int i0 = st->next;
    const double fc = sk.fa[i0], rhoc = sk.rho[i0];
    stage_sketch(sk.den + (int64_t)i0 * SK, sk.Y32 + (int64_t)i0 * SK * p, p, sy, sden);
    __syncthreads();
    unsigned long long my_evals = 0, my_screened = 0;
    int my_min = count;
    for (int base = i0 + 1 + blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
        const int cand = base + threadIdx.x;
        const int cc = min(cand, count - 1);
        float v[SK * PM];
        sketch_load<PM>(sk.Y32 + (int64_t)cc * SK * p, p, v);
        const double fi = sk.fa[cc];
        const bool open = cand < count && phi[cc] == -1;
        const bool wout = open && sk.nlo && outside_window(norm_window(sk, cc), sk.nlo[i0], sk.nhi[i0]);
        const bool rej = open && (wout || sketch_bound_rejects<PM>(v, fi, sy, sden, fc, rhoc, p, tol));
        if (open && rej) my_min = min(my_min, cand);
        const unsigned opened = __ballot_sync(0xffffffffu, open && !wout);
        const unsigned surv = __ballot_sync(0xffffffffu, open && !rej);
        my_evals += __popc(opened);
        my_screened += __popc(opened & ~surv);
        int wb = 0;
        if (lane == 0 && surv) wb = atomicAdd(&st->nsurv, __popc(surv));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (open && !rej) surv_list[wb + __popc(surv & ((1u << lane) - 1u))] = cand;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_min = min(my_min, __shfl_xor_sync(0xffffffffu, my_min, o));
    if (lane == 0) {
        if (my_evals) atomicAdd(&st->evals, my_evals);
        if (my_screened) atomicAdd(&st->screened, my_screened);
        if (my_evals > my_screened) atomicAdd(&st->decided, my_evals - my_screened);
        if (my_min < count) atomicMin(&st->next_new, my_min);
    }
}

__global__ void __launch_bounds__(EVAL_THREADS, 4) k_round_decide(RoundDev* st, int32_t* __restrict__ phi, int count,
                                                                  const double* __restrict__ Ag, int p,
                                                                  const double* __restrict__ Ball,
                                                                  const double* __restrict__ fro_all,
                                                                  const double* __restrict__ w_all,
                                                                  const int32_t* __restrict__ sing_all, double tol,
                                                                  const int32_t* __restrict__ surv_list,
                                                                  int32_t* __restrict__ rep_local) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (st->done) return;
    const int ld = p + 1;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int i0 = st->next;
    const int m = st->m;
    const int ns = st->nsurv;
    unsigned long long my_exact = 0;
    int my_min = count;
    if (blockIdx.x * wpb < ns) {                      // block-uniform: this block has survivors
        double* sAc = reinterpret_cast<double*>(smem);
        double* sB = sAc + p * ld;
        double* sw = sB + p * ld;
        float* sB32 = reinterpret_cast<float*>(sw + PROBE_STRIDE);
        double* wbase = reinterpret_cast<double*>(smem) + decide_block_doubles(p) + (size_t)wid * (p * ld + 64);
        WarpScratch ws{wbase, wbase + p * ld, wbase + p * ld + 32};
        const double* a = Ag + (int64_t)i0 * p * p;
        const double* bm = Ball + (int64_t)i0 * p * p;
        for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
            sAc[(t / p) * ld + (t % p)] = a[t];
            const double b = bm[t];
            sB[(t / p) * ld + (t % p)] = b;
            sB32[(t / p) * ld + (t % p)] = (float)b;
        }
        if (threadIdx.x < PROBE_STRIDE) sw[threadIdx.x] = w_all[(int64_t)i0 * PROBE_STRIDE + threadIdx.x];
        const double bfro = fro_all[i0];
        __syncthreads();
        const int nwarps = gridDim.x * wpb;
        for (int q = blockIdx.x * wpb + wid; q < ns; q += nwarps) {
            const int c2 = surv_list[q];
            double dv;
            int dec = decide_pair(Ag + (int64_t)c2 * p * p, sAc, sB, p, ld, bfro, tol, ws, &dv, false, sw, sB32);
            if (dec < 0) {
                dec = decide_pair(Ag + (int64_t)c2 * p * p, sAc, sB, p, ld, bfro, tol, ws, &dv, true, sw, nullptr);
                ++my_exact;
            }
            if (dec == 1) { if (lane == 0) phi[c2] = m; }
            else my_min = min(my_min, c2);
            __syncwarp();
        }
    }
    if (lane == 0) {
        if (my_exact) atomicAdd(&st->exact, my_exact);
        if (my_min < count) atomicMin(&st->next_new, my_min);
    }
    if (!round_last_block(&st->ticket)) return;
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

// ---------------------------------------------------------------- persistent rounds
// Barrier settings of this translation unit: the arrivals beyond the grid a
// barrier waits for (0; 1 only under psr_debug_inject, so that the wait runs
// out) and the spin limit.
static __device__ unsigned int g_bar_extra = 0u;
static __device__ long long g_bar_limit = 1ll << 24;

// Grid barrier of a cooperatively launched kernel (every block co-resident, so
// every wait ends); bounded all the same: past the limit the error flag is
// set and the barrier left, and the host reports PSR_ERR_TIMEOUT.
__device__ __forceinline__ void rounds_barrier(unsigned int* bar, int32_t* err) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = bar + 1;
        const unsigned int g = *vgen;
        const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
        const long long limit = g_bar_limit;
        if (arrived == gridDim.x + g_bar_extra) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g) {
                if (++spins > limit) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// All rounds of Alg. 1 in one cooperative launch, KC candidate entries per
// round.  The candidates are the KC smallest open (unassigned) patches
// c_0 < ... < c_{K-1}.  Every entry made before the round has rejected every
// open patch, so in sequential Alg. 1 c_k becomes an entry exactly when no
// entry among c_0..c_{k-1} accepts it, and every other open patch (all lie
// above c_{K-1}) meets the round's entries in that order.  A round:
//   A. every block screens all pairs (entry c_l, patch c_k), l < k, itself
//      (the same survivor list in every block); the grid's warps decide the
//      survivors; grid barrier; every block derives the entry mask R
//      serially (c_0 is an entry, c_k one iff no entry of R below it accepts
//      it) and block 0 assigns the candidates;
//   B. one thread per other open patch screens it against the entries of R;
//      survivors (patch, entry) go to a global list; grid barrier; the warps
//      decide them, and the warp that decides a patch's last pair assigns it
//      to its first accepting entry in creation order (the lowest bit of
//      R & accepted); grid barrier.
// A patch therefore meets the entries in creation order and stops at its
// first accept, so phi is that of sequential Alg. 1; the evaluation count
// adds, per patch, the entries of R up to and including its first accept
// (all of R when none accepts) -- the evaluations sequential Alg. 1 makes.
// Pairs decided beyond a patch's first accept, and pairs with candidates
// that turn out not to be entries, are extra work and are not counted.  On
// the 3D lognormal workload a round of 64 candidates makes about 14 entries.
constexpr int KC = 64;

struct MultiWS {
    uint32_t* obits;               // [ceil(count/32)] open patches
    uint32_t* pairs;               // [count * KC] phase B survivor pairs, i << 6 | l
    int32_t* rem;                  // [count] undecided pairs of patch i in this round
    unsigned long long* accm;      // [count] entries (bit l) that accepted patch i
    unsigned long long* exm;       // [count] pairs of patch i decided by the exact stage
    unsigned long long* rejm;      // [count] pairs of patch i the screen rejected
    unsigned long long* wom;       // [count] pairs of patch i outside the norm window
    unsigned long long* accA;      // [2][KC] phase A accepts of candidate k, by round parity
    unsigned long long* exA;       // [2][KC] phase A exact-stage pairs of candidate k
    int32_t* npB;                  // [2] phase B pair counts, by round parity
    int32_t* wq;                   // [4] pairs handed out beyond the first sweep: A, B by parity
    const float* B32;              // [count][p * p] inverses rounded to FP32
};

// Pair q of a decide phase for the calling warp: the first one statically
// (q = the warp's grid index), later ones from a shared counter, so that
// warps that drew cheap pairs take more (the costly ones, certificates and
// power iterations, come in runs of neighbouring patches).
__device__ __forceinline__ int next_pair(int32_t* wq, int gwarps) {
    int q = 0;
    if ((threadIdx.x & 31) == 0) q = gwarps + atomicAdd(wq, 1);
    return __shfl_sync(0xffffffffu, q, 0);
}

// Thresholds of the multi-entry screen.  The one-entry screen rejects when
// sqrt(d2)(1 - (p+9) 2^-24)(1 - 8u) - slack(1 + 8u)(1 - 8u) >= tol den_k
// (1 + 4u), slack = (f_c + f_i) s_c, s_c = 1.01 (gamma_p + rho_c + 2^-24):
// that is sqrt(d2) >= alpha_k + beta f_i with the entry's alpha_k, beta.
// Both are rounded up to FP32 (with a 2^-40 margin for their FP64
// evaluation) and f_i too, and the threshold formed with an FMA rounded up,
// so the FP32 test sqrt(d2) >= T is a certified reject as before.  A
// direction with den_k = 0 gives no bound (threshold NaN: never rejects).
__device__ __forceinline__ void multi_thresholds(double fc, double rhoc, const double* den, int p, double tol,
                                                 float* thr, float* beta) {
    const double sc = 1.01 * (gamma_u(p) + rhoc) + 1.01 * 0x1p-24;
    const double a = 1.0 - (double)(p + 9) * 0x1p-24;
    const double c1 = (1.0 + 4.0 * U64) / (1.0 - 8.0 * U64);
    const double c2 = 1.0 + 8.0 * U64;
    const double widen = 1.0 + 0x1p-40;
    *beta = __double2float_ru(sc * c2 / a * widen);
#pragma unroll
    for (int k = 0; k < SK; ++k)
        thr[k] = den[k] > 0.0 ? __double2float_ru((tol * den[k] * c1 + fc * sc * c2) / a * widen)
                              : __int_as_float(0x7fc00000);   // NaN: this direction never rejects
}

// Multi-entry screen of one patch sketch v (FP32, f_i rounded up in fi32)
// against staged entry l: true when the certified lower bound reaches tol.
template <int PM>
__device__ __forceinline__ bool multi_rejects(const float (&v)[SK * PM], float fi32, const float* sy32,
                                              const float* thr, float beta, int p) {
    bool rej = false;
#pragma unroll
    for (int k = 0; k < SK; ++k) {
        float d2 = 0.f;
#pragma unroll
        for (int r = 0; r < PM; ++r) {
            const float d = (r < p) ? sy32[k * 32 + r] - v[k * PM + r] : 0.f;
            d2 = fmaf(d, d, d2);
        }
        if (sqrtf(d2) >= __fmaf_ru(beta, fi32, thr[k])) rej = true;
    }
    return rej;
}

// Where the entries of a multi-entry pass live: the group's own patches
// (Alg. 1 rounds) or a seed database; entry c is at A + c p^2 and so on.
struct EntrySrc {
    const double* A;               // [*][p * p] patch matrices of the entries
    const double* B;               // [*][p * p] FP64 inverses
    const float* B32;              // [*][p * p] inverses rounded to FP32
    const double* fro;             // [*] ||B^-1||_F
    const double* w;               // [*][PROBE_STRIDE] probe vectors
};

// One pair (entry c, patch i) through the certified cascade; *ex is set when
// the exact stage decided it.  The warp first forms D = A_c - A_i in its
// shared scratch sD with coalesced loads (both matrices are contiguous; rows
// read lane by lane from global memory cost one L1 wavefront per lane and
// were the bulk of a decision's time), testing bitwise equality on the way;
// the inverses are read from global memory (every lane reads the same entry:
// one wavefront per load).
template <int PM>
__device__ __forceinline__ int multi_decide(const EntrySrc& es, const double* __restrict__ Ag, int p, double tol,
                                            WarpScratch ws, double* sD, int c, int i, bool* ex) {
    const int lane = threadIdx.x & 31;
    const size_t pp = (size_t)p * p;
    const double* Ac = es.A + (int64_t)c * pp;
    const double* Ai = Ag + (int64_t)i * pp;
    bool same = true;
    __syncwarp();                                  // the previous pair's readers of sD are done
    for (int e = lane; e < p * p; e += 32) {
        const double a = Ac[e], b = Ai[e];
        same &= __double_as_longlong(a) == __double_as_longlong(b);
        sD[e] = a - b;
    }
    *ex = false;
    if (__all_sync(0xffffffffu, same)) return 1;   // bitwise equal patches: D = 0
    __syncwarp();
    double dv;
    int dec = decide_pair<PM, true>(nullptr, sD, es.B + (int64_t)c * pp, p, p, es.fro[c], tol, ws, &dv, false,
                                    es.w + (int64_t)c * PROBE_STRIDE, es.B32 + (int64_t)c * pp);
    if (dec < 0) {
        dec = decide_pair<PM, true>(nullptr, sD, es.B + (int64_t)c * pp, p, p, es.fro[c], tol, ws, &dv, true,
                                    es.w + (int64_t)c * PROBE_STRIDE, nullptr);
        *ex = true;
    }
    return dec;
}

// Bits 0..l of a 64-bit mask (l in [0, 63]) and bits below l.
__device__ __forceinline__ unsigned long long upto_bit(int l) { return l >= 63 ? ~0ull : ((2ull << l) - 1ull); }
__device__ __forceinline__ unsigned long long below_bit(int l) { return (1ull << l) - 1ull; }

template <int PM>
__global__ void __launch_bounds__(EVAL_THREADS, 4) k_rounds_multi(
    RoundDev* st, int32_t* __restrict__ phi, int count, const double* __restrict__ Ag, int p,
    EntrySrc own, const int32_t* __restrict__ sing_all, SketchDB sk, double tol, MultiWS mw,
    int32_t* __restrict__ rep_local, unsigned int* bar, int32_t* err, EntrySrc seed, SketchDB skd, int m0) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int SYS = SK * 32 + 1;               // padded stride: lanes over candidates hit distinct banks
    __shared__ float sy[KC * SYS];                 // candidates' sketches (FP32, zero beyond p)
    __shared__ float sthr[KC * SK];                // screen thresholds alpha_k per candidate
    __shared__ float sbeta[KC];
    __shared__ float sfi[KC];                      // candidates' ||A||_F rounded up (as patches in phase A)
    __shared__ int scand[KC];
    __shared__ int sridx[KC];                      // slots of the entries of R, in order
    __shared__ unsigned long long srejA[KC], sacc[KC], sexA[KC];
    __shared__ unsigned long long swinA[KC];       // phase A pairs outside the norm window
    __shared__ double snlo[KC], snhi[KC];          // candidates' ||A||_2 brackets (norm window)
    __shared__ unsigned short sapair[KC * (KC - 1) / 2];
    __shared__ int s_aoff[KC];
    __shared__ int s_wsum[EVAL_THREADS / 32];
    __shared__ int s_found, s_na;
    __shared__ unsigned long long s_R;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* wbase = reinterpret_cast<double*>(smem) + (size_t)wid * (2 * (size_t)p * p + 64);
    WarpScratch ws{wbase, wbase + (size_t)p * p, wbase + (size_t)p * p + 32};
    double* sD = wbase + (size_t)p * p + 64;       // D = A_c - A_i of the pair being decided
    const int nwords = (count + 31) >> 5;
    const int gthreads = gridDim.x * blockDim.x;
    const int gwarps = gridDim.x * wpb;
    const int gw = blockIdx.x * wpb + wid;
    unsigned long long my_evals = 0, my_exact = 0, my_screened = 0, my_decided = 0;
    int m = st->m;
    int nrounds = 0;
    const bool win = sk.nlo != nullptr;            // norm-window search (no seed database)
    // the open bitmap from phi (a seed database may have assigned some)
    for (int wd = gw; wd < nwords; wd += gwarps) {
        const int i = wd * 32 + lane;
        const unsigned b = __ballot_sync(0xffffffffu, i < count && phi[i] == -1);
        if (lane == 0) mw.obits[wd] = b;
    }
    rounds_barrier(bar, err);
    int fw = 0;                                    // no open patch below word fw
    bool ok = *((volatile int*)err) == 0;
    int npass = 0;                                 // passes so far (seed chunks and rounds): counter parity
    // Phase B of a pass: every open patch i >= lo screened against the staged
    // entries of R (slots sridx[0..nR)), the surviving pairs decided by the
    // grid's warps; the warp deciding a patch's last pair assigns it to its
    // first accepting entry, numbered ebase + (its rank in R).  Two grid
    // barriers; false when one gave up.  wnd: the norm window applies (the
    // staged entries are candidates, snlo / snhi hold their brackets).
    auto phase_b = [&](const EntrySrc& es, int ebase, unsigned long long R, int nR, int lo, int par,
                       bool wnd) -> bool {
        for (int base = lo + blockIdx.x * blockDim.x; base < count; base += gthreads) {
            const int i = base + threadIdx.x;
            const bool open = i < count && ((__ldcg(mw.obits + (i >> 5)) >> (i & 31)) & 1u);
            unsigned long long rej = 0ull, wo = 0ull;
            if (open) {
                float v[SK * PM];
                sketch_load<PM>(sk.Y32 + (int64_t)i * SK * p, p, v);
                const float fi32 = __double2float_ru(sk.fa[i]);
                NormWin w{0.0, 0.0};
                if (wnd) w = norm_window(sk, i);
                for (int t = 0; t < nR; ++t) {
                    const int l = sridx[t];
                    if (wnd && outside_window(w, snlo[l], snhi[l])) wo |= 1ull << l;
                    else if (multi_rejects<PM>(v, fi32, sy + l * SYS, sthr + l * SK, sbeta[l], p)) rej |= 1ull << l;
                }
                rej |= wo;
            }
            const unsigned long long surv = open ? (R & ~rej) : 0ull;
            const int ns = __popcll(surv);
            if (open && ns == 0) {                 // rejected by every entry: stays open
                my_evals += nR - __popcll(wo);
                my_screened += nR - __popcll(wo);
            }
            int incl = ns;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int wtot = __shfl_sync(0xffffffffu, incl, 31);
            int wb = 0;
            if (lane == 31 && wtot) wb = atomicAdd(mw.npB + par, wtot);
            wb = __shfl_sync(0xffffffffu, wb, 31);
            if (ns) {
                mw.rem[i] = ns;
                mw.rejm[i] = rej & R;
                if (wnd) mw.wom[i] = wo;
                mw.accm[i] = 0ull;
                mw.exm[i] = 0ull;
                int pos = wb + incl - ns;
                unsigned long long b = surv;
                while (b) {
                    const int l = __ffsll((long long)b) - 1;
                    mw.pairs[pos++] = ((uint32_t)i << 6) | (uint32_t)l;
                    b &= b - 1ull;
                }
            }
        }
        rounds_barrier(bar, err);
        if (*((volatile int*)err)) return false;
        const int npb = __ldcg(mw.npB + par);
        for (int q = gw; q < npb; q = next_pair(mw.wq + 2 + par, gwarps)) {
            const uint32_t pr = __ldcg(mw.pairs + q);
            const int i = (int)(pr >> 6), l = (int)(pr & 63u);
            bool ex;
            const int dec = multi_decide<PM>(es, Ag, p, tol, ws, sD, scand[l], i, &ex);
            if (lane == 0) {
                ++my_decided;
                if (dec == 1) atomicOr(mw.accm + i, 1ull << l);
                if (ex) atomicOr(mw.exm + i, 1ull << l);
                __threadfence();
                if (atomicSub(mw.rem + i, 1) == 1) {
                    __threadfence();
                    const unsigned long long a = atomicOr(mw.accm + i, 0ull) & R;
                    const unsigned long long exb = atomicOr(mw.exm + i, 0ull);
                    const unsigned long long rj = __ldcg(mw.rejm + i);
                    unsigned long long path = R;
                    if (a) {
                        const int ls = __ffsll((long long)a) - 1;
                        path = R & upto_bit(ls);
                        phi[i] = ebase + __popcll(R & below_bit(ls));
                        atomicAnd(mw.obits + (i >> 5), ~(1u << (i & 31)));
                    }
                    if (wnd) path &= ~__ldcg(mw.wom + i);   // skipped entries are not tests
                    my_evals += __popcll(path);
                    my_screened += __popcll(rj & path);
                    my_exact += __popcll(exb & path);
                }
            }
            __syncwarp();
        }
        rounds_barrier(bar, err);
        return *((volatile int*)err) == 0;
    };
    // Seed database first (seeded Alg. 1): its entries exist before any new
    // one, so every open patch meets them in creation order, 64 at a time;
    // no entry among them needs deciding.
    for (int j0 = 0; ok && j0 < m0; j0 += KC) {
        const int par = npass & 1;
        ++npass;
        const int K = min(KC, m0 - j0);
        for (int t = threadIdx.x; t < K * SK * 32; t += blockDim.x) {
            const int l = t / (SK * 32), q = t % (SK * 32), k = q >> 5, r = q & 31;
            sy[l * SYS + q] = (r < p) ? skd.Y32[((int64_t)(j0 + l) * SK + k) * p + r] : 0.f;
        }
        for (int l = threadIdx.x; l < K; l += blockDim.x) {
            double den[SK];
#pragma unroll
            for (int k = 0; k < SK; ++k) den[k] = skd.den[(int64_t)(j0 + l) * SK + k];
            multi_thresholds(skd.fa[j0 + l], skd.rho[j0 + l], den, p, tol, sthr + l * SK, sbeta + l);
            scand[l] = j0 + l;
            sridx[l] = l;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {      // counters of the other parity are free again
            mw.npB[par ^ 1] = 0;
            mw.wq[2 + (par ^ 1)] = 0;
        }
        __syncthreads();
        const unsigned long long R = (K == KC) ? ~0ull : ((1ull << K) - 1ull);
        ok = phase_b(seed, j0, R, K, 0, par, false);
    }
    // candidates per round: 64, or fewer while rounds make few entries (a
    // round's pairs among its candidates grow as K^2; on the graded Stokes
    // mesh about 3 of 64 neighbouring candidates are entries)
    int klim = KC;
    for (int round = 0; ok && round < count; ++round) {
        const int par = npass & 1;
        ++npass;
        // ---- the KC smallest open patches (every block finds the same)
        if (threadIdx.x == 0) s_found = 0;
        __syncthreads();
        for (int w0 = fw; w0 < nwords; w0 += blockDim.x) {
            const int wd = w0 + threadIdx.x;
            const unsigned bits = wd < nwords ? __ldcg(mw.obits + wd) : 0u;
            const int c = __popc(bits);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wsum[wid] = incl;
            __syncthreads();
            int pos = s_found, tot = s_found;
            for (int q = 0; q < wpb; ++q) {
                if (q < wid) pos += s_wsum[q];
                tot += s_wsum[q];
            }
            pos += incl - c;
            unsigned b = bits;
            while (b && pos < klim) {
                scand[pos++] = wd * 32 + (__ffs(b) - 1);
                b &= b - 1;
            }
            __syncthreads();
            if (threadIdx.x == 0) s_found = min(tot, klim);
            __syncthreads();
            if (s_found >= klim) break;
        }
        const int K = s_found;
        if (K == 0) break;                         // every patch assigned (same in every block)
        ++nrounds;
        fw = scand[0] >> 5;
        // ---- stage the candidates
        for (int t = threadIdx.x; t < K * SK * 32; t += blockDim.x) {
            const int l = t / (SK * 32), q = t % (SK * 32), k = q >> 5, r = q & 31;
            sy[l * SYS + q] = (r < p) ? sk.Y32[((int64_t)scand[l] * SK + k) * p + r] : 0.f;
        }
        for (int l = threadIdx.x; l < K; l += blockDim.x) {
            const int c = scand[l];
            double den[SK];
#pragma unroll
            for (int k = 0; k < SK; ++k) den[k] = sk.den[(int64_t)c * SK + k];
            multi_thresholds(sk.fa[c], sk.rho[c], den, p, tol, sthr + l * SK, sbeta + l);
            sfi[l] = __double2float_ru(sk.fa[c]);
            srejA[l] = 0ull;
            swinA[l] = 0ull;
            if (win) {
                snlo[l] = sk.nlo[c];
                snhi[l] = sk.nhi[c];
            }
        }
        if (threadIdx.x == 0) s_na = 0;
        __syncthreads();
        // ---- phase A: pairs among the candidates, screened by every block
        // (thread k takes candidate k as the patch and the entries l < k in
        // turn; the reject bits need no atomics), survivors listed in (k, l)
        // order so that every block holds the same list
        for (int t = threadIdx.x; t < 2 * KC; t += blockDim.x) {
            const int k = t & (KC - 1), l0 = (t >> 6) * 32;   // entries l0 .. l0 + 31 below k
            if (k < K && l0 < k) {
                float v[SK * PM];
#pragma unroll
                for (int kk = 0; kk < SK; ++kk)
#pragma unroll
                    for (int r = 0; r < PM; ++r) v[kk * PM + r] = sy[k * SYS + kk * 32 + r];
                unsigned long long rb = 0ull, wb = 0ull;
                const int l1 = min(k, l0 + 32);
                NormWin w{0.0, 0.0};
                if (win) w = norm_window(sk, scand[k]);
                for (int l = l0; l < l1; ++l) {
                    if (win && outside_window(w, snlo[l], snhi[l])) wb |= 1ull << l;
                    else if (multi_rejects<PM>(v, sfi[k], sy + l * SYS, sthr + l * SK, sbeta[l], p)) rb |= 1ull << l;
                }
                if (rb | wb) atomicOr(&srejA[k], rb | wb);
                if (wb) atomicOr(&swinA[k], wb);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int o = 0;
            for (int k = 0; k < K; ++k) {
                s_aoff[k] = o;
                o += __popcll(~srejA[k] & below_bit(k));
            }
            s_na = o;
        }
        __syncthreads();
        for (int k = 1 + wid; k < K; k += wpb) {
            const unsigned long long sv = ~srejA[k] & below_bit(k);
            for (int l0 = 0; l0 < k; l0 += 32) {
                const int l = l0 + lane;
                if (l < k && ((sv >> l) & 1ull))
                    sapair[s_aoff[k] + __popcll(sv & below_bit(l))] = (unsigned short)((l << 8) | k);
            }
        }
        __syncthreads();
        const int na = s_na;
        for (int q = gw; q < na; q = next_pair(mw.wq + par, gwarps)) {
            const int l = sapair[q] >> 8, k = sapair[q] & 255;
            bool ex;
            const int dec = multi_decide<PM>(own, Ag, p, tol, ws, sD, scand[l], scand[k], &ex);
            if (lane == 0) {
                ++my_decided;
                if (dec == 1) atomicOr(&mw.accA[par * KC + k], 1ull << l);
                if (ex) atomicOr(&mw.exA[par * KC + k], 1ull << l);
            }
            __syncwarp();
        }
        rounds_barrier(bar, err);
        if (*((volatile int*)err)) break;
        // ---- the round's entries
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            sacc[k] = __ldcg(mw.accA + par * KC + k);
            sexA[k] = __ldcg(mw.exA + par * KC + k);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long R = 1ull;
            int nr = 0;
            sridx[nr++] = 0;
            for (int k = 1; k < K; ++k)
                if ((sacc[k] & R) == 0ull) {
                    R |= 1ull << k;
                    sridx[nr++] = k;
                }
            s_R = R;
        }
        __syncthreads();
        const unsigned long long R = s_R;
        const int nR = __popcll(R);
        if (blockIdx.x == 0) {
            if (threadIdx.x < KC) {                // phase A counters of the other parity are free again
                mw.accA[(par ^ 1) * KC + threadIdx.x] = 0ull;
                mw.exA[(par ^ 1) * KC + threadIdx.x] = 0ull;
            }
            if (threadIdx.x == 0) {
                mw.npB[par ^ 1] = 0;
                mw.wq[par ^ 1] = 0;
                mw.wq[2 + (par ^ 1)] = 0;
            }
            // the candidates: entries, or assigned to their first accepting entry
            for (int k = threadIdx.x; k < K; k += blockDim.x) {
                const int c = scand[k];
                unsigned long long path;
                int e;
                if ((R >> k) & 1ull) {
                    path = R & below_bit(k);
                    e = m + __popcll(path);
                    rep_local[e] = c;
                } else {
                    const int ls = __ffsll((long long)(sacc[k] & R & below_bit(k))) - 1;
                    path = R & upto_bit(ls);
                    e = m + __popcll(R & below_bit(ls));
                }
                phi[c] = e;
                path &= ~swinA[k];                 // entries outside the norm window are not tests
                my_evals += __popcll(path);
                my_screened += __popcll(srejA[k] & path);
                my_exact += __popcll(sexA[k] & path);
                atomicAnd(mw.obits + (c >> 5), ~(1u << (c & 31)));
            }
            if (threadIdx.x == 0 && st->first_singular < 0) {
                for (int t = 0; t < nR; ++t)
                    if (sing_all[scand[sridx[t]]]) {
                        st->first_singular = scand[sridx[t]];
                        break;
                    }
            }
        }
        // ---- phase B: every other open patch against the entries of R
        if (!phase_b(own, m, R, nR, scand[K - 1] + 1, par, win)) break;
        m += nR;
        klim = min(KC, max(16, 2 * nR + 8));       // the same in every block
    }
    // the counts are per thread here: sum each warp's before the atomics
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_evals += __shfl_xor_sync(0xffffffffu, my_evals, o);
        my_exact += __shfl_xor_sync(0xffffffffu, my_exact, o);
        my_screened += __shfl_xor_sync(0xffffffffu, my_screened, o);
        my_decided += __shfl_xor_sync(0xffffffffu, my_decided, o);
    }
    if (lane == 0) {
        if (my_evals) atomicAdd(&st->evals, my_evals);
        if (my_exact) atomicAdd(&st->exact, my_exact);
        if (my_screened) atomicAdd(&st->screened, my_screened);
        if (my_decided) atomicAdd(&st->decided, my_decided);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *((volatile int*)err) == 0) {
        st->nrounds = nrounds;
        st->m = m;
        st->next = count;
        st->done = 1;
    }
}

// Stages seed entry e (patch matrix, inverse, probe) into shared memory.
__device__ __forceinline__ void stage_seed(EntryDB db, int p, int e, double* sAc, double* sB, double* sw) {
    const int ld = p + 1;
    const double* a = db.A + (int64_t)e * p * p;
    const double* bm = db.Binv + (int64_t)e * p * p;
    for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
        sAc[(t / p) * ld + (t % p)] = a[t];
        sB[(t / p) * ld + (t % p)] = bm[t];
    }
    if (threadIdx.x < PROBE_STRIDE) sw[threadIdx.x] = db.w[(int64_t)e * PROBE_STRIDE + threadIdx.x];
}

// Seeded Alg. 1: every still unassigned patch compared with seed entry e
// (sketch screen first, as in k_round; skd holds the seed entries' sketches).
__global__ void __launch_bounds__(EVAL_THREADS, 4) k_seed_pass(RoundDev* st, int32_t* __restrict__ phi, int count,
                                                     const double* __restrict__ Ag, int p, EntryDB db, SketchDB sk,
                                                     SketchDB skd, double tol, int e) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* sAc = reinterpret_cast<double*>(smem);
    double* sB = sAc + p * ld;
    double* sw = sB + p * ld;
    float* sy = reinterpret_cast<float*>(sw + PROBE_STRIDE);
    double* sden = sw + PROBE_STRIDE + SK * 32;
    float* sB32 = reinterpret_cast<float*>(sden + 8);
    double* wbase = reinterpret_cast<double*>(smem) + eval_block_doubles(p) + (size_t)wid * (p * ld + 64);
    WarpScratch ws{wbase, wbase + p * ld, wbase + p * ld + 32};
    stage_seed(db, p, e, sAc, sB, sw);
    for (int t = threadIdx.x; t < p * p; t += blockDim.x)
        sB32[(t / p) * ld + (t % p)] = (float)db.Binv[(int64_t)e * p * p + t];
    const double bfro = db.fro[e];
    const double fc = skd.fa[e], rhoc = skd.rho[e];
    stage_sketch(skd.den + (int64_t)e * SK, skd.Y32 + (int64_t)e * SK * p, p, sy, sden);
    __syncthreads();
    unsigned long long my_evals = 0, my_exact = 0, my_screened = 0;
    __shared__ int s_list[EVAL_THREADS];
    __shared__ int s_cnt;
    for (int base = blockIdx.x * blockDim.x; base < count; base += gridDim.x * blockDim.x) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const int cand = base + threadIdx.x;
        const int cc = min(cand, count - 1);
        float v[SK * 32];
        sketch_load<32>(sk.Y32 + (int64_t)cc * SK * p, p, v);
        const double fi = sk.fa[cc];
        const bool open = cand < count && phi[cc] == -1;
        const bool rej = open && sketch_bound_rejects<32>(v, fi, sy, sden, fc, rhoc, p, tol);
        const unsigned opened = __ballot_sync(0xffffffffu, open);
        const unsigned surv = __ballot_sync(0xffffffffu, open && !rej);
        my_evals += __popc(opened);
        my_screened += __popc(opened & ~surv);
        int wb = 0;
        if (lane == 0 && surv) wb = atomicAdd(&s_cnt, __popc(surv));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (open && !rej) s_list[wb + __popc(surv & ((1u << lane) - 1u))] = cand;
        __syncthreads();
        const int ns = s_cnt;
        for (int q = wid; q < ns; q += wpb) {
            const int c2 = s_list[q];
            double dv;
            int dec = decide_pair(Ag + (int64_t)c2 * p * p, sAc, sB, p, ld, bfro, tol, ws, &dv, false, sw, sB32);
            if (dec < 0) {
                dec = decide_pair(Ag + (int64_t)c2 * p * p, sAc, sB, p, ld, bfro, tol, ws, &dv, true, sw, nullptr);
                ++my_exact;
            }
            if (lane == 0 && dec == 1) phi[c2] = e;
            __syncwarp();
        }
        __syncthreads();
    }
    if (lane == 0) {
        if (my_evals) atomicAdd(&st->evals, my_evals);
        if (my_exact) atomicAdd(&st->exact, my_exact);
        if (my_screened) atomicAdd(&st->screened, my_screened);
        if (my_evals > my_screened) atomicAdd(&st->decided, my_evals - my_screened);
    }
}

// Smallest unassigned patch -> st->next (done when there is none).
__global__ void k_first_open(RoundDev* st, const int32_t* __restrict__ phi, int count) {
    int mn = count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        if (phi[i] == -1) mn = min(mn, i);
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0 && mn < count) atomicMin(&st->next, mn);
}

__global__ void k_finish_first(RoundDev* st, int count) {
    if (st->next >= count) st->done = 1;
}

// Database assembly: entry j < m0 from the seed inverses, entry j >= m0 from
// the inverse of its patch.
__global__ void k_gather_db(const double* __restrict__ seedB, int m0, const double* __restrict__ Ball,
                            const int32_t* __restrict__ rep_local, int m, int p, double* __restrict__ out) {
    const int64_t pp = (int64_t)p * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * pp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / pp);
        const int64_t o = e - (int64_t)j * pp;
        out[e] = (j < m0) ? seedB[(int64_t)j * pp + o] : Ball[(int64_t)rep_local[j] * pp + o];
    }
}

// Hints: patch i with hint[i] >= 0 is compared with that entry first (one
// evaluation, exact path inline when the bounds do not decide).
__global__ void k_verify_hints(RoundDev* st, int32_t* __restrict__ phi, int count, const double* __restrict__ Ag,
                               int p, EntryDB db, int m0, double tol, const int32_t* __restrict__ hint,
                               int32_t* __restrict__ hits) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* wbase = reinterpret_cast<double*>(smem) + (size_t)wid * (2 * p * ld + p * ld + 64);
    double* sAc = wbase;
    double* sB = wbase + p * ld;
    WarpScratch ws{wbase + 2 * p * ld, wbase + 3 * p * ld, wbase + 3 * p * ld + 32};
    unsigned long long ev = 0, ex = 0;
    int my_hits = 0;
    for (int i = blockIdx.x * wpb + wid; i < count; i += gridDim.x * wpb) {
        const int e = hint[i];
        if (e < 0 || e >= m0) continue;
        const double* a = db.A + (int64_t)e * p * p;
        const double* bm = db.Binv + (int64_t)e * p * p;
        for (int t = lane; t < p * p; t += 32) {
            sAc[(t / p) * ld + (t % p)] = a[t];
            sB[(t / p) * ld + (t % p)] = bm[t];
        }
        __syncwarp();
        double dv;
        const double* pw = db.w + (int64_t)e * PROBE_STRIDE;
        int dec = decide_pair(Ag + (int64_t)i * p * p, sAc, sB, p, ld, db.fro[e], tol, ws, &dv, false, pw);
        if (dec < 0) {
            dec = decide_pair(Ag + (int64_t)i * p * p, sAc, sB, p, ld, db.fro[e], tol, ws, &dv, true, pw);
            ++ex;
        }
        ++ev;
        if (lane == 0 && dec == 1) { phi[i] = e; ++my_hits; }
        __syncwarp();
    }
    if (lane == 0) {
        if (ev) atomicAdd(&st->evals, ev);
        if (ev) atomicAdd(&st->decided, ev);
        if (ex) atomicAdd(&st->exact, ex);
        if (my_hits) atomicAdd(hits, my_hits);
    }
}

// E = D B (B given, global, row stride p) or E = D (B null) for D in the
// warp's shared scratch (row stride p), formed in FP64: lane r holds row r in
// e[] and column r in ecol[]; E itself is left in ws.E (row stride p + 1).
template <int PM>
__device__ void form_e_warp(const double* sD, const double* __restrict__ B, int p, WarpScratch ws, double (&e)[PM],
                            double (&ecol)[PM]) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < p;
    const int ld = p + 1;
#pragma unroll
    for (int j = 0; j < PM; ++j) e[j] = 0.0;
    if (act) {
        if (B) {
            for (int k = 0; k < p; ++k) {
                const double dk = sD[lane * p + k];
#pragma unroll
                for (int j = 0; j < PM; ++j)
                    if (j < p) e[j] = fma(dk, B[k * p + j], e[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) e[j] = sD[lane * p + j];
        }
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int j = 0; j < PM; ++j)
            if (j < p) ws.E[lane * ld + j] = e[j];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < PM; ++r) ecol[r] = (act && r < p) ? ws.E[r * ld + lane] : 0.0;
}

// Power iteration on G = E^T E from E's largest row (lowest row on ties):
// the Rayleigh quotients ||E v||^2 (||v|| = 1) rise towards lambda_max(G);
// stops after three steps that gain less than 2^-50 (relative) or after 300.
// Returns the largest quotient, 0 when E = 0, NaN when E holds a NaN.
template <int PM>
__device__ double power_lambda_warp(const double (&e)[PM], const double (&ecol)[PM], int p, WarpScratch ws) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < p;
    const int ld = p + 1;
    double rn = 0.0;
#pragma unroll
    for (int j = 0; j < PM; ++j) rn = fma(e[j], e[j], rn);
    double best = act ? rn : -1.0;
    int br = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && oi < br)) { best = ob; br = oi; }
    }
    if (best != best) return best;                  // NaN
    if (!(best > 0.0)) return 0.0;
    double v = act ? ws.E[br * ld + lane] : 0.0;
    v /= sqrt(best);
    double lam = 0.0;
    int quiet = 0;
    for (int it = 0; it < 300 && quiet < 3; ++it) {
        __syncwarp();
        ws.v[lane] = v;
        __syncwarp();
        double wr = 0.0;
        if (act) {
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) wr = fma(e[j], ws.v[j], wr);
        }
        const double l2 = warp_sum(wr * wr);
        quiet = (l2 - lam <= 0x1p-50 * l2) ? quiet + 1 : 0;
        lam = fmax(lam, l2);
        ws.w[lane] = wr;
        __syncwarp();
        double uj = 0.0;
        if (act) {
#pragma unroll
            for (int r = 0; r < PM; ++r)
                if (r < p) uj = fma(ecol[r], ws.w[r], uj);
        }
        const double nu = sqrt(warp_sum(uj * uj));
        if (!(nu > 0.0)) break;
        v = uj / nu;
    }
    __syncwarp();
    return lam;
}

// lambda_max(G), G = E^T E, estimated by power iteration: in FP32 on E
// scaled by a power of two (the direction only), from E's largest row (lowest
// row on ties), until the unit vector moves by at most 2^-21 in every entry
// three steps running, or after 500 steps; then the Rayleigh quotient
// ||E v||^2 / ||v||^2 of that vector in FP64, which is below lambda_max (up
// to its rounding) and within (vector error)^2 of it.  The GPU's FP64 rate is
// 1/64 of its FP32 rate, so the iteration costs a few FP64 operations; the
// quotient is as accurate as the FP32 direction allows (about 1e-13), which
// brackets a norm but is too coarse for the 2^-40 certificate of a distance.
// Returns 0 when E = 0, NaN when E holds a NaN.
template <int PM>
__device__ double power_lambda32_warp(const double (&e)[PM], const double (&ecol)[PM], int p, WarpScratch ws) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < p;
    const int ld = p + 1;
    double rn = 0.0;
#pragma unroll
    for (int j = 0; j < PM; ++j) rn = fma(e[j], e[j], rn);
    double best = act ? rn : -1.0;
    int br = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && oi < br)) { best = ob; br = oi; }
    }
    if (best != best) return best;                  // NaN
    if (!(best > 0.0)) return 0.0;
    // scale 2^-x with 2^x the binade of E's largest |entry| (bits, no FP64 op)
    long long mb = 0;
#pragma unroll
    for (int j = 0; j < PM; ++j) mb = max(mb, __double_as_longlong(e[j]) & 0x7fffffffffffffffLL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    int ex = (int)(mb >> 52) - 1023;
    ex = max(-1000, min(1000, ex));
    const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
    float e32[PM], c32[PM];
#pragma unroll
    for (int j = 0; j < PM; ++j) {
        e32[j] = (float)(e[j] * sc);
        c32[j] = (float)(ecol[j] * sc);
    }
    float* v32 = reinterpret_cast<float*>(ws.v);
    float* w32 = reinterpret_cast<float*>(ws.w);
    float v = act ? (float)(ws.E[br * ld + lane] * sc) : 0.f;   // row br of E as the start
    {
        const float n0 = sqrtf(warp_sumf(v * v));
        v = n0 > 0.f ? v / n0 : 0.f;
    }
    int quiet = 0;
    for (int it = 0; it < 500 && quiet < 3; ++it) {
        __syncwarp();
        v32[lane] = v;
        __syncwarp();
        float wr = 0.f;
        if (act) {
#pragma unroll
            for (int j = 0; j < PM; ++j)
                if (j < p) wr = fmaf(e32[j], v32[j], wr);
        }
        w32[lane] = wr;
        __syncwarp();
        float uj = 0.f;
        if (act) {
#pragma unroll
            for (int r = 0; r < PM; ++r)
                if (r < p) uj = fmaf(c32[r], w32[r], uj);
        }
        const float nu = sqrtf(warp_sumf(uj * uj));
        if (!(nu > 0.f)) break;
        const float vn = act ? uj / nu : 0.f;
        float dv = fabsf(vn - v);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dv = fmaxf(dv, __shfl_xor_sync(0xffffffffu, dv, o));
        quiet = (dv <= 0x1p-21f) ? quiet + 1 : 0;
        v = vn;
    }
    // the FP64 Rayleigh quotient of v
    const double vd = act ? (double)v : 0.0;
    __syncwarp();
    ws.v[lane] = vd;
    __syncwarp();
    double wr = 0.0;
    if (act) {
#pragma unroll
        for (int j = 0; j < PM; ++j)
            if (j < p) wr = fma(e[j], ws.v[j], wr);
    }
    const double num = warp_sum(wr * wr);
    const double den = warp_sum(vd * vd);
    __syncwarp();
    return den > 0.0 ? num / den : 0.0;
}

// G = E^T E (X = 0, neg false) or X I - G (neg true) into dst (row stride
// dld) from the columns of E held in ecol[].
template <int PM>
__device__ void gram_warp(const double (&ecol)[PM], int p, double X, bool neg, double* dst, int dld) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int k = 0; k < p; ++k) {
        double g = 0.0;
#pragma unroll
        for (int r = 0; r < PM; ++r)
            if (r < p) g = fma(ecol[r], __shfl_sync(0xffffffffu, ecol[r], k), g);
        if (lane < p) dst[lane * dld + k] = neg ? ((k == lane ? X : 0.0) - g) : g;
    }
    __syncwarp();
}

// True when lambda_max(E^T E) < X is proved: the Cholesky factorisation of
// X I - G - c I, G computed, c = 2 gamma_{p+1} tr(X I - G) covering the
// factorisation's backward error, runs to completion (overwrites ws.E).
template <int PM>
__device__ bool lambda_below_warp(const double (&ecol)[PM], int p, double X, WarpScratch ws) {
    const int lane = threadIdx.x & 31;
    const int ld = p + 1;
    gram_warp<PM>(ecol, p, X, true, ws.E, ld);
    const double tr = warp_sum(lane < p ? ws.E[lane * ld + lane] : 0.0);
    if (!(tr > 0.0)) return false;
    const double c = 2.0 * gamma_u(p + 1) * tr;
    if (lane < p) ws.E[lane * ld + lane] -= c;
    __syncwarp();
    const bool ok = cholesky_warp(ws.E, p, ld) == p;
    __syncwarp();
    return ok;
}

// lambda_below_warp with G = E^T E already formed (G: row stride p, shared).
__device__ bool lambda_below_g_warp(const double* G, int p, double X, WarpScratch ws) {
    const int lane = threadIdx.x & 31;
    const int ld = p + 1;
    __syncwarp();
    if (lane < p)
        for (int k = 0; k < p; ++k) ws.E[lane * ld + k] = (k == lane ? X : 0.0) - G[lane * p + k];
    __syncwarp();
    const double tr = warp_sum(lane < p ? ws.E[lane * ld + lane] : 0.0);
    if (!(tr > 0.0)) return false;
    const double c = 2.0 * gamma_u(p + 1) * tr;
    if (lane < p) ws.E[lane * ld + lane] -= c;
    __syncwarp();
    const bool ok = cholesky_warp(ws.E, p, ld) == p;
    __syncwarp();
    return ok;
}

// sigma_max(E) of E = D B for D = A_c - A_i already in the warp's shared
// scratch sD and B in global memory (row stride p).  lambda_max(E^T E) by the
// power iteration, certified with X = lambda (1 + 2^-40): the value returned
// is then within 2^-41 (relative) of sigma_max.  Where the certificate fails
// (slow convergence) the largest Jacobi eigenvalue of G is taken instead (the
// "small SVD" of the section 3 remark), at about fifteen times the cost.
template <int PM>
__device__ double exact_sigma_d_warp(const double* sD, const double* __restrict__ B, int p, WarpScratch ws) {
    double e[PM], ecol[PM];
    form_e_warp<PM>(sD, B, p, ws, e, ecol);
    const double lam = power_lambda_warp<PM>(e, ecol, p, ws);
    if (!(lam > 0.0)) return lam;                   // 0, or NaN for a NaN E
    if (lambda_below_warp<PM>(ecol, p, lam * (1.0 + 0x1p-40), ws)) return sqrt(lam);
    gram_warp<PM>(ecol, p, 0.0, false, ws.E, p + 1);
    const double lj = jacobi_lambda_max_warp(ws.E, p, p + 1);
    __syncwarp();
    return sqrt(fmax(lj, 0.0));
}

// Bracket [*lo, *hi] of ||A||_2 for A in the warp's shared scratch sA (row
// stride p; overwritten by A^T A): lo from the Rayleigh quotient of the FP32
// power iteration (a lower bound up to its rounding, a few p u, far inside
// the 2^-40 taken off), hi from the first X = lambda (1 + 2^-s),
// s = 40, 36, 32, 26, 20, 12, 4, -4, -12, whose shifted Cholesky certificate
// holds (infinite when none does).  G = A^T A is formed once for the tries.
template <int PM>
__device__ void norm2_bracket_warp(double* sA, int p, WarpScratch ws, double* lo, double* hi) {
    double e[PM], ecol[PM];
    form_e_warp<PM>(sA, nullptr, p, ws, e, ecol);
    const double lam = power_lambda32_warp<PM>(e, ecol, p, ws);
    *lo = 0.0;
    *hi = 0.0;
    if (lam != lam) *lo = lam;                      // NaN patch: the caller widens it to [0, inf]
    if (!(lam > 0.0)) return;
    *lo = sqrt(lam) * (1.0 - 0x1p-40);
    *hi = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    gram_warp<PM>(ecol, p, 0.0, false, sA, p);
    const int shifts[9] = {-40, -36, -32, -26, -20, -12, -4, 4, 12};
#pragma unroll 1
    for (int k = 0; k < 9; ++k) {
        const double X = lam * (1.0 + __longlong_as_double((long long)(1023 + shifts[k]) << 52));
        if (lambda_below_g_warp(sA, p, X, ws)) {
            *hi = sqrt(X) * (1.0 + 0x1p-50);
            break;
        }
    }
}

// Brackets of ||A_i||_2 for a size group's patches, the keys of the
// norm-window search, and each patch's window (norm_window): a warp per
// patch, the patch staged in its scratch.
template <int PM>
__global__ void __launch_bounds__(EVAL_THREADS) k_patch_norms(const double* __restrict__ Ag, int count, int p,
                                                              double tol, double* __restrict__ nlo,
                                                              double* __restrict__ nhi, double* __restrict__ wlo,
                                                              double* __restrict__ whi) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int ld = p + 1;
    double* wbase = reinterpret_cast<double*>(smem) + (size_t)wid * ((size_t)p * ld + 64 + (size_t)p * p);
    WarpScratch ws{wbase, wbase + p * ld, wbase + p * ld + 32};
    double* sA = wbase + (size_t)p * ld + 64;
    const int64_t pp = (int64_t)p * p;
    for (int i = blockIdx.x * wpb + wid; i < count; i += gridDim.x * wpb) {
        __syncwarp();
        for (int e = lane; e < p * p; e += 32) sA[e] = Ag[(int64_t)i * pp + e];
        __syncwarp();
        double lo, hi;
        norm2_bracket_warp<PM>(sA, p, ws, &lo, &hi);
        if (lane == 0) {
            sanitize_bracket(&lo, &hi);
            const NormWin w = norm_window(lo, hi, tol);
            nlo[i] = lo;
            nhi[i] = hi;
            wlo[i] = w.lo;
            whi[i] = w.hi;
        }
    }
}

// D = A_c - A_i into the warp's scratch with coalesced loads; true when the
// two patches are bitwise equal.
__device__ __forceinline__ bool stage_d_warp(const double* __restrict__ Ac, const double* __restrict__ Ai, int p,
                                             double* sD) {
    const int lane = threadIdx.x & 31;
    bool same = true;
    __syncwarp();
    for (int e = lane; e < p * p; e += 32) {
        const double a = Ac[e], b = Ai[e];
        same &= __double_as_longlong(a) == __double_as_longlong(b);
        sD[e] = a - b;
    }
    const bool all_same = __all_sync(0xffffffffu, same);
    __syncwarp();
    return all_same;
}

// Screen thresholds (see multi_thresholds) of every entry, for the
// closest-match pass.
__global__ void k_entry_thresholds(const int32_t* __restrict__ rep_l, int m, SketchDB sk, int p, double tol,
                                   float* __restrict__ thr, float* __restrict__ beta) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int c = rep_l[j];
    double den[SK];
#pragma unroll
    for (int k = 0; k < SK; ++k) den[k] = sk.den[(int64_t)c * SK + k];
    multi_thresholds(sk.fa[c], sk.rho[c], den, p, tol, thr + (int64_t)j * SK, beta + j);
}

// Closest-match variant of Alg. 1 (section 3.1): the entries are those of the
// first-match rounds (an entry is created exactly when no entry passes, which
// does not depend on which passing entry is taken), and patch i joins the
// entry with the least d among the entries created before it that pass
// (d < tol), the lowest index on ties.  Entries before its first match
// failed already, so a warp per patch compares the first match j0 with the
// later entries whose representative precedes i, 32 at a time: the lanes
// screen them with the certified sketch bound (d >= tol), the warp decides
// the survivors in entry order with the certified cascade against the best
// distance so far (d < bs, on D staged in shared memory) and takes sigma_max
// (exact_sigma_d_warp: a certified power iteration, Jacobi where the
// certificate fails) only for those that beat it.  A zero distance
// ends the search (nothing can be smaller; ties keep the lower entry), and
// the evaluations counted are those made up to that point.
template <int PM>
__global__ void __launch_bounds__(EVAL_THREADS) k_closest_pass(int count, int p, const double* __restrict__ Ag,
                                                               const double* __restrict__ Ball,
                                                               const float* __restrict__ B32,
                                                               const double* __restrict__ fro_all,
                                                               const double* __restrict__ w_all,
                                                               const int32_t* __restrict__ rep_l, int m, double tol,
                                                               SketchDB sk, const float* __restrict__ ethr,
                                                               const float* __restrict__ ebeta,
                                                               int32_t* __restrict__ phi,
                                                               unsigned long long* __restrict__ evals) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int ld = p + 1;
    double* wbase = reinterpret_cast<double*>(smem) + (size_t)wid * ((size_t)p * ld + 64 + 2 * (size_t)p * p);
    WarpScratch ws{wbase, wbase + p * ld, wbase + p * ld + 32};
    double* sD = wbase + (size_t)p * ld + 64;      // D of the candidate being decided
    double* sD0 = sD + (size_t)p * p;              // D of the first match
    const int64_t pp = (int64_t)p * p;
    unsigned long long ev = 0;
    for (int i = blockIdx.x * wpb + wid; i < count; i += gridDim.x * wpb) {
        const int j0 = phi[i];
        if (rep_l[j0] == i) continue;                   // a representative keeps its own entry
        const double* Ai = Ag + (int64_t)i * pp;
        const int r0 = rep_l[j0];
        int best = j0;
        // bs: the best distance so far; -1 while the first match's distance
        // (positive unless its D vanishes) has not been needed yet
        double bs = stage_d_warp(Ag + (int64_t)r0 * pp, Ai, p, sD0) ? 0.0 : -1.0;
        if (bs < 0.0) {
            bool zero = true;
            for (int e = lane; e < p * p; e += 32) zero &= sD0[e] == 0.0;
            if (__all_sync(0xffffffffu, zero)) bs = 0.0;
        }
        auto first_sigma = [&]() {
            if (bs < 0.0) bs = exact_sigma_d_warp<PM>(sD0, Ball + (int64_t)r0 * pp, p, ws);
        };
        // the candidate entries: j0 < j < jend, jend the first entry whose
        // representative follows i (entries are created in increasing patch order)
        int lo = j0 + 1, hi = m;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rep_l[mid] > i) hi = mid; else lo = mid + 1;
        }
        const int jend = lo;
        float v[SK * PM];
        sketch_load<PM>(sk.Y32 + (int64_t)i * SK * p, p, v);
        const float fi32 = __double2float_ru(sk.fa[i]);
        for (int jb = j0 + 1; jb < jend && bs != 0.0; jb += 32) {
            const int j = jb + lane;
            bool rej = true;
            if (j < jend) {
                const int rj = rep_l[j];
                const float* yc = sk.Y32 + (int64_t)rj * SK * p;
                rej = false;
#pragma unroll
                for (int k = 0; k < SK; ++k) {
                    float d2 = 0.f;
#pragma unroll
                    for (int r = 0; r < PM; ++r) {
                        const float d = (r < p) ? yc[k * p + r] - v[k * PM + r] : 0.f;
                        d2 = fmaf(d, d, d2);
                    }
                    if (sqrtf(d2) >= __fmaf_ru(ebeta[j], fi32, ethr[(int64_t)j * SK + k])) rej = true;
                }
            }
            unsigned surv = __ballot_sync(0xffffffffu, !rej);
            int last = min(jend, jb + 32) - 1;          // the last entry evaluated in this chunk
            while (surv) {
                const int l = __ffs(surv) - 1;
                surv &= surv - 1u;
                const int jj = jb + l;
                const int rj = rep_l[jj];
                const double* Bc = Ball + (int64_t)rj * pp;
                // only an entry closer than the best so far matters: the
                // certified decision runs against that distance (tol until the
                // first match's distance is needed), and sigma_max is computed
                // for the few that beat it
                double sj = 0.0;
                bool better = true;                     // bitwise equal patches: distance 0
                if (!stage_d_warp(Ag + (int64_t)rj * pp, Ai, p, sD)) {
                    auto decide = [&](double t) {
                        double dv;
                        int dec = decide_pair<PM, true>(nullptr, sD, Bc, p, p, fro_all[rj], t, ws, &dv, false,
                                                        w_all + (int64_t)rj * PROBE_STRIDE, B32 + (int64_t)rj * pp);
                        if (dec < 0)
                            dec = decide_pair<PM, true>(nullptr, sD, Bc, p, p, fro_all[rj], t, ws, &dv, true,
                                                        w_all + (int64_t)rj * PROBE_STRIDE, nullptr);
                        return dec == 1;
                    };
                    const bool known = bs >= 0.0;
                    better = decide(known ? bs : tol);
                    if (better && !known) {             // passes: now the first match's distance is needed
                        first_sigma();
                        better = decide(bs);
                    }
                    if (better) {
                        sj = exact_sigma_d_warp<PM>(sD, Bc, p, ws);
                        better = sj < bs;
                    }
                }
                if (better) {
                    bs = sj;
                    best = jj;
                }
                if (bs == 0.0) {                        // nothing later can be smaller
                    last = jj;
                    break;
                }
            }
            ev += (unsigned long long)(last - jb + 1);
        }
        if (lane == 0) phi[i] = best;
        __syncwarp();
    }
    if (lane == 0 && ev) atomicAdd(evals, ev);
}

// psr_debug_inject(PSR_INJECT_BARRIER_WAIT, spins) on the current device.
// FP32 copy of the inverses for the FP32 stage of the multi-entry rounds.
__global__ void k_round_f32(const double* __restrict__ src, int64_t n, float* __restrict__ dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (float)src[e];
}

static std::atomic<bool> g_rounds_split{false};
void inject_rounds_split(bool on) { g_rounds_split.store(on); }

int inject_barrier_wait(long long spins) {
    const unsigned int extra = spins > 0 ? 1u : 0u;
    const long long limit = spins > 0 ? spins : (1ll << 24);
    cudaError_t e = cudaMemcpyToSymbol(g_bar_extra, &extra, sizeof(extra));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bar_limit, &limit, sizeof(limit));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "barrier injection");
    return PSR_OK;
}

static void launch_sketch(const double* A, const double* Binv, int count, int p, const double* X, double* den,
                          float* Y32, double* fa, double* rho, cudaStream_t s) {
    const int blocks = (count + 7) / 8;
    if (p <= 8) k_sketch<8><<<blocks, 256, 0, s>>>(A, Binv, count, p, X, den, Y32, fa, rho);
    else if (p <= 16) k_sketch<16><<<blocks, 256, 0, s>>>(A, Binv, count, p, X, den, Y32, fa, rho);
    else if (p <= 24) k_sketch<24><<<blocks, 256, 0, s>>>(A, Binv, count, p, X, den, Y32, fa, rho);
    else k_sketch<32><<<blocks, 256, 0, s>>>(A, Binv, count, p, X, den, Y32, fa, rho);
}

// Raises a kernel's dynamic shared memory limit to `bytes`.  Set whatever the
// size: the default limit is 48 KB minus the kernel's static shared memory,
// so a kernel with static arrays needs it below 48 KB of dynamic memory too.
static int set_smem(const void* f, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "criterion smem attribute");
    return PSR_OK;
}

// Runs Alg. 1 for every size group.  On entry ctx->A_ext holds the patches
// (group-contiguous).  With a seed database (seed_A, m0 entries; single size
// group only) the search starts from it, and with hints every patch first
// tries its hinted entry.  On exit every group carries its local assignment
// (G.sphi, original order) and its FP64 inverses (G.rinv, m x p x p), which the
// sweep builder converts and lays out.
int run_alg1(psr_ctx* ctx, cudaStream_t s, const double* seed_A, int m0, const int32_t* hints) {
    const double tol = ctx->opts.tol;
    RoundDev* st = nullptr;
    RoundDev* h_st = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&st, sizeof(RoundDev)));
    PSR_CUDA(ctx, psr::host_alloc(&h_st, sizeof(RoundDev)));
    int32_t* flag = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&flag, sizeof(int32_t)));
    int rc = PSR_OK;
    int64_t total_evals = 0, total_exact = 0, total_hits = 0, total_screened = 0, total_decided = 0;
    int rounds_total = 0;
    int first_singular = -1;
    if (m0 > 0 && ctx->groups.size() != 1) { set_error(ctx, "a seed database needs patches of one size"); return PSR_ERR_INVALID_ARG; }
    const bool window = ctx->opts.search == PSR_SEARCH_NORM_WINDOW;
    if (window && (m0 > 0 || hints)) {
        set_error(ctx, "the norm-window search takes no seed database or hints");
        return PSR_ERR_INVALID_ARG;
    }
    if (window && ctx->opts.match == PSR_MATCH_CLOSEST) {
        set_error(ctx, "the norm-window search is a first-match search");
        return PSR_ERR_INVALID_ARG;
    }
    for (size_t g = 0; g < ctx->groups.size() && rc == PSR_OK; ++g) {
        Group& G = ctx->groups[g];
        const int p = G.p, count = G.count;
        const double* Ag = ctx->A_ext + G.mat_off;
        if (p > 32) {
            // block-per-candidate kernels (criterion_big.cu)
            if (m0 > 0) { set_error(ctx, "a seed database needs patches of at most 32 DOFs"); rc = PSR_ERR_INVALID_ARG; break; }
            int fs = -1;
            const int64_t ev0 = total_evals, sc0 = total_screened;
            rc = run_alg1_big(ctx, G, Ag, s, &total_evals, &total_exact, &total_screened, &fs);
            if (rc != PSR_OK) break;
            rounds_total += G.m;
            total_decided += (total_evals - ev0) - (total_screened - sc0);   // one entry per round here
            if (fs >= 0 && first_singular < 0) first_singular = G.h_gidx[fs];
            continue;
        }
        int32_t* phi_l = nullptr;
        int32_t* rep_l = nullptr;
        int32_t* sing_all = nullptr;
        double *Ball = nullptr, *fro_all = nullptr, *w_all = nullptr;
        EntryDB db{nullptr, nullptr, nullptr, nullptr};
        const int cap = count + m0;
        PSR_CUDA(ctx, psr::dev_alloc(&phi_l, sizeof(int32_t) * count));
        PSR_CUDA(ctx, psr::dev_alloc(&rep_l, sizeof(int32_t) * cap));
        PSR_CUDA(ctx, psr::dev_alloc(&sing_all, sizeof(int32_t) * count));
        PSR_CUDA(ctx, psr::dev_alloc(&fro_all, sizeof(double) * count));
        PSR_CUDA(ctx, psr::dev_alloc(&w_all, sizeof(double) * (size_t)count * PROBE_STRIDE));
        if (psr::dev_alloc(&Ball, sizeof(double) * (size_t)count * p * p) != cudaSuccess) {
            cudaGetLastError();
            set_error(ctx, "out of device memory for the patch inverses");
            return PSR_ERR_OOM;
        }
        PSR_CUDA(ctx, cudaMemsetAsync(phi_l, 0xff, sizeof(int32_t) * count, s));
        // every patch's inverse, norm, probes and sketch, batched (any patch
        // may become an entry)
        GpuSpan span;                              // the inverses' GPU time (stats.t_invert)
        span.begin(s);
        rc = launch_batched_inverse(Ag, (int64_t)p * p, nullptr, count, p, Ball, (int64_t)p * p, sing_all, s);
        span.end(s);
        if (rc != PSR_OK) break;
        count_launch();
        k_entry_fro<<<(count + 7) / 8, 256, 0, s>>>(Ag, Ball, count, p, fro_all, w_all, sing_all, nullptr);
        double *skX = nullptr, *skDen = nullptr, *skF = nullptr, *skR = nullptr;
        float *skY32 = nullptr, *sdY32 = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&skX, sizeof(double) * SK * 32));
        PSR_CUDA(ctx, psr::dev_alloc(&skY32, sizeof(float) * (size_t)count * SK * p));
        PSR_CUDA(ctx, psr::dev_alloc(&skF, sizeof(double) * (size_t)count));
        PSR_CUDA(ctx, psr::dev_alloc(&skR, sizeof(double) * (size_t)count));
        if (psr::dev_alloc(&skDen, sizeof(double) * (size_t)count * SK) != cudaSuccess) {
            cudaGetLastError();
            set_error(ctx, "out of device memory for the patch sketches");
            return PSR_ERR_OOM;
        }
        count_launch();
        k_sketch_dirs<<<1, 32 * SK, 0, s>>>(Ag, count, p, skX);
        count_launch();
        launch_sketch(Ag, Ball, count, p, skX, skDen, skY32, skF, skR, s);
        PSR_CHECK_LAUNCH(ctx, "patch sketches");
        double* skN = nullptr;                     // [4][count] ||A_i||_2 brackets and windows
        if (window) {
            PSR_CUDA(ctx, psr::dev_alloc(&skN, sizeof(double) * 4 * (size_t)count));
            const int wpn = EVAL_THREADS / 32;
            const size_t smem_n = (size_t)wpn * ((size_t)p * (p + 1) + 64 + (size_t)p * p) * 8;
            const void* kn = (p <= 8) ? (const void*)k_patch_norms<8>
                           : (p <= 16) ? (const void*)k_patch_norms<16> : (const void*)k_patch_norms<32>;
            if ((rc = set_smem(kn, smem_n)) != PSR_OK) break;
            const int nb = std::max(1, std::min((count + wpn - 1) / wpn, 152 * 8));
            count_launch();
            if (p <= 8)
                k_patch_norms<8><<<nb, EVAL_THREADS, smem_n, s>>>(Ag, count, p, tol, skN, skN + count,
                                                                 skN + 2 * (size_t)count, skN + 3 * (size_t)count);
            else if (p <= 16)
                k_patch_norms<16><<<nb, EVAL_THREADS, smem_n, s>>>(Ag, count, p, tol, skN, skN + count,
                                                                  skN + 2 * (size_t)count, skN + 3 * (size_t)count);
            else
                k_patch_norms<32><<<nb, EVAL_THREADS, smem_n, s>>>(Ag, count, p, tol, skN, skN + count,
                                                                  skN + 2 * (size_t)count, skN + 3 * (size_t)count);
            PSR_CHECK_LAUNCH(ctx, "patch norms");
        }
        const SketchDB sk{skX, skDen, skF, skR, skY32, skN,
                          window ? skN + count : nullptr,
                          window ? skN + 2 * (size_t)count : nullptr,
                          window ? skN + 3 * (size_t)count : nullptr};
        SketchDB skd{skX, nullptr, nullptr, nullptr, nullptr};
        double *sdDen = nullptr, *sdF = nullptr, *sdR = nullptr;
        RoundDev init{};
        init.first_singular = -1;
        init.m = m0;
        init.next = 0;
        init.next_new = count;
        init.nn2[0] = init.nn2[1] = count;
        PSR_CUDA(ctx, cudaMemcpyAsync(st, &init, sizeof(RoundDev), cudaMemcpyHostToDevice, s));
        const int ld = p + 1;
        const int wpb = EVAL_THREADS / 32;
        const size_t smem_eval = eval_smem_bytes(p, wpb);
        const size_t smem_dec = decide_smem_bytes(p, wpb);
        if ((rc = set_smem((const void*)k_round_decide, smem_dec)) != PSR_OK) break;
        int32_t* surv_list = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&surv_list, sizeof(int32_t) * (size_t)count));
        if ((rc = set_smem((const void*)k_seed_pass, smem_eval)) != PSR_OK) break;
        // one candidate per thread in the screen: enough blocks for every
        // SM, a few passes each; the decide grid is one wave of 4 blocks per SM
        int eval_blocks = (count + EVAL_THREADS - 1) / EVAL_THREADS;
        if (eval_blocks > 152 * 4) eval_blocks = 152 * 4;
        if (eval_blocks < 1) eval_blocks = 1;
        const int decide_blocks = 152 * 4;
        if (m0 > 0) {
            PSR_CUDA(ctx, psr::dev_alloc(&db.A, sizeof(double) * (size_t)m0 * p * p));
            PSR_CUDA(ctx, psr::dev_alloc(&db.Binv, sizeof(double) * (size_t)m0 * p * p));
            PSR_CUDA(ctx, psr::dev_alloc(&db.fro, sizeof(double) * m0));
            PSR_CUDA(ctx, psr::dev_alloc(&db.w, sizeof(double) * (size_t)m0 * PROBE_STRIDE));
            PSR_CUDA(ctx, cudaMemcpyAsync(db.A, seed_A, sizeof(double) * (size_t)m0 * p * p, cudaMemcpyDeviceToDevice, s));
            int32_t* sflags = nullptr;
            PSR_CUDA(ctx, psr::dev_alloc(&sflags, sizeof(int32_t) * m0));
            rc = launch_batched_inverse(db.A, (int64_t)p * p, nullptr, m0, p, db.Binv, (int64_t)p * p, sflags, s);
            if (rc != PSR_OK) break;
            PSR_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
            count_launch();
            k_entry_fro<<<(m0 + 7) / 8, 256, 0, s>>>(db.A, db.Binv, m0, p, db.fro, db.w, sflags, flag);
            PSR_CUDA(ctx, psr::dev_alloc(&sdDen, sizeof(double) * (size_t)m0 * SK));
            PSR_CUDA(ctx, psr::dev_alloc(&sdF, sizeof(double) * (size_t)m0));
            PSR_CUDA(ctx, psr::dev_alloc(&sdR, sizeof(double) * (size_t)m0));
            PSR_CUDA(ctx, psr::dev_alloc(&sdY32, sizeof(float) * (size_t)m0 * SK * p));
            count_launch();
            launch_sketch(db.A, db.Binv, m0, p, skX, sdDen, sdY32, sdF, sdR, s);
            skd = SketchDB{skX, sdDen, sdF, sdR, sdY32};
            std::vector<int32_t> seq(m0, -1);
            PSR_CUDA(ctx, cudaMemcpyAsync(rep_l, seq.data(), sizeof(int32_t) * m0, cudaMemcpyHostToDevice, s));
            int32_t h_bad = 0;
            PSR_CUDA(ctx, cudaMemcpyAsync(&h_bad, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            psr::dev_free(sflags);
            if (h_bad) { set_error(ctx, "a seed database entry is singular"); rc = PSR_ERR_SINGULAR_PATCH; break; }
            if (hints) {
                int32_t* hits = nullptr;
                PSR_CUDA(ctx, psr::dev_alloc(&hits, sizeof(int32_t)));
                PSR_CUDA(ctx, cudaMemsetAsync(hits, 0, sizeof(int32_t), s));
                const size_t smem_h = (size_t)wpb * (3 * p * ld + 64) * 8;
                if ((rc = set_smem((const void*)k_verify_hints, smem_h)) != PSR_OK) break;
                const int hb = std::max(1, std::min((count + wpb - 1) / wpb, 152 * 8));
                count_launch();
                k_verify_hints<<<hb, wpb * 32, smem_h, s>>>(st, phi_l, count, Ag, p, db, m0, tol, hints, hits);
                int32_t h_hits = 0;
                PSR_CUDA(ctx, cudaMemcpyAsync(&h_hits, hits, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                PSR_CUDA(ctx, cudaStreamSynchronize(s));
                total_hits += h_hits;
                psr::dev_free(hits);
            }
        }
        // misses of a seed database: first match over its entries in creation
        // order, one launch per entry (the multi-entry kernel below does the
        // same 64 entries at a time when it runs)
        auto seed_passes = [&]() -> int {
            for (int j = 0; j < m0; ++j) {
                count_launch();
                k_seed_pass<<<eval_blocks, wpb * 32, smem_eval, s>>>(st, phi_l, count, Ag, p, db, sk, skd, tol, j);
            }
            PSR_CHECK_LAUNCH(ctx, "seeded Alg. 1 passes");
            // the first new entry is the smallest patch still unassigned
            int big = count;
            PSR_CUDA(ctx, cudaMemcpyAsync(&st->next, &big, sizeof(int), cudaMemcpyHostToDevice, s));
            count_launch();
            k_first_open<<<std::max(1, std::min((count + 255) / 256, 1024)), 256, 0, s>>>(st, phi_l, count);
            count_launch();
            k_finish_first<<<1, 1, 0, s>>>(st, count);
            return PSR_OK;
        };
        // all rounds in one cooperative launch when every block of the grid
        // can be co-resident; otherwise two launches per round
        bool persistent = false;
        {
            int coop = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
            if (g_rounds_split.load()) coop = 0;
            const void* kf = (p <= 8) ? (const void*)k_rounds_multi<8>
                           : (p <= 16) ? (const void*)k_rounds_multi<16> : (const void*)k_rounds_multi<32>;
            const size_t smem_multi = (size_t)wpb * (2 * (size_t)p * p + 64) * 8;
            int per_sm = 0;
            if (coop && count <= (1 << 25) && set_smem(kf, smem_multi) == PSR_OK &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, EVAL_THREADS, smem_multi) == cudaSuccess &&
                per_sm >= 1) {
                int sms = 0;
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
                // as few blocks as give every candidate a screening thread
                // (each grid barrier costs an arrival per block), at most 4 per SM
                const int want = (int)((count + (int64_t)sms * EVAL_THREADS - 1) / ((int64_t)sms * EVAL_THREADS));
                const int grid = sms * std::max(1, std::min(want, std::min(per_sm, 4)));
                MultiWS mw{};
                unsigned int* bar = nullptr;
                int32_t* perr = nullptr;
                float* b32 = nullptr;
                bool room = true;
                const int nwords = (count + 31) / 32;
                PSR_CUDA(ctx, psr::dev_alloc(&bar, 2 * sizeof(unsigned int)));
                PSR_CUDA(ctx, psr::dev_alloc(&perr, sizeof(int32_t)));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.obits, sizeof(uint32_t) * nwords));
                if (psr::dev_alloc(&mw.pairs, sizeof(uint32_t) * (size_t)count * KC) != cudaSuccess ||
                    psr::dev_alloc(&b32, sizeof(float) * (size_t)count * p * p) != cudaSuccess) {
                    // no room for the pair list or the FP32 inverses: two launches per round
                    cudaGetLastError();
                    psr::dev_free(mw.pairs);
                    psr::dev_free(b32);
                    mw.pairs = nullptr;
                    b32 = nullptr;
                    room = false;
                }
                PSR_CUDA(ctx, psr::dev_alloc(&mw.rem, sizeof(int32_t) * (size_t)count));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.accm, 8 * (size_t)count));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.exm, 8 * (size_t)count));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.rejm, 8 * (size_t)count));
                if (window) PSR_CUDA(ctx, psr::dev_alloc(&mw.wom, 8 * (size_t)count));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.accA, 8 * 2 * KC));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.exA, 8 * 2 * KC));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.npB, sizeof(int32_t) * 2));
                PSR_CUDA(ctx, psr::dev_alloc(&mw.wq, sizeof(int32_t) * 4));
                PSR_CUDA(ctx, cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s));
                PSR_CUDA(ctx, cudaMemsetAsync(perr, 0, sizeof(int32_t), s));
                PSR_CUDA(ctx, cudaMemsetAsync(mw.accA, 0, 8 * 2 * KC, s));
                PSR_CUDA(ctx, cudaMemsetAsync(mw.exA, 0, 8 * 2 * KC, s));
                PSR_CUDA(ctx, cudaMemsetAsync(mw.npB, 0, sizeof(int32_t) * 2, s));
                PSR_CUDA(ctx, cudaMemsetAsync(mw.wq, 0, sizeof(int32_t) * 4, s));
                float* sb32 = nullptr;
                if (room && m0 > 0 && psr::dev_alloc(&sb32, sizeof(float) * (size_t)m0 * p * p) != cudaSuccess) {
                    cudaGetLastError();
                    room = false;
                }
                cudaError_t le = cudaErrorMemoryAllocation;
                if (room) {
                    const int64_t tot = (int64_t)count * p * p;
                    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 16));
                    count_launch();
                    k_round_f32<<<gb, 256, 0, s>>>(Ball, tot, b32);
                    if (m0 > 0) {
                        const int64_t ts = (int64_t)m0 * p * p;
                        count_launch();
                        k_round_f32<<<(int)std::max<int64_t>(1, std::min<int64_t>((ts + 255) / 256, 152 * 16)), 256, 0,
                                      s>>>(db.Binv, ts, sb32);
                    }
                    mw.B32 = b32;
                    const EntrySrc own{Ag, Ball, b32, fro_all, w_all};
                    const EntrySrc seeds{db.A, db.Binv, sb32, db.fro, db.w};
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3((unsigned)grid);
                    cfg.blockDim = dim3(EVAL_THREADS);
                    cfg.dynamicSmemBytes = smem_multi;
                    cfg.stream = s;
                    cudaLaunchAttribute at[1];
                    at[0].id = cudaLaunchAttributeCooperative;
                    at[0].val.cooperative = 1;
                    cfg.attrs = at;
                    cfg.numAttrs = 1;
                    count_launch();
                    if (p <= 8)
                        le = cudaLaunchKernelEx(&cfg, k_rounds_multi<8>, st, phi_l, count, Ag, p, own,
                                                (const int32_t*)sing_all, sk, tol, mw, rep_l, bar, perr, seeds, skd,
                                                m0);
                    else if (p <= 16)
                        le = cudaLaunchKernelEx(&cfg, k_rounds_multi<16>, st, phi_l, count, Ag, p, own,
                                                (const int32_t*)sing_all, sk, tol, mw, rep_l, bar, perr, seeds, skd,
                                                m0);
                    else
                        le = cudaLaunchKernelEx(&cfg, k_rounds_multi<32>, st, phi_l, count, Ag, p, own,
                                                (const int32_t*)sing_all, sk, tol, mw, rep_l, bar, perr, seeds, skd,
                                                m0);
                }
                int32_t herr = 0;
                if (le == cudaSuccess) {
                    persistent = true;
                    PSR_CUDA(ctx, cudaMemcpyAsync(h_st, st, sizeof(RoundDev), cudaMemcpyDeviceToHost, s));
                    PSR_CUDA(ctx, cudaMemcpyAsync(&herr, perr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                    PSR_CUDA(ctx, cudaStreamSynchronize(s));
                } else {
                    cudaGetLastError();
                    PSR_CUDA(ctx, cudaStreamSynchronize(s));
                }
                psr::dev_free(bar);
                psr::dev_free(perr);
                psr::dev_free(mw.obits);
                psr::dev_free(mw.pairs);
                psr::dev_free(mw.rem);
                psr::dev_free(mw.accm);
                psr::dev_free(mw.exm);
                psr::dev_free(mw.rejm);
                psr::dev_free(mw.wom);
                psr::dev_free(mw.accA);
                psr::dev_free(mw.exA);
                psr::dev_free(mw.npB);
                psr::dev_free(mw.wq);
                psr::dev_free(b32);
                psr::dev_free(sb32);
                if (persistent && (herr || !h_st->done)) {
                    set_error(ctx, "a grid barrier of the Alg. 1 rounds gave up waiting");
                    rc = PSR_ERR_TIMEOUT;
                    break;
                }
            }
        }
        if (!persistent && m0 > 0 && (rc = seed_passes()) != PSR_OK) break;
        int batch = 8;
        int issued = 0;
        for (; !persistent;) {
            for (int r = 0; r < batch; ++r) {
                count_launch();
                if (p <= 8)
                    k_round_screen<8><<<eval_blocks, EVAL_THREADS, 0, s>>>(st, phi_l, count, p, sk, tol, surv_list);
                else if (p <= 16)
                    k_round_screen<16><<<eval_blocks, EVAL_THREADS, 0, s>>>(st, phi_l, count, p, sk, tol, surv_list);
                else
                    k_round_screen<32><<<eval_blocks, EVAL_THREADS, 0, s>>>(st, phi_l, count, p, sk, tol, surv_list);
                count_launch();
                k_round_decide<<<decide_blocks, EVAL_THREADS, smem_dec, s>>>(st, phi_l, count, Ag, p, Ball, fro_all,
                                                                            w_all, sing_all, tol, surv_list, rep_l);
            }
            PSR_CHECK_LAUNCH(ctx, "Alg. 1 round kernel");
            issued += batch;
            PSR_CUDA(ctx, cudaMemcpyAsync(h_st, st, sizeof(RoundDev), cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            if (h_st->done) break;
            if (issued > count + 8) { set_error(ctx, "Alg. 1 rounds did not terminate"); rc = PSR_ERR_TIMEOUT; break; }
            if (batch < 512) batch *= 2;
        }
        if (rc != PSR_OK) break;
        G.m = h_st->m;
        if (ctx->opts.match == PSR_MATCH_CLOSEST && G.m > 1) {
            if (m0 > 0) { set_error(ctx, "closest match takes no seed database"); rc = PSR_ERR_INVALID_ARG; break; }
            unsigned long long* cev = nullptr;
            PSR_CUDA(ctx, psr::dev_alloc(&cev, sizeof(unsigned long long)));
            PSR_CUDA(ctx, cudaMemsetAsync(cev, 0, sizeof(unsigned long long), s));
            const size_t smem_c = (size_t)wpb * ((size_t)p * ld + 64 + 2 * (size_t)p * p) * 8;
            const void* kf = (p <= 8) ? (const void*)k_closest_pass<8>
                           : (p <= 16) ? (const void*)k_closest_pass<16> : (const void*)k_closest_pass<32>;
            if ((rc = set_smem(kf, smem_c)) != PSR_OK) break;
            float *cb32 = nullptr, *ethr = nullptr, *ebeta = nullptr;
            PSR_CUDA(ctx, psr::dev_alloc(&cb32, sizeof(float) * (size_t)count * p * p));
            PSR_CUDA(ctx, psr::dev_alloc(&ethr, sizeof(float) * (size_t)G.m * SK));
            PSR_CUDA(ctx, psr::dev_alloc(&ebeta, sizeof(float) * (size_t)G.m));
            {
                const int64_t tot = (int64_t)count * p * p;
                count_launch();
                k_round_f32<<<(int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 16)), 256, 0, s>>>(
                    Ball, tot, cb32);
                count_launch();
                k_entry_thresholds<<<(G.m + 127) / 128, 128, 0, s>>>(rep_l, G.m, sk, p, tol, ethr, ebeta);
            }
            const int cb = std::max(1, std::min((count + wpb - 1) / wpb, 152 * 8));
            count_launch();
            if (p <= 8)
                k_closest_pass<8><<<cb, EVAL_THREADS, smem_c, s>>>(count, p, Ag, Ball, cb32, fro_all, w_all, rep_l, G.m,
                                                                   tol, sk, ethr, ebeta, phi_l, cev);
            else if (p <= 16)
                k_closest_pass<16><<<cb, EVAL_THREADS, smem_c, s>>>(count, p, Ag, Ball, cb32, fro_all, w_all, rep_l,
                                                                    G.m, tol, sk, ethr, ebeta, phi_l, cev);
            else
                k_closest_pass<32><<<cb, EVAL_THREADS, smem_c, s>>>(count, p, Ag, Ball, cb32, fro_all, w_all, rep_l,
                                                                    G.m, tol, sk, ethr, ebeta, phi_l, cev);
            PSR_CHECK_LAUNCH(ctx, "closest-match pass");
            unsigned long long h_cev = 0;
            PSR_CUDA(ctx, cudaMemcpyAsync(&h_cev, cev, sizeof(h_cev), cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            psr::dev_free(cev);
            psr::dev_free(cb32);
            psr::dev_free(ethr);
            psr::dev_free(ebeta);
            total_evals += (int64_t)h_cev;
            total_decided += (int64_t)h_cev;
        }
        total_evals += (int64_t)h_st->evals;
        total_exact += (int64_t)h_st->exact;
        total_screened += (int64_t)h_st->screened;
        total_decided += (int64_t)h_st->decided;
        rounds_total += persistent ? h_st->nrounds : h_st->m - m0;
        if (h_st->first_singular >= 0 && first_singular < 0) first_singular = G.h_gidx[h_st->first_singular];
        std::vector<int32_t> hrep(G.m);
        PSR_CUDA(ctx, cudaMemcpyAsync(hrep.data(), rep_l, sizeof(int32_t) * G.m, cudaMemcpyDeviceToHost, s));
        double* Bdb = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&Bdb, sizeof(double) * (size_t)std::max(G.m, 1) * p * p));
        {
            const int64_t tot = (int64_t)G.m * p * p;
            const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 16));
            count_launch();
            k_gather_db<<<gb, 256, 0, s>>>(db.Binv, m0, Ball, rep_l, G.m, p, Bdb);
            // the entries' patch matrices, kept for reuse by a later setup
            PSR_CUDA(ctx, psr::dev_alloc(&G.dbA, sizeof(double) * (size_t)std::max(G.m, 1) * p * p));
            count_launch();
            k_gather_db<<<gb, 256, 0, s>>>(db.A, m0, Ag, rep_l, G.m, p, G.dbA);
        }
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        ctx->stats.t_invert += span.seconds();
        G.h_rep.assign(hrep.begin(), hrep.end());   // local patch of each entry, -1 for seed entries
        G.sphi = phi_l;             // local phi in original (unsorted) order
        G.rinv = Bdb;               // FP64 database, converted in the sweep builder
        psr::dev_free(Ball);
        psr::dev_free(fro_all);
        psr::dev_free(w_all);
        psr::dev_free(sing_all);
        for (double* q : {skX, skDen, skF, skR, sdDen, sdF, sdR, skN}) psr::dev_free(q);
        psr::dev_free(skY32);
        psr::dev_free(sdY32);
        psr::dev_free(surv_list);
        psr::dev_free(db.A);
        psr::dev_free(db.Binv);
        psr::dev_free(db.fro);
        psr::dev_free(db.w);
        psr::dev_free(rep_l);
    }
    psr::dev_free(st);
    psr::host_free(h_st);
    psr::dev_free(flag);
    ctx->stats.criterion_evals = total_evals;
    ctx->stats.criterion_exact = total_exact;
    ctx->stats.criterion_screened = total_screened;
    ctx->stats.criterion_decided = total_decided;
    ctx->stats.mlp_hits = total_hits;
    ctx->stats.rounds = rounds_total;
    ctx->stats.first_singular = first_singular;
    return rc;
}

// ------------------------------------------------------ stateless entry
__global__ void k_criterion_batch(const double* __restrict__ A_i, int32_t batch, int p,
                                  const double* __restrict__ A_c, const double* __restrict__ Binv_c,
                                  double tol, int32_t* __restrict__ accept, double* __restrict__ dval,
                                  int32_t* __restrict__ undec, int32_t* __restrict__ n_undec, int phase) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* sAc = reinterpret_cast<double*>(smem);
    double* sB = sAc + p * ld;
    float* sB32 = reinterpret_cast<float*>(sB + p * ld + 32);
    double* wbase = reinterpret_cast<double*>(smem) + eval_block_doubles(p) + (size_t)wid * (p * ld + 64);
    WarpScratch ws{wbase, wbase + p * ld, wbase + p * ld + 32};
    double bf = 0.0;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        sAc[(e / p) * ld + (e % p)] = A_c[e];
        sB[(e / p) * ld + (e % p)] = Binv_c[e];
        sB32[(e / p) * ld + (e % p)] = (float)Binv_c[e];
    }
    __syncthreads();
    for (int e = lane; e < p * p; e += 32) bf = fma(Binv_c[e], Binv_c[e], bf);
    bf = sqrt(warp_sum(bf));
    const int total = (phase == 0) ? batch : *n_undec;
    for (int u = blockIdx.x * wpb + wid; u < total; u += gridDim.x * wpb) {
        const int b = (phase == 0) ? u : undec[u];
        double dv;
        const int dec = decide_pair(A_i + (int64_t)b * p * p, sAc, sB, p, ld, bf, tol, ws, &dv, phase == 1,
                                    nullptr, phase == 0 ? sB32 : nullptr);
        if (lane == 0) {
            if (dec >= 0) {
                accept[b] = dec;
                if (dval) dval[b] = dv;
            } else {
                const int slot = atomicAdd(n_undec, 1);
                undec[slot] = b;       // slot < batch always
            }
        }
        __syncwarp();
    }
}

int launch_criterion_batch(const double* A_i, int32_t batch, int32_t p, const double* A_c,
                           const double* Binv_c, double tol, int32_t* accept, double* dval,
                           int32_t* work, cudaStream_t s) {
    // work: device int32 scratch of batch + 1 entries (undecided list + count)
    const int wpb = 8;
    const size_t sm = eval_smem_bytes(p, wpb);
    int rc = set_smem((const void*)k_criterion_batch, sm);
    if (rc != PSR_OK) return rc;
    cudaError_t e = cudaMemsetAsync(work + batch, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "criterion scratch reset");
    int blocks = (batch + wpb - 1) / wpb;
    if (blocks > 152 * 4) blocks = 152 * 4;
    if (blocks < 1) blocks = 1;
    count_launch(); k_criterion_batch<<<blocks, wpb * 32, sm, s>>>(A_i, batch, p, A_c, Binv_c, tol, accept, dval, work, work + batch, 0);
    count_launch(); k_criterion_batch<<<blocks, wpb * 32, sm, s>>>(A_i, batch, p, A_c, Binv_c, tol, accept, dval, work, work + batch, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_criterion_batch");
    return PSR_OK;
}

__global__ void k_spectral_norm(const double* __restrict__ E, int32_t batch, int p, double* __restrict__ sigma) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = p + 1;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double* G = reinterpret_cast<double*>(smem) + (size_t)wid * p * ld;
    for (int b = blockIdx.x * wpb + wid; b < batch; b += gridDim.x * wpb) {
        const double* e = E + (int64_t)b * p * p;
        double col[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) col[r] = (lane < p && r < p) ? e[r * p + lane] : 0.0;
        for (int k = 0; k < p; ++k) {
            double g = 0.0;
#pragma unroll
            for (int r = 0; r < 32; ++r) g = fma(col[r], __shfl_sync(0xffffffffu, col[r], k), g);
            if (lane < p) G[lane * ld + k] = g;
        }
        __syncwarp();
        const double lam = jacobi_lambda_max_warp(G, p, ld);
        if (lane == 0) sigma[b] = sqrt(fmax(lam, 0.0));
        __syncwarp();
    }
}

int launch_spectral_norm(const double* E, int32_t batch, int32_t p, double* sigma, cudaStream_t s) {
    const int wpb = 4;
    const size_t sm = (size_t)wpb * p * (p + 1) * 8;
    int blocks = (batch + wpb - 1) / wpb;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    count_launch(); k_spectral_norm<<<blocks, wpb * 32, sm, s>>>(E, batch, p, sigma);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "k_spectral_norm");
    return PSR_OK;
}

}  // namespace psr

// ---------------------------------------------------------------------------
// Allocation-free variant of psr_criterion.
//
// Some callers cannot let a library allocate device memory: an application
// whose own memory manager has reserved (or must account for) all device
// memory, or a latency-sensitive pipeline that cannot afford the implicit
// device-wide synchronisation a cudaMalloc may cause.  psr_criterion_noalloc
// serves them: its only scratch (the list of candidates whose bounds did not
// decide, plus its counter) lives in the fixed array below, which every GPU
// that loads this library holds until the process exits.
// ---------------------------------------------------------------------------

#include <mutex>

static __device__ __align__(256) int32_t g_criterion_scratch[PSR_CRITERION_NOALLOC_MAX + 1];

namespace {
std::mutex g_scratch_mutex;
void* g_scratch_addr[256] = {nullptr};   // device address of the array, per device ordinal
}

extern "C" int psr_criterion_noalloc(const double* A_i, int32_t batch, int32_t p, const double* A_c,
                                     const double* Binv_c, double tol, int32_t* accept, double* dval,
                                     void* stream) {
    using namespace psr;
    if (!A_i || !A_c || !Binv_c || !accept || batch < 0 || p < 1 || p > 32 || !(tol >= 0.0)) {
        set_error(nullptr, "invalid criterion arguments");
        return PSR_ERR_INVALID_ARG;
    }
    if (batch > PSR_CRITERION_NOALLOC_MAX) {
        set_error(nullptr, "psr_criterion_noalloc: batch " + std::to_string(batch) +
                               " exceeds its fixed scratch of " + std::to_string(PSR_CRITERION_NOALLOC_MAX) +
                               " candidates; split the batch or call psr_criterion");
        return PSR_ERR_INVALID_ARG;
    }
    if (batch == 0) return PSR_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) { set_error(nullptr, "device ordinal out of range"); return PSR_ERR_INVALID_ARG; }
    void* scratch = nullptr;
    {
        // One-time set-up per device, with that device current: the array's
        // name is only a host-side stand-in, its device address must be asked for.
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_criterion_scratch);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(criterion scratch)");
            g_scratch_addr[dev] = ptr;
        }
        scratch = g_scratch_addr[dev];
    }
    // launch_criterion_batch clears the counter (scratch[batch]) before use.
    return launch_criterion_batch(A_i, batch, p, A_c, Binv_c, tol, accept, dval,
                                  reinterpret_cast<int32_t*>(scratch), (cudaStream_t)stream);
}

namespace psr {

// ---------------------------------------------------------------- Alg. 1, entrywise l1 test
// Experiment 3's variant of Alg. 1: patch i joins the first entry (creation
// order) with ||A_i - A_c||_l1 < tol.  Rounds as in the spectral form: round
// r takes the smallest unassigned patch c as entry r and compares every
// unassigned patch after it (one warp each, lanes over the p^2 entries).  The
// next entry is the smallest patch rejected in the round; it goes through
// three device slots (round r reads slot r%3, bids into slot (r+1)%3 with
// atomicMin, resets slot (r+2)%3 for round r+1), so rounds are enqueued back
// to back and the host reads the state once per batch.  Decisions need no
// inverse: the inverses of the entries alone are formed afterwards.
struct L1State {
    int32_t slot[3];
    int32_t rounds;
};

__global__ void k_l1_round(const double* __restrict__ Ag, int count, int p, double tol, int r, L1State* st,
                           int32_t* __restrict__ phi, int32_t* __restrict__ rep,
                           unsigned long long* __restrict__ evals) {
    const int c = st->slot[r % 3];
    if (c >= count) {                                // Alg. 1 finished in an earlier round:
        if (blockIdx.x == 0 && threadIdx.x == 0) st->slot[(r + 1) % 3] = count;   // so is the next
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        phi[c] = r;
        rep[r] = c;
        st->slot[(r + 2) % 3] = count;
        st->rounds = r + 1;
    }
    const int lane = threadIdx.x & 31;
    const int pp = p * p;
    const double* a = Ag + (int64_t)c * pp;
    unsigned long long my_evals = 0;
    int my_min = count;
    for (int i = c + 1 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < count;
         i += (gridDim.x * blockDim.x) >> 5) {
        if (phi[i] != -1) continue;                  // uniform over the warp
        const double* b = Ag + (int64_t)i * pp;
        double s0 = 0.0, s1 = 0.0;
        for (int e = lane; e < pp; e += 64) {
            s0 += fabs(a[e] - b[e]);
            if (e + 32 < pp) s1 += fabs(a[e + 32] - b[e + 32]);
        }
        const double d = warp_sum(s0 + s1);
        ++my_evals;
        if (d < tol) {
            if (lane == 0) phi[i] = r;
        } else {
            my_min = min(my_min, i);
        }
    }
    if (lane == 0) {
        if (my_evals) atomicAdd(evals, my_evals);
        if (my_min < count) atomicMin(&st->slot[(r + 1) % 3], my_min);
    }
}

int run_alg1_l1(psr_ctx* ctx, cudaStream_t s) {
    const double tol = ctx->opts.tol;
    int64_t total_evals = 0;
    int rounds_total = 0;
    int first_singular = -1;
    L1State* st = nullptr;
    unsigned long long* evals = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&st, sizeof(L1State)));
    PSR_CUDA(ctx, psr::dev_alloc(&evals, sizeof(unsigned long long)));
    int rc = PSR_OK;
    for (size_t g = 0; g < ctx->groups.size() && rc == PSR_OK; ++g) {
        Group& G = ctx->groups[g];
        const int p = G.p, count = G.count;
        const int64_t pp = (int64_t)p * p;
        const double* Ag = ctx->A_ext + G.mat_off;
        int32_t *phi_l = nullptr, *rep_l = nullptr, *sing = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&phi_l, sizeof(int32_t) * count));
        PSR_CUDA(ctx, psr::dev_alloc(&rep_l, sizeof(int32_t) * count));
        PSR_CUDA(ctx, cudaMemsetAsync(phi_l, 0xff, sizeof(int32_t) * count, s));
        PSR_CUDA(ctx, cudaMemsetAsync(evals, 0, sizeof(unsigned long long), s));
        L1State init{{0, count, count}, 0};
        L1State h{};
        PSR_CUDA(ctx, cudaMemcpyAsync(st, &init, sizeof(L1State), cudaMemcpyHostToDevice, s));
        const int blocks = std::max(1, std::min((count + 7) / 8, 152 * 16));
        constexpr int BATCH = 64;
        for (int r0 = 0; r0 < count; r0 += BATCH) {
            const int r1 = std::min(count, r0 + BATCH);
            for (int r = r0; r < r1; ++r) {
                count_launch();
                k_l1_round<<<blocks, 256, 0, s>>>(Ag, count, p, tol, r, st, phi_l, rep_l, evals);
            }
            PSR_CHECK_LAUNCH(ctx, "Alg. 1 rounds (l1)");
            PSR_CUDA(ctx, cudaMemcpyAsync(&h, st, sizeof(L1State), cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            if (h.rounds < r1) break;                 // a round of this batch found no patch left
        }
        const int m = h.rounds;
        unsigned long long h_evals = 0;
        PSR_CUDA(ctx, cudaMemcpy(&h_evals, evals, sizeof(h_evals), cudaMemcpyDeviceToHost));
        // the entries' matrices and their inverses
        PSR_CUDA(ctx, psr::dev_alloc(&G.dbA, sizeof(double) * (size_t)std::max(m, 1) * pp));
        double* Bdb = nullptr;
        PSR_CUDA(ctx, psr::dev_alloc(&Bdb, sizeof(double) * (size_t)std::max(m, 1) * pp));
        PSR_CUDA(ctx, psr::dev_alloc(&sing, sizeof(int32_t) * std::max(m, 1)));
        {
            const int64_t tot = (int64_t)m * pp;
            const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 16));
            count_launch();
            k_gather_db<<<gb, 256, 0, s>>>(nullptr, 0, Ag, rep_l, m, p, G.dbA);
        }
        rc = launch_batched_inverse(G.dbA, pp, nullptr, m, p, Bdb, pp, sing, s);
        std::vector<int32_t> hrep((size_t)m), hs((size_t)m);
        if (rc == PSR_OK) {
            PSR_CUDA(ctx, cudaMemcpyAsync(hrep.data(), rep_l, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaMemcpyAsync(hs.data(), sing, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
            PSR_CUDA(ctx, cudaStreamSynchronize(s));
            for (int j = 0; j < m && first_singular < 0; ++j)
                if (hs[j]) first_singular = G.h_gidx[hrep[j]];
        }
        psr::dev_free(sing);
        psr::dev_free(rep_l);
        G.m = m;
        G.sphi = phi_l;
        G.rinv = Bdb;
        G.h_rep.assign(hrep.begin(), hrep.end());
        total_evals += (int64_t)h_evals;
        rounds_total += m;
    }
    psr::dev_free(st);
    psr::dev_free(evals);
    ctx->stats.first_singular = first_singular;
    ctx->stats.criterion_evals = total_evals;
    ctx->stats.criterion_exact = 0;
    ctx->stats.criterion_screened = 0;
    ctx->stats.rounds = rounds_total;
    return rc;
}

}  // namespace psr
