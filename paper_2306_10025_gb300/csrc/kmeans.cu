// Alg. 2 of section 3.2: the database size m_p is fixed beforehand, B_j the
// entrywise mean of its cluster (Eq. 6), the stored inverse that of the
// mean; d(A_i, B_j) = ||A_i - B_j||_l1 (entrywise variant) or
// ||I - A_i B_j^-1||_2 (spectral variant), chosen by psr_opts.criterion.
//
// Starts from the means B_j = A_{init[j]} (the caller draws the m_p distinct
// patches).  A sweep assigns every patch to its nearest mean in parallel
// (the assignments of one sweep do not depend on each other: the means only
// change between sweeps), ties to the lowest j; when an assignment changed,
// the means are recomputed and the next sweep follows.  Means sum their
// members in increasing patch index, one thread per matrix entry, so they
// are bitwise those of a sequential loop; a cluster left empty keeps its
// mean.
#include "psr_internal.cuh"
#include "dense.cuh"

#include <algorithm>
#include <vector>

namespace psr {

// One warp per patch: entrywise l1 distance to every mean (lanes over the
// p^2 entries, warp sum), strict minimum (the lowest j wins ties); counts the
// patches whose assignment changed.
__global__ void k_kmeans_assign(const double* __restrict__ A, int count, int pp, const double* __restrict__ B,
                                int m, int32_t* __restrict__ phi, int32_t* __restrict__ changes) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= count) return;                                   // warp-uniform
    const double* a = A + (int64_t)i * pp;
    double best = 0.0;
    int arg = 0;
    for (int j = 0; j < m; ++j) {
        const double* b = B + (int64_t)j * pp;
        double s = 0.0;
        for (int e = lane; e < pp; e += 32) s += fabs(a[e] - b[e]);
        s = warp_sum(s);
        if (j == 0 || s < best) {
            best = s;
            arg = j;
        }
    }
    if (lane == 0 && phi[i] != arg) {
        phi[i] = arg;
        atomicAdd(changes, 1);
    }
}

// Spectral variant: d(A_i, B_j) = ||I - A_i B_j^-1||_2, evaluated in the
// difference form ||(B_j - A_i) B_j^-1||_2 = sqrt(lambda_max(E^T E)) with
// Bi = the inverses of the current means.  One warp per patch (p <= 32):
// lane r forms row r of E into the warp's shared scratch, then holds column
// r of E, G = E^T E is built with shuffles over the scratch and its largest
// eigenvalue taken by the cyclic Jacobi of the criterion's exact path;
// strict minimum (the lowest j wins ties).
__global__ void __launch_bounds__(128) k_kmeans_assign_spectral(const double* __restrict__ A, int count, int p,
                                                                 const double* __restrict__ B,
                                                                 const double* __restrict__ Bi, int m,
                                                                 int32_t* __restrict__ phi,
                                                                 int32_t* __restrict__ changes) {
    extern __shared__ double kscratch[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int ld = p + 1, pp = p * p;
    double* G = kscratch + (size_t)wid * p * ld;
    for (int i = blockIdx.x * wpb + wid; i < count; i += gridDim.x * wpb) {
        const double* a = A + (int64_t)i * pp;
        double best = 0.0;
        int arg = 0;
        for (int j = 0; j < m; ++j) {
            const double* b = B + (int64_t)j * pp;
            const double* bi = Bi + (int64_t)j * pp;
            double drow[32];
#pragma unroll
            for (int l = 0; l < 32; ++l) drow[l] = (lane < p && l < p) ? b[lane * p + l] - a[lane * p + l] : 0.0;
            if (lane < p)
                for (int k = 0; k < p; ++k) {
                    double e = 0.0;
#pragma unroll
                    for (int l = 0; l < 32; ++l)
                        if (l < p) e = fma(drow[l], bi[l * p + k], e);
                    G[lane * ld + k] = e;
                }
            __syncwarp();
            double ecol[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) ecol[r] = (lane < p && r < p) ? G[r * ld + lane] : 0.0;
            __syncwarp();
            for (int k = 0; k < p; ++k) {
                double g = 0.0;
#pragma unroll
                for (int r = 0; r < 32; ++r) g = fma(ecol[r], __shfl_sync(0xffffffffu, ecol[r], k), g);
                if (lane < p) G[lane * ld + k] = g;
            }
            __syncwarp();
            const double sig = sqrt(fmax(jacobi_lambda_max_warp(G, p, ld), 0.0));
            __syncwarp();
            if (j == 0 || sig < best) {
                best = sig;
                arg = j;
            }
        }
        if (lane == 0 && phi[i] != arg) {
            phi[i] = arg;
            atomicAdd(changes, 1);
        }
    }
}

// Means of Eq. (6): thread (j, e) sums entry e over the members of cluster
// j (member list in increasing patch index), empty clusters keep theirs.
__global__ void k_kmeans_means(const double* __restrict__ A, int pp, const int32_t* __restrict__ moff,
                               const int32_t* __restrict__ mlist, int m, double* __restrict__ B) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * pp) return;
    const int j = (int)(t / pp), e = (int)(t % pp);
    const int b = moff[j], c = moff[j + 1] - b;
    if (c == 0) return;
    double acc = 0.0;
    for (int q = 0; q < c; ++q) acc = acc + A[(int64_t)mlist[b + q] * pp + e];
    B[(int64_t)j * pp + e] = acc / (double)c;
}

__global__ void k_kmeans_init(const double* __restrict__ A, int pp, const int32_t* __restrict__ init, int m,
                              double* __restrict__ B) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * pp) return;
    const int j = (int)(t / pp), e = (int)(t % pp);
    B[t] = A[(int64_t)init[j] * pp + e];
}

// Database and assignment of the (single) size group by entrywise k-means.
// init: host, m distinct local patch indices.  Leaves G.m, G.sphi (device,
// local phi), G.rinv (FP64 inverses of the means, m x p x p), G.h_rep (-1:
// no entry is a patch), and the number of sweeps in ctx->stats.rounds.
int run_kmeans(psr_ctx* ctx, cudaStream_t s, int m, const std::vector<int32_t>& init, int max_iter) {
    Group& G = ctx->groups[0];
    const int p = G.p, pp = p * p, count = G.count;
    const bool spectral = ctx->opts.criterion == PSR_CRITERION_SPECTRAL;
    if (spectral && p > 32) {
        set_error(ctx, "spectral k-means handles patches of at most 32 DOFs");
        return PSR_ERR_INVALID_ARG;
    }
    const double* Ag = ctx->A_ext + G.mat_off;
    double* B = nullptr;
    int32_t *phi = nullptr, *d_init = nullptr, *changes = nullptr, *moff = nullptr, *mlist = nullptr;
    PSR_CUDA(ctx, cudaMalloc(&B, sizeof(double) * (size_t)m * pp));
    PSR_CUDA(ctx, cudaMalloc(&phi, sizeof(int32_t) * (size_t)count));
    PSR_CUDA(ctx, cudaMalloc(&d_init, sizeof(int32_t) * (size_t)m));
    PSR_CUDA(ctx, cudaMalloc(&changes, sizeof(int32_t)));
    PSR_CUDA(ctx, cudaMalloc(&moff, sizeof(int32_t) * (size_t)(m + 1)));
    PSR_CUDA(ctx, cudaMalloc(&mlist, sizeof(int32_t) * (size_t)count));
    double* Bcur = nullptr;                   // spectral: inverses of the current means
    int32_t* sing_cur = nullptr;
    if (spectral) {
        PSR_CUDA(ctx, cudaMalloc(&Bcur, sizeof(double) * (size_t)m * pp));
        PSR_CUDA(ctx, cudaMalloc(&sing_cur, sizeof(int32_t) * (size_t)m));
    }
    PSR_CUDA(ctx, cudaMemcpyAsync(d_init, init.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    PSR_CUDA(ctx, cudaMemsetAsync(phi, 0xff, sizeof(int32_t) * (size_t)count, s));
    const int eb = (int)std::max<int64_t>(1, ((int64_t)m * pp + 255) / 256);
    count_launch();
    k_kmeans_init<<<eb, 256, 0, s>>>(Ag, pp, d_init, m, B);
    std::vector<int32_t> hphi((size_t)count), hoff((size_t)m + 1), hlist((size_t)count);
    int sweeps = 0;
    int rc = PSR_OK;
    while (sweeps < max_iter) {
        ++sweeps;
        PSR_CUDA(ctx, cudaMemsetAsync(changes, 0, sizeof(int32_t), s));
        if (spectral) {
            // inverses of the current means (a singular mean is reported after the loop)
            int rci = launch_batched_inverse(B, pp, nullptr, m, p, Bcur, pp, sing_cur, s);
            if (rci != PSR_OK) { rc = rci; break; }
            count_launch();
            const int kb = std::max(1, std::min((count + 3) / 4, 152 * 16));
            k_kmeans_assign_spectral<<<kb, 128, sizeof(double) * 4 * p * (p + 1), s>>>(Ag, count, p, B, Bcur, m,
                                                                                       phi, changes);
        } else {
            count_launch();
            k_kmeans_assign<<<(count + 7) / 8, 256, 0, s>>>(Ag, count, pp, B, m, phi, changes);
        }
        int32_t h_changes = 0;
        PSR_CUDA(ctx, cudaMemcpyAsync(&h_changes, changes, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaMemcpyAsync(hphi.data(), phi, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        if (h_changes == 0) break;
        // members of every cluster in increasing patch index (counting sort)
        std::fill(hoff.begin(), hoff.end(), 0);
        for (int i = 0; i < count; ++i) ++hoff[(size_t)hphi[i] + 1];
        for (int j = 0; j < m; ++j) hoff[(size_t)j + 1] += hoff[j];
        std::vector<int32_t> fill(hoff.begin(), hoff.end() - 1);
        for (int i = 0; i < count; ++i) hlist[(size_t)fill[hphi[i]]++] = i;
        PSR_CUDA(ctx, cudaMemcpyAsync(moff, hoff.data(), sizeof(int32_t) * hoff.size(), cudaMemcpyHostToDevice, s));
        PSR_CUDA(ctx, cudaMemcpyAsync(mlist, hlist.data(), sizeof(int32_t) * hlist.size(), cudaMemcpyHostToDevice, s));
        count_launch();
        k_kmeans_means<<<eb, 256, 0, s>>>(Ag, pp, moff, mlist, m, B);
        PSR_CHECK_LAUNCH(ctx, "k-means means");
        // the host copies above read hoff / hlist before the next sweep rewrites them
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
    }
    // inverses of the means (FP64 Gauss-Jordan with partial pivoting)
    double* Bdb = nullptr;
    int32_t* sing = nullptr;
    PSR_CUDA(ctx, cudaMalloc(&Bdb, sizeof(double) * (size_t)m * pp));
    PSR_CUDA(ctx, cudaMalloc(&sing, sizeof(int32_t) * (size_t)m));
    if (rc == PSR_OK) rc = launch_batched_inverse(B, pp, nullptr, m, p, Bdb, pp, sing, s);
    std::vector<int32_t> hs((size_t)m);
    if (rc == PSR_OK) {
        PSR_CUDA(ctx, cudaMemcpyAsync(hs.data(), sing, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        for (int j = 0; j < m; ++j)
            if (hs[j]) {
                set_error(ctx, "k-means mean " + std::to_string(j) + " failed the pivot test (singular)");
                rc = PSR_ERR_SINGULAR_PATCH;
                break;
            }
    }
    cudaFree(d_init);
    cudaFree(Bcur);
    cudaFree(sing_cur);
    cudaFree(changes);
    cudaFree(moff);
    cudaFree(mlist);
    cudaFree(sing);
    if (rc != PSR_OK) {
        cudaFree(B);
        cudaFree(phi);
        cudaFree(Bdb);
        return rc;
    }
    G.dbA = B;                      // the means: the entries' matrices, kept for reuse
    G.m = m;
    G.sphi = phi;
    G.rinv = Bdb;
    G.h_rep.assign((size_t)m, -1);
    ctx->stats.rounds = sweeps;
    ctx->stats.criterion_evals = 0;
    return PSR_OK;
}

}  // namespace psr
