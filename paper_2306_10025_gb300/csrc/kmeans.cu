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
#include <map>
#include <vector>

namespace psr {

// One warp per patch: entrywise l1 distance to every mean (lanes over the
// p^2 entries, warp sum), strict minimum (the lowest j wins ties); counts the
// patches whose assignment changed.
// pcls / mcls (both null, or both set): class of every patch and of every
// mean; a patch is assigned only among the means of its class (the boundary
// partition of section 3.2).
__global__ void k_kmeans_assign(const double* __restrict__ A, int count, int pp, const double* __restrict__ B,
                                int m, int32_t* __restrict__ phi, int32_t* __restrict__ changes,
                                const int32_t* __restrict__ pcls, const int32_t* __restrict__ mcls) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= count) return;                                   // warp-uniform
    const double* a = A + (int64_t)i * pp;
    const int ci = pcls ? pcls[i] : 0;
    double best = 0.0;
    int arg = -1;
    for (int j = 0; j < m; ++j) {
        if (pcls && mcls[j] != ci) continue;                  // warp-uniform
        const double* b = B + (int64_t)j * pp;
        double s = 0.0;
        for (int e = lane; e < pp; e += 32) s += fabs(a[e] - b[e]);
        s = warp_sum(s);
        if (arg < 0 || s < best) {
            best = s;
            arg = j;
        }
    }
    if (arg < 0) arg = 0;                                     // every class has a mean (checked on the host)
    if (lane == 0 && phi[i] != arg) {
        phi[i] = arg;
        atomicAdd(changes, 1);
    }
}

// d(A_i, B) = ||I - A_i B^-1||_2 in the difference form ||(B - A_i) B^-1||_2
// = sqrt(lambda_max(E^T E)), by one warp (p <= 32): lane r forms row r of E
// into the warp's shared scratch G (p x (p+1)), then holds column r of E;
// G = E^T E is built with shuffles and its largest eigenvalue taken by the
// cyclic Jacobi of the criterion's exact path.  Every lane gets the value.
__device__ double spectral_dist_warp(const double* __restrict__ a, const double* __restrict__ b,
                                     const double* __restrict__ bi, int p, double* G) {
    const int lane = threadIdx.x & 31;
    const int ld = p + 1;
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
    return sig;
}

// Spectral and variance-minimising variants: d(A_i, B_j) = ||I - A_i B_j^-1||_2
// with Bi the inverses of the current representatives (the means, or the
// chosen members).  One warp per patch; strict minimum (the lowest j wins ties).
__global__ void __launch_bounds__(128) k_kmeans_assign_spectral(const double* __restrict__ A, int count, int p,
                                                                 const double* __restrict__ B,
                                                                 const double* __restrict__ Bi, int m,
                                                                 int32_t* __restrict__ phi,
                                                                 int32_t* __restrict__ changes,
                                                                 const int32_t* __restrict__ pcls,
                                                                 const int32_t* __restrict__ mcls) {
    extern __shared__ double kscratch[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int pp = p * p;
    double* G = kscratch + (size_t)wid * p * (p + 1);
    for (int i = blockIdx.x * wpb + wid; i < count; i += gridDim.x * wpb) {
        const int ci = pcls ? pcls[i] : 0;
        double best = 0.0;
        int arg = -1;
        for (int j = 0; j < m; ++j) {
            if (pcls && mcls[j] != ci) continue;              // warp-uniform
            const double sig = spectral_dist_warp(A + (int64_t)i * pp, B + (int64_t)j * pp, Bi + (int64_t)j * pp, p, G);
            if (arg < 0 || sig < best) {
                best = sig;
                arg = j;
            }
        }
        if (arg < 0) arg = 0;                                 // every class has a mean (checked on the host)
        if (lane == 0 && phi[i] != arg) {
            phi[i] = arg;
            atomicAdd(changes, 1);
        }
    }
}

// Variance-minimising variant: V[m] = sum over the members k of m's cluster
// (in increasing k) of d(A_k, A_m)^2, one warp per patch m.
__global__ void __launch_bounds__(128) k_kmeans_variance(const double* __restrict__ A,
                                                          const double* __restrict__ Ainv, int count, int p,
                                                          const int32_t* __restrict__ phi,
                                                          const int32_t* __restrict__ moff,
                                                          const int32_t* __restrict__ mlist, double* __restrict__ V) {
    extern __shared__ double kscratch[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int pp = p * p;
    double* G = kscratch + (size_t)wid * p * (p + 1);
    for (int mm = blockIdx.x * wpb + wid; mm < count; mm += gridDim.x * wpb) {
        const int j = phi[mm];
        double acc = 0.0;
        for (int q = moff[j]; q < moff[j + 1]; ++q) {
            const int k = mlist[q];
            const double d = spectral_dist_warp(A + (int64_t)k * pp, A + (int64_t)mm * pp, Ainv + (int64_t)mm * pp, p, G);
            acc = acc + d * d;
        }
        if (lane == 0) V[mm] = acc;
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
// out[j] = src[idx[j]] for matrices of pp entries
__global__ void k_kmeans_gather(const double* __restrict__ src, const int32_t* __restrict__ idx, int m, int pp,
                                double* __restrict__ out) {
    const int64_t total = (int64_t)m * pp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / pp);
        out[e] = src[(int64_t)idx[j] * pp + (e - (int64_t)j * pp)];
    }
}

// Variance-minimising variant of Alg. 2 (section 3.2): representatives are
// members (init the first ones); a sweep assigns every patch to the nearest
// representative by ||I - A_i B_j^-1||_2, then every cluster takes the
// member with the smallest variance sum_k d(A_k, A_m)^2 (sums in member
// order on the device, the lowest member on ties chosen on the host).  The
// inverses of all patches are formed once; the database keeps the
// representatives' patches and inverses.
// Device copies of the class of every patch and of every mean (the class of
// its seed) for the partitioned assignment; nothing when cls is null.
struct ClassFilter {
    int32_t* pcls = nullptr;
    int32_t* mcls = nullptr;
    ~ClassFilter() {
        dev_free(pcls);
        dev_free(mcls);
    }
    int upload(psr_ctx* ctx, const std::vector<int32_t>* cls, const std::vector<int32_t>& init, cudaStream_t s) {
        if (!cls) return PSR_OK;
        std::vector<int32_t> hm(init.size());
        for (size_t j = 0; j < init.size(); ++j) hm[j] = (*cls)[(size_t)init[j]];
        PSR_CUDA(ctx, dev_alloc(&pcls, sizeof(int32_t) * std::max<size_t>(cls->size(), 1)));
        PSR_CUDA(ctx, dev_alloc(&mcls, sizeof(int32_t) * std::max<size_t>(hm.size(), 1)));
        PSR_CUDA(ctx, cudaMemcpyAsync(pcls, cls->data(), sizeof(int32_t) * cls->size(), cudaMemcpyHostToDevice, s));
        PSR_CUDA(ctx, cudaMemcpyAsync(mcls, hm.data(), sizeof(int32_t) * hm.size(), cudaMemcpyHostToDevice, s));
        return PSR_OK;
    }
};

static int run_kmeans_varmin(psr_ctx* ctx, cudaStream_t s, int m, const std::vector<int32_t>& init, int max_iter,
                             const std::vector<int32_t>* cls) {
    Group& G = ctx->groups[0];
    const int p = G.p, pp = p * p, count = G.count;
    if (p > 32) {
        set_error(ctx, "variance-minimising k-means handles patches of at most 32 DOFs");
        return PSR_ERR_INVALID_ARG;
    }
    const double* Ag = ctx->A_ext + G.mat_off;
    ClassFilter cf;
    if (int rcf = cf.upload(ctx, cls, init, s)) return rcf;
    double *Ainv = nullptr, *B = nullptr, *Bcur = nullptr, *V = nullptr;
    int32_t *sing_all = nullptr, *phi = nullptr, *changes = nullptr, *moff = nullptr, *mlist = nullptr,
            *d_reps = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&Ainv, sizeof(double) * (size_t)count * pp));
    PSR_CUDA(ctx, psr::dev_alloc(&sing_all, sizeof(int32_t) * (size_t)count));
    PSR_CUDA(ctx, psr::dev_alloc(&B, sizeof(double) * (size_t)m * pp));
    PSR_CUDA(ctx, psr::dev_alloc(&Bcur, sizeof(double) * (size_t)m * pp));
    PSR_CUDA(ctx, psr::dev_alloc(&V, sizeof(double) * (size_t)count));
    PSR_CUDA(ctx, psr::dev_alloc(&phi, sizeof(int32_t) * (size_t)count));
    PSR_CUDA(ctx, psr::dev_alloc(&changes, sizeof(int32_t)));
    PSR_CUDA(ctx, psr::dev_alloc(&moff, sizeof(int32_t) * (size_t)(m + 1)));
    PSR_CUDA(ctx, psr::dev_alloc(&mlist, sizeof(int32_t) * (size_t)count));
    PSR_CUDA(ctx, psr::dev_alloc(&d_reps, sizeof(int32_t) * (size_t)m));
    int rc = launch_batched_inverse(Ag, pp, nullptr, count, p, Ainv, pp, sing_all, s);
    std::vector<int32_t> reps(init.begin(), init.end());
    std::vector<int32_t> hphi((size_t)count), hoff((size_t)m + 1), hlist((size_t)count);
    std::vector<double> hV((size_t)count);
    PSR_CUDA(ctx, cudaMemsetAsync(phi, 0xff, sizeof(int32_t) * (size_t)count, s));
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)m * pp + 255) / 256, 152 * 16));
    const int kb = std::max(1, std::min((count + 3) / 4, 152 * 16));
    const size_t scratch = sizeof(double) * 4 * p * (p + 1);
    int sweeps = 0;
    while (rc == PSR_OK && sweeps < max_iter) {
        ++sweeps;
        PSR_CUDA(ctx, cudaMemcpyAsync(d_reps, reps.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        count_launch(); k_kmeans_gather<<<gb, 256, 0, s>>>(Ag, d_reps, m, pp, B);
        count_launch(); k_kmeans_gather<<<gb, 256, 0, s>>>(Ainv, d_reps, m, pp, Bcur);
        PSR_CUDA(ctx, cudaMemsetAsync(changes, 0, sizeof(int32_t), s));
        count_launch();
        k_kmeans_assign_spectral<<<kb, 128, scratch, s>>>(Ag, count, p, B, Bcur, m, phi, changes, cf.pcls, cf.mcls);
        int32_t h_changes = 0;
        PSR_CUDA(ctx, cudaMemcpyAsync(&h_changes, changes, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaMemcpyAsync(hphi.data(), phi, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        if (h_changes == 0) break;
        std::fill(hoff.begin(), hoff.end(), 0);
        for (int i = 0; i < count; ++i) ++hoff[(size_t)hphi[i] + 1];
        for (int j = 0; j < m; ++j) hoff[(size_t)j + 1] += hoff[j];
        std::vector<int32_t> fill(hoff.begin(), hoff.end() - 1);
        for (int i = 0; i < count; ++i) hlist[(size_t)fill[hphi[i]]++] = i;
        PSR_CUDA(ctx, cudaMemcpyAsync(moff, hoff.data(), sizeof(int32_t) * hoff.size(), cudaMemcpyHostToDevice, s));
        PSR_CUDA(ctx, cudaMemcpyAsync(mlist, hlist.data(), sizeof(int32_t) * hlist.size(), cudaMemcpyHostToDevice, s));
        count_launch();
        k_kmeans_variance<<<kb, 128, scratch, s>>>(Ag, Ainv, count, p, phi, moff, mlist, V);
        PSR_CHECK_LAUNCH(ctx, "k-means variances");
        PSR_CUDA(ctx, cudaMemcpyAsync(hV.data(), V, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        for (int j = 0; j < m; ++j) {
            int best = -1;
            for (int q = hoff[j]; q < hoff[j + 1]; ++q)
                if (best < 0 || hV[hlist[q]] < hV[best]) best = hlist[q];
            if (best >= 0) reps[j] = best;         // an empty cluster keeps its representative
        }
    }
    // the database: the representatives' patches and inverses
    double* Bdb = nullptr;
    std::vector<int32_t> hsing((size_t)count);
    if (rc == PSR_OK) {
        PSR_CUDA(ctx, cudaMemcpyAsync(d_reps, reps.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        PSR_CUDA(ctx, psr::dev_alloc(&Bdb, sizeof(double) * (size_t)m * pp));
        count_launch(); k_kmeans_gather<<<gb, 256, 0, s>>>(Ag, d_reps, m, pp, B);
        count_launch(); k_kmeans_gather<<<gb, 256, 0, s>>>(Ainv, d_reps, m, pp, Bdb);
        PSR_CUDA(ctx, cudaMemcpyAsync(hsing.data(), sing_all, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToHost, s));
        PSR_CUDA(ctx, cudaStreamSynchronize(s));
        for (int j = 0; j < m; ++j)
            if (hsing[reps[j]]) {
                set_error(ctx, "representative patch " + std::to_string(G.h_gidx[reps[j]]) +
                                   " failed the pivot test (singular)");
                rc = PSR_ERR_SINGULAR_PATCH;
                break;
            }
    }
    for (void* q : {(void*)Ainv, (void*)sing_all, (void*)Bcur, (void*)V, (void*)changes, (void*)moff, (void*)mlist,
                    (void*)d_reps})
        psr::dev_free(q);
    if (rc != PSR_OK) {
        psr::dev_free(B);
        psr::dev_free(phi);
        psr::dev_free(Bdb);
        return rc;
    }
    G.dbA = B;
    G.m = m;
    G.sphi = phi;
    G.rinv = Bdb;
    G.h_rep.assign(reps.begin(), reps.end());
    ctx->stats.rounds = sweeps;
    ctx->stats.criterion_evals = 0;
    return PSR_OK;
}

int run_kmeans(psr_ctx* ctx, cudaStream_t s, int m, const std::vector<int32_t>& init, int max_iter,
               const std::vector<int32_t>* cls) {
    if (ctx->opts.criterion == PSR_CRITERION_VARMIN) return run_kmeans_varmin(ctx, s, m, init, max_iter, cls);
    Group& G = ctx->groups[0];
    const int p = G.p, pp = p * p, count = G.count;
    const bool spectral = ctx->opts.criterion == PSR_CRITERION_SPECTRAL;
    if (spectral && p > 32) {
        set_error(ctx, "spectral k-means handles patches of at most 32 DOFs");
        return PSR_ERR_INVALID_ARG;
    }
    const double* Ag = ctx->A_ext + G.mat_off;
    ClassFilter cf;
    if (int rcf = cf.upload(ctx, cls, init, s)) return rcf;
    double* B = nullptr;
    int32_t *phi = nullptr, *d_init = nullptr, *changes = nullptr, *moff = nullptr, *mlist = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&B, sizeof(double) * (size_t)m * pp));
    PSR_CUDA(ctx, psr::dev_alloc(&phi, sizeof(int32_t) * (size_t)count));
    PSR_CUDA(ctx, psr::dev_alloc(&d_init, sizeof(int32_t) * (size_t)m));
    PSR_CUDA(ctx, psr::dev_alloc(&changes, sizeof(int32_t)));
    PSR_CUDA(ctx, psr::dev_alloc(&moff, sizeof(int32_t) * (size_t)(m + 1)));
    PSR_CUDA(ctx, psr::dev_alloc(&mlist, sizeof(int32_t) * (size_t)count));
    double* Bcur = nullptr;                   // spectral: inverses of the current means
    int32_t* sing_cur = nullptr;
    if (spectral) {
        PSR_CUDA(ctx, psr::dev_alloc(&Bcur, sizeof(double) * (size_t)m * pp));
        PSR_CUDA(ctx, psr::dev_alloc(&sing_cur, sizeof(int32_t) * (size_t)m));
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
                                                                                       phi, changes, cf.pcls, cf.mcls);
        } else {
            count_launch();
            k_kmeans_assign<<<(count + 7) / 8, 256, 0, s>>>(Ag, count, pp, B, m, phi, changes, cf.pcls, cf.mcls);
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
    PSR_CUDA(ctx, psr::dev_alloc(&Bdb, sizeof(double) * (size_t)m * pp));
    PSR_CUDA(ctx, psr::dev_alloc(&sing, sizeof(int32_t) * (size_t)m));
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
    psr::dev_free(d_init);
    psr::dev_free(Bcur);
    psr::dev_free(sing_cur);
    psr::dev_free(changes);
    psr::dev_free(moff);
    psr::dev_free(mlist);
    psr::dev_free(sing);
    if (rc != PSR_OK) {
        psr::dev_free(B);
        psr::dev_free(phi);
        psr::dev_free(Bdb);
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

// Boundary partition (section 3.2): bit a of mask[k] is set when row a of the
// patch matrix A_k has exactly one nonzero entry (a boundary condition);
// one warp per patch, p <= 64.
__global__ void k_bc_mask(const double* __restrict__ Aext, const int64_t* __restrict__ mat_off,
                          const int32_t* __restrict__ offsets, int np, int pu,
                          unsigned long long* __restrict__ mask) {
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= np) return;                                      // warp-uniform
    const int p = pu > 0 ? pu : offsets[k + 1] - offsets[k];
    const double* a = Aext + (pu > 0 ? (int64_t)k * p * p : mat_off[k]);
    unsigned lo = 0u, hi = 0u;
    for (int r = lane; r < p; r += 32) {
        int nz = 0;
        for (int c = 0; c < p; ++c) nz += a[(int64_t)r * p + c] != 0.0;
        if (nz == 1) {
            if (r < 32) lo |= 1u << r;
            else hi |= 1u << (r - 32);
        }
    }
    lo = __reduce_or_sync(0xffffffffu, lo);
    hi = __reduce_or_sync(0xffffffffu, hi);
    if (lane == 0) mask[k] = ((unsigned long long)hi << 32) | lo;
}

}  // namespace psr

extern "C" int psr_boundary_classes(const psr_csr* A, const psr_patches* P, int32_t* patch_class,
                                    int32_t* n_classes, void* stream) {
    using namespace psr;
    if (!A || !P || !patch_class || !n_classes || A->n <= 0 || P->n_patches <= 0 || !P->dofs ||
        (P->uniform_size <= 0 && !P->offsets) || P->uniform_size > 64) {
        set_error(nullptr, "psr_boundary_classes: invalid argument (patches of at most 64 DOFs)");
        return PSR_ERR_INVALID_ARG;
    }
    *n_classes = 0;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = P->n_patches;
    std::vector<int32_t> ho((size_t)np + 1);
    std::vector<int64_t> hm((size_t)np + 1, 0);
    if (P->uniform_size > 0) {
        for (int k = 0; k <= np; ++k) ho[(size_t)k] = k * P->uniform_size;
    } else {
        PSR_CUDA(nullptr, cudaMemcpyAsync(ho.data(), P->offsets, sizeof(int32_t) * (size_t)(np + 1),
                                          cudaMemcpyDeviceToHost, s));
        PSR_CUDA(nullptr, cudaStreamSynchronize(s));
    }
    for (int k = 0; k < np; ++k) {
        const int64_t pk = ho[(size_t)k + 1] - ho[(size_t)k];
        if (pk < 1 || pk > 64) {
            set_error(nullptr, "psr_boundary_classes: patch sizes must lie in 1..64");
            return PSR_ERR_INVALID_ARG;
        }
        hm[(size_t)k + 1] = hm[(size_t)k] + pk * pk;
    }
    double* Aext = nullptr;
    int64_t* mo = nullptr;
    unsigned long long* mask = nullptr;
    int rc = PSR_OK;
    if (dev_alloc(&Aext, sizeof(double) * (size_t)std::max<int64_t>(hm[(size_t)np], 1)) != cudaSuccess ||
        dev_alloc(&mo, sizeof(int64_t) * (size_t)(np + 1)) != cudaSuccess ||
        dev_alloc(&mask, sizeof(unsigned long long) * (size_t)np) != cudaSuccess) {
        cudaGetLastError();
        set_error(nullptr, "psr_boundary_classes: out of device memory");
        rc = PSR_ERR_OOM;
    }
    // the patch matrices (validates the CSR and the map)
    if (rc == PSR_OK) rc = psr_extract(A, P, Aext, nullptr, nullptr, stream);
    std::vector<unsigned long long> hmask((size_t)np);
    if (rc == PSR_OK) {
        cudaError_t e = cudaMemcpyAsync(mo, hm.data(), sizeof(int64_t) * (size_t)(np + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            count_launch();
            k_bc_mask<<<(np + 7) / 8, 256, 0, s>>>(Aext, mo, P->uniform_size > 0 ? nullptr : P->offsets, np,
                                                   P->uniform_size, mask);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hmask.data(), mask, sizeof(unsigned long long) * (size_t)np, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(nullptr, e, "psr_boundary_classes");
    }
    if (rc == PSR_OK) {
        // classes numbered in the order of their first patch
        std::map<unsigned long long, int32_t> ids;
        std::vector<int32_t> hc((size_t)np);
        for (int k = 0; k < np; ++k) {
            auto it = ids.emplace(hmask[(size_t)k], (int32_t)ids.size()).first;
            hc[(size_t)k] = it->second;
        }
        cudaError_t e = cudaMemcpyAsync(patch_class, hc.data(), sizeof(int32_t) * (size_t)np, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(nullptr, e, "psr_boundary_classes");
        else *n_classes = (int32_t)ids.size();
    }
    cudaStreamSynchronize(s);
    dev_free(Aext);
    dev_free(mo);
    dev_free(mask);
    return rc;
}
