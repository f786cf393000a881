// C ABI entry points (include/psr.h): setup / apply / solve / queries and the
// stateless single-step calls.  No C++ exception crosses this boundary.
#include "psr_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

namespace psr {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;

void count_launch(long long k) {
    if (!g_capturing) g_launches.fetch_add(k, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }

void set_error(psr_ctx* ctx, const std::string& msg) {
    g_last_error = msg;
    if (ctx) ctx->err = msg;
}

int cuda_fail(psr_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    set_error(ctx, m);
    return (e == cudaErrorMemoryAllocation) ? PSR_ERR_OOM : PSR_ERR_CUDA;
}

int build_sweep_layout(psr_ctx* ctx, const std::vector<std::vector<int32_t>>& gidx, cudaStream_t s);
int sweep_prepare(psr_ctx* ctx);

__global__ void k_iota(int32_t* a, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

__global__ void k_any(const int32_t* flags, int n, int32_t* first) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (flags[i]) atomicMin(first, i);
}

// NVTX ranges around the setup phases (visible in a profiler timeline; no
// cost without one).  The depth is tracked so a failing setup closes them.
static thread_local int g_nvtx_depth = 0;
static void phase_begin(const char* name) {
    nvtxRangePushA(name);
    ++g_nvtx_depth;
}
static void phase_end() {
    if (g_nvtx_depth > 0) {
        nvtxRangePop();
        --g_nvtx_depth;
    }
}
static void phases_close(int depth) {
    while (g_nvtx_depth > depth) phase_end();
}

static double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

static void destroy_ctx(psr_ctx* ctx) {
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != ctx->device) cudaSetDevice(ctx->device);
    free_sweep(ctx);
    coarse_free(ctx);
    krylov_free(ctx);
    psr::dev_free(ctx->rowptr);
    psr::dev_free(ctx->colidx);
    psr::dev_free(ctx->vals);
    psr::dev_free(ctx->offsets);
    psr::dev_free(ctx->dofs);
    psr::dev_free(ctx->mat_off);
    psr::dev_free(ctx->A_ext);
    psr::dev_free(ctx->W);
    if (ctx->Wg && ctx->Wg != ctx->W) psr::dev_free(ctx->Wg);
    psr::dev_free(ctx->phi);
    psr::dev_free(ctx->rep_ids);
    psr::dev_free(ctx->status);
    if (ctx->mlp) psr_mlp_destroy(ctx->mlp);
    if (cur != ctx->device) cudaSetDevice(cur);
    delete ctx;
}

static int check_status(psr_ctx* ctx, cudaStream_t s) {
    int32_t st = 0;
    PSR_CUDA(ctx, cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    if (st & ST_UNSORTED) { set_error(ctx, "CSR columns not sorted/unique or out of range"); return PSR_ERR_UNSORTED_CSR; }
    if (st & ST_OOB) { set_error(ctx, "patch map holds a DOF outside [0, n) or decreasing offsets"); return PSR_ERR_INVALID_ARG; }
    if (st & ST_UNCOVERED) { set_error(ctx, "a DOF belongs to no patch: W = (sum V^T V)^-1 is undefined"); return PSR_ERR_UNCOVERED_DOF; }
    return PSR_OK;
}

// Database construction of the setup: Alg. 1 (default; seeded and hinted
// when seed_A / hints are given) or entrywise k-means (km_m > 0).
struct AssignMode {
    const double* seed_A = nullptr;
    int m0 = 0;
    const int32_t* hints = nullptr;
    int km_m = 0;
    const std::vector<int32_t>* km_init = nullptr;
    int km_iter = 0;
    const std::vector<int32_t>* km_cls = nullptr;   // class of every patch (boundary partition) or null
    psr_mlp* mlp = nullptr;          // predictions of this network become the hints
    const float* features = nullptr; // its inputs (device) or null: computed from the patch matrices
};

static int setup_impl(const psr_csr* A, const psr_patches* P, const psr_opts* o, cudaStream_t s, psr_ctx** out,
                      const AssignMode& mode) {
    const double* seed_A = mode.seed_A;
    const int m0 = mode.m0;
    const int32_t* hints = mode.hints;
    auto t_all = std::chrono::steady_clock::now();
    const int nvtx_base = g_nvtx_depth;
    phase_begin("psr_setup");
    AllocScope scope;                              // a failed setup frees what its steps still hold
    psr_ctx* ctx = new psr_ctx();
    *out = nullptr;
    if (o) ctx->opts = *o; else psr_default_opts(&ctx->opts);
    psr_opts& op = ctx->opts;
    if (op.restart < 1 || op.restart > 32 || op.maxit < 1 || !(op.rtol > 0.0) || op.tol < 0.0 ||
        op.store_prec < 0 || op.store_prec > 2 || op.weighting < 0 || op.weighting > 1 || op.krylov < 0 || op.krylov > 1 ||
        op.sweep_kernel < PSR_SWEEP_AUTO || op.sweep_kernel > PSR_SWEEP_TENSOR || op.ortho < PSR_ORTHO_AUTO ||
        op.ortho > PSR_ORTHO_SPLIT || op.criterion < PSR_CRITERION_SPECTRAL || op.criterion > PSR_CRITERION_VARMIN ||
        op.fp64_arith < PSR_FP64_PAIRS || op.fp64_arith > PSR_FP64_NATIVE || op.match < PSR_MATCH_FIRST ||
        op.match > PSR_MATCH_CLOSEST || !(op.prec_check >= 0.0) || op.search < PSR_SEARCH_CREATION ||
        op.search > PSR_SEARCH_NORM_WINDOW) {
        set_error(ctx, "invalid option value");
        destroy_ctx(ctx);
        return PSR_ERR_INVALID_ARG;
    }
    cudaGetDevice(&ctx->device);
    const int n = A->n;
    ctx->n = n;
    ctx->nnz = A->nnz;
    ctx->n_patches = P->n_patches;
    ctx->stats.first_singular = -1;
    int rc = PSR_OK;
#define FAIL(code) do { rc = (code); goto fail; } while (0)
#define CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { rc = cuda_fail(ctx, e_, #call); goto fail; } } while (0)
    {
        // --- copies of the inputs
        CK(psr::dev_alloc(&ctx->status, sizeof(int32_t)));
        CK(cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), s));
        CK(psr::dev_alloc(&ctx->rowptr, sizeof(int32_t) * (size_t)(n + 1)));
        CK(psr::dev_alloc(&ctx->colidx, sizeof(int32_t) * (size_t)std::max<int64_t>(A->nnz, 1)));
        CK(psr::dev_alloc(&ctx->vals, sizeof(double) * (size_t)std::max<int64_t>(A->nnz, 1)));
        CK(cudaMemcpyAsync(ctx->rowptr, A->rowptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->colidx, A->colidx, sizeof(int32_t) * (size_t)A->nnz, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->vals, A->vals, sizeof(double) * (size_t)A->nnz, cudaMemcpyDeviceToDevice, s));
        const int np = P->n_patches;
        ctx->h_offsets.resize((size_t)np + 1);
        if (P->uniform_size > 0) {
            for (int k = 0; k <= np; ++k) ctx->h_offsets[k] = k * P->uniform_size;
            if ((int64_t)np * P->uniform_size >= (1ll << 31)) { set_error(ctx, "sum of patch sizes exceeds int32"); FAIL(PSR_ERR_INVALID_ARG); }
        } else {
            CK(cudaMemcpyAsync(ctx->h_offsets.data(), P->offsets, sizeof(int32_t) * (size_t)(np + 1), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (ctx->h_offsets[0] != 0) { set_error(ctx, "offsets[0] must be 0"); FAIL(PSR_ERR_INVALID_ARG); }
            for (int k = 0; k < np; ++k)
                if (ctx->h_offsets[k + 1] <= ctx->h_offsets[k]) { set_error(ctx, "patch sizes must be positive"); FAIL(PSR_ERR_INVALID_ARG); }
        }
        const int64_t total = ctx->h_offsets[np];
        CK(psr::dev_alloc(&ctx->offsets, sizeof(int32_t) * (size_t)(np + 1)));
        CK(cudaMemcpyAsync(ctx->offsets, ctx->h_offsets.data(), sizeof(int32_t) * (size_t)(np + 1), cudaMemcpyHostToDevice, s));
        CK(psr::dev_alloc(&ctx->dofs, sizeof(int32_t) * (size_t)total));
        CK(cudaMemcpyAsync(ctx->dofs, P->dofs, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToDevice, s));
        // --- validation
        rc = validate_inputs(ctx, A, ctx->offsets, ctx->dofs, np, total, ctx->status, s);
        if (rc != PSR_OK) goto fail;
        rc = check_status(ctx, s);
        if (rc != PSR_OK) goto fail;
        // --- size groups (Remark after Eq. 1), group-contiguous patch storage
        std::map<int, std::vector<int32_t>> bysize;
        for (int k = 0; k < np; ++k) bysize[ctx->h_offsets[k + 1] - ctx->h_offsets[k]].push_back(k);
        std::vector<std::vector<int32_t>> gidx;
        std::vector<int64_t> h_mat_off((size_t)np + 1, 0);
        int64_t off = 0;
        // larger patches first: the grouped kernel's heavy tiles are dealt out early
        for (auto it = bysize.rbegin(); it != bysize.rend(); ++it) {
            Group G;
            G.p = it->first;
            G.count = (int)it->second.size();
            G.mat_off = off;
            if (G.p > 128) { set_error(ctx, "patches larger than 128 DOFs are not supported"); FAIL(PSR_ERR_INVALID_ARG); }
            for (int l = 0; l < G.count; ++l) h_mat_off[it->second[l]] = off + (int64_t)l * G.p * G.p;
            off += (int64_t)G.count * G.p * G.p;
            G.h_gidx = it->second;
            ctx->groups.push_back(G);
            gidx.push_back(it->second);
        }
        h_mat_off[np] = off;
        ctx->A_ext_len = off;
        CK(psr::dev_alloc(&ctx->mat_off, sizeof(int64_t) * (size_t)(np + 1)));
        CK(cudaMemcpyAsync(ctx->mat_off, h_mat_off.data(), sizeof(int64_t) * (size_t)(np + 1), cudaMemcpyHostToDevice, s));
        {
            cudaError_t ea = psr::dev_alloc(&ctx->A_ext, sizeof(double) * (size_t)off);
            if (ea != cudaSuccess) { cudaGetLastError(); set_error(ctx, "out of device memory for the patch matrices"); FAIL(PSR_ERR_OOM); }
        }
        // --- a1: extraction
        phase_begin("psr_setup: extraction and weights");
        auto t0 = std::chrono::steady_clock::now();
        rc = launch_extract(ctx->rowptr, ctx->colidx, ctx->vals, ctx->offsets, ctx->dofs, ctx->mat_off, np,
                            0, total, ctx->A_ext, s);
        if (rc != PSR_OK) goto fail;
        // --- a1': multiplicity and weights
        {
            int32_t* mult = nullptr;
            double* w1 = nullptr;
            double* w2 = nullptr;
            CK(psr::dev_alloc(&mult, sizeof(int32_t) * (size_t)n));
            CK(psr::dev_alloc(&w1, sizeof(double) * (size_t)n));
            CK(psr::dev_alloc(&w2, sizeof(double) * (size_t)n));
            rc = launch_multiplicity(ctx->dofs, total, n, mult, w1, w2, ctx->status, s);
            if (rc != PSR_OK) { psr::dev_free(mult); psr::dev_free(w1); psr::dev_free(w2); goto fail; }
            CK(cudaStreamSynchronize(s));
            psr::dev_free(mult);
            if (op.weighting == PSR_WEIGHT_SYM) {
                psr::dev_free(w1);
                ctx->W = w2;
                ctx->Wg = w2;
            } else {
                psr::dev_free(w2);
                ctx->W = w1;
                ctx->Wg = nullptr;
            }
        }
        rc = check_status(ctx, s);
        if (rc != PSR_OK) goto fail;
        ctx->stats.t_extract = seconds_since(t0);
        phase_end();
        phase_begin("psr_setup: database and inverses");
        // --- a2 / a3: database and assignment
        CK(psr::dev_alloc(&ctx->phi, sizeof(int32_t) * (size_t)np));
        // seed entries come on top of at most one new entry per patch
        CK(psr::dev_alloc(&ctx->rep_ids, sizeof(int32_t) * ((size_t)np + (size_t)std::max(m0, 0))));
        t0 = std::chrono::steady_clock::now();
        if (mode.km_m == 0 && op.criterion == PSR_CRITERION_VARMIN) {
            set_error(ctx, "the variance-minimising criterion is an Alg. 2 variant (psr_setup_kmeans)");
            FAIL(PSR_ERR_INVALID_ARG);
        }
        if (mode.km_m > 0) {
            rc = run_kmeans(ctx, s, mode.km_m, *mode.km_init, mode.km_iter, mode.km_cls);
            if (rc != PSR_OK) goto fail;
        } else if (op.tol == 0.0 && m0 == 0) {
            // strict "< 0" never holds: every patch is its own entry (Eq. 1)
            int32_t* sing = nullptr;
            int32_t* first = nullptr;
            CK(psr::dev_alloc(&sing, sizeof(int32_t) * (size_t)np));
            CK(psr::dev_alloc(&first, sizeof(int32_t)));
            // FP64 pairs, p > 32: the inverses go straight into the streamed
            // sweep's layout (the sweep layout finds the group streamed)
            const bool fused = op.store_prec == PSR_PREC_FP64 && op.fp64_arith == PSR_FP64_PAIRS;
            GpuSpan span;                          // the inverses' GPU time (stats.t_invert)
            for (auto& G : ctx->groups) {
                double* base = ctx->A_ext + G.mat_off;
                if (fused && G.p > 32) {
                    const size_t ne = (size_t)G.count * G.p * G.p;
                    float2* dst = nullptr;
                    if (psr::dev_alloc(&dst, sizeof(float2) * std::max<size_t>(ne, 1)) != cudaSuccess) {
                        cudaGetLastError();
                        psr::dev_free(sing);
                        psr::dev_free(first);
                        set_error(ctx, "out of device memory for the streamed inverses");
                        FAIL(PSR_ERR_OOM);
                    }
                    CK(psr::dev_alloc(&G.bexp, sizeof(int32_t) * (size_t)std::max(G.count, 1)));
                    span.begin(s);
                    rc = launch_batched_inverse_pairs(base, G.count, G.p, dst, G.bexp, sing, s);
                    span.end(s);
                    G.stream = true;
                    G.rinv = dst;
                } else {
                    span.begin(s);
                    rc = launch_batched_inverse(base, (int64_t)G.p * G.p, nullptr, G.count, G.p, base,
                                                (int64_t)G.p * G.p, sing, s);
                    span.end(s);
                    G.rinv = base;
                }
                if (rc != PSR_OK) { psr::dev_free(sing); psr::dev_free(first); goto fail; }
                int32_t big = 0x7fffffff;
                CK(cudaMemcpyAsync(first, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
                count_launch(); k_any<<<std::max(1, std::min(G.count / 256 + 1, 1024)), 256, 0, s>>>(sing, G.count, first);
                int32_t h_first = 0;
                CK(cudaMemcpyAsync(&h_first, first, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                ctx->stats.t_invert += span.seconds();
                G.m = G.count;
                CK(psr::dev_alloc(&G.sphi, sizeof(int32_t) * (size_t)G.count));
                count_launch(); k_iota<<<std::max(1, std::min(G.count / 256 + 1, 1024)), 256, 0, s>>>(G.sphi, G.count);
                G.h_rep.resize(G.count);
                for (int l = 0; l < G.count; ++l) G.h_rep[l] = l;
                if (h_first != 0x7fffffff && ctx->stats.first_singular < 0) ctx->stats.first_singular = gidx[&G - &ctx->groups[0]][h_first];
            }
            psr::dev_free(sing);
            psr::dev_free(first);
            ctx->stats.rounds = 0;
            ctx->stats.criterion_evals = 0;
        } else if (op.criterion == PSR_CRITERION_L1) {
            if (m0 > 0 || hints) { set_error(ctx, "the l1 criterion takes no seed database or hints"); FAIL(PSR_ERR_INVALID_ARG); }
            if (op.search != PSR_SEARCH_CREATION) {
                set_error(ctx, "the norm-window search is for the spectral criterion");
                FAIL(PSR_ERR_INVALID_ARG);
            }
            rc = run_alg1_l1(ctx, s);
            if (rc != PSR_OK) goto fail;
        } else {
            int32_t* pred = nullptr;
            if (mode.mlp) {
                // learned assignment: the network's entry for every patch becomes its hint
                const Group& G0 = ctx->groups[0];
                const int d = G0.p * G0.p + 2;
                float* X = nullptr;
                CK(psr::dev_alloc(&pred, sizeof(int32_t) * (size_t)np));
                const float* feat = mode.features;
                if (!feat) {
                    CK(psr::dev_alloc(&X, sizeof(float) * (size_t)np * d));
                    rc = psr_features(ctx->A_ext + G0.mat_off, np, G0.p, nullptr, X, s);
                    if (rc != PSR_OK) { psr::dev_free(X); psr::dev_free(pred); goto fail; }
                    feat = X;
                }
                rc = psr_mlp_predict(mode.mlp, feat, np, pred, nullptr, s);
                CK(cudaStreamSynchronize(s));
                psr::dev_free(X);
                if (rc != PSR_OK) { psr::dev_free(pred); goto fail; }
                hints = pred;
            }
            rc = run_alg1(ctx, s, seed_A, m0, hints);
            psr::dev_free(pred);
            if (rc != PSR_OK) goto fail;
        }
        CK(cudaStreamSynchronize(s));
        ctx->stats.t_rounds = seconds_since(t0);
        phase_end();
        if (ctx->stats.first_singular >= 0) {
            set_error(ctx, "patch " + std::to_string(ctx->stats.first_singular) +
                           " failed the pivot test |u_kk| <= p * 2^-53 * max|A_k| (singular)");
            FAIL(PSR_ERR_SINGULAR_PATCH);
        }
        phase_begin("psr_setup: storage and sweep layout");
        t0 = std::chrono::steady_clock::now();
        rc = build_sweep_layout(ctx, gidx, s);
        if (rc != PSR_OK) goto fail;
        rc = sweep_prepare(ctx);
        if (rc != PSR_OK) goto fail;
        ctx->stats.t_convert = seconds_since(t0);
        phase_end();
        // the patch matrices are no longer needed unless they hold the inverses
        {
            bool in_use = false;
            for (auto& G : ctx->groups)
                if (reinterpret_cast<double*>(G.rinv) >= ctx->A_ext &&
                    reinterpret_cast<double*>(G.rinv) < ctx->A_ext + std::max<int64_t>(ctx->A_ext_len, 1))
                    in_use = true;
            if (!in_use) {
                psr::dev_free(ctx->A_ext);
                ctx->A_ext = nullptr;
                ctx->A_ext_len = 0;
            }
        }
        rc = krylov_alloc(ctx, s);
        if (rc != PSR_OK) goto fail;
        phase_begin("psr_setup: sweep autotuner");
        t0 = std::chrono::steady_clock::now();
        rc = autotune_sweep(ctx, s);
        if (rc != PSR_OK) goto fail;
        CK(cudaStreamSynchronize(s));
        ctx->stats.t_autotune = seconds_since(t0);
        phase_end();
        ctx->stats.n = n;
        ctx->stats.n_patches = np;
        ctx->stats.n_groups = (int)ctx->groups.size();
        (void)t_all;
        *out = ctx;
        phases_close(nvtx_base);
        scope.commit();
        return PSR_OK;
    }
fail:
    destroy_ctx(ctx);
    phases_close(nvtx_base);
    return rc;
#undef FAIL
#undef CK
}

}  // namespace psr

using namespace psr;

extern "C" {

void psr_default_opts(psr_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 0.0;
    o->store_prec = PSR_PREC_FP64;
    o->weighting = PSR_WEIGHT_SYM;
    o->krylov = PSR_KRYLOV_CG;
    o->restart = 30;
    o->rtol = 1e-8;
    o->maxit = 10000;
    o->use_graph = 1;
    o->sweep_kernel = PSR_SWEEP_AUTO;
    o->autotune = 1;
    o->symmetrize = 1;
    o->use_mlp = 0;
    o->ortho = PSR_ORTHO_AUTO;
    o->criterion = PSR_CRITERION_SPECTRAL;
    o->fp64_arith = PSR_FP64_PAIRS;
    o->match = PSR_MATCH_FIRST;
    o->seed = 0;
    o->prec_check = 0.5;
    o->search = PSR_SEARCH_CREATION;
}

int psr_setup(const psr_csr* A, const psr_patches* patches, const psr_opts* opts, void* stream, psr_ctx** out) {
    if (!out) { set_error(nullptr, "out is NULL"); return PSR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!A || !patches || !A->rowptr || !A->vals || !A->colidx || A->n <= 0 || A->nnz < 0 ||
        patches->n_patches <= 0 || !patches->dofs || (patches->uniform_size <= 0 && !patches->offsets)) {
        set_error(nullptr, "invalid matrix or patch description");
        return PSR_ERR_INVALID_ARG;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        set_error(nullptr, "no CUDA device: the library has no CPU fallback");
        return PSR_ERR_CUDA;
    }
    try {
        return setup_impl(A, patches, opts, (cudaStream_t)stream, out, AssignMode{});
    } catch (const std::bad_alloc&) {
        set_error(nullptr, "host allocation failed");
        return PSR_ERR_OOM;
    } catch (...) {
        set_error(nullptr, "unexpected host exception in psr_setup");
        return PSR_ERR_CUDA;
    }
}

int psr_setup_seeded(const psr_csr* A, const psr_patches* patches, const psr_opts* opts, const double* seed_A,
                     int32_t m0, const int32_t* hints, void* stream, psr_ctx** out) {
    if (!out) { set_error(nullptr, "out is NULL"); return PSR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!A || !patches || !A->rowptr || !A->vals || !A->colidx || A->n <= 0 || patches->n_patches <= 0 ||
        !patches->dofs || patches->uniform_size <= 0 || patches->uniform_size > 32 || m0 < 0 ||
        (m0 > 0 && !seed_A) || (hints && m0 == 0)) {
        set_error(nullptr, "invalid seeded setup arguments (uniform patches of at most 32 DOFs, m0 >= 0)");
        return PSR_ERR_INVALID_ARG;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        set_error(nullptr, "no CUDA device: the library has no CPU fallback");
        return PSR_ERR_CUDA;
    }
    psr_opts o;
    if (opts) o = *opts; else psr_default_opts(&o);
    if (!(o.tol > 0.0)) { set_error(nullptr, "a seeded setup needs tol > 0"); return PSR_ERR_INVALID_ARG; }
    try {
        AssignMode mode;
        mode.seed_A = seed_A;
        mode.m0 = m0;
        mode.hints = hints;
        return setup_impl(A, patches, &o, (cudaStream_t)stream, out, mode);
    } catch (...) {
        set_error(nullptr, "unexpected host exception in psr_setup_seeded");
        return PSR_ERR_CUDA;
    }
}

int psr_setup_learned(const psr_csr* A, const psr_patches* patches, const psr_opts* opts, const psr_ctx* trained,
                      const float* features, void* stream, psr_ctx** out) {
    if (!out) { set_error(nullptr, "out is NULL"); return PSR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!trained || trained->groups.size() != 1 || !trained->groups[0].dbA || trained->m_p < 1) {
        set_error(nullptr, "psr_setup_learned needs a trained context with a one-size database");
        return PSR_ERR_INVALID_ARG;
    }
    const int p = trained->groups[0].p;
    if (!A || !patches || !A->rowptr || !A->vals || !A->colidx || A->n <= 0 || patches->n_patches <= 0 ||
        !patches->dofs || patches->uniform_size != p || p > 32) {
        set_error(nullptr, "psr_setup_learned: uniform patches of the trained context's size (at most 32 DOFs)");
        return PSR_ERR_INVALID_ARG;
    }
    psr_opts o;
    if (opts) o = *opts; else psr_default_opts(&o);
    if (!(o.tol > 0.0)) { set_error(nullptr, "a learned setup needs tol > 0"); return PSR_ERR_INVALID_ARG; }
    if (o.use_mlp && (!trained->mlp || trained->mlp_classes != trained->m_p)) {
        set_error(nullptr, "use_mlp: the trained context has no network for its database (psr_mlp_train)");
        return PSR_ERR_INVALID_ARG;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        set_error(nullptr, "no CUDA device: the library has no CPU fallback");
        return PSR_ERR_CUDA;
    }
    try {
        AssignMode mode;
        mode.seed_A = trained->groups[0].dbA;
        mode.m0 = trained->m_p;
        if (o.use_mlp) {
            mode.mlp = trained->mlp;
            mode.features = features;
        }
        return setup_impl(A, patches, &o, (cudaStream_t)stream, out, mode);
    } catch (...) {
        set_error(nullptr, "unexpected host exception in psr_setup_learned");
        return PSR_ERR_CUDA;
    }
}

int psr_setup_kmeans(const psr_csr* A, const psr_patches* patches, const psr_opts* opts, int32_t m_p,
                     const int32_t* init, int32_t max_iter, const int32_t* patch_class, void* stream,
                     psr_ctx** out) {
    if (!out) { set_error(nullptr, "out is NULL"); return PSR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!A || !patches || !A->rowptr || !A->vals || !A->colidx || A->n <= 0 || patches->n_patches <= 0 ||
        !patches->dofs || patches->uniform_size <= 0 || patches->uniform_size > 128 || m_p < 1 ||
        m_p > patches->n_patches || !init || max_iter < 1) {
        set_error(nullptr, "invalid k-means setup arguments (uniform patches of at most 128 DOFs, 1 <= m_p <= n_patches, max_iter >= 1)");
        return PSR_ERR_INVALID_ARG;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
        cudaGetLastError();
        set_error(nullptr, "no CUDA device: the library has no CPU fallback");
        return PSR_ERR_CUDA;
    }
    try {
        std::vector<int32_t> h_init((size_t)m_p);
        cudaError_t e = cudaMemcpy(h_init.data(), init, sizeof(int32_t) * (size_t)m_p, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "k-means seeds");
        std::vector<char> seen((size_t)patches->n_patches, 0);
        for (int32_t v : h_init) {
            if (v < 0 || v >= patches->n_patches || seen[(size_t)v]) {
                set_error(nullptr, "k-means seeds must be distinct patch indices in [0, n_patches)");
                return PSR_ERR_INVALID_ARG;
            }
            seen[(size_t)v] = 1;
        }
        // boundary partition: every class needs at least one seed
        std::vector<int32_t> h_cls;
        if (patch_class) {
            h_cls.resize((size_t)patches->n_patches);
            e = cudaMemcpy(h_cls.data(), patch_class, sizeof(int32_t) * h_cls.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "k-means patch classes");
            int32_t cmax = -1;
            for (int32_t c : h_cls) {
                if (c < 0 || c >= patches->n_patches) {
                    set_error(nullptr, "patch classes must lie in [0, n_patches)");
                    return PSR_ERR_INVALID_ARG;
                }
                cmax = std::max(cmax, c);
            }
            std::vector<char> has((size_t)cmax + 1, 0), used((size_t)cmax + 1, 0);
            for (int32_t c : h_cls) used[(size_t)c] = 1;
            for (int32_t v : h_init) has[(size_t)h_cls[(size_t)v]] = 1;
            for (int32_t c = 0; c <= cmax; ++c)
                if (used[(size_t)c] && !has[(size_t)c]) {
                    set_error(nullptr, "patch class " + std::to_string(c) + " has no k-means seed");
                    return PSR_ERR_INVALID_ARG;
                }
        }
        psr_opts o;
        if (opts) o = *opts; else psr_default_opts(&o);
        AssignMode mode;
        mode.km_m = m_p;
        mode.km_init = &h_init;
        mode.km_iter = max_iter;
        mode.km_cls = patch_class ? &h_cls : nullptr;
        return setup_impl(A, patches, &o, (cudaStream_t)stream, out, mode);
    } catch (const std::bad_alloc&) {
        set_error(nullptr, "host allocation failed");
        return PSR_ERR_OOM;
    } catch (...) {
        set_error(nullptr, "unexpected host exception in psr_setup_kmeans");
        return PSR_ERR_CUDA;
    }
}

int psr_apply(psr_ctx* ctx, const double* r, double* z, void* stream) {
    if (!ctx || !r || !z) { set_error(ctx, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    if (r == z) { set_error(ctx, "r and z must not overlap"); return PSR_ERR_INVALID_ARG; }
    return sweep_apply(ctx, r, z, (cudaStream_t)stream);
}

int psr_solve(psr_ctx* ctx, const double* b, double* x, void* stream, psr_solve_info* info) {
    if (!ctx || !b || !x) { set_error(ctx, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    try {
        return krylov_solve(ctx, b, x, (cudaStream_t)stream, info);
    } catch (...) {
        set_error(ctx, "unexpected host exception in psr_solve");
        return PSR_ERR_CUDA;
    }
}

int psr_get_history(psr_ctx* ctx, double* hist, int32_t cap, int32_t* len) {
    if (!ctx || !len) { set_error(ctx, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    const int32_t L = (int32_t)ctx->h_hist.size();
    *len = L;
    if (hist) std::memcpy(hist, ctx->h_hist.data(), sizeof(double) * (size_t)std::min(L, cap));
    return PSR_OK;
}

int psr_get_assignment(psr_ctx* ctx, int32_t* phi, int32_t* rep_ids, int32_t* m_p) {
    if (!ctx) { set_error(nullptr, "NULL context"); return PSR_ERR_INVALID_ARG; }
    if (m_p) *m_p = ctx->m_p;
    if (phi) PSR_CUDA(ctx, cudaMemcpy(phi, ctx->phi, sizeof(int32_t) * (size_t)ctx->n_patches, cudaMemcpyDeviceToDevice));
    if (rep_ids && ctx->m_p > 0)
        PSR_CUDA(ctx, cudaMemcpy(rep_ids, ctx->rep_ids, sizeof(int32_t) * (size_t)ctx->m_p, cudaMemcpyDeviceToDevice));
    return PSR_OK;
}

int psr_export_database(psr_ctx* ctx, double* entries, void* stream) {
    if (!ctx || !entries) { set_error(ctx, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    if (ctx->groups.size() != 1 || !ctx->groups[0].dbA) {
        set_error(ctx, "no database copy: export needs one patch size and an Alg. 1, seeded or Alg. 2 setup");
        return PSR_ERR_INVALID_ARG;
    }
    const Group& G = ctx->groups[0];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PSR_CUDA(ctx, cudaMemcpyAsync(entries, G.dbA, sizeof(double) * (size_t)G.m * G.p * G.p, cudaMemcpyDeviceToDevice, s));
    PSR_CUDA(ctx, cudaStreamSynchronize(s));
    return PSR_OK;
}

int psr_get_stats(psr_ctx* ctx, psr_stats* st) {
    if (!ctx || !st) { set_error(ctx, "NULL argument"); return PSR_ERR_INVALID_ARG; }
    *st = ctx->stats;
    return PSR_OK;
}

const char* psr_last_error(psr_ctx* ctx) {
    if (ctx && !ctx->err.empty()) return ctx->err.c_str();
    return g_last_error.c_str();
}

void psr_destroy(psr_ctx* ctx) { destroy_ctx(ctx); }

int64_t psr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int psr_set_kernel_timing(psr_ctx* ctx, int enable) {
    if (!ctx) {
        set_error(nullptr, "ctx is NULL");
        return PSR_ERR_INVALID_ARG;
    }
    return kernel_timing_enable(ctx, enable != 0);
}

int psr_get_kernel_timing(psr_ctx* ctx, double* ms, int64_t* launches, double* bytes, double* flops, int count) {
    if (!ctx || count < 1 || count > PSR_KT_COUNT) {
        set_error(ctx, "ctx is NULL or count outside 1 .. PSR_KT_COUNT");
        return PSR_ERR_INVALID_ARG;
    }
    for (int k = 0; k < count; ++k) {
        if (ms) ms[k] = ctx->kt_ms[k];
        if (launches) launches[k] = ctx->kt_n[k];
        if (bytes) bytes[k] = ctx->kt_bytes[k];
        if (flops) flops[k] = ctx->kt_flops[k];
    }
    return PSR_OK;
}

int psr_extract(const psr_csr* A, const psr_patches* P, double* A_out, int32_t* mult_out, double* W_out, void* stream) {
    if (!A || !P || A->n <= 0 || P->n_patches <= 0 || !P->dofs || (P->uniform_size <= 0 && !P->offsets)) {
        set_error(nullptr, "invalid matrix or patch description");
        return PSR_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int np = P->n_patches;
    std::vector<int32_t> ho((size_t)np + 1);
    if (P->uniform_size > 0) {
        for (int k = 0; k <= np; ++k) ho[k] = k * P->uniform_size;
    } else {
        PSR_CUDA(nullptr, cudaMemcpyAsync(ho.data(), P->offsets, sizeof(int32_t) * (size_t)(np + 1), cudaMemcpyDeviceToHost, s));
        PSR_CUDA(nullptr, cudaStreamSynchronize(s));
    }
    const int64_t total = ho[np];
    int32_t* status = nullptr;
    PSR_CUDA(nullptr, psr::dev_alloc(&status, sizeof(int32_t)));
    PSR_CUDA(nullptr, cudaMemsetAsync(status, 0, sizeof(int32_t), s));
    int rc = validate_inputs(nullptr, A, P->uniform_size > 0 ? nullptr : P->offsets, P->dofs, np, total, status, s);
    int32_t st = 0;
    if (rc == PSR_OK) {
        cudaMemcpyAsync(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (st & ST_UNSORTED) rc = PSR_ERR_UNSORTED_CSR;
        else if (st & ST_OOB) rc = PSR_ERR_INVALID_ARG;
        if (rc != PSR_OK) set_error(nullptr, "invalid CSR or patch map");
    }
    int64_t* mo = nullptr;
    if (rc == PSR_OK && A_out) {
        if (P->uniform_size > 0) {
            rc = launch_extract(A->rowptr, A->colidx, A->vals, nullptr, P->dofs, nullptr, np, P->uniform_size, total, A_out, s);
        } else {
            std::vector<int64_t> hm((size_t)np + 1, 0);
            for (int k = 0; k < np; ++k) {
                const int64_t pk = ho[k + 1] - ho[k];
                hm[k + 1] = hm[k] + pk * pk;
            }
            if (psr::dev_alloc(&mo, sizeof(int64_t) * (size_t)(np + 1)) != cudaSuccess) rc = PSR_ERR_OOM;
            else {
                cudaMemcpyAsync(mo, hm.data(), sizeof(int64_t) * (size_t)(np + 1), cudaMemcpyHostToDevice, s);
                rc = launch_extract(A->rowptr, A->colidx, A->vals, P->offsets, P->dofs, mo, np, 0, total, A_out, s);
            }
        }
    }
    if (rc == PSR_OK && (mult_out || W_out)) {
        int32_t* mult = mult_out;
        if (!mult && psr::dev_alloc(&mult, sizeof(int32_t) * (size_t)A->n) != cudaSuccess) rc = PSR_ERR_OOM;
        if (rc == PSR_OK) rc = launch_multiplicity(P->dofs, total, A->n, mult, W_out, nullptr, status, s);
        if (rc == PSR_OK && W_out) {
            cudaMemcpyAsync(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            if (st & ST_UNCOVERED) { rc = PSR_ERR_UNCOVERED_DOF; set_error(nullptr, "a DOF belongs to no patch"); }
        }
        if (mult && !mult_out) { cudaStreamSynchronize(s); psr::dev_free(mult); }
    }
    cudaStreamSynchronize(s);
    psr::dev_free(mo);
    psr::dev_free(status);
    return rc;
}

int psr_batched_inverse(const double* A, int32_t batch, int32_t p, double* Ainv, int32_t* singular, void* stream) {
    if (!A || !Ainv || batch < 0 || p < 1 || p > 128) { set_error(nullptr, "invalid batched inverse arguments"); return PSR_ERR_INVALID_ARG; }
    return launch_batched_inverse(A, (int64_t)p * p, nullptr, batch, p, Ainv, (int64_t)p * p, singular, (cudaStream_t)stream);
}

int psr_criterion(const double* A_i, int32_t batch, int32_t p, const double* A_c, const double* Binv_c, double tol,
                  int32_t* accept, double* dval, void* stream) {
    if (!A_i || !A_c || !Binv_c || !accept || batch < 0 || p < 1 || p > 128 || !(tol >= 0.0)) {
        set_error(nullptr, "invalid criterion arguments");
        return PSR_ERR_INVALID_ARG;
    }
    if (batch == 0) return PSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (p > 32) return launch_criterion_big(A_i, batch, p, A_c, Binv_c, tol, accept, dval, s);
    int32_t* work = nullptr;
    PSR_CUDA(nullptr, cudaMallocAsync((void**)&work, sizeof(int32_t) * ((size_t)batch + 1), s));
    int rc = launch_criterion_batch(A_i, batch, p, A_c, Binv_c, tol, accept, dval, work, s);
    cudaFreeAsync(work, s);
    return rc;
}

int psr_debug_inject(int32_t what, int64_t value) {
    if (value < 0) { set_error(nullptr, "psr_debug_inject: negative value"); return PSR_ERR_INVALID_ARG; }
    if (what == PSR_INJECT_ALLOC_FAIL) {
        inject_alloc_fail((long long)value);
        return PSR_OK;
    }
    if (what == PSR_INJECT_BARRIER_WAIT) {
        int dev_count = 0;
        if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
            cudaGetLastError();
            set_error(nullptr, "no CUDA device");
            return PSR_ERR_CUDA;
        }
        return inject_barrier_wait((long long)value);
    }
    if (what == PSR_INJECT_ROUNDS_SPLIT) {
        inject_rounds_split(value != 0);
        return PSR_OK;
    }
    set_error(nullptr, "psr_debug_inject: unknown kind");
    return PSR_ERR_INVALID_ARG;
}

int psr_spectral_norm(const double* E, int32_t batch, int32_t p, double* sigma, void* stream) {
    if (!E || !sigma || batch < 0 || p < 1 || p > 32) { set_error(nullptr, "invalid spectral norm arguments"); return PSR_ERR_INVALID_ARG; }
    if (batch == 0) return PSR_OK;
    return launch_spectral_norm(E, batch, p, sigma, (cudaStream_t)stream);
}

}  // extern "C"
