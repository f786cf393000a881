// Internal declarations shared by the CUDA translation units of the
// compressed patch-relaxation library (Harper & Tuminaro, arXiv 2306.10025).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/psr.h"

namespace psr {

// ---------------------------------------------------------------- errors
void set_error(psr_ctx* ctx, const std::string& msg);
int cuda_fail(psr_ctx* ctx, cudaError_t e, const char* what);

// Kernel-launch instrumentation: every host launch site calls count_launch();
// graph launches add the number of kernel nodes; nothing is counted while a
// stream is being captured (set_capturing).
void count_launch(long long k = 1);
void set_capturing(bool on);

#define PSR_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return psr::cuda_fail((ctx), e_, #call); \
    } while (0)

#define PSR_CHECK_LAUNCH(ctx, what)                           \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) return psr::cuda_fail((ctx), e_, what); \
    } while (0)

// GPU time of a launch sequence on one stream (two CUDA events): begin() and
// end() around the launches, seconds() once the stream has been synchronised.
struct GpuSpan {
    cudaEvent_t a = nullptr, b = nullptr;
    GpuSpan() {
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) cudaGetLastError();
    }
    ~GpuSpan() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    GpuSpan(const GpuSpan&) = delete;
    GpuSpan& operator=(const GpuSpan&) = delete;
    void begin(cudaStream_t s) { if (a) cudaEventRecord(a, s); }
    void end(cudaStream_t s) { if (b) cudaEventRecord(b, s); }
    double seconds() const {
        float ms = 0.f;
        if (!a || !b || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            cudaGetLastError();
            return 0.0;
        }
        return ms * 1e-3;
    }
};

// Device and pinned host memory of the library go through a caching
// allocator (memory.cu): freed blocks are kept and handed out again, after a
// device synchronisation when they were freed since the last one.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
cudaError_t host_alloc(void** p, size_t bytes);
cudaError_t host_free(void* p);
void inject_alloc_fail(long long k);      // psr_debug_inject(PSR_INJECT_ALLOC_FAIL, k)
int inject_barrier_wait(long long spins); // criterion.cu
void inject_rounds_split(bool on);        // criterion.cu: psr_debug_inject(PSR_INJECT_ROUNDS_SPLIT, 1)
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) { return dev_alloc(reinterpret_cast<void**>(p), bytes); }
template <class T>
inline cudaError_t host_alloc(T** p, size_t bytes) { return host_alloc(reinterpret_cast<void**>(p), bytes); }

// Blocks handed out on this thread while an AllocScope is open are recorded
// in it and a free removes them; a scope that ends without commit() frees
// the blocks it still holds (the locals of a call that failed part-way), a
// committed one passes them to the enclosing scope.  AllocPause stops the
// recording for buffers of objects that outlive the call (a network's
// activations grown during a setup).
class AllocScope {
public:
    AllocScope();
    ~AllocScope();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;
    void commit() { committed_ = true; }
private:
    std::unordered_map<void*, bool> held_;   // block -> pinned host (else device)
    std::unordered_map<void*, bool>* prev_;
    bool committed_ = false;
};
class AllocPause {
public:
    AllocPause();
    ~AllocPause();
    AllocPause(const AllocPause&) = delete;
    AllocPause& operator=(const AllocPause&) = delete;
private:
    std::unordered_map<void*, bool>* prev_;
};

// ------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Norm window of Alg. 1's sorted search (section 3.1, after Alg. 1).  Since
// d(A_i, B_c) = ||(A_c - A_i) B_c^-1||_2 >= ||A_c - A_i||_2 / ||A_c||_2 >=
// | ||A_c||_2 - ||A_i||_2 | / ||A_c||_2, entry c can pass only when
// ||A_i|| / (1 + tol) < ||A_c|| < ||A_i|| / (1 - tol); the window is widened
// by 1e-12 (relative) against rounding.  With ||A_i|| known as a bracket
// [alo, ahi], the window spans every value in it; an entry whose own bracket
// [klo, khi] lies wholly outside is skipped: neither tested nor counted.
// The window is computed once per patch; the per-pair test compares the bit
// patterns of the (non-negative, non-NaN) bounds as integers, which order
// like the values and keep the test off the GPU's narrow FP64 pipe.
struct NormWin {
    double lo, hi;
};
__device__ __forceinline__ NormWin norm_window(double alo, double ahi, double tol) {
    NormWin w;
    w.lo = __dmul_rn(__ddiv_rn(alo, 1.0 + tol), 1.0 - 1e-12);
    w.hi = tol < 1.0 ? __dmul_rn(__ddiv_rn(ahi, 1.0 - tol), 1.0 + 1e-12)
                     : __longlong_as_double(0x7ff0000000000000ll);
    return w;
}
__device__ __forceinline__ bool outside_window(const NormWin& w, double klo, double khi) {
    return __double_as_longlong(khi) < __double_as_longlong(w.lo) ||
           __double_as_longlong(klo) > __double_as_longlong(w.hi);
}
// A bracket [lo, hi] of a 2-norm made safe for outside_window: a NaN bound
// (a non-finite patch) becomes the bracket [0, inf], never outside.
__device__ __forceinline__ void sanitize_bracket(double* lo, double* hi) {
    if (!(*lo >= 0.0) || !(*hi >= 0.0)) {
        *lo = 0.0;
        *hi = __longlong_as_double(0x7ff0000000000000ll);
    }
}

// Device-side status word bits (written by kernels, read by the host).
enum : int {
    ST_UNSORTED = 1,
    ST_OOB = 2,
    ST_UNCOVERED = 4,
    ST_SINGULAR = 8,
    ST_NAN = 16,
    ST_HASH = 32,       // patch detection: two column sets with one hash
};

// ------------------------------------------------------------ size group
// Patches of one size p (Remark after Eq. 1: groups of equal size are handled
// independently).  Patches inside a group are ordered by database entry
// (stable), so a tile of consecutive patches shares one inverse.
struct Group {
    int p = 0;
    int count = 0;                 // patches in the group
    int m = 0;                     // database entries of this size
    int32_t* patch = nullptr;      // [count] global patch index, sorted by entry
    int32_t* sdofs = nullptr;      // [count * p] DOFs in sorted order
    int32_t* sphi = nullptr;       // [count] group-local entry of each sorted patch
    void* rinv = nullptr;          // [m * p * p] inverses in storage precision
    double* dbA = nullptr;         // [m * p * p] patch matrix of each entry (Alg. 1 / seeded / Alg. 2), for reuse
    int64_t mat_off = 0;           // offset of the group's patches in A_ext (doubles)
    // tiles: (entry, first sorted patch, count)
    int32_t* tiles = nullptr;      // [ntiles * 3]
    int ntiles = 0;
    int tile_patches = 32;         // chosen by the autotuner
    int warps = 4;
    bool tc = false;               // BF16 entries applied on the tensor cores
    bool tpp = false;              // clustered p <= 32: one patch per thread
    bool stream = false;           // every patch its own entry: column-major inverses streamed
                                   // by k_sweep_stream (thread per row)
    int32_t* bexp = nullptr;       // [m] power-of-two scale of each entry (FP64 pairs only)
    void* rinv_pair = nullptr;     // [m * p * p] clustered FP64 entries as scaled (hi, lo) FP32
                                   // pairs, column-major (thread-per-patch kernel on pairs)
    // entries whose rounded inverse failed the precision check (psr_opts.prec_check):
    // their tiles run separately on an FP64 copy of the database
    std::vector<char> h_hi;        // [m] 1 = entry applied in FP64
    double* rinv_hi = nullptr;     // [m * p * p] FP64 inverses (read for the flagged entries)
    int32_t* tiles_hi = nullptr;   // [ntiles_hi * 3] tiles of the flagged entries
    int ntiles_hi = 0;
    int32_t* sdofs_t = nullptr;    // [p * count] DOFs, local-DOF major (tpp kernel)
    int32_t* wtiles = nullptr;     // [nwt * 3] warp tiles (entry, first, count <= 32)
    int nwt = 0;
    std::vector<int> h_rep;        // local patch of each entry (-1: seed entry)
    std::vector<int32_t> h_gidx;   // global patch index of each local patch
    std::vector<int32_t> h_sorted_phi;  // entry of each patch in sweep order
};

struct KrylovWS {
    double* x = nullptr;   // iterate
    double* b = nullptr;   // right-hand side copy
    double* r = nullptr;
    double* z = nullptr;
    double* p = nullptr;
    double* q = nullptr;
    double* V = nullptr;   // FGMRES basis (m+1) x n
    double* Z = nullptr;   // FGMRES preconditioned basis m x n
    double* partial = nullptr;  // reduction partials
    double* scal = nullptr;     // device scalars (see krylov.cu)
    double* hist = nullptr;     // [maxit + 1]
    int32_t* ictl = nullptr;    // device control ints
    int32_t* rflag = nullptr;   // [64] FGMRES: second Gram-Schmidt pass taken at step j
    double* part_arn = nullptr; // partials of the fused Arnoldi step, 4 regions x 33 x sms
    float2* Vs = nullptr;       // pair copy (hi, lo FP32) of the FGMRES basis, (m+1) x n, fused step only
    unsigned int* bar = nullptr;  // grid barrier of the fused Arnoldi step (count, generation)
    bool coop = false;          // fused Arnoldi step (cooperative launch) available
    int64_t* sell_ptr = nullptr;  // SELL-32 copy of A: slice offsets [nslices + 1]
    int32_t* sell_cols = nullptr;
    double* sell_vals = nullptr;
    int32_t* sell_row = nullptr;  // padded SELL row -> row of A (-1: none), or null when rows are in order
    int nslices = 0;
    int nblk = 0;
    int nspmv = 0;
    int sms = 0;           // streaming multiprocessors of the device
};

// One timed launch of the solve: class, iteration inside the enqueued block
// (the launch did work iff the block ran more than j iterations) and its
// algorithmic bytes.  Events 2i and 2i+1 of psr_ctx::kt_ev bracket mark i.
struct KtMark {
    int kind;
    int j;
    double bytes;
    double bytes_reorth;   // added when step j took the second Gram-Schmidt pass
    double flops;          // algorithmic FP64 flops
    double flops_reorth;
};

}  // namespace psr

namespace psr {
struct Coarse;
}

struct psr_ctx {
    int device = 0;
    psr_opts opts{};
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t *rowptr = nullptr, *colidx = nullptr;
    double* vals = nullptr;
    int32_t n_patches = 0;
    int32_t* offsets = nullptr;   // device n_patches+1
    int32_t* dofs = nullptr;      // device flat
    std::vector<int32_t> h_offsets;
    int64_t* mat_off = nullptr;   // device n_patches+1 (offset of A_k in A_ext)
    double* A_ext = nullptr;      // extracted patches, FP64
    int64_t A_ext_len = 0;
    double* W = nullptr;          // scale applied at the scatter
    double* Wg = nullptr;         // scale applied at the gather (SYM) or nullptr
    int32_t* phi = nullptr;       // device n_patches
    int32_t* rep_ids = nullptr;   // device n_patches + seed entries (first m_p used)
    int32_t m_p = 0;
    std::vector<int32_t> h_rep_ids;
    std::vector<psr::Group> groups;
    int32_t* status = nullptr;    // device status word
    psr::KrylovWS ws;
    std::vector<double> h_hist;
    int32_t last_iters = 0;
    psr_stats stats{};
    std::string err;
    // graphs
    cudaGraphExec_t g_cycle = nullptr;   // one FGMRES cycle / CG block
    psr::Coarse* coarse = nullptr;       // two-level term of Eq. (2), psr_set_coarse
    cudaStream_t g_stream = nullptr;
    int graph_block = 0;
    // grouped persistent sweep
    int32_t* gtiles = nullptr;    // all tiles of all groups: (group, entry, start, count)
    int gntiles = 0;
    void* gdesc = nullptr;        // device group descriptors
    int32_t* gcounter = nullptr;  // work counter for the persistent sweep
    int sweep_mode = PSR_SWEEP_PERGROUP;
    int grouped_blocks = 0;
    // streaming sweep of the full-storage groups (one launch over all of them)
    void* sdesc = nullptr;        // device StreamDesc per streamed group
    int n_stream = 0;             // streamed groups
    int stream_rb = 0;            // 32-row blocks over all streamed groups
    int stream_blocks = 0;        // grid of k_sweep_stream (autotuned)
    // per-kernel timing of the solve (psr_set_kernel_timing)
    bool kt_on = false;
    std::vector<cudaEvent_t> kt_ev;       // two per mark
    std::vector<psr::KtMark> kt_marks;    // marks of the enqueued block / captured graph
    double kt_ms[PSR_KT_COUNT] = {};
    int64_t kt_n[PSR_KT_COUNT] = {};
    double kt_bytes[PSR_KT_COUNT] = {};
    double kt_flops[PSR_KT_COUNT] = {};
    // learned assignment: network trained on this setup (psr_mlp_train)
    psr_mlp* mlp = nullptr;
    int32_t mlp_classes = 0;      // its output width (the m_p it was trained for)
};

namespace psr {

// extract.cu
int validate_inputs(psr_ctx* ctx, const psr_csr* A, const int32_t* offsets, const int32_t* dofs,
                    int32_t n_patches, int64_t total_dofs, int32_t* status, cudaStream_t s);
int launch_extract(const int32_t* rowptr, const int32_t* colidx, const double* vals,
                   const int32_t* offsets, const int32_t* dofs, const int64_t* mat_off,
                   int32_t n_patches, int32_t pmax, int64_t total, double* A_out, cudaStream_t s);
int launch_multiplicity(const int32_t* dofs, int64_t total, int32_t n, int32_t* mult,
                        double* W, double* sqrtW, int32_t* status, cudaStream_t s);

// inverse.cu
int launch_batched_inverse(const double* A, int64_t stride_in, const int32_t* index,
                           int32_t batch, int32_t p, double* Ainv, int64_t stride_out,
                           int32_t* singular, cudaStream_t s);
// 33 <= p <= 128: inverses written in the streamed sweep's FP64-pair layout
// (column-major scaled (hi, lo) pairs and their exponents), no FP64 copy
int launch_batched_inverse_pairs(const double* A, int32_t batch, int32_t p, float2* pout, int32_t* pexp,
                                 int32_t* singular, cudaStream_t s);

// criterion.cu
struct RoundState;
int run_alg1(psr_ctx* ctx, cudaStream_t s, const double* seed_A, int m0, const int32_t* hints);
int launch_criterion_batch(const double* A_i, int32_t batch, int32_t p, const double* A_c,
                           const double* Binv_c, double tol, int32_t* accept, double* dval,
                           int32_t* work, cudaStream_t s);
int launch_spectral_norm(const double* E, int32_t batch, int32_t p, double* sigma, cudaStream_t s);

// criterion_big.cu (33 <= p <= 128: a block per candidate)
int run_alg1_big(psr_ctx* ctx, Group& G, const double* Ag, cudaStream_t s, int64_t* evals, int64_t* exact,
                 int64_t* screened, int* first_singular_local);
int launch_criterion_big(const double* A_i, int32_t batch, int32_t p, const double* A_c, const double* Binv_c,
                         double tol, int32_t* accept, double* dval, cudaStream_t s);

// sweep.cu
int build_sweep(psr_ctx* ctx, cudaStream_t s);
int sweep_apply(psr_ctx* ctx, const double* r, double* z, cudaStream_t s);
int autotune_sweep(psr_ctx* ctx, cudaStream_t s);
// z_zeroed: z is already zero (the caller cleared it), the sweep skips its memset
int sweep_apply_ex(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s,
                   bool z_zeroed = false);
int build_grouped_tables(psr_ctx* ctx);
void free_sweep(psr_ctx* ctx);

// sweep_stream.cu (full-storage groups: column-major inverses, thread per row)
// entry_of (device, count, may be NULL): the entry of each sorted patch, for
// a clustered group applied like full storage (one streamed inverse per patch)
int stream_convert(psr_ctx* ctx, Group& G, const double* db64, cudaStream_t s, int64_t* bytes,
                   const int32_t* entry_of = nullptr);
int stream_build_table(psr_ctx* ctx);
int launch_sweep_stream(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s);
// Clustered FP64 database of a group (p <= 32) as scaled FP32 pairs
// (G.rinv_pair, G.bexp) and its thread-per-patch sweep on pair arithmetic.
int pair_db_convert(psr_ctx* ctx, Group& G, const double* db64, cudaStream_t s);
int launch_sweep_tpp_pair(psr_ctx* ctx, const Group& G, const double* r, double* z, const int32_t* stop,
                          cudaStream_t s);
void stream_free(psr_ctx* ctx);
int coarse_apply(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s);
int run_alg1_l1(psr_ctx* ctx, cudaStream_t s);
void coarse_free(psr_ctx* ctx);

// sweep_tc.cu (BF16 entries on tcgen05 tensor cores)
int tc_pad(int p);
int tc_prepare();
int convert_tc(const double* src, int m, int p, int sym, __nv_bfloat16** out, cudaStream_t s);
int launch_sweep_tc(const int32_t* tiles, int ntiles, int p, const __nv_bfloat16* rinv, const int32_t* sdofs,
                    const double* r, const double* wg, const double* wsc, double* z, const int32_t* stop,
                    int32_t* err, cudaStream_t s);

// kmeans.cu
// cls: class of every patch (boundary partition) or null
int run_kmeans(psr_ctx* ctx, cudaStream_t s, int m, const std::vector<int32_t>& init, int max_iter,
               const std::vector<int32_t>* cls);

// krylov.cu
int krylov_alloc(psr_ctx* ctx, cudaStream_t s);
int krylov_solve(psr_ctx* ctx, const double* b, double* x, cudaStream_t s, psr_solve_info* info);
void krylov_free(psr_ctx* ctx);
int kernel_timing_enable(psr_ctx* ctx, bool on);

}  // namespace psr
