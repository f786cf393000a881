/*
 * psr.h -- C ABI of the GB300 compressed patch-relaxation library.
 *
 * Method: Harper & Tuminaro, "Compression and Reduced Representation
 * Techniques for Patch-Based Relaxation" (arXiv 2306.10025).
 *
 *   Patch matrices     A_k = V_k A V_k^T                        (section 2)
 *   Weights            W   = (sum_l V_l^T V_l)^{-1}             (section 2)
 *   Full preconditioner M^{-1}  = W sum_k V_k^T A_k^{-1} V_k    (Eq. 1)
 *   Compressed         M~^{-1} = W sum_k V_k^T B_phi(k)^{-1} V_k (Eq. 3)
 *   Database / map     B = {B_1^-1..B_mp^-1}, phi built by Alg. 1 with the
 *                      criterion d(A_i, B_j) = ||I - A_i B_j^{-1}||_2 < tol
 *   Outer solve        A x = b by PCG or FGMRES(m), x0 = 0, stop when
 *                      ||r_k||_2 <= rtol ||r_0||_2 (section 4, Exp. 1)
 *
 * Conventions (all entry points):
 *   - Every call returns int: PSR_OK (0) or a negative PSR_ERR_* code; no C++
 *     exception crosses the ABI.  psr_last_error() gives a message.
 *   - Pointers documented "device" are CUDA device pointers owned by the
 *     caller (e.g. PyTorch tensors); the library never frees them.  Storage
 *     derived by the library (patch matrices, inverses, Krylov basis) is owned
 *     by the psr_ctx and released by psr_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; only psr_setup and psr_solve block the
 *     host (setup to read small control scalars, solve to read the stopping
 *     flag).  There is no CPU fallback: without a CUDA device every compute
 *     entry point returns PSR_ERR_CUDA.
 *   - Indices are int32 (n < 2^31, sum of patch sizes < 2^31); values FP64.
 *   - Compute entry points run on the current CUDA device of the calling
 *     thread; a psr_ctx must be used on the device it was created on.
 */
#ifndef PSR_H
#define PSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PSR_OK                  0
#define PSR_ERR_INVALID_ARG    -1  /* bad pointer / size / option            */
#define PSR_ERR_UNSORTED_CSR   -2  /* CSR columns not sorted+unique, or out of range */
#define PSR_ERR_SINGULAR_PATCH -3  /* a stored patch failed the pivot test   */
#define PSR_ERR_NOT_CONVERGED  -4  /* solve hit maxit before rtol            */
#define PSR_ERR_CUDA           -5  /* CUDA runtime error (message in psr_last_error) */
#define PSR_ERR_OOM            -6  /* device allocation failed               */
#define PSR_ERR_TIMEOUT        -7  /* a bounded device-side wait gave up     */
#define PSR_ERR_UNCOVERED_DOF  -8  /* a DOF lies in no patch: W undefined    */

/* ---- option values ----------------------------------------------------- */
#define PSR_PREC_FP64 0            /* representative inverses stored FP64    */
#define PSR_PREC_FP32 1            /* stored FP32, applied in FP32           */
#define PSR_PREC_BF16 2            /* stored BF16, applied on tensor cores   */

#define PSR_WEIGHT_LEFT 0          /* z = W sum V^T B^-1 V r (Eq. 1 / Eq. 3)  */
#define PSR_WEIGHT_SYM  1          /* z = W^.5 sum V^T B^-1 V W^.5 r (SPD)    */

#define PSR_KRYLOV_CG     0
#define PSR_KRYLOV_FGMRES 1

#define PSR_SWEEP_AUTO     0       /* library chooses                         */
#define PSR_SWEEP_GROUPED  1       /* one persistent launch over all size groups */
#define PSR_SWEEP_PERGROUP 2       /* one launch per patch-size group         */
#define PSR_SWEEP_TENSOR   3       /* per group; BF16 clustered groups always on the
                                      tensor cores (AUTO uses them only when their
                                      128-patch tiles are at least 1/4 full) */

#define PSR_CRITERION_SPECTRAL 0   /* Alg. 1 with ||I - A_i B_j^-1||_2 < tol (Eq. 4)        */
#define PSR_CRITERION_L1       1   /* Alg. 1 with ||A_i - A_j||_l1 < tol (entrywise, Exp. 3) */
#define PSR_CRITERION_VARMIN   2   /* Alg. 2 only: spectral distance, representatives the
                                      members of least in-cluster variance (section 3.2) */

#define PSR_ORTHO_AUTO   0        /* FGMRES Gram-Schmidt: one fused cooperative launch per
                                      step with dots and updates on FP32 pairs (about 48
                                      significant bits; FP64 when ||w|| is outside
                                      [2^-80, 2^60]); the FP64 kernels without cooperative launch */
#define PSR_ORTHO_FP64   1         /* the fused launch in FP64 arithmetic                  */
#define PSR_ORTHO_SPLIT  2         /* one launch per pass, FP64 arithmetic                 */

#define PSR_FP64_PAIRS   0         /* FP64 inverses of full-storage groups kept as (hi, lo)
                                      FP32 pairs (8 bytes, 48-bit significand, a power-of-two
                                      scale per patch) and applied in compensated FP32 pair
                                      arithmetic: the GPU's FP64 units are 1/64 of its FP32
                                      rate and would bound the sweep instead of HBM          */
#define PSR_FP64_NATIVE  1         /* FP64 inverses applied with FP64 fused multiply-adds      */

#define PSR_MATCH_FIRST   0        /* Alg. 1 as printed: the first entry with d < tol          */
#define PSR_MATCH_CLOSEST 1        /* section 3.1 variant: of the entries existing when the
                                      patch is reached, the one with the least d (< tol)       */

#define PSR_SEARCH_CREATION    0   /* Alg. 1 tests the entries in creation order           */
#define PSR_SEARCH_NORM_WINDOW 1   /* section 3.1 sorted search: only entries with
                                      ||A_i||/(1+tol) < ||B_j|| < ||A_i||/(1-tol) (the 2-norms
                                      of the patch and of the entry's patch, widened by 1e-12)
                                      are tested, in creation order; the others cannot pass
                                      (d >= | ||B_j|| - ||A_i|| | / ||B_j||), so phi and the
                                      entries are those of the creation-order search and only
                                      the evaluation count drops.  Spectral criterion, first
                                      match, no seed database or hints; any patch size.    */

typedef struct psr_ctx psr_ctx;    /* opaque, library-owned */

/* Assembled matrix A (section 2: A x = b), CSR, device pointers. */
typedef struct {
    int32_t        n;        /* rows == columns                                  */
    int64_t        nnz;      /* entries                                          */
    const int32_t* rowptr;   /* device, n+1, rowptr[0] = 0, nondecreasing        */
    const int32_t* colidx;   /* device, nnz, sorted and unique within each row   */
    const double*  vals;     /* device, nnz                                      */
} psr_csr;

/* Patches: the boolean restrictions V_k as a cell -> DOF map (section 2:
 * (V_k)_{ij} = 1 iff global DOF j is local DOF i of patch k).  Local order is
 * the order in which the DOFs are listed. */
typedef struct {
    int32_t        n_patches;
    int32_t        uniform_size;  /* p_s when every patch has p_s DOFs, else 0   */
    const int32_t* offsets;       /* device, n_patches+1 (ignored when uniform_size > 0) */
    const int32_t* dofs;          /* device, flat list, patch k at [offsets[k], offsets[k+1]) */
} psr_patches;

typedef struct {
    double  tol;          /* Alg. 1 epsilon; 0 => full storage (phi = identity)  */
    int32_t store_prec;   /* PSR_PREC_*                                           */
    int32_t weighting;    /* PSR_WEIGHT_*                                         */
    int32_t krylov;       /* PSR_KRYLOV_*                                         */
    int32_t restart;      /* FGMRES restart length m (1..32)                      */
    double  rtol;         /* relative residual target                             */
    int32_t maxit;        /* outer iteration cap                                  */
    int32_t use_graph;    /* 1: capture Krylov cycles in CUDA graphs              */
    int32_t sweep_kernel; /* PSR_SWEEP_*                                          */
    int32_t autotune;     /* 1: time candidate sweep tile shapes at setup         */
    int32_t symmetrize;   /* 1: store (B^-1 + B^-T)/2 before rounding to FP32/BF16 */
    int32_t use_mlp;      /* psr_setup_learned: 1 = verify the trained network's
                             predicted entries first (the other setups ignore it)  */
    int32_t ortho;        /* PSR_ORTHO_* (FGMRES only)                            */
    int32_t criterion;    /* PSR_CRITERION_* of Alg. 1 (L1: psr_setup only)        */
    int32_t fp64_arith;   /* PSR_FP64_* arithmetic of the FP64 full-storage sweep  */
    int32_t match;        /* PSR_MATCH_* rule of Alg. 1 (spectral criterion)       */
    uint64_t seed;        /* seed of the library's own random draws (MLP weights,
                             training order of psr_mlp_train)                     */
    double  prec_check;   /* FP32 / BF16 storage of a database built by Alg. 1 or 2:
                             an entry whose rounded (symmetrised) inverse B~ has
                             ||B~ A_c - I||_F > prec_check, or (CG) is not positive
                             definite, is kept and applied in FP64 instead;
                             0 disables the check                                  */
    int32_t search;       /* PSR_SEARCH_* of Alg. 1 (psr_setup with the spectral
                             criterion; the learned and seeded setups take only
                             PSR_SEARCH_CREATION)                                  */
} psr_opts;

/* Fill `o` with defaults: tol 0, FP64, SYM, CG, restart 30, rtol 1e-8,
 * maxit 10000, graphs on, AUTO sweep, autotune on, symmetrize on, no MLP,
 * AUTO orthogonalisation, spectral criterion, FP64 pairs, first match,
 * seed 0, precision check 0.5, creation-order search. */
void psr_default_opts(psr_opts* o);

/* A rectangular CSR matrix (the interpolation P0 of Eq. 2), device pointers. */
typedef struct {
    int32_t        n_rows;
    int32_t        n_cols;
    int64_t        nnz;
    const int32_t* rowptr;   /* device, n_rows+1 */
    const int32_t* colidx;   /* device, nnz, in [0, n_cols) */
    const double*  vals;     /* device, nnz */
} psr_csr_rect;

#define PSR_COARSE_MAX 16384       /* coarse dimension n0 (A0^-1 is kept dense) */

/* ---- whole method ------------------------------------------------------- */

/* Setup of M~^{-1} (Eq. 3): validate the CSR and map, extract every A_k,
 * compute W, build B and phi with Alg. 1 at opts->tol (tol = 0 stores every
 * patch, Eq. 1), invert the representatives (FP64 LU-equivalent Gauss-Jordan
 * with partial pivoting), convert them to opts->store_prec and lay out the
 * sweep.  Patches of up to 128 DOFs; every size forms its own group (the
 * remark after Eq. 1) with its own database, numbered group after group,
 * larger sizes first.  Groups in which every patch is its own entry are
 * stored column-major and streamed (one launch over all of them).  The CSR
 * and map are copied; the caller may free them afterwards.
 * opts->match and opts->search pick Alg. 1's rule (first or closest match)
 * and search (creation order or the norm window); the norm window takes
 * first match and the spectral criterion (INVALID_ARG otherwise).
 * On success *out owns all derived storage; on failure every block the call
 * took is given back.  Errors: INVALID_ARG, UNSORTED_CSR, UNCOVERED_DOF,
 * SINGULAR_PATCH (psr_last_error names the patch), OOM, TIMEOUT (a bounded
 * wait of the Alg. 1 rounds gave up), CUDA.  Blocks the host. */
int psr_setup(const psr_csr* A, const psr_patches* patches, const psr_opts* opts,
              void* stream, psr_ctx** out);

/* Setup whose Alg. 1 starts from a given database and optional hints
 * (learned assignment; no counterpart in the paper beyond its closing remark
 * on deep-learning assisted clustering).  seed_A: device, m0 x p x p patch
 * matrices forming database entries 0..m0-1 (inverted here).  hints: device,
 * n_patches entries in [-1, m0); patch i with hints[i] >= 0 is first compared
 * with that entry (one criterion evaluation) and assigned to it when
 * d < tol; every other patch runs Alg. 1 against the database in creation
 * order (seed entries first) and may append new entries.  Needs tol > 0,
 * patches of one size p <= 32, first match and the creation-order search.
 * psr_get_stats reports the hits. */
int psr_setup_seeded(const psr_csr* A, const psr_patches* patches, const psr_opts* opts,
                     const double* seed_A, int32_t m0, const int32_t* hints, void* stream,
                     psr_ctx** out);

/* Setup whose database comes from Alg. 2 (section 3.2) instead of Alg. 1:
 * m_p entries fixed beforehand, B_j the entrywise mean of its cluster
 * (Eq. 6), the stored inverse that of the mean; the distance by
 * opts->criterion: PSR_CRITERION_L1 the entrywise ||A_i - B_j||_l1,
 * PSR_CRITERION_SPECTRAL ||I - A_i B_j^-1||_2 (p <= 32).  With
 * PSR_CRITERION_VARMIN (p <= 32) B_j is instead the member of cluster j with
 * the least sum over the cluster of d(A_k, B_j)^2 (d spectral), stored with
 * its own inverse (variance-minimising clustering).  init: device, m_p distinct
 * patch indices (drawn at random by the caller, as Alg. 2's randperm) whose
 * patches are the initial means.  Every sweep assigns each patch to its
 * nearest mean (ties to the lowest index); the means are recomputed (members
 * summed in increasing patch index; an emptied cluster keeps its mean) until
 * a sweep changes nothing or after max_iter sweeps.  opts->tol is ignored;
 * psr_get_stats reports the sweeps in `rounds`.  Needs patches of one size
 * p <= 128.  patch_class (device, n_patches int32, or NULL): the boundary
 * partition of psr_boundary_classes -- a patch is then assigned only among
 * the means seeded in its class, every class needing a seed.  Errors:
 * INVALID_ARG (arguments, seeds not distinct or out of range, a class
 * without a seed), SINGULAR_PATCH (a mean failed the pivot test), OOM, CUDA. */
int psr_setup_kmeans(const psr_csr* A, const psr_patches* patches, const psr_opts* opts, int32_t m_p,
                     const int32_t* init, int32_t max_iter, const int32_t* patch_class, void* stream,
                     psr_ctx** out);

/* Boundary partition for Alg. 2 (section 3.2): boundary conditions appear in
 * a patch matrix as rows with exactly one nonzero entry, and averaging a
 * patch that has them with one that has not destroys them, so the patches
 * are partitioned by the set of such rows and each partition is clustered
 * on its own (9 partitions on a square, 27 on a cube).  patch_class (device,
 * n_patches int32, written) gets the partition of every patch, numbered in
 * the order of its first patch; n_classes (host) their number.  Pass the
 * classes as psr_setup_kmeans's patch_class, with init holding at least one
 * seed of every class (the paper divides the clusters in proportion to the
 * partition sizes).  Patches of at most 64 DOFs.  Errors: INVALID_ARG,
 * UNSORTED_CSR, OOM, CUDA.  Blocks the host until done. */
int psr_boundary_classes(const psr_csr* A, const psr_patches* patches, int32_t* patch_class,
                         int32_t* n_classes, void* stream);

/* z = M~^{-1} r (Eq. 3 with the context's weighting).  r, z: device, length n,
 * must not overlap.  Stream-ordered, no host synchronisation, no allocation. */
int psr_apply(psr_ctx* ctx, const double* r, double* z, void* stream);

typedef struct {
    int32_t iterations;   /* outer iterations performed                        */
    int32_t converged;    /* 1 when ||r_k|| <= rtol ||r_0||                     */
    double  relres;       /* final ||r_k|| / ||r_0|| (recursively updated)      */
    double  seconds;      /* device time of the solve (CUDA events)            */
} psr_solve_info;

/* Solve A x = b (x0 = 0) with the context's Krylov method preconditioned on
 * the right by M~^{-1}.  b, x: device, length n.  Returns NOT_CONVERGED when
 * maxit is hit (x then holds the last iterate).  `info` may be NULL. */
int psr_solve(psr_ctx* ctx, const double* b, double* x, void* stream, psr_solve_info* info);

/* Residual history of the last solve: hist[k] = ||r_k||/||r_0||, k = 0..len-1
 * (host buffer of capacity cap).  *len receives the number of entries. */
int psr_get_history(psr_ctx* ctx, double* hist, int32_t cap, int32_t* len);

/* Alg. 1 output: phi (device, n_patches, 0-based database index per patch),
 * rep_ids (device, m_p, patch index of each database entry in creation
 * order, or NULL) and *m_p (host). */
int psr_get_assignment(psr_ctx* ctx, int32_t* phi, int32_t* rep_ids, int32_t* m_p);

/* Smoothing iteration of Experiment 3: `sweeps` times
 * x <- x + omega M^-1 (b - A x), M^-1 as in psr_apply (the patch method of
 * Eq. 3, plus the coarse term of Eq. 2 when set).  b, x: device, n FP64; x
 * is updated in place.  sweeps = 0 leaves x unchanged.  Errors:
 * INVALID_ARG (NULL, sweeps < 0, omega NaN), CUDA.  Blocks the host. */
int psr_smooth(psr_ctx* ctx, const double* b, double* x, double omega, int32_t sweeps, void* stream);

/* Two-level combination preconditioner (Eq. 2): after this call psr_apply
 * and psr_solve use M_combo^-1 = M^-1 + P0 A0^-1 R0 with M^-1 the patch method
 * (Eq. 3), R0 = P0^T and A0 = R0 A P0 formed here and inverted (a direct
 * coarse solve in place of the first-order AMG, as in Experiment 1).
 * P0: device CSR, n x n0 (n0 <= PSR_COARSE_MAX), copied; for Experiment 1
 * the bilinear interpolation from the mesh vertices to the high-order nodes.
 * A0 must be symmetric positive definite (A SPD, P0 of full rank): its
 * Gauss-Jordan inverse takes no pivots.  The coarse term is added after the
 * patch sweep without a weight.  Errors: INVALID_ARG (shape, indices), OOM,
 * CUDA.  Replaces an earlier coarse space; blocks the host. */
int psr_set_coarse(psr_ctx* ctx, const psr_csr_rect* P0, void* stream);

/* The database of a finished setup, for reuse in a later setup of a related
 * matrix (section 3.2, linear problem sequences: a database initialised from
 * the previous setup; pass the entries as seed_A of psr_setup_seeded and the
 * previous phi, from psr_get_assignment, as hints).  entries: device,
 * m_p x p x p FP64, row-major per entry, in creation order: the patch matrix
 * of each entry's representative, a seed entry's matrix, or an Alg. 2 mean.
 * Setups with patches of one size built by Alg. 1 (tol > 0), seeded Alg. 1
 * or Alg. 2 only; INVALID_ARG otherwise (tol = 0 keeps no database copy).
 * Blocks the host until the copy is done. */
int psr_export_database(psr_ctx* ctx, double* entries, void* stream);

typedef struct {
    int32_t n, n_patches, m_p, n_groups;
    int64_t criterion_evals;      /* d(A_i, B_j) evaluations in Alg. 1 order   */
    int64_t criterion_exact;      /* of which needed the exact SVD-class path   */
    int64_t mlp_hits;             /* patches whose predicted entry verified      */
    int64_t factor_bytes;         /* bytes of stored inverses                   */
    int64_t index_bytes;          /* bytes of phi + maps used by the sweep      */
    double  t_extract, t_rounds, t_invert, t_convert, t_autotune; /* setup seconds; t_invert:
                                     GPU time (CUDA events) of the batched inverses,
                                     every patch's at tol 0 and before Alg. 1 (part
                                     of t_rounds)                                  */
    int32_t first_singular;       /* patch index or -1                          */
    int32_t rounds;               /* Alg. 1 rounds: passes of the round kernels
                                     (one makes up to 64 entries for patches of
                                     at most 32 DOFs, one entry above); Alg. 2
                                     and the l1 test: their own passes          */
    int32_t tc_groups;            /* size groups applied on the tensor cores (BF16
                                     storage, 128-patch tiles at least 1/4 full) */
    int32_t prec_fallback;        /* database entries kept in FP64 because their rounded
                                     inverse failed psr_opts.prec_check */
    int64_t criterion_screened;   /* of the evaluations, rejected by the per-patch
                                     sketch screen without reading the candidate */
    int64_t criterion_decided;    /* pairs the warp / block cascade decided, also
                                     those Alg. 1 does not count (candidates of a
                                     round that are not entries, pairs past a
                                     patch's first accept)                       */
} psr_stats;

int psr_get_stats(psr_ctx* ctx, psr_stats* st);

/* Message of the last failing call on this thread (ctx may be NULL). */
const char* psr_last_error(psr_ctx* ctx);

void psr_destroy(psr_ctx* ctx);

/* Patch detection (section 2, after Figure 1): cell-restricted patches found
 * from the matrix alone.  A row with exactly row_nnz = q (p+1)^d stored
 * entries (q components, tensor-product cells of degree p in d dimensions)
 * couples only with the DOFs of its own cell, so its column set is that
 * cell's DOF set; every distinct set of such rows is one patch.  The stored
 * pattern must be the symbolic one (boundary conditions that remove entries
 * hide the boundary cells).
 *   A:           device CSR (vals unused); only rows of length row_nnz are
 *                read, and their columns must be sorted, unique, in range.
 *   row_nnz:     1..1024.
 *   dofs:        device int32 [max_patches * row_nnz], or NULL to only count.
 *                Patch k (ordered by the smallest row having its set) is
 *                dofs[k * row_nnz .. k * row_nnz + row_nnz), ascending, and
 *                goes to psr_setup as a uniform-size patch map.
 *   n_patches:   host; the number of patches found (also when dofs is NULL
 *                or too small).
 * Errors: INVALID_ARG (bad argument, more patches than max_patches, or two
 * different column sets with equal 64-bit hashes), UNSORTED_CSR, CUDA.
 * Blocks the host until done. */
int psr_detect_patches(const psr_csr* A, int32_t row_nnz, int32_t* dofs, int32_t max_patches,
                       int32_t* n_patches, void* stream);

/* Memory: the library keeps the device and pinned host blocks that a destroy
 * (or a setup's temporaries) frees and hands them out again to later
 * allocations of a similar size (1x to 1.25x), after one device
 * synchronisation when they were freed since the last; at most 16 GiB per
 * device is kept, and on out-of-memory the cache is released and the
 * allocation retried.  This call synchronises every device the library
 * allocated on and returns all cached blocks to the driver (blocks still in
 * use by live contexts are not touched).  Returns PSR_OK or PSR_ERR_CUDA. */
int psr_release_cached_memory(void);

/* Bytes of device and of pinned host memory the library's allocator has
 * handed out and not taken back (cached blocks excluded): contexts, networks
 * and the buffers of calls in progress on any thread.  A setup that fails
 * frees what its steps held, so the figures return to their value before
 * the call.  Either pointer (host) may be NULL.  Returns PSR_OK. */
int psr_memory_in_use(int64_t* device_bytes, int64_t* host_bytes);

/* Fault injection for tests of the failure paths (the paper has no
 * counterpart).  Nothing here makes a GPU fault: the failures are made on
 * the host or by a bounded wait that runs out.
 *   PSR_INJECT_ALLOC_FAIL, value k >= 1: the k-th next device allocation of
 *     the library (counted from this call, 1 = the next) fails as if the
 *     device were out of memory, without a driver call; the call that made
 *     it returns PSR_ERR_OOM and frees what it held.  0 disables.
 *   PSR_INJECT_BARRIER_WAIT, value s >= 1: the grid barriers of the Alg. 1
 *     rounds kernel launched on the current device from now on wait for one
 *     block more than the grid holds and give up after s spins (about
 *     s x 32 ns); every block then leaves the kernel and the setup returns
 *     PSR_ERR_TIMEOUT.  0 restores the normal barrier (limit 2^24 spins).
 *   PSR_INJECT_ROUNDS_SPLIT, value 1: the Alg. 1 rounds for patches of at
 *     most 32 DOFs take the path used where a cooperative launch is not
 *     available or the pair lists do not fit (one entry per round, a screen
 *     and a decide launch each); 0 restores the cooperative multi-entry
 *     kernel.  Host state; the results are the same.
 * Returns PSR_OK, PSR_ERR_INVALID_ARG (unknown kind, negative value) or
 * PSR_ERR_CUDA (PSR_INJECT_BARRIER_WAIT without a device). */
#define PSR_INJECT_ALLOC_FAIL   1
#define PSR_INJECT_BARRIER_WAIT 2
#define PSR_INJECT_ROUNDS_SPLIT 3
int psr_debug_inject(int32_t what, int64_t value);

/* Instrumentation: number of CUDA kernels this library has launched in the
 * process so far (a graph launch counts its kernel nodes).  Host-only, never
 * fails; used by benchmarks to state how many kernels a timed region ran. */
int64_t psr_kernel_launches(void);

/* Instrumentation (the paper has no counterpart): per-kernel device time of
 * the outer solve.  Classes of the per-iteration kernels: */
#define PSR_KT_SWEEP 0   /* preconditioner application z = M^-1 r (Eq. 1 / Eq. 3) */
#define PSR_KT_SPMV 1    /* A z inside the iteration (CSR, FP64) */
#define PSR_KT_MDOT 2    /* FGMRES Gram-Schmidt: the fused Arnoldi step (one cooperative
                            launch: projection, update(s), normalisation), or without
                            cooperative launch the first projection h = V^T w */
#define PSR_KT_MAXPY 3   /* FGMRES updates w -= V h: the first (fused with the second
                            projection when the step reorthogonalises, else with
                            ||w|| and the Arnoldi finish), and the second update */
#define PSR_KT_VEC 4     /* remaining vector kernels (FGMRES scale; CG updates and dots) */
#define PSR_KT_COUNT 5

/* enable != 0: from the next psr_solve on, every per-iteration kernel launch
 * of the solve is bracketed by two CUDA event records on the solve's stream
 * (inside the captured graph when graphs are on), and after each CG block /
 * FGMRES cycle the elapsed times of the launches that did work (iterations
 * that ran, not ones skipped by the stop flag) are added to per-class totals,
 * with their algorithmic bytes.  Enabling resets the totals; enabling or
 * disabling drops the captured graph (re-captured by the next solve).  The
 * events add a little time per launch: take the solve's own timing from a
 * run with timing disabled.  Returns PSR_OK or PSR_ERR_INVALID_ARG (ctx NULL). */
int psr_set_kernel_timing(psr_ctx* ctx, int enable);

/* Copies the totals since the last enable for classes 0 .. count-1
 * (count <= PSR_KT_COUNT): ms = summed event durations in milliseconds,
 * launches = timed launches, bytes = summed algorithmic bytes of those
 * launches (SpMV: 12 nnz + 4 (n+1) + 16 n; V^T w with j+1 basis vectors:
 * 8 (j+2) n; each w -= V h: 8 (j+3) n, the second one only when step j took
 * the second Gram-Schmidt pass; the fused step the sum of these plus 16 n for
 * the normalisation; sweep: 24 n + 4 sum(p_k) + 4 n_patches +
 * stored factor bytes; FGMRES scale 16 n; CG kernels their vector reads and
 * writes), flops = summed algorithmic FP64 flops (SpMV 2 nnz, plus 2 n for
 * the CG dot; fused step 4 n (j+2) + n, plus 4 n (j+1) with the second pass;
 * first projection 2 n (j+2), updates 2 n (j+2) each; sweep 2 sum(p_k) for
 * the weighted scatter, plus 2 sum(p_k^2) with FP64 inverses; vector
 * kernels 2 flops per element and operation).  Any pointer may be NULL.
 * Host-only; PSR_ERR_INVALID_ARG for a NULL ctx or count outside
 * 1 .. PSR_KT_COUNT. */
int psr_get_kernel_timing(psr_ctx* ctx, double* ms, int64_t* launches, double* bytes, double* flops,
                          int count);

/* ---- single steps of the path (stateless; for testing and reuse) ------- */

/* Step a1/a1': A_out <- every A_k (section 2), row-major, patch k at offset
 * sum_{j<k} p_j^2 doubles; mult_out[i] <- number of patches holding DOF i;
 * W_out[i] <- 1/mult_out[i].  All device; any output may be NULL.
 * Errors: INVALID_ARG, UNSORTED_CSR, UNCOVERED_DOF (only when W_out given). */
int psr_extract(const psr_csr* A, const psr_patches* patches, double* A_out,
                int32_t* mult_out, double* W_out, void* stream);

/* Step a2: Ainv[b] <- A[b]^{-1} for a batch of p x p row-major FP64
 * matrices (device), partial pivoting (largest |entry|, lowest row on ties).
 * singular (device, batch, may be NULL) <- 1 when some pivot has
 * |pivot| <= p * 2^-53 * max|A[b]|; that inverse is then NaN.  1 <= p <= 128. */
int psr_batched_inverse(const double* A, int32_t batch, int32_t p, double* Ainv,
                        int32_t* singular, void* stream);

/* Step a3 for one database entry: for b < batch, decide
 * d(A_i[b], B_c) = ||(A_c - A_i[b]) Binv_c||_2 < tol (the difference form of
 * ||I - A_i B_c^{-1}||_2, Alg. 1 test).  accept (device, batch) <- 0/1;
 * dval (device, batch, may be NULL) <- the value that decided: 0 for an
 * exactly equal patch, a certified upper bound below tol for an accept, a
 * certified lower bound >= tol for a reject, or sigma_max from the exact
 * path (p <= 32: Jacobi eigenvalues of E^T E; 33 <= p <= 128: the power-
 * iteration estimate, the decision taken by one Cholesky of tol^2 I - E^T E
 * for the near ties no certificate settles).  A_i, A_c, Binv_c: device,
 * row-major p x p FP64.  1 <= p <= 128 (p > 32: one block per candidate;
 * the call allocates scratch and blocks the host until done). */
int psr_criterion(const double* A_i, int32_t batch, int32_t p, const double* A_c,
                  const double* Binv_c, double tol, int32_t* accept, double* dval,
                  void* stream);

/* The same decision as psr_criterion, for callers that cannot let the
 * library allocate device memory (an application whose memory manager owns
 * all device memory, or a pipeline that cannot afford the device-wide
 * synchronisation an allocation may cause).  The paper has no counterpart;
 * this is a deployment variant.  It calls no allocator: its scratch is a
 * fixed device array of PSR_CRITERION_NOALLOC_MAX + 1 int32 (about 1 MiB)
 * that every GPU loading the library holds until the process exits.
 *   - batch > PSR_CRITERION_NOALLOC_MAX returns PSR_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address (a
 *     one-time set-up per device, done with that device current); make that
 *     first call before any stream capture on the device.  The address is
 *     kept for the life of the process: after a cudaDeviceReset of that
 *     device it is stale, so a process that resets a device must not call
 *     this entry point on it again.
 *   - All calls share the array (it keeps the last call's contents; the
 *     counter is cleared at the start of every call), so calls whose work
 *     overlaps on the GPU race: order them on one stream or synchronise.
 * Arguments, layout and results as psr_criterion. */
#define PSR_CRITERION_NOALLOC_MAX 262144
int psr_criterion_noalloc(const double* A_i, int32_t batch, int32_t p, const double* A_c,
                          const double* Binv_c, double tol, int32_t* accept, double* dval,
                          void* stream);

/* sigma_max of each p x p matrix (device, row-major) by one-sided Jacobi in
 * FP64 (the "small SVD" of the section 3 remark).  1 <= p <= 32. */
int psr_spectral_norm(const double* E, int32_t batch, int32_t p, double* sigma,
                      void* stream);

/* ---- learned assignment: per-patch features and a small MLP ------------ */

/* X[k] <- (A_k / ||A_k||_F row-major, log ||A_k||_F, log coef[k]) as FP32,
 * row stride p*p + 2.  A: device n_patches x p x p FP64; coef: device FP64
 * cell coefficient per patch or NULL (feature 0). */
int psr_features(const double* A, int32_t n_patches, int32_t p, const double* coef, float* X,
                 void* stream);

typedef struct psr_mlp psr_mlp;   /* opaque, library-owned */

/* d -> h -> h -> m network, ReLU hidden layers, softmax cross-entropy, Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  Parameters are FP32 and packed as
 * W1 (h x d), b1 (h), W2 (h x h), b2 (h), W3 (m x h), b3 (m), row-major;
 * they start at zero until psr_mlp_set_params. */
int psr_mlp_create(int32_t in_dim, int32_t hidden, int32_t classes, psr_mlp** out);
int64_t psr_mlp_num_params(const psr_mlp* net);
/* packed: device, psr_mlp_num_params floats; also resets the Adam state. */
int psr_mlp_set_params(psr_mlp* net, const float* packed, void* stream);
int psr_mlp_get_params(const psr_mlp* net, float* packed, void* stream);
/* Mean loss over the batch (device scalar, may be NULL) and its gradient
 * (device, packed like the parameters, may be NULL).  X: device batch x d
 * FP32, y: device batch labels in [0, m). */
int psr_mlp_loss_grad(psr_mlp* net, const float* X, const int32_t* y, int32_t batch, float* loss,
                      float* grads, void* stream);
/* One Adam step on the batch; loss as above. */
int psr_mlp_train_step(psr_mlp* net, const float* X, const int32_t* y, int32_t batch, float lr,
                       float* loss, void* stream);
/* cls (device, batch, may be NULL) <- argmax of the logits (lowest index on
 * ties); logits (device, batch x m, may be NULL). */
int psr_mlp_predict(psr_mlp* net, const float* X, int32_t batch, int32_t* cls, float* logits,
                    void* stream);
void psr_mlp_destroy(psr_mlp* net);

/* ---- learned assignment inside setup (a network trained on a finished
 * setup predicts the entries of a later one; the paper leaves deep-learning
 * assisted clustering to future work, end of section 3.2) -------------- */

#define PSR_LABEL_ASSIGNMENT 0      /* labels = the context's phi (closest-match phi when
                                       the context was built with PSR_MATCH_CLOSEST) */

typedef struct {
    int32_t hidden;          /* hidden width h of the d -> h -> h -> m_p network        */
    int32_t epochs;          /* full-batch Adam steps                                    */
    float   lr;              /* Adam learning rate                                       */
    float   train_fraction;  /* the first ceil(f n_patches) patches (patch order) train  */
    uint64_t seed;           /* initial weights: N(0, 1/fan_in), biases 0, from this seed */
} psr_train_opts;

typedef struct {
    int32_t n_train;         /* patches trained on                                        */
    int32_t classes;         /* m_p of the context                                        */
    float   final_loss;      /* mean cross-entropy after the last step                    */
    float   train_accuracy;  /* fraction of training patches whose argmax is their label  */
    double  seconds;         /* host wall time of the training (features included)        */
} psr_train_info;

/* Defaults: hidden 256, 300 epochs, lr 1e-3, train_fraction 1, seed 0. */
void psr_default_train_opts(psr_train_opts* t);

/* Trains a network owned by ctx to predict each patch's database entry.
 * ctx: a setup built by Alg. 1 (tol > 0) with patches of one size p <= 32.
 * Inputs: features (device, n_patches x (p*p + 2) FP32, as psr_features), or
 * NULL to compute them from the context's patch matrices without a cell
 * coefficient.  Labels: the context's phi (PSR_LABEL_ASSIGNMENT); build ctx
 * with opts.match = PSR_MATCH_CLOSEST to train on closest representatives.
 * The network (d = p*p + 2 -> hidden -> hidden -> m_p, ReLU, softmax) is
 * trained on the GPU (forward and backward GEMMs on the tensor cores) and
 * replaces an earlier one.  info (host) may be NULL.  Errors: INVALID_ARG,
 * OOM, CUDA.  Blocks the host until done. */
int psr_mlp_train(psr_ctx* ctx, const float* features_or_NULL, const psr_train_opts* t, void* stream,
                  psr_train_info* info);

/* The trained network of ctx (owned by ctx; NULL before psr_mlp_train), for
 * psr_mlp_predict / psr_mlp_get_params. */
psr_mlp* psr_ctx_mlp(psr_ctx* ctx);

/* Setup whose Alg. 1 starts from the database of `trained` (its entries'
 * patch matrices, inverted here) and, when opts->use_mlp is set, first tries
 * for every patch the entry that trained's network predicts: one criterion
 * evaluation, the patch assigned when d < tol; patches whose prediction
 * fails (or all patches, use_mlp = 0) run Alg. 1 against the database in
 * creation order and may append entries -- psr_setup_seeded with the
 * network's predictions as hints.  features: device n_patches x (p*p + 2)
 * FP32 of the new patches, or NULL (computed from the patch matrices without
 * a cell coefficient).  Needs tol > 0 and patches of trained's size
 * (p <= 32).  psr_get_stats reports the verified predictions in mlp_hits and
 * the prediction time inside t_rounds.  Errors as psr_setup_seeded. */
int psr_setup_learned(const psr_csr* A, const psr_patches* patches, const psr_opts* opts, const psr_ctx* trained,
                      const float* features_or_NULL, void* stream, psr_ctx** out);

#ifdef __cplusplus
}
#endif
#endif /* PSR_H */
