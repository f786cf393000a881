// Patch detection from the matrix pattern (section 2, after Figure 1): a row
// with exactly q (p+1)^d stored entries (q components, tensor-product cells
// of degree p in d dimensions) couples only with the DOFs of its own cell, so
// its column set is that cell's DOF set; rows with the same set give one
// cell-restricted patch.
//
//   k_detect_flag    one thread per row: rows of the requested length whose
//                    columns are strictly increasing and in range are
//                    flagged, with a 64-bit hash of their column list;
//   k_detect_insert  every flagged row claims its hash's slot of an
//                    open-addressing table (linear probing, atomicCAS on the
//                    key, at most T probes with T >= 2 x flagged rows) and
//                    lowers the slot's row to its own (atomicMin);
//   k_detect_canon   the slot's row is the smallest row with that hash: a row
//                    is canonical iff it is that row; any other row compares
//                    its columns with it and reports a collision if they
//                    differ; per-block counts of canonical rows;
//   k_detect_write   canonical rows write their columns at their rank (block
//                    offsets from an exclusive scan of the counts), so
//                    patches come in the order of their smallest row.
#include "psr_internal.cuh"

#include <vector>

namespace psr {
namespace {

constexpr int DT = 256;        // threads per block of the rank kernels

// splitmix64 finaliser (Steele, Lea and Flood 2014), chained over the columns
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_detect_flag(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int n, int q,
                              unsigned long long* __restrict__ hash, int32_t* __restrict__ flag,
                              int32_t* __restrict__ status, int32_t* __restrict__ nflag) {
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int r = base + threadIdx.x;
        int f = 0;
        if (r < n) {
            const int a = rowptr[r], b = rowptr[r + 1];
            if (b - a == q) {
                bool ok = true;
                int prev = -1;
                unsigned long long h = 0;
                for (int k = a; k < b; ++k) {
                    const int c = colidx[k];
                    ok &= (c > prev) && (c < n);
                    prev = c;
                    h = mix64(h ^ (unsigned long long)(unsigned int)c);
                }
                if (ok) {
                    f = 1;
                    hash[r] = h | 1ull;                // 0 marks an empty slot
                } else {
                    atomicOr(status, ST_UNSORTED);
                }
            }
            flag[r] = f;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0 && bal) atomicAdd(nflag, __popc(bal));
    }
}

__global__ void k_detect_insert(const unsigned long long* __restrict__ hash, const int32_t* __restrict__ flag, int n,
                                unsigned long long* __restrict__ keys, int32_t* __restrict__ rows, int T,
                                int32_t* __restrict__ status) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        if (!flag[r]) continue;
        const unsigned long long h = hash[r];
        int slot = (int)(h & (unsigned long long)(T - 1));
        int it = 0;
        for (; it < T; ++it) {
            const unsigned long long prev = atomicCAS(&keys[slot], 0ull, h);
            if (prev == 0ull || prev == h) {
                atomicMin(&rows[slot], r);
                break;
            }
            slot = (slot + 1) & (T - 1);
        }
        if (it == T) atomicOr(status, ST_OOB);      // table full: cannot happen with T >= 2 x flagged
    }
}

__global__ void __launch_bounds__(DT) k_detect_canon(const int32_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colidx,
                                                     const unsigned long long* __restrict__ hash,
                                                     const int32_t* __restrict__ flag, int n, int q,
                                                     const unsigned long long* __restrict__ keys,
                                                     const int32_t* __restrict__ rows, int T,
                                                     int32_t* __restrict__ canon, int32_t* __restrict__ bcount,
                                                     int32_t* __restrict__ status) {
    const int r = blockIdx.x * DT + threadIdx.x;
    int f = 0;
    if (r < n && flag[r]) {
        const unsigned long long h = hash[r];
        int slot = (int)(h & (unsigned long long)(T - 1));
        for (int it = 0; it < T && keys[slot] != h; ++it) slot = (slot + 1) & (T - 1);
        const int c = (keys[slot] == h) ? rows[slot] : -1;
        if (c == r) {
            f = 1;
        } else if (c >= 0 && c < n) {
            const int a = rowptr[r], ac = rowptr[c];
            bool same = true;
            for (int k = 0; k < q; ++k) same &= colidx[a + k] == colidx[ac + k];
            if (!same) atomicOr(status, ST_HASH);
        } else {
            atomicOr(status, ST_OOB);
        }
    }
    if (r < n) canon[r] = f;
    const int cnt = __syncthreads_count(f);
    if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(DT) k_detect_write(const int32_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colidx,
                                                     const int32_t* __restrict__ canon, int n, int q,
                                                     const int32_t* __restrict__ boff, int32_t* __restrict__ dofs) {
    __shared__ int wsum[DT / 32];
    const int r = blockIdx.x * DT + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int f = (r < n) ? canon[r] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    if (f) {
        const int64_t pos = (int64_t)boff[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
        const int a = rowptr[r];
        for (int k = 0; k < q; ++k) dofs[pos * q + k] = colidx[a + k];
    }
}

}  // namespace
}  // namespace psr

using namespace psr;

extern "C" int psr_detect_patches(const psr_csr* A, int32_t row_nnz, int32_t* dofs, int32_t max_patches,
                                  int32_t* n_patches, void* stream) {
    if (!A || A->n <= 0 || !A->rowptr || !A->colidx || !n_patches || row_nnz < 1 || row_nnz > 1024 ||
        (dofs && max_patches < 0)) {
        set_error(nullptr, "psr_detect_patches: invalid argument");
        return PSR_ERR_INVALID_ARG;
    }
    *n_patches = 0;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = A->n;
    const int nb = (n + DT - 1) / DT;
    const int gs = std::min(nb, 152 * 8);
    unsigned long long* hash = nullptr;
    unsigned long long* keys = nullptr;
    int32_t *flag = nullptr, *canon = nullptr, *rows = nullptr, *bcount = nullptr, *boff = nullptr, *ctl = nullptr;
    int rc = PSR_OK;
    auto fail = [&](cudaError_t e, const char* what) { rc = cuda_fail(nullptr, e, what); };
    auto finish = [&]() {
        cudaStreamSynchronize(s);
        for (void* p : {(void*)hash, (void*)keys, (void*)flag, (void*)canon, (void*)rows, (void*)bcount, (void*)boff,
                        (void*)ctl})
            dev_free(p);
        return rc;
    };
    cudaError_t e;
    if ((e = dev_alloc(&hash, sizeof(unsigned long long) * (size_t)n)) != cudaSuccess ||
        (e = dev_alloc(&flag, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
        (e = dev_alloc(&canon, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
        (e = dev_alloc(&bcount, sizeof(int32_t) * (size_t)nb)) != cudaSuccess ||
        (e = dev_alloc(&boff, sizeof(int32_t) * (size_t)nb)) != cudaSuccess ||
        (e = dev_alloc(&ctl, sizeof(int32_t) * 2)) != cudaSuccess) {
        fail(e, "psr_detect_patches allocation");
        return finish();
    }
    int32_t hctl[2] = {0, 0};       // status, flagged rows
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(int32_t) * 2, s)) != cudaSuccess) { fail(e, "memset"); return finish(); }
    count_launch();
    k_detect_flag<<<gs, DT, 0, s>>>(A->rowptr, A->colidx, n, row_nnz, hash, flag, ctl, ctl + 1);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        fail(e, "k_detect_flag");
        return finish();
    }
    if (hctl[0] & ST_UNSORTED) {
        set_error(nullptr, "psr_detect_patches: a row of the requested length has unsorted, repeated or out-of-range columns");
        rc = PSR_ERR_UNSORTED_CSR;
        return finish();
    }
    const int nflag = hctl[1];
    if (nflag == 0) return finish();
    if (nflag > (1 << 28)) {
        set_error(nullptr, "psr_detect_patches: more than 2^28 rows of the requested length");
        rc = PSR_ERR_INVALID_ARG;
        return finish();
    }
    int T = 64;
    while (T < 2 * nflag) T <<= 1;
    if ((e = dev_alloc(&keys, sizeof(unsigned long long) * (size_t)T)) != cudaSuccess ||
        (e = dev_alloc(&rows, sizeof(int32_t) * (size_t)T)) != cudaSuccess ||
        (e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)T, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(rows, 0x7f, sizeof(int32_t) * (size_t)T, s)) != cudaSuccess) {
        fail(e, "psr_detect_patches table");
        return finish();
    }
    count_launch();
    k_detect_insert<<<gs, DT, 0, s>>>(hash, flag, n, keys, rows, T, ctl);
    count_launch();
    k_detect_canon<<<nb, DT, 0, s>>>(A->rowptr, A->colidx, hash, flag, n, row_nnz, keys, rows, T, canon, bcount, ctl);
    std::vector<int32_t> hb((size_t)nb);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hb.data(), bcount, sizeof(int32_t) * (size_t)nb, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hctl, ctl, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        fail(e, "k_detect_canon");
        return finish();
    }
    if (hctl[0] & (ST_HASH | ST_OOB)) {
        set_error(nullptr, "psr_detect_patches: two different column sets share a 64-bit hash");
        rc = PSR_ERR_INVALID_ARG;
        return finish();
    }
    int64_t total = 0;
    for (int b = 0; b < nb; ++b) {
        const int c = hb[b];
        hb[b] = (int32_t)total;
        total += c;
    }
    *n_patches = (int32_t)total;
    if (!dofs) return finish();
    if (total > max_patches) {
        set_error(nullptr, "psr_detect_patches: more patches than max_patches (their number is in *n_patches)");
        rc = PSR_ERR_INVALID_ARG;
        return finish();
    }
    if ((e = cudaMemcpyAsync(boff, hb.data(), sizeof(int32_t) * (size_t)nb, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        fail(e, "psr_detect_patches offsets");
        return finish();
    }
    count_launch();
    k_detect_write<<<nb, DT, 0, s>>>(A->rowptr, A->colidx, canon, n, row_nnz, boff, dofs);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
        fail(e, "k_detect_write");
    return finish();
}
