// Step a4 for groups in which every patch is its own database entry (full
// storage, Eq. 1, or a tolerance that merged nothing): each inverse is read
// exactly once per apply, so there is nothing to stage and the sweep is a
// stream of p x p matrices, one matrix-vector product each.
//
// Layout.  Entry i (= sorted patch i of the group) is stored column-major,
// element (a, b) at i p^2 + b p + a, so that the 32 lanes of a warp owning 32
// consecutive rows read 32 consecutive elements of one column: every load of
// the inverse is coalesced and no element is read twice.  One launch covers
// every streamed size group (the remark after Eq. 1: groups of equal size
// handled independently): the rows of all groups are cut into blocks of 32,
// a warp takes a block, gathers the residual of the (at most floor(31/p) + 2)
// patches its rows touch into shared memory, and lane l forms row l of the
// block, y_a = sum_b B[a][b] x_b, and scatter-adds W y_a.
//
// Arithmetic.  GB300 issues FP64 fused multiply-adds at 1/64 of its FP32
// rate: the FP64 form of this stream (2 p^2 flops per 8 p^2 bytes) would be
// bound by the FP64 units at about 1.4x the time HBM needs.  FP64 entries are
// therefore kept as (hi, lo) FP32 pairs of B 2^-s (s per entry, so the
// largest scaled entry is below 1), the gathered x is split the same way with
// integer operations (a shift per 32-row block), and the row sum is formed in
// compensated FP32 pair arithmetic: every product hi*hi exact (FMA), its
// accumulation exact (TwoSum), the cross products and the error terms summed
// in FP32.  The result carries about 47 significant bits (PSR_FP64_PAIRS);
// PSR_FP64_NATIVE keeps FP64 entries and FP64 FMAs.  FP32 and BF16 storage
// multiply in FP32 with x rounded to FP32.
#include "psr_internal.cuh"
#include "pairs.cuh"

#include <algorithm>

namespace psr {

enum { SM_PAIR = 0, SM_F64 = 1, SM_F32 = 2, SM_BF16 = 3 };

struct StreamDesc {
    const void* Bt;         // count x p x p, column-major per entry, storage type of the mode
    const int32_t* bexp;    // SM_PAIR: entry i holds B_i 2^-bexp[i]
    const int32_t* sdofs;   // DOFs in sweep order (sorted patch i <-> entry i)
    int count;
    int p;
    int rb_begin;           // first 32-row block of the group in the launch
    int pad;
};

constexpr int STREAM_MAX_GROUPS = 32;

template <int MODE> struct StreamT;
template <> struct StreamT<SM_PAIR> { using st = float2; using xt = float2; };
template <> struct StreamT<SM_F64> { using st = double; using xt = double; };
template <> struct StreamT<SM_F32> { using st = float; using xt = float; };
template <> struct StreamT<SM_BF16> { using st = __nv_bfloat16; using xt = float; };

// Read-only loads kept in program order (volatile), so that a batch of them
// is in flight together before the first use.
__device__ __forceinline__ float2 ld_stream(const float2* q) {
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(q));
    return v;
}
__device__ __forceinline__ double ld_stream(const double* q) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ float ld_stream(const float* q) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ float ld_stream(const __nv_bfloat16* q) {
    unsigned short h;
    asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(h) : "l"(q));
    return __uint_as_float((unsigned)h << 16);          // BF16 -> FP32 is exact
}

// Two BF16 of one row (columns 2c and 2c + 1, the lower address first) as FP32.
__device__ __forceinline__ float2 ld_stream_bf16x2(const unsigned* q) {
    unsigned w;
    asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(w) : "l"(q));
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

template <int MODE>
__global__ void __launch_bounds__(256) k_sweep_stream(const StreamDesc* __restrict__ gdesc, int ng, int total_rb,
                                                      const double* __restrict__ r, const double* __restrict__ wg,
                                                      const double* __restrict__ wsc, double* __restrict__ z,
                                                      const int32_t* __restrict__ stop, int slot) {
    using ST = typename StreamT<MODE>::st;
    using XT = typename StreamT<MODE>::xt;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ StreamDesc sd[STREAM_MAX_GROUPS];
    if (stop && *stop) return;
    for (int t = threadIdx.x; t < ng; t += blockDim.x) sd[t] = gdesc[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    XT* xs = reinterpret_cast<XT*>(smem) + (size_t)wid * slot;
    const int nw = gridDim.x * wpb;
    for (int rb = blockIdx.x * wpb + wid; rb < total_rb; rb += nw) {
        int g = 0;
        while (g + 1 < ng && rb >= sd[g + 1].rb_begin) ++g;
        const int p = sd[g].p;
        const int count = sd[g].count;
        const int32_t* sdofs = sd[g].sdofs;
        const ST* Bt = reinterpret_cast<const ST*>(sd[g].Bt);
        const int64_t R = (int64_t)count * p;
        const int64_t g0 = (int64_t)(rb - sd[g].rb_begin) * 32;
        const int k0 = (int)(g0 / p);
        const int64_t klast = (g0 + 31) / p;
        const int k1 = (int)(klast < (int64_t)count - 1 ? klast : (int64_t)count - 1);
        const int nx = (k1 - k0 + 1) * p;                // <= 2 p + 31 <= slot
        const int32_t* dk0 = sdofs + (int64_t)k0 * p;
        // gather x = (W^1/2) r at the DOFs of the patches of this block
        unsigned emax = 0;
        for (int e0 = 0; e0 < nx; e0 += 128) {
            int d[4];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + lane + 32 * u;
                d[u] = __ldg(dk0 + min(e, nx - 1));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldg(r + d[u]);
            if (wg) {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] *= __ldg(wg + d[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + lane + 32 * u;
                if (e < nx) {
                    if constexpr (MODE == SM_PAIR) {
                        reinterpret_cast<double*>(xs)[e] = v[u];
                        const unsigned ex = (unsigned)(__double2hiint(v[u]) >> 20) & 0x7ffu;
                        if (ex != 0x7ffu) emax = max(emax, ex);
                    } else if constexpr (MODE == SM_F64) {
                        xs[e] = v[u];
                    } else {
                        xs[e] = __double2float_rn(v[u]);
                    }
                }
            }
        }
        int shift = 0;
        if constexpr (MODE == SM_PAIR) {
            emax = __reduce_max_sync(0xffffffffu, emax);
            shift = (int)emax - 1023;
            __syncwarp();
            for (int e = lane; e < nx; e += 32) xs[e] = split_scaled(reinterpret_cast<const double*>(xs)[e], shift);
        }
        __syncwarp();
        const int64_t gr = g0 + lane;
        if (gr < R) {
            const int k = (int)(gr / p);
            const int a = (int)(gr - (int64_t)k * p);
            const ST* col = Bt + (int64_t)k * p * p + a;   // BF16: column pairs, indexed below
            const XT* xk = xs + (k - k0) * p;
            const int dof = __ldg(sdofs + (int64_t)k * p + a);
            double y;
            if constexpr (MODE == SM_PAIR) {
                float s = 0.f, c = 0.f;
                int b = 0;
                for (; b + 8 <= p; b += 8) {
                    float2 bv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) bv[u] = ld_stream(col + (int64_t)(b + u) * p);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float2 xv = xk[b + u];
                        pair_fma(s, c, bv[u].x, bv[u].y, xv.x, xv.y);
                    }
                }
                for (; b < p; ++b) {
                    const float2 bv = ld_stream(col + (int64_t)b * p);
                    const float2 xv = xk[b];
                    pair_fma(s, c, bv.x, bv.y, xv.x, xv.y);
                }
                y = ldexp((double)s + (double)c, shift + __ldg(sd[g].bexp + k));
            } else {
                using CT = typename StreamT<MODE>::xt;
                CT acc = (CT)0;
                if constexpr (MODE == SM_BF16) {
                    // columns in pairs: lane a reads (B[a][2c], B[a][2c+1]) as
                    // one 4-byte word, 128 bytes per warp load
                    const int pc = (p + 1) >> 1;
                    const unsigned* col2 = reinterpret_cast<const unsigned*>(Bt) + (int64_t)k * p * pc + a;
                    const int full = p >> 1;
                    int c = 0;
                    for (; c + 4 <= full; c += 4) {
                        float2 bv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) bv[u] = ld_stream_bf16x2(col2 + (int64_t)(c + u) * p);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            acc = fma(bv[u].x, xk[2 * (c + u)], acc);
                            acc = fma(bv[u].y, xk[2 * (c + u) + 1], acc);
                        }
                    }
                    for (; c < full; ++c) {
                        const float2 bv = ld_stream_bf16x2(col2 + (int64_t)c * p);
                        acc = fma(bv.x, xk[2 * c], acc);
                        acc = fma(bv.y, xk[2 * c + 1], acc);
                    }
                    if (p & 1) acc = fma(ld_stream_bf16x2(col2 + (int64_t)full * p).x, xk[p - 1], acc);
                } else {
                    int b = 0;
                    for (; b + 8 <= p; b += 8) {
                        CT bv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) bv[u] = (CT)ld_stream(col + (int64_t)(b + u) * p);
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc = fma(bv[u], xk[b + u], acc);
                    }
                    for (; b < p; ++b) acc = fma((CT)ld_stream(col + (int64_t)b * p), xk[b], acc);
                }
                y = (double)acc;
            }
            atomicAdd(&z[dof], y * __ldg(wsc + dof));
        }
        __syncwarp();
    }
}

// FP64 row-major entries -> the column-major storage of the mode; one block
// per output matrix (output i from entry idx[i], or entry i without idx).  SM_PAIR: the scale exponent s with max|B| 2^-s in [1/2, 1)
// (0 for a zero matrix), hi = fl32(B 2^-s), lo = fl32(B 2^-s - hi).
// sym (FP32 / BF16 only): (B + B^T) / 2 before rounding.
template <int MODE>
__global__ void __launch_bounds__(256) k_to_stream(const double* __restrict__ src, int m, int p, int sym,
                                                   void* __restrict__ dst, int32_t* __restrict__ bexp,
                                                   const int32_t* __restrict__ idx) {
    using ST = typename StreamT<MODE>::st;
    __shared__ double red[8];
    const int pp = p * p;
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        const double* B = src + (int64_t)(idx ? idx[i] : i) * pp;
        ST* out = reinterpret_cast<ST*>(dst) + (int64_t)i * pp;
        int ex = 0;
        if constexpr (MODE == SM_PAIR) {
            double mx = 0.0;
            for (int t = threadIdx.x; t < pp; t += blockDim.x) mx = fmax(mx, fabs(B[t]));
            mx = warp_max(mx);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
            __syncthreads();
            mx = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
            if (mx > 0.0 && mx <= 1.79e308) frexp(mx, &ex);
            if (threadIdx.x == 0) bexp[i] = ex;
        }
        if constexpr (MODE == SM_BF16) {
            // column pairs: (B[a][2c], B[a][2c+1]) adjacent, a zero column
            // after the last one when p is odd
            const int pc = (p + 1) >> 1;
            __nv_bfloat16* o2 = reinterpret_cast<__nv_bfloat16*>(dst) + (int64_t)i * 2 * p * pc;
            for (int t = threadIdx.x; t < 2 * p * pc; t += blockDim.x) {
                const int c = t / (2 * p), q = t - c * 2 * p, a = q >> 1, b = 2 * c + (q & 1);
                double v = 0.0;
                if (b < p) {
                    v = B[a * p + b];
                    if (sym) v = 0.5 * (v + B[b * p + a]);
                }
                o2[t] = __float2bfloat16_rn(__double2float_rn(v));
            }
            __syncthreads();
            continue;
        }
        for (int t = threadIdx.x; t < pp; t += blockDim.x) {
            const int b = t / p, a = t - b * p;           // out[t] = B[a][b]
            double v = B[a * p + b];
            if constexpr (MODE == SM_PAIR) {
                const double vs = ldexp(v, -ex);
                const float hi = __double2float_rn(vs);
                out[t] = make_float2(hi, __double2float_rn(vs - (double)hi));
            } else if constexpr (MODE == SM_F64) {
                out[t] = v;
            } else {
                if (sym) v = 0.5 * (v + B[b * p + a]);
                if constexpr (MODE == SM_F32) out[t] = __double2float_rn(v);
                else out[t] = __float2bfloat16_rn(__double2float_rn(v));
            }
        }
        __syncthreads();
    }
}

static int stream_mode(const psr_ctx* ctx) {
    const int prec = ctx->opts.store_prec;
    if (prec == PSR_PREC_FP64) return ctx->opts.fp64_arith == PSR_FP64_NATIVE ? SM_F64 : SM_PAIR;
    return prec == PSR_PREC_FP32 ? SM_F32 : SM_BF16;
}

static size_t stream_elem_bytes(int mode) {
    return (mode == SM_PAIR || mode == SM_F64) ? 8 : (mode == SM_F32 ? 4 : 2);
}

int stream_convert(psr_ctx* ctx, Group& G, const double* db64, cudaStream_t s, int64_t* bytes,
                   const int32_t* entry_of) {
    const int mode = stream_mode(ctx);
    const int nmat = entry_of ? G.count : G.m;
    // BF16 keeps the columns in pairs (p (p + 1) / 2 pairs for odd p)
    const int64_t ne = (int64_t)nmat * G.p * (mode == SM_BF16 ? 2 * ((G.p + 1) / 2) : G.p);
    const size_t es = stream_elem_bytes(mode);
    void* dst = nullptr;
    if (psr::dev_alloc(&dst, es * (size_t)std::max<int64_t>(ne, 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error(ctx, "out of device memory for the streamed inverses");
        return PSR_ERR_OOM;
    }
    int32_t* bexp = nullptr;
    if (mode == SM_PAIR) PSR_CUDA(ctx, psr::dev_alloc(&bexp, sizeof(int32_t) * (size_t)std::max(nmat, 1)));
    const int blocks = std::max(1, std::min(nmat, 152 * 16));
    const int sym = ctx->opts.symmetrize;
    count_launch();
    switch (mode) {
        case SM_PAIR: k_to_stream<SM_PAIR><<<blocks, 256, 0, s>>>(db64, nmat, G.p, sym, dst, bexp, entry_of); break;
        case SM_F64: k_to_stream<SM_F64><<<blocks, 256, 0, s>>>(db64, nmat, G.p, sym, dst, bexp, entry_of); break;
        case SM_F32: k_to_stream<SM_F32><<<blocks, 256, 0, s>>>(db64, nmat, G.p, sym, dst, bexp, entry_of); break;
        default: k_to_stream<SM_BF16><<<blocks, 256, 0, s>>>(db64, nmat, G.p, sym, dst, bexp, entry_of); break;
    }
    PSR_CHECK_LAUNCH(ctx, "k_to_stream");
    G.rinv = dst;
    G.bexp = bexp;
    G.stream = true;
    *bytes = ne * (int64_t)es;
    return PSR_OK;
}

// Clustered FP64 entries (m of them) as scaled pairs in the column-major
// layout of the stream: the same conversion, applied to the database.
int pair_db_convert(psr_ctx* ctx, Group& G, const double* db64, cudaStream_t s) {
    const int64_t ne = (int64_t)G.m * G.p * G.p;
    float2* dst = nullptr;
    PSR_CUDA(ctx, psr::dev_alloc(&dst, sizeof(float2) * (size_t)std::max<int64_t>(ne, 1)));
    PSR_CUDA(ctx, psr::dev_alloc(&G.bexp, sizeof(int32_t) * (size_t)std::max(G.m, 1)));
    const int blocks = std::max(1, std::min(G.m, 152 * 8));
    count_launch();
    k_to_stream<SM_PAIR><<<blocks, 256, 0, s>>>(db64, G.m, G.p, 0, dst, G.bexp, nullptr);
    PSR_CHECK_LAUNCH(ctx, "pair database conversion");
    G.rinv_pair = dst;
    return PSR_OK;
}

// Clustered sweep, p <= 32, FP64 entries on FP32 pair arithmetic: one patch
// per thread (warp tiles of patches sharing one entry, as k_sweep_tpp), the
// entry read as pairs (every lane reads the same element: one transaction),
// the patch's weighted residual split into pairs after a power-of-two shift
// that brings its largest entry into [1, 2), each row of B^-1 r_k summed
// with compensated products, the result unshifted in FP64.  The FP64 pipe
// keeps the gathers' weighting, the row results and their weighting (about
// 6p FP64 operations per patch instead of the p^2 FMAs of the FP64 form).
template <int PM>
__global__ void __launch_bounds__(256) k_sweep_tpp_pair(const int32_t* __restrict__ wtiles, int nwt, int p, int count,
                                                        const float2* __restrict__ Bt, const int32_t* __restrict__ bexp,
                                                        const int32_t* __restrict__ sdofs_t,
                                                        const double* __restrict__ r, const double* __restrict__ wg,
                                                        const double* __restrict__ wsc, double* __restrict__ z,
                                                        const int32_t* __restrict__ stop) {
    if (stop && *stop) return;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nwt; t += nw) {
        const int c = wtiles[3 * t], start = wtiles[3 * t + 1], cnt = wtiles[3 * t + 2];
        const bool live = lane < cnt;
        const int k = start + (live ? lane : 0);
        int dof[PM];
#pragma unroll
        for (int a = 0; a < PM; ++a) dof[a] = __ldg(sdofs_t + (int64_t)min(a, p - 1) * count + k);
        double rv[PM];
#pragma unroll
        for (int a = 0; a < PM; ++a) rv[a] = __ldg(r + dof[a]);
        if (wg) {
#pragma unroll
            for (int a = 0; a < PM; ++a) rv[a] *= __ldg(wg + dof[a]);
        }
        unsigned emax = 0;
#pragma unroll
        for (int a = 0; a < PM; ++a) {
            const unsigned ex = (unsigned)(__double2hiint(rv[a]) >> 20) & 0x7ffu;
            if (a < p && ex != 0x7ffu) emax = max(emax, ex);
        }
        const int shift = (int)emax - 1023;
        float2 x[PM];
#pragma unroll
        for (int a = 0; a < PM; ++a) x[a] = (live && a < p) ? split_scaled(rv[a], shift) : make_float2(0.f, 0.f);
        const float2* B = Bt + (int64_t)c * p * p;       // B[a][b] at b * p + a
        const int sc = shift + __ldg(bexp + c);
#pragma unroll 1
        for (int a = 0; a < p; ++a) {
            float sh = 0.f, sl = 0.f;
#pragma unroll
            for (int b = 0; b < PM; ++b) {
                if (b < p) {
                    const float2 bv = __ldg(B + b * p + a);
                    pair_fma(sh, sl, bv.x, bv.y, x[b].x, x[b].y);
                }
            }
            if (live) {
                const int d = dof[a];
                atomicAdd(&z[d], ldexp((double)sh + (double)sl, sc) * __ldg(wsc + d));
            }
        }
    }
}

int launch_sweep_tpp_pair(psr_ctx* ctx, const Group& G, const double* r, double* z, const int32_t* stop,
                          cudaStream_t s) {
    const int tb = std::max(1, std::min((G.nwt + 7) / 8, 152 * 16));
    const float2* Bt = reinterpret_cast<const float2*>(G.rinv_pair);
    if (G.p <= 16) {
        count_launch();
        k_sweep_tpp_pair<16><<<tb, 256, 0, s>>>(G.wtiles, G.nwt, G.p, G.count, Bt, G.bexp, G.sdofs_t, r, ctx->Wg,
                                                ctx->W, z, stop);
    } else {
        count_launch();
        k_sweep_tpp_pair<32><<<tb, 256, 0, s>>>(G.wtiles, G.nwt, G.p, G.count, Bt, G.bexp, G.sdofs_t, r, ctx->Wg,
                                                ctx->W, z, stop);
    }
    PSR_CHECK_LAUNCH(ctx, "sweep kernel (thread per patch, FP64 pairs)");
    return PSR_OK;
}

static int stream_slot(int pmax) { return 2 * pmax + 32; }

int stream_build_table(psr_ctx* ctx) {
    std::vector<StreamDesc> t;
    int rb = 0;
    for (auto& G : ctx->groups) {
        if (!G.stream) continue;
        StreamDesc d{G.rinv, G.bexp, G.sdofs, G.count, G.p, rb, 0};
        t.push_back(d);
        const int64_t rows = (int64_t)G.count * G.p;
        rb += (int)((rows + 31) / 32);
    }
    psr::dev_free(ctx->sdesc);
    ctx->sdesc = nullptr;
    ctx->n_stream = (int)t.size();
    ctx->stream_rb = rb;
    if (t.empty()) return PSR_OK;
    if ((int)t.size() > STREAM_MAX_GROUPS) {
        set_error(ctx, "too many patch sizes for the streaming sweep (at most 32)");
        return PSR_ERR_INVALID_ARG;
    }
    PSR_CUDA(ctx, psr::dev_alloc(&ctx->sdesc, sizeof(StreamDesc) * t.size()));
    PSR_CUDA(ctx, cudaMemcpy(ctx->sdesc, t.data(), sizeof(StreamDesc) * t.size(), cudaMemcpyHostToDevice));
    if (ctx->stream_blocks <= 0) ctx->stream_blocks = 152 * 8;
    return PSR_OK;
}

int launch_sweep_stream(psr_ctx* ctx, const double* r, double* z, const int32_t* stop, cudaStream_t s) {
    if (ctx->n_stream == 0 || ctx->stream_rb == 0) return PSR_OK;
    int pmax = 1;
    for (auto& G : ctx->groups)
        if (G.stream) pmax = std::max(pmax, G.p);
    const int mode = stream_mode(ctx);
    const int slot = stream_slot(pmax);
    const size_t xsz = (mode == SM_PAIR || mode == SM_F64) ? 8 : 4;
    const int warps = 8;
    const size_t sm = (size_t)warps * slot * xsz;
    const int blocks = std::max(1, std::min(ctx->stream_blocks, (ctx->stream_rb + warps - 1) / warps));
    const StreamDesc* gd = reinterpret_cast<const StreamDesc*>(ctx->sdesc);
    count_launch();
    switch (mode) {
        case SM_PAIR:
            k_sweep_stream<SM_PAIR><<<blocks, warps * 32, sm, s>>>(gd, ctx->n_stream, ctx->stream_rb, r, ctx->Wg, ctx->W, z, stop, slot);
            break;
        case SM_F64:
            k_sweep_stream<SM_F64><<<blocks, warps * 32, sm, s>>>(gd, ctx->n_stream, ctx->stream_rb, r, ctx->Wg, ctx->W, z, stop, slot);
            break;
        case SM_F32:
            k_sweep_stream<SM_F32><<<blocks, warps * 32, sm, s>>>(gd, ctx->n_stream, ctx->stream_rb, r, ctx->Wg, ctx->W, z, stop, slot);
            break;
        default:
            k_sweep_stream<SM_BF16><<<blocks, warps * 32, sm, s>>>(gd, ctx->n_stream, ctx->stream_rb, r, ctx->Wg, ctx->W, z, stop, slot);
            break;
    }
    PSR_CHECK_LAUNCH(ctx, "k_sweep_stream");
    return PSR_OK;
}

void stream_free(psr_ctx* ctx) {
    psr::dev_free(ctx->sdesc);
    ctx->sdesc = nullptr;
    ctx->n_stream = 0;
    ctx->stream_rb = 0;
}

}  // namespace psr
