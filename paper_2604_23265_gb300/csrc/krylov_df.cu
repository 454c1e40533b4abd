// Gram-Schmidt of the flexible-GMRES Arnoldi step on df64 vectors (FP32 pipe).
//
// The Krylov basis V (K vectors) and the vector w are df64 (df64.h: planar
// hi / lo floats, 48 significant bits, 8 bytes per element like a double).
// Classical Gram-Schmidt with one reorthogonalisation in three passes, each
// bound by HBM:
//   pass 1  h1 = V^T w
//   pass 2  w <- w - V h1,  h2 = V^T w          (V read from HBM once)
//   pass 3  w <- w - V h2,  ||w||^2
// A pass is a persistent grid of blocks of eight consumer warps and one
// producer warp.  Block b owns the 128-element chunks c = b, b + nb, ...; the
// producer loads a chunk's rows into a shared-memory stage with two TMA
// tensor copies (one box of the 2K basis rows, hi and lo planes, one of w),
// completing on the stage's "full" mbarrier, up to NS stages ahead, and
// reuses a stage once the warps that consumed it arrived on its "empty"
// mbarrier.  A box past n is zero-filled by the copy.  The consumers form two
// groups of four warps that take alternate chunks, so a group's barriers
// never wait for the other group and two chunks are in work at once.  On a
// staged chunk, in group g:
//   phase A (passes 2, 3): warp w owns the element pairs 16 w .. 16 w + 15;
//     its two half warps sum h_k V_k over the even and the odd rows (two
//     chains each), a shuffle adds the halves, and w_t <- w_t - sum_k h_k V_kt
//     (df64) goes to HBM and back into the stage (pass 2: group barrier);
//   phase B (passes 1, 2): half warp h of warp w owns the rows k = w + 4 h,
//     w + 4 h + 8, ...; lane l accumulates V_ke w_e over its elements
//     e = 2 l + 32 t, 2 l + 32 t + 1 (t < 4) into one df64 sum per owned row,
//     kept in registers for the whole pass.
// Lanes work on element pairs with the packed .f32x2 instructions and rows
// past K read a zero row.  So the re-read of V that the update and the
// projection of pass 2 need comes from shared memory, not from HBM.  Each
// block adds its two groups' sums in FP64 in a fixed order and the last block
// (atomic ticket) adds the block partials in block order: the result depends
// only on (K, n), never on scheduling.
//
// Waits are bounded: a wait that does not complete in 2^24 polls ends the
// group's loop (its warps agree on it through a barrier reduction), sets
// g_krylov_timeout, waits (bounded) for the copies still in flight, and
// writes NaN partial sums, so the step's Hessenberg column is NaN and the
// solver treats the step as failed.
#include <cuda.h>

#include <mutex>

#include "async_ptx.h"
#include "df64.h"
#include "rte_internal.h"

namespace rte {

__device__ int g_krylov_timeout = 0;

namespace {

constexpr int kE = 128;                       // elements per chunk
constexpr int kCons = 8;                      // consumer warps
constexpr int kConsThr = kCons * 32;          // consumer threads
constexpr int kThr = kConsThr + 32;           // plus one producer warp
constexpr int kGroups = 2;                    // consumer groups: group g takes the chunks i = g mod 2
constexpr int kGW = kCons / kGroups;          // warps of a group
constexpr int kGroupThr = kGW * 32;
constexpr int kOwnB = kMaxKrylov / (2 * kGW); // phase B rows of a half warp (k = w + 4 half mod 8)
constexpr int kMaxStages = 8;
constexpr int kRowBytes = kE * 8;             // one staged row: hi then lo, 128 floats each
constexpr int kStageBudget = 102 * 1024;      // shared memory the stages of a block aim at

enum Mode { kDot = 0, kUpdateDot = 1, kUpdateNorm = 2 };

using namespace ::rte::ptx;

// named barrier 2 + g among the warps of consumer group g (immediate ids,
// so the block reserves only the barriers it uses)
__device__ __forceinline__ void group_sync(int g) {
    if (g == 0)
        asm volatile("bar.sync 2, %0;" ::"n"(kGroupThr) : "memory");
    else
        asm volatile("bar.sync 3, %0;" ::"n"(kGroupThr) : "memory");
}

// the same barrier, returning the AND of v over the group
__device__ __forceinline__ bool group_all(int g, bool v) {
    unsigned r;
    if (g == 0)
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.ne.u32 q, %1, 0;\n\t"
            "bar.red.and.pred p, 2, %2, q;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(r)
            : "r"((unsigned)v), "n"(kGroupThr)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.ne.u32 q, %1, 0;\n\t"
            "bar.red.and.pred p, 3, %2, q;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(r)
            : "r"((unsigned)v), "n"(kGroupThr)
            : "memory");
    return r != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// sum over the 16 lanes of each half warp (lane 0 and lane 16 hold the sums)
__device__ __forceinline__ double half_warp_sum(double v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, 16);
    return v;
}

// Pipeline depth of a block for K basis rows: as many stages as fit the
// budget, an even number in 2..8, so that every stage serves one consumer
// group (chunk i: stage i mod NS, group i mod 2).  With an odd count a stage
// would alternate between the groups, and a group could wait on a stage's
// "full" barrier two phases ahead of the other group's use of it, which the
// parity wait cannot tell from a completed phase.  Shared memory of the
// block: NS stages of (K + 1) rows.
__host__ __device__ __forceinline__ int gs_stages(int K) {
    const int stage = (K + 1) * kRowBytes;
    int ns = (kStageBudget / stage) & ~1;
    return ns < 2 ? 2 : (ns > kMaxStages ? kMaxStages : ns);
}
__host__ __device__ __forceinline__ size_t gs_smem(int K) {
    // stages, one zero row, and slack for aligning the stages to 128 bytes
    return (size_t)gs_stages(K) * (K + 1) * kRowBytes + kRowBytes + 128;
}

struct GsArgs {
    const float* V;           // K df64 vectors, vector k at V + 2 k n
    int K;
    int64_t n;
    float* w;                 // df64 [n]
    const double* hin;        // passes 2, 3: the projection subtracted
    const double* h1;         // pass 3: out[k] = h1[k] + hin[k]
    double* partials;         // [nb][kMaxKrylov]
    unsigned* counter;
    double* out;              // pass 1, 2: [K]; pass 3: [K + 1]
};

// Tensor maps of one pass: the K basis vectors as 2K rows of n floats (row
// 2k the hi plane of vector k, 2k + 1 its lo plane; box 128 x 2K) and w as 2
// rows (box 128 x 2).  A box past n is zero-filled.
struct GsMaps {
    CUtensorMap v, w;
};

template <int MODE>
__device__ void gs_run(const GsArgs& a, const CUtensorMap* mv, const CUtensorMap* mw, bool global_maps, int bid,
                       int nb, unsigned char* smem) {
    using df::f2;
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ float hh[kMaxKrylov + 8], hl[kMaxKrylov + 8];      // rows past K: h = 0
    __shared__ int s_issued;
    __shared__ bool s_last;
    const int K = a.K, tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
    const bool producer = wq == kCons;
    const int64_t n = a.n;
    const int NS = gs_stages(K);
    const int stage_bytes = (K + 1) * kRowBytes;
    const int64_t nchunks = (n + kE - 1) / kE;
    const int mine = bid < nchunks ? (int)((nchunks - 1 - bid) / nb + 1) : 0;
    float* zero_row = reinterpret_cast<float*>(smem + (size_t)NS * stage_bytes);

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kGW);
        }
        mbar_init_fence();
        s_issued = 0;
    }
    for (int e = tid; e < 2 * kE; e += kThr) zero_row[e] = 0.f;
    for (int k = tid; k < kMaxKrylov + 8; k += kThr) {
        float x = 0.f, y = 0.f;
        if (MODE != kDot && k < K) df::from_double(a.hin[k], x, y);
        hh[k] = x;
        hl[k] = y;
    }
    __syncthreads();

    bool ok = true;
    const int g = (wq / kGW) & 1, gw = wq % kGW;                  // consumer group, warp in the group
    const int half = lane >> 4, l16 = lane & 15;
    f2 S2[kOwnB], C2[kOwnB];
#pragma unroll
    for (int r = 0; r < kOwnB; ++r) S2[r] = C2[r] = 0ull;
    float nS = 0.f, nC = 0.f;

    if (producer) {
        // chunk i into stage i % NS once its group released the stage: one
        // TMA box for the basis rows and one for w
        if (lane == 0) {
            if (global_maps) {
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mv) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mw) : "memory");
            }
            int i = 0;
            for (; i < mine; ++i) {
                const int s = i % NS;
                if (i >= NS && !mbar_wait(&empty[s], (unsigned)((i / NS) + 1) & 1u)) {
                    ok = false;
                    break;
                }
                const int x = (int)((int64_t)(bid + (int64_t)i * nb) * kE);
                unsigned char* st = smem + (size_t)s * stage_bytes;
                mbar_expect(&full[s], (uint32_t)stage_bytes);
                fence_proxy_async();
                tma_load_2d(st, mv, x, 0, &full[s]);
                tma_load_2d(st + K * kRowBytes, mw, x, 0, &full[s]);
            }
            s_issued = i;
        }
        __syncwarp();
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    } else {
        const int RA = (K + 1) / 2;                                // phase A rows of a half warp (k = half mod 2)
        const int RB = (K + 2 * kGW - 1) / (2 * kGW);              // phase B rows of a half warp
        for (int i = g; i < mine; i += kGroups) {
            const int s = i % NS;
            const bool got = mbar_wait(&full[s], (unsigned)(i / NS) & 1u);
            if (!group_all(g, got)) {
                ok = false;
                break;
            }
            const int64_t base = (int64_t)(bid + (int64_t)i * nb) * kE;
            const int rem = (int)(n - base < kE ? n - base : kE);
            float* st = reinterpret_cast<float*>(smem + (size_t)s * stage_bytes);
            float* wrow = st + K * (kRowBytes / 4);
            auto row_of = [&](int k) -> const float* { return k < K ? st + k * 2 * kE : zero_row; };
            if (MODE != kDot) {
                // phase A: warp gw owns the element pairs 16 gw + l16; half warp
                // `half` sums h_k V_k over the rows k = half + 2 j in two chains,
                // and the halves are added by a shuffle: no cross-warp sum
                const int e0 = 32 * gw + 2 * l16;
                f2 uS[2] = {0ull, 0ull}, uC[2] = {0ull, 0ull};
                for (int j = 0; j < RA; j += 2) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int k = half + 2 * (j + c);
                        const float* row = row_of(k);
                        const f2 bh = df::pk(hh[k], hh[k]);
                        const f2 nbh = df::pk(-hh[k], -hh[k]), nbl = df::pk(-hl[k], -hl[k]);
                        const f2 vh = *reinterpret_cast<const f2*>(row + e0);
                        const f2 vl = *reinterpret_cast<const f2*>(row + kE + e0);
                        df::mac2(uS[c], uC[c], vh, vl, nbh, nbl, bh);
                    }
                }
                f2 us, ut;
                df::two_sum2(uS[0], uS[1], us, ut);
                f2 uc = df::add2(ut, df::add2(uC[0], uC[1]));
                const f2 os = __shfl_xor_sync(0xffffffffu, us, 16), oc = __shfl_xor_sync(0xffffffffu, uc, 16);
                f2 u2, ut2;
                df::two_sum2(us, os, u2, ut2);
                uc = df::add2(ut2, df::add2(uc, oc));
                df::renorm2(u2, uc);
                if (half == 0) {
                    // w <- w - u for the pair, into the stage and HBM
                    float uh[2], ul[2], wh[2], wl[2];
                    df::upk(u2, uh[0], uh[1]);
                    df::upk(uc, ul[0], ul[1]);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        df::sub(wrow[e0 + q], wrow[kE + e0 + q], uh[q], ul[q], wh[q], wl[q]);
                        wrow[e0 + q] = wh[q];
                        wrow[kE + e0 + q] = wl[q];
                    }
                    if (e0 < rem) {                          // rem is a multiple of 4
                        *reinterpret_cast<float2*>(a.w + base + e0) = make_float2(wh[0], wh[1]);
                        *reinterpret_cast<float2*>(a.w + n + base + e0) = make_float2(wl[0], wl[1]);
                        if (MODE == kUpdateNorm) {
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                float p, e;
                                df::mul(wh[q], wl[q], wh[q], wl[q], p, e);
                                df::acc(nS, nC, p, e);
                            }
                            df::renorm(nS, nC);
                        }
                    }
                }
                if (MODE == kUpdateDot) group_sync(g);
            }
            if (MODE != kUpdateNorm) {
                // phase B: half warp `half` of warp gw owns the rows
                // k = gw + 4 half + 8 r; lane l16 the pairs l16 + 16 t
                f2 wh2[4], wl2[4], nwh2[4], nwl2[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e0 = 2 * (l16 + 16 * t);
                    wh2[t] = *reinterpret_cast<const f2*>(wrow + e0);
                    wl2[t] = *reinterpret_cast<const f2*>(wrow + kE + e0);
                    nwh2[t] = df::sub2(0ull, wh2[t]);
                    nwl2[t] = df::sub2(0ull, wl2[t]);
                }
#pragma unroll
                for (int r = 0; r < kOwnB; ++r) {
                    if (r < RB) {
                        const float* row = row_of(gw + kGW * half + 2 * kGW * r);
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int e0 = 2 * (l16 + 16 * t);
                            const f2 vh = *reinterpret_cast<const f2*>(row + e0);
                            const f2 vl = *reinterpret_cast<const f2*>(row + kE + e0);
                            df::mac2(S2[r], C2[r], vh, vl, nwh2[t], nwl2[t], wh2[t]);
                        }
                        df::renorm2(S2[r], C2[r]);
                    }
                }
            }
            // this warp is done with stage s
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    if (!__syncthreads_and(ok)) {
        // wait (bounded) for the last copy issued into every stage
        if (tid == 0) {
            atomicExch(&g_krylov_timeout, 1);
            const int iss = s_issued;
            for (int s = 0; s < NS && s < iss; ++s) {
                const int last = s + ((iss - 1 - s) / NS) * NS;
                mbar_wait(&full[s], (unsigned)(last / NS) & 1u);
            }
        }
        ok = false;
    }
    __syncthreads();

    // block sums (FP64, fixed order) into the first stage, then the last
    // block adds the blocks
    double* red = reinterpret_cast<double*>(smem);                 // [kGroups][kMaxKrylov]
    const double bad = ok ? 0.0 : __longlong_as_double(0x7ff8000000000000LL);
    if (MODE != kUpdateNorm) {
        if (!producer) {
#pragma unroll
            for (int r = 0; r < kOwnB; ++r) {
                const int k = gw + kGW * half + 2 * kGW * r;
                float sx, sy, cx, cy;
                df::upk(S2[r], sx, sy);
                df::upk(C2[r], cx, cy);
                const double v = half_warp_sum(df::to_double(sx, cx) + df::to_double(sy, cy));
                if (l16 == 0 && k < K) red[g * kMaxKrylov + k] = v;
            }
        }
        __syncthreads();
        for (int k = tid; k < K; k += kThr)
            a.partials[(size_t)bid * kMaxKrylov + k] = red[k] + red[kMaxKrylov + k] + bad;
    } else {
        const double v = producer ? 0.0 : warp_sum(df::to_double(nS, nC));
        if (lane == 0) red[wq] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < kCons; ++q) t += red[q];
            a.partials[(size_t)bid * kMaxKrylov] = t + bad;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.counter, 1u) == (unsigned)nb - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int R = MODE == kUpdateNorm ? 1 : K;
    for (int k = wq; k < R; k += kThr / 32) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(a.partials + (size_t)b * kMaxKrylov + k);
        t = warp_sum(t);
        if (lane == 0) {
            if (MODE == kUpdateNorm)
                a.out[K] = sqrt(t);
            else
                a.out[k] = t;
        }
    }
    if (MODE == kUpdateNorm)
        for (int k = tid; k < K; k += kThr) a.out[k] = a.h1[k] + a.hin[k];
    if (tid == 0) *a.counter = 0u;
}

template <int MODE>
__global__ void __launch_bounds__(kThr, 2) k_gs(const __grid_constant__ GsArgs a, const __grid_constant__ GsMaps m) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations: 128-byte aligned (the launch adds 128 bytes of slack)
    unsigned char* smem = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
    gs_run<MODE>(a, &m.v, &m.w, false, blockIdx.x, gridDim.x, smem);
}

// v = w / s[0] (s[0] == 0: v = w), df64 in and out
__device__ void scale_df_run(const float* __restrict__ w, const double* __restrict__ s, int64_t n,
                             float* __restrict__ v, int bid, int nb) {
    __shared__ float ih, il;
    if (threadIdx.x == 0) {
        const double d = s[0];
        df::from_double(d != 0.0 ? 1.0 / d : 1.0, ih, il);
    }
    __syncthreads();
    const float bh = ih, bl = il;
    for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x) {
        float p, e, h, l;
        df::mul(w[i], w[n + i], bh, bl, p, e);
        df::two_sum(p, e, h, l);
        v[i] = h;
        v[n + i] = l;
    }
}

__global__ void __launch_bounds__(256) k_scale_df(const float* __restrict__ w, const double* __restrict__ s,
                                                  int64_t n, float* __restrict__ v) {
    scale_df_run(w, s, n, v, blockIdx.x, gridDim.x);
}

// out = x / s[0] as df64 (s == nullptr: out = x)
__global__ void k_split_df(const double* __restrict__ x, const double* __restrict__ s, int64_t n,
                           float* __restrict__ out) {
    const double inv = s ? (s[0] != 0.0 ? 1.0 / s[0] : 1.0) : 1.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        df::from_double(x[i] * inv, h, l);
        out[i] = h;
        out[n + i] = l;
    }
}

// out = x as double
__global__ void k_compose_df(const float* __restrict__ x, int64_t n, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df::to_double(x[i], x[n + i]);
}

// out = sum_k V_k y_k (df64 sums, double out)
__global__ void k_lincomb_df(const float* __restrict__ V, int K, int64_t n, const double* __restrict__ y,
                             double* __restrict__ out) {
    __shared__ float yh[kMaxKrylov], yl[kMaxKrylov];
    for (int k = threadIdx.x; k < K; k += blockDim.x) df::from_double(y[k], yh[k], yl[k]);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float S = 0.f, C = 0.f;
        for (int k = 0; k < K; ++k) {
            const float* v = V + (size_t)2 * k * n;
            float p, e;
            df::mul(v[i], v[n + i], yh[k], yl[k], p, e);
            df::acc(S, C, p, e);
        }
        out[i] = df::to_double(S, C);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThr, 2) k_gs_group(const GroupItem* __restrict__ items, int count,
                                                       const GsMaps* __restrict__ maps) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
    int q;
    if (MODE == kDot)
        q = group_item_of<&GroupItem::b_md>(items, count);
    else if (MODE == kUpdateDot)
        q = group_item_of<&GroupItem::b_ud>(items, count);
    else
        q = group_item_of<&GroupItem::b_rd>(items, count);
    const GroupItem& it = items[q];
    GsArgs a;
    a.V = it.V;
    a.K = it.K;
    a.n = it.n;
    a.w = it.w;
    a.partials = it.partials;
    a.counter = it.counter;
    if (MODE == kDot) {
        a.hin = nullptr;
        a.h1 = nullptr;
        a.out = it.h1;
        gs_run<MODE>(a, &maps[q].v, &maps[q].w, true, blockIdx.x - it.b_md, it.n_md, smem);
    } else if (MODE == kUpdateDot) {
        a.hin = it.h1;
        a.h1 = nullptr;
        a.out = it.h2;
        gs_run<MODE>(a, &maps[q].v, &maps[q].w, true, blockIdx.x - it.b_ud, it.n_ud, smem);
    } else {
        a.hin = it.h2;
        a.h1 = it.h1;
        a.out = it.hcol;
        gs_run<MODE>(a, &maps[q].v, &maps[q].w, true, blockIdx.x - it.b_rd, it.n_rd, smem);
    }
}

__global__ void __launch_bounds__(256) k_scale_df_group(const GroupItem* __restrict__ items, int count) {
    const GroupItem& it = items[group_item_of<&GroupItem::b_sc>(items, count)];
    scale_df_run(it.w, it.hcol + it.K, it.n, it.Vnext, blockIdx.x - it.b_sc, it.n_sc);
}

template <int MODE>
void set_smem_limit() {
    size_t m = 0;
    for (int K = 1; K <= kMaxKrylov; ++K) m = gs_smem(K) > m ? gs_smem(K) : m;
    raise_smem_limit((const void*)k_gs<MODE>, m);
    raise_smem_limit((const void*)k_gs_group<MODE>, m);
}

void set_all_smem_limits() {
    static std::once_flag once;
    std::call_once(once, [] {
        set_smem_limit<kDot>();
        set_smem_limit<kUpdateDot>();
        set_smem_limit<kUpdateNorm>();
    });
}

// blocks of one pass: one per chunk, at most 4 resident blocks per SM (the
// lone launch's geometry; a grouped launch gives every item the same count)
template <int MODE>
int gs_blocks(rte_ctx* ctx, int K, int64_t n) {
    set_all_smem_limits();
    int per_sm = 0;
    check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs<MODE>, kThr, gs_smem(K)), "occupancy");
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    const int64_t chunks = (n + kE - 1) / kE;
    const int64_t cap = (int64_t)ctx->num_sms * per_sm;
    return (int)(chunks < cap ? (chunks > 0 ? chunks : 1) : cap);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tiled_encoder() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        check(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q),
              "cudaGetDriverEntryPointByVersion");
        if (q != cudaDriverEntryPointSuccess || !p)
            throw StatusError{RTE_ECUDA, "cuTensorMapEncodeTiled is not available"};
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// rows x n floats at base (row stride n floats), box 128 x rows
void encode_rows(CUtensorMap* map, const float* base, int64_t n, int rows) {
    if (reinterpret_cast<uintptr_t>(base) % 16 || n % 4)
        throw StatusError{RTE_EINVAL, "df64 vectors must be 16-byte aligned with n a multiple of 4"};
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kE, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult cr = tiled_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) throw StatusError{RTE_ECUDA, "cuTensorMapEncodeTiled failed (df64 Gram-Schmidt)"};
}

void encode_maps(GsMaps* m, const float* V, int K, const float* w, int64_t n) {
    encode_rows(&m->v, V, n, 2 * K);
    encode_rows(&m->w, w, n, 2);
}

int ew_grid(rte_ctx* ctx, int64_t n) {
    const int64_t want = (n + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

void launch_orthogonalise_df(rte_ctx* ctx, const float* V, int K, float* w, double* h1, double* h2,
                             double* hcol) {
    if (K < 1 || K > kMaxKrylov) throw StatusError{RTE_EINVAL, "Gram-Schmidt: K out of range"};
    const int64_t n = ctx->n;
    GsArgs a;
    a.V = V;
    a.K = K;
    a.n = n;
    a.w = w;
    a.partials = ctx->partials;
    a.counter = ctx->counter;
    const size_t smem = gs_smem(K);
    GsMaps maps;
    encode_maps(&maps, V, K, w, n);
    {
        const int g = gs_blocks<kDot>(ctx, K, n);
        ProfScope ps(ctx, K_MDOT, (double)(K + 1) * n * 8, 1, 2.0 * K * n);
        a.hin = nullptr;
        a.h1 = nullptr;
        a.out = h1;
        k_gs<kDot><<<g, kThr, smem, ctx->stream>>>(a, maps);
        check(cudaGetLastError(), "k_gs (V^T w)");
    }
    {
        const int g = gs_blocks<kUpdateDot>(ctx, K, n);
        ProfScope ps(ctx, K_UPDATE_DOT, (double)(K + 2) * n * 8, 1, 4.0 * K * n);
        a.hin = h1;
        a.out = h2;
        k_gs<kUpdateDot><<<g, kThr, smem, ctx->stream>>>(a, maps);
        check(cudaGetLastError(), "k_gs (update, V^T w)");
    }
    {
        const int g = gs_blocks<kUpdateNorm>(ctx, K, n);
        ProfScope ps(ctx, K_UPDATE_NORM, (double)(K + 2) * n * 8, 1, (2.0 * K + 2.0) * n);
        a.hin = h2;
        a.h1 = h1;
        a.out = hcol;
        k_gs<kUpdateNorm><<<g, kThr, smem, ctx->stream>>>(a, maps);
        check(cudaGetLastError(), "k_gs (update, norm)");
    }
}

void launch_scale_df(rte_ctx* ctx, const float* w, const double* s, float* v) {
    ProfScope ps(ctx, K_SCALE, (double)ctx->n * 16);
    k_scale_df<<<ew_grid(ctx, ctx->n), 256, 0, ctx->stream>>>(w, s, ctx->n, v);
    check(cudaGetLastError(), "k_scale_df");
}

void launch_split_df(rte_ctx* ctx, const double* x, const double* s, float* out) {
    ProfScope ps(ctx, K_SCALE, (double)ctx->n * 16);
    k_split_df<<<ew_grid(ctx, ctx->n), 256, 0, ctx->stream>>>(x, s, ctx->n, out);
    check(cudaGetLastError(), "k_split_df");
}

void launch_compose_df(rte_ctx* ctx, const float* x, double* out) {
    ProfScope ps(ctx, K_SCALE, (double)ctx->n * 16);
    k_compose_df<<<ew_grid(ctx, ctx->n), 256, 0, ctx->stream>>>(x, ctx->n, out);
    check(cudaGetLastError(), "k_compose_df");
}

void launch_lincomb_df(rte_ctx* ctx, const float* V, int K, const double* y, double* out) {
    ProfScope ps(ctx, K_XUPDATE, (double)ctx->n * (8 + 8 * K));
    k_lincomb_df<<<ew_grid(ctx, ctx->n), 256, 0, ctx->stream>>>(V, K, ctx->n, y, out);
    check(cudaGetLastError(), "k_lincomb_df");
}

void group_ortho_geometry_df(rte_ctx* ctx, int K, int* n_md, int* n_ud, int* n_rd, int* n_sc) {
    *n_md = gs_blocks<kDot>(ctx, K, ctx->n);
    *n_ud = gs_blocks<kUpdateDot>(ctx, K, ctx->n);
    *n_rd = gs_blocks<kUpdateNorm>(ctx, K, ctx->n);
    *n_sc = ew_grid(ctx, ctx->n);
}

size_t group_gs_maps_bytes() { return sizeof(GsMaps); }

void encode_group_gs_maps(const GroupItem* items_host, int count, void* maps_host) {
    GsMaps* m = static_cast<GsMaps*>(maps_host);
    for (int q = 0; q < count; ++q) encode_maps(&m[q], items_host[q].V, items_host[q].K, items_host[q].w, items_host[q].n);
}

void launch_group_orthogonalise_df(const GroupItem* items_dev, const void* maps_dev, int count, int blocks_md,
                                   int blocks_ud, int blocks_rd, int blocks_sc, int kmax, cudaStream_t st) {
    const GsMaps* maps = static_cast<const GsMaps*>(maps_dev);
    set_all_smem_limits();
    // every item's stages within the shared memory of the launch
    size_t smem = 0;
    for (int K = 1; K <= kmax; ++K) smem = gs_smem(K) > smem ? gs_smem(K) : smem;
    k_gs_group<kDot><<<blocks_md, kThr, smem, st>>>(items_dev, count, maps);
    k_gs_group<kUpdateDot><<<blocks_ud, kThr, smem, st>>>(items_dev, count, maps);
    k_gs_group<kUpdateNorm><<<blocks_rd, kThr, smem, st>>>(items_dev, count, maps);
    k_scale_df_group<<<blocks_sc, 256, 0, st>>>(items_dev, count);
    check(cudaGetLastError(), "grouped Gram-Schmidt (df64)");
}

int krylov_timeout_flag(bool reset) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_krylov_timeout, sizeof(int)) != cudaSuccess) return -1;
    if (reset && v) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_krylov_timeout, &z, sizeof(int)) != cudaSuccess) return -1;
    }
    return v;
}

}  // namespace rte
