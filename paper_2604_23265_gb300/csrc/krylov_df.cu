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

// kDot, kUpdateDot, kUpdateNorm: the three passes of CGS2 (below).  The
// solver's deferred form uses two passes a step (launch_cgs2_deferred_df):
//   kFixDot        v_j = (u_j - V c) / beta on the staged row j (the previous
//                  step's second projection, deferred), then h1 = V^T w.
//                  h1 is formed in FP32 from the hi planes (about 1e-5 of
//                  ||w||): the step subtracts exactly the h1 it formed (the
//                  next pass, in df64), and the second projection h2 = V^T w'
//                  is df64, so h1 + h2 is V^T w and the basis orthogonal to
//                  df64 accuracy as long as ||w'|| is not below about 1e-4
//                  ||w|| (below, the loss of orthogonality grows as
//                  1e-4 ||w|| / ||w'|| times 2^-48)
//   kUpdateDotNorm w' = w - V h1 into the slot of u_{j+1}, then h2 = V^T w'
//                  and ||w'||^2
enum Mode { kDot = 0, kUpdateDot = 1, kUpdateNorm = 2, kFixDot = 3, kUpdateDotNorm = 4 };

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
// budget, 2..8 (chunk i: stage i mod NS, group i mod 2).  With an odd count a
// stage serves the two groups in turn, and a group could reach a stage's
// "full" barrier two phases ahead of the other group's use of it, which the
// parity wait cannot tell from a completed phase; so there a group first
// waits for the other group's release of the stage's previous chunk (its
// "empty" phase, which cannot be two phases behind).  Shared memory of the
// block: NS stages of (K + 1) rows.
__host__ __device__ __forceinline__ int gs_stages(int K) {
    const int stage = (K + 1) * kRowBytes;
    const int ns = kStageBudget / stage;
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
    double* partials;         // [nb][kMaxKrylov], then [nb] (pass 1: ||w||^2)
    unsigned* counter;
    double* out;              // pass 1, 2: [K]; pass 3: [K + 1]
    float* wout;              // phase A result (df64): kFixDot the fixed row j, else w' (null: w)
    const double* beta;       // kFixDot: v_j = (u_j - V c) / beta[0]
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
    // the coefficients of phase A as packed pairs, per row: (h, h), (-h, -h)
    // for the hi part and (-l, -l) for the lo part; rows past K: h = 0
    __shared__ __align__(16) df::f2 hc[kMaxKrylov + 8][4];
    __shared__ int s_issued;
    __shared__ bool s_last;
    __shared__ float s_bh, s_bl;                                   // kFixDot: 1 / beta
    constexpr bool kUpdate = MODE != kDot;                          // has phase A
    constexpr bool kDots = MODE != kUpdateNorm;                     // has phase B
    constexpr bool kNorm = MODE == kUpdateNorm || MODE == kUpdateDotNorm;
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
    // phase A coefficients: kFixDot c over the rows before the fixed one
    const int KA = MODE == kFixDot ? K - 1 : K;
    if (MODE == kFixDot && tid == 0) df::from_double(1.0 / a.beta[0], s_bh, s_bl);
    for (int k = tid; k < kMaxKrylov + 8; k += kThr) {
        float x = 0.f, y = 0.f;
        if (kUpdate && k < KA) df::from_double(a.hin[k], x, y);
        hc[k][0] = df::pk(x, x);
        hc[k][1] = df::pk(-x, -x);
        hc[k][2] = df::pk(-y, -y);
        hc[k][3] = 0ull;
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
            bool got = true;
            if ((NS & 1) && i >= NS) got = mbar_wait(&empty[s], (unsigned)((i / NS) - 1) & 1u);
            got = got && mbar_wait(&full[s], (unsigned)(i / NS) & 1u);
            if (!group_all(g, got)) {
                ok = false;
                break;
            }
            const int64_t base = (int64_t)(bid + (int64_t)i * nb) * kE;
            const int rem = (int)(n - base < kE ? n - base : kE);
            float* st = reinterpret_cast<float*>(smem + (size_t)s * stage_bytes);
            float* wrow = st + K * (kRowBytes / 4);
            auto row_of = [&](int k) -> const float* { return k < K ? st + k * 2 * kE : zero_row; };
            if (kUpdate) {
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
                        const f2 bh = hc[k][0], nbh = hc[k][1], nbl = hc[k][2];
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
                    // t <- t - u for the pair (kFixDot: times 1 / beta), into
                    // the stage and HBM; t is w, or the row being fixed
                    float* trow = MODE == kFixDot ? st + (K - 1) * 2 * kE : wrow;
                    float* gout = a.wout ? a.wout : a.w;
                    float uh[2], ul[2], wh[2], wl[2];
                    df::upk(u2, uh[0], uh[1]);
                    df::upk(uc, ul[0], ul[1]);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        df::sub(trow[e0 + q], trow[kE + e0 + q], uh[q], ul[q], wh[q], wl[q]);
                        if (MODE == kFixDot) {
                            float p, e;
                            df::mul(wh[q], wl[q], s_bh, s_bl, p, e);
                            df::two_sum(p, e, wh[q], wl[q]);
                        }
                        trow[e0 + q] = wh[q];
                        trow[kE + e0 + q] = wl[q];
                    }
                    if (e0 < rem) {                          // rem is a multiple of 4
                        *reinterpret_cast<float2*>(gout + base + e0) = make_float2(wh[0], wh[1]);
                        *reinterpret_cast<float2*>(gout + n + base + e0) = make_float2(wl[0], wl[1]);
                        if (kNorm) {
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
                if (kDots) group_sync(g);
            }
            if (kDots) {
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
                        if (MODE == kFixDot) {
                            // the first projection h1 of the deferred step:
                            // FP32 products of the hi planes, summed in FP32
                            // per lane (see kFixDot above)
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const f2 vh = *reinterpret_cast<const f2*>(row + 2 * (l16 + 16 * t));
                                S2[r] = df::fma2(vh, wh2[t], S2[r]);
                            }
                        } else {
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const int e0 = 2 * (l16 + 16 * t);
                                const f2 vh = *reinterpret_cast<const f2*>(row + e0);
                                const f2 vl = *reinterpret_cast<const f2*>(row + kE + e0);
                                df::mac2(S2[r], C2[r], vh, vl, nwh2[t], nwl2[t], wh2[t]);
                            }
                            // renormalised every second chunk of the group
                            // (the small parts of eight products at most)
                            if ((i >> 1) & 1) df::renorm2(S2[r], C2[r]);
                        }
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
    if (kDots) {
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
            if (kNorm) {
                const double v = warp_sum(df::to_double(nS, nC));
                if (lane == 0) red[2 * kMaxKrylov + wq] = v;
            }
        }
        __syncthreads();
        for (int k = tid; k < K; k += kThr)
            a.partials[(size_t)bid * kMaxKrylov + k] = red[k] + red[kMaxKrylov + k] + bad;
        if (kNorm && tid == 0) {
            double t = 0.0;
            for (int q = 0; q < kCons; ++q) t += red[2 * kMaxKrylov + q];
            a.partials[(size_t)nb * kMaxKrylov + bid] = t + bad;
        }
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
        // four independent chains, so the loads of a lane are in flight together
        const double* pk = a.partials + k;
        double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
        int b = lane;
        for (; b + 96 < nb; b += 128) {
            t0 += __ldcg(pk + (size_t)b * kMaxKrylov);
            t1 += __ldcg(pk + (size_t)(b + 32) * kMaxKrylov);
            t2 += __ldcg(pk + (size_t)(b + 64) * kMaxKrylov);
            t3 += __ldcg(pk + (size_t)(b + 96) * kMaxKrylov);
        }
        for (; b < nb; b += 32) t0 += __ldcg(pk + (size_t)b * kMaxKrylov);
        double t = warp_sum((t0 + t1) + (t2 + t3));
        if (lane == 0) {
            if (MODE == kUpdateNorm)
                a.out[K] = sqrt(t);
            else
                a.out[k] = t;
        }
    }
    if (MODE == kUpdateNorm)
        for (int k = tid; k < K; k += kThr) a.out[k] = a.h1[k] + a.hin[k];
    if (MODE == kUpdateDotNorm && wq == 0) {
        // ||w'||^2 over the blocks into out[K]
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(a.partials + (size_t)nb * kMaxKrylov + b);
        t = warp_sum(t);
        if (lane == 0) a.out[K] = t;
    }
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

// grouped solves: the two passes of the deferred step for every item
template <int MODE>
__global__ void __launch_bounds__(kThr, 2) k_gs_group(const GroupItem* __restrict__ items, int count,
                                                       const GsMaps* __restrict__ maps) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
    static_assert(MODE == kFixDot || MODE == kUpdateDotNorm, "grouped passes: the deferred step");
    const int q = MODE == kFixDot ? group_item_of<&GroupItem::b_md>(items, count)
                                  : group_item_of<&GroupItem::b_ud>(items, count);
    const GroupItem& it = items[q];
    GsArgs a;
    a.V = it.V;
    a.K = it.K;
    a.n = it.n;
    a.w = it.w;
    a.partials = it.partials;
    a.counter = it.counter;
    a.h1 = nullptr;
    float* V = const_cast<float*>(it.V);
    if (MODE == kFixDot) {
        a.hin = it.cfix;
        a.out = it.h1;
        a.wout = V + (size_t)2 * (it.K - 1) * it.n;
        a.beta = it.betas + (it.K - 1);
        gs_run<MODE>(a, &maps[q].v, &maps[q].w, true, blockIdx.x - it.b_md, it.n_md, smem);
    } else {
        a.hin = it.h1;
        a.out = it.h2;
        a.wout = V + (size_t)2 * it.K * it.n;
        a.beta = nullptr;
        gs_run<MODE>(a, &maps[q].v, &maps[q].w, true, blockIdx.x - it.b_ud, it.n_ud, smem);
    }
}

size_t gs_smem_max() {
    size_t m = 0;
    for (int K = 1; K <= kMaxKrylov; ++K) m = gs_smem(K) > m ? gs_smem(K) : m;
    return m;
}

template <int MODE>
void set_smem_limit() {
    raise_smem_limit((const void*)k_gs<MODE>, gs_smem_max());
}

void set_all_smem_limits() {
    static std::once_flag once;
    std::call_once(once, [] {
        set_smem_limit<kDot>();
        set_smem_limit<kUpdateDot>();
        set_smem_limit<kUpdateNorm>();
        set_smem_limit<kFixDot>();
        set_smem_limit<kUpdateDotNorm>();
        raise_smem_limit((const void*)k_gs_group<kFixDot>, gs_smem_max());
        raise_smem_limit((const void*)k_gs_group<kUpdateDotNorm>, gs_smem_max());
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
    a.wout = nullptr;
    a.beta = nullptr;
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

void launch_cgs2_deferred_df(rte_ctx* ctx, float* V, int j, const float* w, const double* c,
                             const double* beta_j, double* h1, double* h2nu) {
    const int K = j + 1;
    if (K < 1 || K > kMaxKrylov) throw StatusError{RTE_EINVAL, "Gram-Schmidt: K out of range"};
    const int64_t n = ctx->n;
    GsArgs a;
    a.V = V;
    a.K = K;
    a.n = n;
    a.w = const_cast<float*>(w);
    a.partials = ctx->partials;
    a.counter = ctx->counter;
    a.h1 = nullptr;
    const size_t smem = gs_smem(K);
    GsMaps maps;
    encode_maps(&maps, V, K, w, n);
    {
        const int g = gs_blocks<kFixDot>(ctx, K, n);
        ProfScope ps(ctx, K_FIX_DOT, (double)(K + 2) * n * 8, 1, (4.0 * K - 2.0) * n);
        a.hin = c;
        a.out = h1;
        a.wout = V + (size_t)2 * j * n;
        a.beta = beta_j;
        k_gs<kFixDot><<<g, kThr, smem, ctx->stream>>>(a, maps);
        check(cudaGetLastError(), "k_gs (fix v_j, V^T w)");
    }
    {
        const int g = gs_blocks<kUpdateDotNorm>(ctx, K, n);
        ProfScope ps(ctx, K_UPDATE_DOT_NORM, (double)(K + 2) * n * 8, 1, (4.0 * K + 2.0) * n);
        a.hin = h1;
        a.out = h2nu;
        a.wout = V + (size_t)2 * (j + 1) * n;
        a.beta = nullptr;
        k_gs<kUpdateDotNorm><<<g, kThr, smem, ctx->stream>>>(a, maps);
        check(cudaGetLastError(), "k_gs (update, V^T w', ||w'||)");
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

void group_ortho_geometry_df(rte_ctx* ctx, int K, int* n_md, int* n_ud) {
    *n_md = gs_blocks<kFixDot>(ctx, K, ctx->n);
    *n_ud = gs_blocks<kUpdateDotNorm>(ctx, K, ctx->n);
}

size_t group_gs_maps_bytes() { return sizeof(GsMaps); }

void encode_group_gs_maps(const GroupItem* items_host, int count, void* maps_host) {
    GsMaps* m = static_cast<GsMaps*>(maps_host);
    for (int q = 0; q < count; ++q) encode_maps(&m[q], items_host[q].V, items_host[q].K, items_host[q].w, items_host[q].n);
}

void launch_group_orthogonalise_df(const GroupItem* items_dev, const void* maps_dev, int count, int blocks_md,
                                   int blocks_ud, int kmax, cudaStream_t st) {
    const GsMaps* maps = static_cast<const GsMaps*>(maps_dev);
    set_all_smem_limits();
    // every item's stages within the shared memory of the launch
    size_t smem = 0;
    for (int K = 1; K <= kmax; ++K) smem = gs_smem(K) > smem ? gs_smem(K) : smem;
    k_gs_group<kFixDot><<<blocks_md, kThr, smem, st>>>(items_dev, count, maps);
    k_gs_group<kUpdateDotNorm><<<blocks_ud, kThr, smem, st>>>(items_dev, count, maps);
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
