// Tensor-core gather convolution of the MgNet forward pass (Sec. 3.3) at
// inference: BF16 operands, FP32 accumulation in tensor memory (tcgen05).
//
// Implicit GEMM over tap tables:
//   D[p][o] = sum_t sum_i X[b][i][S gy_p + dy_t][S gx_p + dx_t] W[t][i][o]
// with M = 128 class-grid pixels per CTA (pixel row m of the tile owns TMEM
// lane m), N = output channels rounded up to 16 (TMEM columns), and one MMA of
// K = 16 input channels per (tap, channel pair).
//
// Activations between the layers are BF16 in a channel-chunked layout
// "C8" = [B][ceil(C/8)][H][W][8]: the 8 channels of one pixel are one 16-byte
// row of an MMA core matrix.  Both operands use the no-swizzle K-major
// canonical layout (8 rows x 16 bytes per core matrix).
//
// Input staging, by layer:
//  * halo (stride-1 taps within +-1: the 3 x 3 smoothers, the four parity
//    classes of the transposed prolongation, the 1 x 1 projection): one TMA
//    tensor load brings the tile's rows with a one-pixel halo, [KC][BH][BW]
//    x 16 bytes, zero outside the image.  The tile is R rows x SW columns of
//    the class grid (SW = min(W, 128), BW = SW + 2, BH = R + 2) and MMA row m
//    is halo pixel (m / BW + 1, m mod BW + 1), so the A operand of tap
//    (dy, dx) is the same buffer shifted by dy BW + dx rows: no copy per tap.
//    Rows with m mod BW >= SW are computed and discarded.
//  * gather (the stride-2 restriction): tap t of the tile is one 16-byte
//    cp.async per (pixel, chunk), all taps in flight at once when they fit in
//    shared memory, else a ring of three stages overlapping the MMAs.
//  * FP64 (the lift from the Krylov vector [2M][I][I]): loaded and converted
//    by the threads.
//  * streamed (layers whose weights do not stay resident: more than
//    kResidentWeightBytes per CTA, or more than 256 output channels): a ring
//    of stages, stage u = (tap, block of KB channel chunks), each holding the
//    gathered activation rows and the matching weight slice (one bulk copy);
//    output channels beyond 256 are split into equal slices over blockIdx.z.
// The weights of a layer are packed once per weight version into the MMA
// layout (tc_pack) and arrive by bulk async copies of 8 KB.
//
// The four parity classes of a transposed convolution run as one launch
// (blockIdx.y = class, each with its own taps, weights and output offset).
// Layers are chained by programmatic dependent launch: a layer allocates its
// tensor memory and copies its weights while the previous layer runs, waits
// for the previous grid's completion only before touching activations, and
// lets the next layer launch right after that wait.
//
// The epilogue reads the accumulators back with tcgen05.ld (warp w sees lanes
// 32 (w mod 4) ...; the two warps on the same lanes take alternate 16-column
// blocks) and applies v = sign (acc o gate) (+ base) before the store.
// Every wait is bounded: on expiry the CTA records the failure in a device
// flag, writes NaN outputs, releases its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "async_ptx.h"
#include "nn_internal.h"

namespace rte {
namespace nn {
namespace {

constexpr int kRows = 128;           // pixels per CTA = MMA M = TMEM lanes
constexpr int kThreads = 256;
constexpr int kMaxStages = 3;
constexpr size_t kResidentWeightBytes = 112 * 1024;   // per CTA, else streamed
constexpr int kStreamChunks = 8;                       // KB: channel chunks of 8 per stage
constexpr int kMaxSlice = 256;                         // output channels per CTA (MMA N)

enum Mode { kGather = 0, kF64 = 1, kHalo = 2, kStream = 3 };

constexpr int kLiftGroup = 4;        // channel chunks a thread loads at once in the lift

using namespace ::rte::ptx;

__device__ int g_tc_status;          // 1 once a bounded wait expired

// 16-byte async copy global -> shared; bytes beyond src_bytes are zero
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

__device__ __forceinline__ void unpack8(uint4 u, float (&v)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[2 * i] = __uint_as_float(w[i] << 16);
        v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
}

// ReLU of the BF16 pairs of 16 bytes of shared memory
__device__ __forceinline__ void relu16(uint32_t addr) {
    uint32_t w[4];
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                 : "r"(addr));
#pragma unroll
    for (int i = 0; i < 4; ++i) {      // clear negative halves
        const uint32_t lo = (w[i] & 0x8000u) ? 0u : (w[i] & 0xFFFFu);
        const uint32_t hi = (w[i] & 0x80000000u) ? 0u : (w[i] & 0xFFFF0000u);
        w[i] = lo | hi;
    }
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
}

// Issues the MMAs of one accumulation (the first overwrites the accumulator).
struct Chain {
    uint32_t d;
    uint32_t acc = 0;
    __device__ explicit Chain(uint32_t tmem) : d(tmem) {}
    __device__ __forceinline__ void mma(uint64_t ad, uint64_t bd, uint32_t idesc) {
        tc_mma(d, ad, bd, idesc, acc);
        acc = 1;
    }
};

// Geometry of one launch (host computed).
// KC: channel chunks of 8 per MMA row (even); Npad: output channels of this
// CTA (its slice) rounded up to 16; NS: stages (gather and streamed modes);
// ncols: TMEM columns (power of two >= Npad); halo mode: tile SW x R
// class-grid pixels, halo box BW x BH, tiles_x tiles across the width,
// tiles_y down the height; streamed mode: KB chunks per stage, NKB blocks
// per tap; xoff: byte offset of the input staging area (1024-aligned).
struct Geo {
    int KC, Npad, NS;
    uint32_t ncols;
    int SW, R, BW, BH, tiles_x, tiles_y;
    int KB, NKB;
    uint32_t xoff;
};

// Two CTAs per SM (at most 128 registers a thread): on the finest levels the
// grid is several times the SM count, and a second resident CTA overlaps one
// tile's loads and MMAs with the other's epilogue (a third costs spills).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_conv_tc(const __grid_constant__ TcConv a, const Geo g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mma_bar[kMaxStages];
    __shared__ __align__(8) uint64_t wst_bar[kMaxStages];   // streamed mode: weight slice of a stage
    __shared__ __align__(8) uint64_t w_bar, x_bar;
    __shared__ uint32_t tslot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int KC = g.KC, Npad = g.Npad, NS = g.NS;
    const int T = a.T, cls = blockIdx.y;
    const uint32_t tap_bytes = (uint32_t)Npad * KC * 16;
    const uint32_t stage_bytes = (uint32_t)KC * 2048;
    const uint32_t wbytes = (uint32_t)T * tap_bytes;
    const uint32_t wbase = saddr(smem), xbase = wbase + g.xoff;
    const int KCi = (a.Ci + 7) / 8;
    const int OY0 = a.oy0[cls], OX0 = a.ox0[cls];
    const int zs = blockIdx.z, cbase = zs * Npad;       // output channels cbase .. cbase + Npad - 1

    // tile of this CTA: halo mode, rows y0 .. y0 + R - 1, columns x0 .. x0 + SW - 1
    // of batch entry tb; gather modes, 128 consecutive pixels from p0
    int tb = 0, y0 = 0, x0 = 0;
    int64_t p0 = 0;
    const int64_t total = (int64_t)a.B * a.Hg * a.Wg;
    if (MODE == kHalo) {
        int q = blockIdx.x;
        const int tx = q % g.tiles_x;
        q /= g.tiles_x;
        const int ty = q % g.tiles_y;
        tb = q / g.tiles_y;
        y0 = ty * g.R;
        x0 = tx * g.SW;
    } else {
        p0 = (int64_t)blockIdx.x * kRows;
    }
    // class-grid pixel of MMA row m (false: no output there)
    auto pixel = [&](int m, int& b, int& gy, int& gx) -> bool {
        if (MODE == kHalo) {
            const int yy = m / g.BW, xx = m - yy * g.BW;
            b = tb;
            gy = y0 + yy;
            gx = x0 + xx;
            return xx < g.SW && yy < g.R && gy < a.Hg && gx < a.Wg;
        }
        const int64_t p = p0 + m;
        if (p >= total) return false;
        gx = (int)(p % a.Wg);
        gy = (int)((p / a.Wg) % a.Hg);
        b = (int)(p / ((int64_t)a.Wg * a.Hg));
        return true;
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tslot)),
                     "r"(g.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        fail = 0;
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(&mma_bar[s], 1);
            mbar_init(&wst_bar[s], 1);
        }
        mbar_init(&w_bar, 1);
        mbar_init(&x_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    if (MODE != kStream && tid == 0) {   // this class's packed weights: bulk copies of 8 KB tracked by w_bar
        mbar_expect(&w_bar, wbytes);
        const char* src = static_cast<const char*>(a.w) + (size_t)cls * wbytes;
        for (uint32_t off = 0; off < wbytes; off += 8192) {
            const uint32_t n = wbytes - off < 8192 ? wbytes - off : 8192;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    wbase + off),
                "l"(src + off), "r"(n), "r"(saddr(&w_bar))
                : "memory");
        }
    }
    // the inputs are the previous layer's outputs: wait for that grid to
    // complete (its writes are visible after this).  Then let the next layer
    // launch: its CTAs set up (tensor memory, barriers, weight copies) while
    // this one computes, and its own wait holds its reads until this grid has
    // completed, so the trigger's place only moves the launch latency off the
    // chain of dependent layers.  The next grid launches once every CTA of
    // this one has reached this point (a CTA of it may wait in tcgen05.alloc
    // until a CTA of this grid on its SM releases its columns).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (MODE == kHalo && tid == 0) {
        mbar_expect(&x_bar, (uint32_t)KCi * g.BH * g.BW * 16);
        tma_load_4d(xbase, &a.tmap, 0, x0 - 1, y0 - 1, tb * KCi, &x_bar);
    }

    // epilogue row of this thread (warp w reads TMEM lanes 32 (w mod 4) ...;
    // the two warps on the same lanes take alternate 16-column blocks)
    const int quad = warp & 3, first_c16 = warp >> 2;
    int eb = 0, egy = 0, egx = 0;
    const bool elive = pixel(quad * 32 + (tid & 31), eb, egy, egx);
    const int oy = a.OS * egy + OY0, ox = a.OS * egx + OX0;
    const size_t oplane = (size_t)a.Ho * a.Wo;
    const size_t opix = elive ? (size_t)oy * a.Wo + ox : 0;
    const int KCo = (a.Co + 7) / 8;
    // gate and base of a 16-column block (read-only in this kernel)
    auto load_epi = [&](int c16, float (&gt)[16], float (&bb)[16]) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            gt[i] = 1.f;
            bb[i] = 0.f;
        }
        if (!elive) return;
        if (a.gate || (a.batched && a.gate_b[0])) {
            const float* gsrc = a.batched ? a.gate_b[eb] : a.gate;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int co = cbase + c16 * 16 + i;
                if (co < a.Co) gt[i] = __ldg(gsrc + (size_t)co * oplane + opix);
            }
        }
        if (a.base8) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kc = (cbase >> 3) + c16 * 2 + h;
                if (kc < KCo) {
                    float t8[8];
                    unpack8(__ldg(reinterpret_cast<const uint4*>(a.base8) + ((size_t)eb * KCo + kc) * oplane + opix),
                            t8);
#pragma unroll
                    for (int i = 0; i < 8; ++i) bb[h * 8 + i] = t8[i];
                }
            }
        } else if (a.base64 || (a.batched && a.base64_b[0])) {
            const double* bsrc = a.batched ? a.base64_b[eb] : a.base64 + (size_t)eb * a.Co * oplane;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int co = cbase + c16 * 16 + i;
                if (co < a.Co) bb[i] = (float)__ldg(bsrc + (size_t)co * oplane + opix);
            }
        } else if (a.batched && a.base32_b[0]) {
            const float* bsrc = a.base32_b[eb];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int co = cbase + c16 * 16 + i;
                if (co < a.Co) bb[i] = __ldg(bsrc + (size_t)co * oplane + opix);
            }
        }
    };
    float eg[16], eb8[16];
    if (first_c16 < Npad / 16) load_epi(first_c16, eg, eb8);

    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Npad >> 3) << 17) |
                           ((uint32_t)(kRows >> 4) << 24);
    bool ok = true;

    if (MODE == kHalo) {
        // the halo is written by the async proxy and read by it: only ReLU
        // or the zero chunk of an odd channel count touch it from the threads
        const uint32_t plane_bytes = (uint32_t)g.BH * g.BW * 16;
        if (a.relu_in || KC > KCi) {
            if (!mbar_wait(&x_bar, 0)) ok = false;
            if (a.relu_in)
                for (uint32_t o = tid * 16; o < (uint32_t)KCi * plane_bytes; o += kThreads * 16) relu16(xbase + o);
            for (uint32_t o = KCi * plane_bytes + tid * 16; o < (uint32_t)KC * plane_bytes; o += kThreads * 16)
                asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(xbase + o), "r"(0u) : "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (tid == 0) {
            if (!mbar_wait(&w_bar, 0) || !mbar_wait(&x_bar, 0)) ok = false;
            if (ok) {
                tc_fence_after();
                // descriptors differ only in the start-address field (bits 0-13,
                // no carry below 256 KB), so each MMA costs two adds
                const uint64_t a0 = sdesc(xbase, plane_bytes, 128), b0 = sdesc(wbase, 128, KC * 128);
                const uint64_t astep = (2 * plane_bytes) >> 4;
                Chain chain(tmem);
                for (int t = 0; t < T; ++t) {
                    const int tt = cls * T + t;
                    uint64_t ad = a0 + (((1 + a.dy[tt]) * g.BW + (1 + a.dx[tt])) & 0xFFFF);
                    uint64_t bd = b0 + ((t * tap_bytes) >> 4);
                    for (int j = 0; j < KC / 2; ++j, ad += astep, bd += 16) chain.mma(ad, bd, idesc);
                }
            }
            tc_commit(&mma_bar[0]);
        }
        if (!mbar_wait(&mma_bar[0], 0)) ok = false;
    } else if (MODE == kStream) {
        // stage u = (tap t, block kb of KB chunks): this thread gathers row r,
        // chunks half, half + 2, ... of the block; thread 0 copies the weight
        // slice [tap][slice][kb] (b_bytes) behind the rows; the gather of stage
        // u overlaps the MMAs of stage u - 1
        const int KB = g.KB, NKB = g.NKB, U = T * NKB;
        const uint32_t a_bytes = (uint32_t)KB * 2048, b_bytes = (uint32_t)Npad * KB * 16;
        const uint32_t sbytes = a_bytes + b_bytes;
        const int r = tid & (kRows - 1), half = tid >> 7;
        int b = 0, gy = 0, gx = 0;
        const bool live = pixel(r, b, gy, gx);
        const uint32_t row_off = (uint32_t)((r >> 3) * KB) * 128 + (uint32_t)(r & 7) * 16;
        const char* wsrc = static_cast<const char*>(a.w);
        const size_t plane = (size_t)a.Hi * a.Wi;
        const uint4* xp = reinterpret_cast<const uint4*>(a.x8);
        auto load = [&](int u, int s) {
            const int t = u / NKB, kb = u - t * NKB, tt = cls * T + t;
            const uint32_t sa = xbase + (uint32_t)s * sbytes;
            if (tid == 0) {
                const size_t off = (((size_t)tt * gridDim.z + zs) * NKB + kb) * b_bytes;
                mbar_expect(&wst_bar[s], b_bytes);
                for (uint32_t o = 0; o < b_bytes; o += 8192) {
                    const uint32_t nb = b_bytes - o < 8192 ? b_bytes - o : 8192;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            sa + a_bytes + o),
                        "l"(wsrc + off + o), "r"(nb), "r"(saddr(&wst_bar[s]))
                        : "memory");
                }
            }
            const int iy = a.S * gy + a.dy[tt], ix = a.S * gx + a.dx[tt];
            const bool in = live && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
            const size_t pix = in ? (size_t)iy * a.Wi + ix : 0;
            for (int kcl = half; kcl < KB; kcl += 2) {
                const int kc = kb * KB + kcl;
                const bool okc = in && kc < KCi;
                const uint4* src = okc ? xp + ((size_t)b * KCi + kc) * plane + pix : xp;
                cp_async16(sa + row_off + kcl * 128, src, okc ? 16u : 0u);
            }
            cp_async_commit();
        };
        Chain chain(tmem);               // used by thread 0 only
        auto consume = [&](int u, bool last) {
            const int s = u % NS;
            const uint32_t sa = xbase + (uint32_t)s * sbytes;
            if (last) cp_async_wait<0>(); else cp_async_wait<1>();
            if (a.relu_in)
                for (int kcl = half; kcl < KB; kcl += 2) relu16(sa + row_off + kcl * 128);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                if (!mbar_wait(&wst_bar[s], (unsigned)(u / NS) & 1u)) ok = false;
                if (ok) {
                    tc_fence_after();
                    uint64_t ad = sdesc(sa, 128, KB * 128), bd = sdesc(sa + a_bytes, 128, KB * 128);
                    for (int j = 0; j < KB / 2; ++j, ad += 16, bd += 16) chain.mma(ad, bd, idesc);
                }
                tc_commit(&mma_bar[s]);
            }
        };
        for (int u = 0; u < U; ++u) {
            const int s = u % NS;
            if (u >= NS && !mbar_wait(&mma_bar[s], (unsigned)((u / NS) - 1) & 1u)) ok = false;
            load(u, s);
            if (u > 0) consume(u - 1, false);
        }
        consume(U - 1, true);
        if (!mbar_wait(&mma_bar[(U - 1) % NS], (unsigned)((U - 1) / NS) & 1u)) ok = false;
    } else {
        // this thread gathers row r, channel chunks kc = half, half + 2, ...
        const int r = tid & (kRows - 1), half = tid >> 7;
        int b = 0, gy = 0, gx = 0;
        const bool live = pixel(r, b, gy, gx);
        const uint32_t row_off = (uint32_t)((r >> 3) * KC) * 128 + (uint32_t)(r & 7) * 16;
        auto gather = [&](int t, int s) {
            const int tt = cls * T + t;
            const int iy = a.S * gy + a.dy[tt], ix = a.S * gx + a.dx[tt];
            const bool in = live && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
            const uint32_t dst = xbase + (uint32_t)s * stage_bytes + row_off;
            const size_t plane = (size_t)a.Hi * a.Wi;
            if (MODE == kF64) {
                // FP64 or FP32 input vector (x64 / x64_b, or x32_b), rounded on load
                const bool f32 = a.batched && a.x32_b[0];
                const size_t pix = in ? (size_t)iy * a.Wi + ix : 0;
                const double* xp = f32 ? nullptr : (a.batched ? a.x64_b[b] : a.x64 + (size_t)b * a.Ci * plane) + pix;
                const float* xq = f32 ? a.x32_b[b] + pix : nullptr;
                // groups of kLiftGroup chunks: every load of a group is issued
                // before its shared-memory stores (which the compiler keeps in
                // order with the loads), so a thread has 8 kLiftGroup loads in flight
                for (int kc0 = half; kc0 < KC; kc0 += 2 * kLiftGroup) {
                    float v[kLiftGroup][8];
#pragma unroll
                    for (int q = 0; q < kLiftGroup; ++q) {
                        const int kc = kc0 + 2 * q;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int ci = kc * 8 + j;
                            float x = 0.f;
                            if (in && kc < KC && ci < a.Ci)
                                x = f32 ? __ldg(xq + (size_t)ci * plane) : (float)__ldg(xp + (size_t)ci * plane);
                            v[q][j] = a.relu_in ? fmaxf(x, 0.f) : x;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kLiftGroup; ++q) {
                        const int kc = kc0 + 2 * q;
                        if (kc < KC) {
                            const uint4 pk = pack8(v[q]);
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + kc * 128),
                                         "r"(pk.x), "r"(pk.y), "r"(pk.z), "r"(pk.w)
                                         : "memory");
                        }
                    }
                }
            } else {
                const uint4* xp = reinterpret_cast<const uint4*>(a.x8);
                const size_t pix = in ? (size_t)iy * a.Wi + ix : 0;
                for (int kc = half; kc < KC; kc += 2) {
                    const bool okc = in && kc < KCi;
                    const uint4* src = okc ? xp + ((size_t)b * KCi + kc) * plane + pix : xp;
                    cp_async16(dst + kc * 128, src, okc ? 16u : 0u);
                }
            }
            cp_async_commit();
        };
        // ReLU of this thread's own (landed) rows of stage s
        auto relu_stage = [&](int s) {
            if (MODE == kGather && a.relu_in) {
                const uint32_t dst = xbase + (uint32_t)s * stage_bytes + row_off;
                for (int kc = half; kc < KC; kc += 2) relu16(dst + kc * 128);
            }
        };
        Chain chain(tmem);               // used by thread 0 only
        auto issue = [&](int u) {       // one thread: the MMAs of tap u
            uint64_t ad = sdesc(xbase + (u % NS) * stage_bytes, 128, KC * 128);
            uint64_t bd = sdesc(wbase + u * tap_bytes, 128, KC * 128);
            for (int j = 0; j < KC / 2; ++j, ad += 16, bd += 16) chain.mma(ad, bd, idesc);
        };
        // after this thread's copies of tap u have landed: ReLU them if asked,
        // hand them to the async proxy, then one thread issues the tap's MMAs
        auto finish = [&](int u, bool last) {
            const int s = u % NS;
            if (last) cp_async_wait<0>(); else cp_async_wait<1>();
            relu_stage(s);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                if (u == 0 && !mbar_wait(&w_bar, 0)) ok = false;
                if (ok) {
                    tc_fence_after();
                    issue(u);
                }
                tc_commit(&mma_bar[s]);
            }
        };
        if (NS == T) {
            // every tap has its own stage: all gathers in flight at once, one
            // wait, then all MMAs back to back
            for (int t = 0; t < T; ++t) gather(t, t);
            cp_async_wait<0>();
            for (int t = 0; t < T; ++t) relu_stage(t);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                if (!mbar_wait(&w_bar, 0)) ok = false;
                if (ok) {
                    tc_fence_after();
                    for (int t = 0; t < T; ++t) issue(t);
                }
                tc_commit(&mma_bar[0]);
            }
            if (!mbar_wait(&mma_bar[0], 0)) ok = false;
        } else {
            // ring of NS stages: the gather of tap t overlaps the MMAs of tap t - 1
            for (int t = 0; t < T; ++t) {
                const int s = t % NS;
                if (t >= NS && !mbar_wait(&mma_bar[s], (unsigned)((t / NS) - 1) & 1u)) ok = false;
                gather(t, s);
                if (t > 0) finish(t - 1, false);
            }
            finish(T - 1, true);
            if (!mbar_wait(&mma_bar[(T - 1) % NS], (unsigned)((T - 1) / NS) & 1u)) ok = false;
        }
    }
    if (MODE != kStream && tid == 0 && !mbar_wait(&w_bar, 0)) ok = false;   // the weight copy has landed
    if (MODE == kHalo && tid == 0 && !mbar_wait(&x_bar, 0)) ok = false;
    tc_fence_after();
    if (!ok) {
        fail = 1;
        atomicExch(&g_tc_status, 1);
    }
    __syncthreads();
    ok = fail == 0;

    // epilogue: block c16 of 16 columns; the operands of the next block are
    // loaded before the current one is stored, so each thread has one round
    // trip in flight per block instead of one per element
    const float nanv = __int_as_float(0x7fc00000);
    for (int c16 = first_c16; c16 < Npad / 16; c16 += 2) {
        float acc[16];
        tc_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c16 * 16), acc);
        float gn[16], bn[16];
        if (c16 + 2 < Npad / 16) load_epi(c16 + 2, gn, bn);
        if (elive) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kc = (cbase >> 3) + c16 * 2 + h;
                if (kc >= KCo) break;
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int co = kc * 8 + i;
                    const float x = a.sign * (acc[h * 8 + i] * eg[h * 8 + i]) + eb8[h * 8 + i];
                    v[i] = co < a.Co ? (ok ? x : nanv) : 0.f;
                }
                if (a.y8) {
                    reinterpret_cast<uint4*>(a.y8)[((size_t)eb * KCo + kc) * oplane + opix] = pack8(v);
                } else {
                    float* ysrc = a.batched ? a.y32_b[eb] : a.y32 + (size_t)eb * a.Co * oplane;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int co = kc * 8 + i;
                        if (co < a.Co) ysrc[(size_t)co * oplane + opix] = v[i];
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            eg[i] = gn[i];
            eb8[i] = bn[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.ncols) : "memory");
    }
}

// packed weights: entry ((t (Npad/8) + g) KC + kc) 8 + rr holds
// W[t][kc*8 .. kc*8+7][8 g + rr] as 8 BF16 (zero outside Ci x Co)
__global__ void k_tc_pack(const float* __restrict__ w, int so, int si, int KK, Taps tp, int Ci, int Co, int KC,
                          int Npad, uint4* __restrict__ out) {
    const int groupsN = Npad / 8;
    const int n = tp.T * groupsN * KC * 8;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int q = e;
        const int rr = q % 8;
        q /= 8;
        const int kc = q % KC;
        q /= KC;
        const int g = q % groupsN, t = q / groupsN;
        const int co = g * 8 + rr;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ci = kc * 8 + j;
            v[j] = (co < Co && ci < Ci) ? w[((size_t)co * so + (size_t)ci * si) * KK + tp.wi[t]] : 0.f;
        }
        out[e] = pack8(v);
    }
}

// streamed layout: entry ((((t Z + z) NKB + kb) (Ns/8) + g) KB + kcl) 8 + rr holds
// W[t][(kb KB + kcl) 8 .. +7][z Ns + 8 g + rr] (zero outside Ci x Co), so the
// weight slice of stage (t, z, kb) is one contiguous block of Ns KB 16 bytes
__global__ void k_tc_pack_stream(const float* __restrict__ w, int so, int si, int KK, Taps tp, int Ci, int Co,
                                 int Ns, int Z, int KB, int NKB, uint4* __restrict__ out) {
    const int groups = Ns / 8;
    const int64_t n = (int64_t)tp.T * Z * NKB * groups * KB * 8;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = e;
        const int rr = (int)(q % 8);
        q /= 8;
        const int kcl = (int)(q % KB);
        q /= KB;
        const int g = (int)(q % groups);
        q /= groups;
        const int kb = (int)(q % NKB);
        q /= NKB;
        const int z = (int)(q % Z), t = (int)(q / Z);
        const int co = z * Ns + g * 8 + rr, kc = kb * KB + kcl;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ci = kc * 8 + j;
            v[j] = (co < Co && ci < Ci) ? w[((size_t)co * so + (size_t)ci * si) * KK + tp.wi[t]] : 0.f;
        }
        out[e] = pack8(v);
    }
}

int chunks_kc(int Ci) { return ((Ci + 15) / 16) * 2; }
int pad_n(int Co) { return ((Co + 15) / 16) * 16; }

// Output-channel slices of a layer: Z slices of Ns channels (a multiple of
// 16, at most kMaxSlice) covering Co.
void slices(int Co, int& Z, int& Ns) {
    Z = (pad_n(Co) + kMaxSlice - 1) / kMaxSlice;
    Ns = pad_n((Co + Z - 1) / Z);
}

// Weights of one CTA (Tc taps of its class) too large to stay resident.
bool streamed(int Tc, int Ci, int Co) {
    return pad_n(Co) > kMaxSlice || (size_t)Tc * pad_n(Co) * chunks_kc(Ci) * 16 > kResidentWeightBytes;
}

void stream_blocks(int Ci, int& KB, int& NKB) {
    const int KC = chunks_kc(Ci);
    KB = KC < kStreamChunks ? KC : kStreamChunks;
    NKB = (KC + KB - 1) / KB;
}

struct KernelLimits {
    size_t max_dyn = 0;
    size_t floor_bytes[4] = {0, 0, 0, 0};   // by TMEM columns 32, 64, 128, 256
};

// Dynamic shared memory limit (opt-in limit minus static shared memory) and,
// per TMEM column count, the least dynamic shared memory that keeps the
// resident CTAs of one SM within the 512 TMEM columns (a CTA would otherwise
// wait in tcgen05.alloc).
template <int MODE>
const KernelLimits& limits() {
    static KernelLimits L;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, optin = 0, per_sm = 0;
        check(cudaGetDevice(&dev), "cudaGetDevice");
        check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attribute");
        check(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev), "attribute");
        cudaFuncAttributes fa{};
        check(cudaFuncGetAttributes(&fa, k_conv_tc<MODE>), "cudaFuncGetAttributes");
        L.max_dyn = (size_t)optin - fa.sharedSizeBytes;
        check(cudaFuncSetAttribute(k_conv_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.max_dyn),
              "cudaFuncSetAttribute");
        for (int k = 0; k < 4; ++k) {
            const int allowed = 512 / (32 << k);
            size_t s = 0;
            for (;;) {
                int nb = 0;
                check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_tc<MODE>, kThreads, s), "occupancy");
                if (nb <= allowed) break;
                s = s == 0 ? (size_t)per_sm / (allowed + 1) : s + 4096;
                if (s > L.max_dyn) throw StatusError{RTE_EINVAL, "cannot bound tensor-core occupancy"};
            }
            L.floor_bytes[k] = s;
        }
    });
    return L;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, reached through the runtime (no libcuda link)
EncodeTiled encoder() {
    static EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        check(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q),
              "cudaGetDriverEntryPointByVersion");
        if (q != cudaDriverEntryPointSuccess || !p)
            throw StatusError{RTE_ECUDA, "cuTensorMapEncodeTiled is not available"};
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

template <int MODE>
void launch(const TcConv& a, Geo g, size_t stage_area, bool pdl, unsigned grid_x, cudaStream_t st,
            unsigned slices_z = 1) {
    g.ncols = 32;
    while (g.ncols < (uint32_t)g.Npad) g.ncols <<= 1;
    int k = 0;
    while ((32u << k) < g.ncols) ++k;
    const KernelLimits& L = limits<MODE>();
    const size_t wbytes = MODE == kStream ? 0 : (size_t)a.T * g.Npad * g.KC * 16;   // resident weights
    g.xoff = (uint32_t)((wbytes + 1023) & ~(size_t)1023);
    size_t smem = g.xoff + stage_area;
    if (smem < L.floor_bytes[k]) smem = L.floor_bytes[k];
    if (smem > L.max_dyn) throw StatusError{RTE_EINVAL, "tensor-core convolution: tile exceeds shared memory"};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_x, (unsigned)a.classes, slices_z);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    check(cudaLaunchKernelEx(&cfg, k_conv_tc<MODE>, a, g), "k_conv_tc");
}

}  // namespace

size_t tc_weight_bytes(int T, int classes, int Ci, int Co) {
    if (streamed(T / classes, Ci, Co)) {
        int Z = 0, Ns = 0, KB = 0, NKB = 0;
        slices(Co, Z, Ns);
        stream_blocks(Ci, KB, NKB);
        return (size_t)T * Z * NKB * Ns * KB * 16;
    }
    return (size_t)T * pad_n(Co) * chunks_kc(Ci) * 16;
}

void tc_pack(const float* w, int so, int si, int KK, const Taps& tp, int classes, int Ci, int Co, void* dst,
             cudaStream_t st) {
    if (streamed(tp.T / classes, Ci, Co)) {
        int Z = 0, Ns = 0, KB = 0, NKB = 0;
        slices(Co, Z, Ns);
        stream_blocks(Ci, KB, NKB);
        const int64_t n = (int64_t)tp.T * Z * NKB * (Ns / 8) * KB * 8;
        const int64_t blocks = (n + 255) / 256;
        k_tc_pack_stream<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, st>>>(
            w, so, si, KK, tp, Ci, Co, Ns, Z, KB, NKB, static_cast<uint4*>(dst));
        check(cudaGetLastError(), "k_tc_pack_stream");
        return;
    }
    const int KC = chunks_kc(Ci), Npad = pad_n(Co);
    const int n = tp.T * (Npad / 8) * KC * 8;
    k_tc_pack<<<(n + 255) / 256, 256, 0, st>>>(w, so, si, KK, tp, Ci, Co, KC, Npad, static_cast<uint4*>(dst));
    check(cudaGetLastError(), "k_tc_pack");
}

void tc_conv(const TcConv& in, bool pdl, cudaStream_t st) {
    TcConv a = in;
    if (a.T < 1 || a.classes < 1 || a.classes > 4 || a.T * a.classes > kMaxTaps || a.S < 1 || a.S > 2 ||
        a.Ci < 1 || a.Co < 1 || !a.w ||
        (!a.x8) == (!(a.x64 || (a.batched && (a.x64_b[0] || a.x32_b[0])))) ||
        (!a.y8) == (!(a.y32 || (a.batched && a.y32_b[0]))) || (a.batched && a.B > kTcMaxBatch))
        throw StatusError{RTE_EINVAL, "tensor-core convolution: bad arguments"};
    const bool stream = streamed(a.T, a.Ci, a.Co);
    if (reinterpret_cast<uintptr_t>(a.w) % 16 || (a.x8 && reinterpret_cast<uintptr_t>(a.x8) % 16) ||
        (a.y8 && reinterpret_cast<uintptr_t>(a.y8) % 16) || (a.base8 && reinterpret_cast<uintptr_t>(a.base8) % 16))
        throw StatusError{RTE_EINVAL, "tensor-core convolution: buffers must be 16-byte aligned"};
    const int64_t total = (int64_t)a.B * a.Hg * a.Wg;
    if (total == 0) return;
    if (tl_counters) {
        tl_counters->launches += 1;
        tl_counters->flops += 2.0 * a.B * a.Co * (double)a.Hg * a.Wg * a.Ci * a.T * a.classes;
    }
    Geo g{};
    g.KC = chunks_kc(a.Ci);
    g.Npad = pad_n(a.Co);
    const int T = a.T;
    if (a.x64 || (a.batched && (a.x64_b[0] || a.x32_b[0]))) {
        if (stream) throw StatusError{RTE_EINVAL, "tensor-core convolution: lift weights too large"};
        g.NS = T;
        launch<kF64>(a, g, (size_t)T * g.KC * 2048, pdl, (unsigned)((total + kRows - 1) / kRows), st);
        return;
    }
    if (stream) {
        int Z = 0;
        slices(a.Co, Z, g.Npad);
        stream_blocks(a.Ci, g.KB, g.NKB);
        const int U = T * g.NKB;
        g.NS = U < kMaxStages ? U : kMaxStages;
        const size_t sbytes = (size_t)g.KB * 2048 + (size_t)g.Npad * g.KB * 16;
        launch<kStream>(a, g, (size_t)g.NS * sbytes, pdl, (unsigned)((total + kRows - 1) / kRows), st,
                        (unsigned)Z);
        return;
    }
    bool halo = a.S == 1 && a.Hg == a.Hi && a.Wg == a.Wi;
    for (int t = 0; t < T * a.classes; ++t)
        halo = halo && a.dy[t] >= -1 && a.dy[t] <= 1 && a.dx[t] >= -1 && a.dx[t] <= 1;
    if (halo) {
        g.SW = a.Wg < kRows ? a.Wg : kRows;
        g.BW = g.SW + 2;
        g.R = (kRows - g.SW) / g.BW + 1;
        if (g.R > a.Hg) g.R = a.Hg;
        g.BH = g.R + 2;
        g.tiles_x = (a.Wg + g.SW - 1) / g.SW;
        g.tiles_y = (a.Hg + g.R - 1) / g.R;
        g.NS = 1;
        const int KCi = (a.Ci + 7) / 8;
        const cuuint64_t dims[4] = {8, (cuuint64_t)a.Wi, (cuuint64_t)a.Hi, (cuuint64_t)a.B * KCi};
        const cuuint64_t strides[3] = {16, (cuuint64_t)a.Wi * 16, (cuuint64_t)a.Hi * a.Wi * 16};
        const cuuint32_t box[4] = {8, (cuuint32_t)g.BW, (cuuint32_t)g.BH, (cuuint32_t)KCi};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult cr = encoder()(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(a.x8), dims,
                                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) throw StatusError{RTE_ECUDA, "cuTensorMapEncodeTiled failed"};
        // halo planes plus the rows the discarded MMA rows of the last plane read
        const size_t area = (size_t)g.KC * g.BH * g.BW * 16 + (size_t)(2 * g.BW + 130) * 16;
        const unsigned tiles = (unsigned)(g.tiles_x * g.tiles_y * a.B);
        launch<kHalo>(a, g, area, pdl, tiles, st);
        return;
    }
    // every tap resident if it fits, else a ring of kMaxStages stages
    const size_t wbytes = (size_t)T * g.Npad * g.KC * 16, stage = (size_t)g.KC * 2048;
    g.NS = T;
    if (((wbytes + 1023) & ~(size_t)1023) + T * stage > limits<kGather>().max_dyn)
        g.NS = T < kMaxStages ? T : kMaxStages;
    launch<kGather>(a, g, (size_t)g.NS * stage, pdl, (unsigned)((total + kRows - 1) / kRows), st);
}

int conv_tc_status(bool reset) {
    int v = 0;
    check(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)), "read tensor-core status");
    if (reset && v) {
        const int zero = 0;
        check(cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int)), "reset tensor-core status");
    }
    return v;
}

}  // namespace nn
}  // namespace rte
