// Tensor-core gather convolution of the MgNet forward pass (Sec. 3.3) at
// inference: BF16 operands, FP32 accumulation in tensor memory (tcgen05).
//
// Implicit GEMM over tap tables:
//   D[p][o] = sum_t sum_i X[b][i][S gy_p + dy_t][S gx_p + dx_t] W[t][i][o]
// with M = 128 class-grid pixels per CTA (pixel r of the tile owns TMEM lane
// r), N = output channels rounded up to 16 (TMEM columns), and one MMA of
// K = 16 input channels per (tap, channel pair group).
//
// Activations between the layers are BF16 in a channel-chunked layout
// "C8" = [B][ceil(C/8)][H][W][8]: the 8 channels of one pixel are one 16-byte
// row of an MMA core matrix, so gathering tap t of the tile is one 16-byte
// cp.async per (pixel, chunk), zero-filled outside the image.  The first layer
// (lift) reads the FP64 Krylov vector [2M][I][I] directly and converts; the
// last (projection) writes FP32 [2M][I][I].
//
// Shared memory: the layer's weights, packed once per weight version into the
// MMA layout (tc_pack) and copied by one bulk async copy, then a ring of NS
// stages of the gathered tile, one tap per stage.  When every tap fits (up to
// 64 input channels with 3 x 3 taps) all gathers are in flight at once and the
// MMAs follow one wait.  Otherwise every thread issues the cp.async of tap t,
// waits for its own copies of tap t - 1, fences them into the async proxy and
// meets the others at a barrier, after which one thread issues tap t - 1's
// MMAs and commits them to the stage's mbarrier; tap t + NS - 1 waits on that
// barrier before reusing the stage.  Launched with programmatic dependent
// launch, a layer allocates its tensor memory and copies its weights while the
// previous layer finishes, and waits for it only before the gather; a layer
// signals its dependents only after its last output store (the signal is what
// makes those stores visible to them).  Operands use the
// no-swizzle K-major canonical layout with 8 x 16-byte core matrices stored
// row-group-major (byte (g KC + kc) 128 + (r mod 8) 16 for row 8 g + r mod 8,
// channel chunk kc; KC chunks per row): leading (K) byte offset 128, stride
// (M/N) byte offset 128 KC.
//
// The epilogue reads the accumulators back with tcgen05.ld (warp w sees lanes
// 32 (w mod 4) ...; the two warps on the same lanes take alternate 16-column
// blocks) and applies v = sign (acc o gate) (+ base) before the store.
// Every wait is bounded: on expiry the CTA records the failure in a device
// flag, writes NaN outputs, releases its tensor memory and returns.
#include <cuda_bf16.h>

#include <mutex>

#include "nn_internal.h"

namespace rte {
namespace nn {
namespace {

constexpr int kRows = 128;           // pixels per CTA = MMA M = TMEM lanes
constexpr int kThreads = 256;
constexpr int kMaxStages = 3;
constexpr long long kSpinLimit = 1ll << 24;

__device__ int g_tc_status;          // 1 once a bounded wait expired

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// waits for the completion of the phase with the given parity, at most
// kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (long long i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     saddr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's lane; the wait is in the same
// statement so no register is read before the load has landed
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

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

// KC: channel chunks of 8 per MMA row (even); Npad: output channels rounded
// up to 16; NS: stages; ncols: allocated TMEM columns (power of two >= Npad).
// F64IN: the input is FP64 [B][Ci][Hi][Wi] (converted while gathering),
// otherwise BF16 C8.
template <bool F64IN>
__global__ void __launch_bounds__(kThreads, 1)
    k_conv_tc(const __grid_constant__ TcConv a, int KC, int Npad, int NS, uint32_t ncols) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mma_bar[kMaxStages];
    __shared__ __align__(8) uint64_t w_bar;
    __shared__ uint32_t tslot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int T = a.T;
    const uint32_t tap_bytes = (uint32_t)Npad * KC * 16;
    const uint32_t stage_bytes = (uint32_t)KC * 2048;
    const uint32_t wbytes = (uint32_t)T * tap_bytes;
    const uint32_t wbase = saddr(smem), xbase = wbase + wbytes;
    const int64_t total = (int64_t)a.B * a.Hg * a.Wg;
    const int64_t p0 = (int64_t)blockIdx.x * kRows;
    const int KCi = (a.Ci + 7) / 8;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        fail = 0;
        for (int s = 0; s < NS; ++s) mbar_init(&mma_bar[s], 1);
        mbar_init(&w_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    if (tid == 0) {      // packed weights: one bulk copy tracked by w_bar
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&w_bar)), "r"(wbytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(wbase),
            "l"(a.w), "r"(wbytes), "r"(saddr(&w_bar))
            : "memory");
    }
    // the inputs are the previous layer's outputs: wait for that grid (its
    // writes before its trigger are visible after this)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // this thread gathers row r, channel chunks kc = half, half + 2, ...
    const int r = tid & (kRows - 1), half = tid >> 7;
    const int64_t p = p0 + r;
    const bool live = p < total;
    int gx = 0, gy = 0, b = 0;
    if (live) {
        gx = (int)(p % a.Wg);
        gy = (int)((p / a.Wg) % a.Hg);
        b = (int)(p / ((int64_t)a.Wg * a.Hg));
    }
    const uint32_t row_off = (uint32_t)((r >> 3) * KC) * 128 + (uint32_t)(r & 7) * 16;

    // epilogue row of this thread (warp w reads TMEM lanes 32 (w mod 4) ...;
    // the two warps on the same lanes take alternate 16-column blocks)
    const int quad = warp & 3, first_c16 = warp >> 2;
    const int64_t pe = p0 + quad * 32 + (tid & 31);
    int oy = 0, ox = 0, eb = 0;
    if (pe < total) {
        const int egx = (int)(pe % a.Wg), egy = (int)((pe / a.Wg) % a.Hg);
        eb = (int)(pe / ((int64_t)a.Wg * a.Hg));
        oy = a.OS * egy + a.OY0;
        ox = a.OS * egx + a.OX0;
    }
    const size_t oplane = (size_t)a.Ho * a.Wo;
    const size_t opix = (size_t)oy * a.Wo + ox;
    const int KCo = (a.Co + 7) / 8;
    // gate and base of a 16-column block (read-only in this kernel)
    auto load_epi = [&](int c16, float (&g)[16], float (&bb)[16]) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            g[i] = 1.f;
            bb[i] = 0.f;
        }
        if (pe >= total) return;
        if (a.gate) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int co = c16 * 16 + i;
                if (co < a.Co) g[i] = __ldg(a.gate + (size_t)co * oplane + opix);
            }
        }
        if (a.base8) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kc = c16 * 2 + h;
                if (kc < KCo) {
                    float t8[8];
                    unpack8(__ldg(reinterpret_cast<const uint4*>(a.base8) + ((size_t)eb * KCo + kc) * oplane + opix),
                            t8);
#pragma unroll
                    for (int i = 0; i < 8; ++i) bb[h * 8 + i] = t8[i];
                }
            }
        } else if (a.base64) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int co = c16 * 16 + i;
                if (co < a.Co) bb[i] = (float)__ldg(a.base64 + ((size_t)eb * a.Co + co) * oplane + opix);
            }
        }
    };
    float eg[16], eb8[16];
    if (first_c16 < Npad / 16) load_epi(first_c16, eg, eb8);

    auto gather = [&](int t, int s) {
        const int iy = a.S * gy + a.dy[t], ix = a.S * gx + a.dx[t];
        const bool in = live && iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
        const uint32_t dst = xbase + (uint32_t)s * stage_bytes + row_off;
        if constexpr (F64IN) {
            const size_t plane = (size_t)a.Hi * a.Wi;
            const double* xp = a.x64 + (size_t)b * a.Ci * plane + (in ? (size_t)iy * a.Wi + ix : 0);
#pragma unroll 4
            for (int kc = half; kc < KC; kc += 2) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ci = kc * 8 + j;
                    const float x = (in && ci < a.Ci) ? (float)__ldg(xp + (size_t)ci * plane) : 0.f;
                    v[j] = a.relu_in ? fmaxf(x, 0.f) : x;
                }
                const uint4 pk = pack8(v);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + kc * 128), "r"(pk.x),
                             "r"(pk.y), "r"(pk.z), "r"(pk.w)
                             : "memory");
            }
        } else {
            const uint4* xp = reinterpret_cast<const uint4*>(a.x8);
            const size_t plane = (size_t)a.Hi * a.Wi;
            const size_t pix = in ? (size_t)iy * a.Wi + ix : 0;
            for (int kc = half; kc < KC; kc += 2) {
                const bool ok = in && kc < KCi;
                const uint4* src = ok ? xp + ((size_t)b * KCi + kc) * plane + pix : xp;
                cp_async16(dst + kc * 128, src, ok ? 16u : 0u);
            }
        }
        cp_async_commit();
    };
    // ReLU of this thread's own (landed) rows of stage s
    auto relu_stage = [&](int s) {
        if (!F64IN && a.relu_in) {
            const uint32_t dst = xbase + (uint32_t)s * stage_bytes + row_off;
            for (int kc = half; kc < KC; kc += 2) {
                uint32_t w[4];
                asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                             : "r"(dst + kc * 128));
#pragma unroll
                for (int i = 0; i < 4; ++i) {      // ReLU of two BF16: clear negative halves
                    const uint32_t lo = (w[i] & 0x8000u) ? 0u : (w[i] & 0xFFFFu);
                    const uint32_t hi = (w[i] & 0x80000000u) ? 0u : (w[i] & 0xFFFF0000u);
                    w[i] = lo | hi;
                }
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + kc * 128), "r"(w[0]),
                             "r"(w[1]), "r"(w[2]), "r"(w[3])
                             : "memory");
            }
        }
    };
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Npad >> 3) << 17) |
                           ((uint32_t)(kRows >> 4) << 24);
    auto issue = [&](int u) {       // one thread: the MMAs of tap u
        const int s = u % NS;
        for (int j = 0; j < KC / 2; ++j) {
            const uint64_t ad = sdesc(xbase + s * stage_bytes + 2 * j * 128, 128, KC * 128);
            const uint64_t bd = sdesc(wbase + u * tap_bytes + 2 * j * 128, 128, KC * 128);
            tc_mma(tmem, ad, bd, idesc, (u > 0 || j > 0) ? 1u : 0u);
        }
    };
    // after this thread's copies of tap u have landed: ReLU them if asked,
    // hand them to the async proxy, then one thread issues the tap's MMAs
    bool ok = true;
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
    if (tid == 0 && !mbar_wait(&w_bar, 0)) ok = false;   // weights landed even if no MMA ran
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
        if (pe < total) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kc = c16 * 2 + h;
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
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int co = kc * 8 + i;
                        if (co < a.Co) a.y32[((size_t)eb * a.Co + co) * oplane + opix] = v[i];
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
    // every output of this CTA is written: the next layer may launch (its
    // CTAs may wait in tcgen05.alloc until this CTA releases its columns)
    tc_fence_before();
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
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

int chunks_kc(int Ci) { return ((Ci + 15) / 16) * 2; }
int pad_n(int Co) { return ((Co + 15) / 16) * 16; }

template <bool F64IN>
struct KernelLimits {
    size_t max_dyn = 0;
    size_t floor_bytes[4] = {0, 0, 0, 0};   // by TMEM columns 32, 64, 128, 256
};

// Dynamic shared memory limit (opt-in limit minus static shared memory) and,
// per TMEM column count, the least dynamic shared memory that keeps the
// resident CTAs of one SM within the 512 TMEM columns (a CTA would otherwise
// wait in tcgen05.alloc).
template <bool F64IN>
const KernelLimits<F64IN>& limits() {
    static KernelLimits<F64IN> L;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, optin = 0, per_sm = 0;
        check(cudaGetDevice(&dev), "cudaGetDevice");
        check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attribute");
        check(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev), "attribute");
        cudaFuncAttributes fa{};
        check(cudaFuncGetAttributes(&fa, k_conv_tc<F64IN>), "cudaFuncGetAttributes");
        L.max_dyn = (size_t)optin - fa.sharedSizeBytes;
        check(cudaFuncSetAttribute(k_conv_tc<F64IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.max_dyn),
              "cudaFuncSetAttribute");
        for (int k = 0; k < 4; ++k) {
            const int allowed = 512 / (32 << k);
            size_t s = 0;
            for (;;) {
                int nb = 0;
                check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_tc<F64IN>, kThreads, s),
                      "occupancy");
                if (nb <= allowed) break;
                s = s == 0 ? (size_t)per_sm / (allowed + 1) : s + 4096;
                if (s > L.max_dyn) throw StatusError{RTE_EINVAL, "cannot bound tensor-core occupancy"};
            }
            L.floor_bytes[k] = s;
        }
    });
    return L;
}

template <bool F64IN>
void launch(const TcConv& a, bool pdl, cudaStream_t st) {
    const int T = a.T;
    const int KC = chunks_kc(a.Ci), Npad = pad_n(a.Co);
    int k = 0;
    while ((32 << k) < Npad) ++k;
    const uint32_t ncols = 32u << k;
    const KernelLimits<F64IN>& L = limits<F64IN>();
    const size_t wbytes = (size_t)T * Npad * KC * 16, stage = (size_t)KC * 2048;
    // every tap resident if it fits, else a ring of kMaxStages stages
    int NS = T;
    if (wbytes + NS * stage > L.max_dyn) NS = T < kMaxStages ? T : kMaxStages;
    size_t smem = wbytes + NS * stage;
    if (smem < L.floor_bytes[k]) smem = L.floor_bytes[k];
    if (smem > L.max_dyn) throw StatusError{RTE_EINVAL, "tensor-core convolution: tile exceeds shared memory"};
    const int64_t total = (int64_t)a.B * a.Hg * a.Wg;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((total + kRows - 1) / kRows));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    check(cudaLaunchKernelEx(&cfg, k_conv_tc<F64IN>, a, KC, Npad, NS, ncols), "k_conv_tc");
}

}  // namespace

size_t tc_weight_bytes(int T, int Ci, int Co) { return (size_t)T * pad_n(Co) * chunks_kc(Ci) * 16; }

void tc_pack(const float* w, int so, int si, int KK, const Taps& tp, int Ci, int Co, void* dst, cudaStream_t st) {
    const int KC = chunks_kc(Ci), Npad = pad_n(Co);
    const int n = tp.T * (Npad / 8) * KC * 8;
    k_tc_pack<<<(n + 255) / 256, 256, 0, st>>>(w, so, si, KK, tp, Ci, Co, KC, Npad, static_cast<uint4*>(dst));
    check(cudaGetLastError(), "k_tc_pack");
}

void tc_conv(const TcConv& a, bool pdl, cudaStream_t st) {
    if (a.T < 1 || a.T > kMaxTaps || a.S < 1 || a.S > 2 || a.Ci < 1 || a.Co < 1 || !a.w ||
        (!a.x8) == (!a.x64) || (!a.y8) == (!a.y32))
        throw StatusError{RTE_EINVAL, "tensor-core convolution: bad arguments"};
    if (pad_n(a.Co) > 256) throw StatusError{RTE_EINVAL, "tensor-core convolution: more than 256 output channels"};
    if (reinterpret_cast<uintptr_t>(a.w) % 16 || (a.x8 && reinterpret_cast<uintptr_t>(a.x8) % 16) ||
        (a.y8 && reinterpret_cast<uintptr_t>(a.y8) % 16) || (a.base8 && reinterpret_cast<uintptr_t>(a.base8) % 16))
        throw StatusError{RTE_EINVAL, "tensor-core convolution: buffers must be 16-byte aligned"};
    if ((int64_t)a.B * a.Hg * a.Wg == 0) return;
    if (tl_counters) {
        tl_counters->launches += 1;
        tl_counters->flops += 2.0 * a.B * a.Co * (double)a.Hg * a.Wg * a.Ci * a.T;
    }
    if (a.x64)
        launch<true>(a, pdl, st);
    else
        launch<false>(a, pdl, st);
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
