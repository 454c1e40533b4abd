// FP64 Krylov kernels: multi-dot, fused Gram-Schmidt passes, norms, scaling
// and the solution update, on double vectors.  They serve the FP64 entry
// points (rte_cgs2, rte_cgs2_noalloc, rte_arnoldi_basis) and the norms of
// FP64 residuals; the solver's own Arnoldi step runs on df64 vectors
// (krylov_df.cu), which stream at the memory bound instead of the FP64 pipe's.
//
// Classical Gram-Schmidt with one reorthogonalisation is done in three passes
// over the basis V (k vectors of n doubles, vector j at V + j*n):
//   pass 1  h1 = V^T w
//   pass 2  w <- w - V h1,  h2 = V^T w        (fused: V streamed from HBM once,
//                                              its re-read served by L1/L2)
//   pass 3  w <- w - V h2,  ||w||^2            (fused)
// Each block walks 1024-element chunks with the chunk of w in registers and
// reduces one dot per basis vector across the warp.
// Reductions are deterministic: every block writes its partial sums, the last
// block to finish (atomic ticket) adds them in block order with a fixed tree,
// so a result does not depend on scheduling -- an instance gives the same
// bits alone or beside others.
#include <mutex>

#include "rte_internal.h"

namespace rte {
namespace {

constexpr int kT = kRedThreads;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Reduce acc[0..K) over the block into partials[blockIdx.x * KMAX + k], then the
// last block sums the partials over blocks into res[k] (res[k] = post(sum)).
template <int KMAX>
__device__ void block_reduce_finish(double (&acc)[KMAX], int K, double* __restrict__ partials,
                                    unsigned* __restrict__ counter, double* __restrict__ res,
                                    bool sqrt_result, int bid, int nb) {
    __shared__ double red[kT / 32][KMAX];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < K) {
            const double v = warp_sum(acc[k]);
            if (lane == 0) red[warp][k] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][k];
        partials[(size_t)bid * KMAX + k] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == nb - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nw = blockDim.x >> 5;
    for (int k = warp; k < K; k += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(partials + (size_t)b * KMAX + k);
        s = warp_sum(s);
        if (lane == 0) res[k] = sqrt_result ? sqrt(s) : s;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Chunked streaming layout: a block owns chunks of kChunk = 8 * kT consecutive
// elements; lane l of warp w holds elements base + 2l + {0,1} + 64 q, q = 0..3,
// of its 256-element slice (four 16-byte loads per vector), so every load
// instruction of a warp covers 512 contiguous bytes.  Only the last chunk
// needs bounds checks.
constexpr int kChunk = 8 * kT;

struct Slice {
    double v[8];
};

__device__ __forceinline__ int64_t slice_base(int64_t chunk) {
    return chunk * kChunk + (int64_t)(threadIdx.x >> 5) * 256 + 2 * (threadIdx.x & 31);
}

template <bool TAIL>
__device__ __forceinline__ Slice load_slice(const double* __restrict__ p, int64_t base, int64_t n) {
    Slice s;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + 64 * q;
        if (!TAIL || i + 1 < n) {
            const double2 a = *reinterpret_cast<const double2*>(p + i);
            s.v[2 * q] = a.x;
            s.v[2 * q + 1] = a.y;
        } else {
            s.v[2 * q] = i < n ? p[i] : 0.0;
            s.v[2 * q + 1] = 0.0;
        }
    }
    return s;
}

template <bool TAIL>
__device__ __forceinline__ void store_slice(double* __restrict__ p, int64_t base, int64_t n,
                                            const Slice& s) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + 64 * q;
        if (!TAIL || i + 1 < n) {
            *reinterpret_cast<double2*>(p + i) = make_double2(s.v[2 * q], s.v[2 * q + 1]);
        } else if (i < n) {
            p[i] = s.v[2 * q];
        }
    }
}

__device__ __forceinline__ double slice_dot(const Slice& a, const Slice& b) {
    double t0 = a.v[0] * b.v[0], t1 = a.v[1] * b.v[1];
#pragma unroll
    for (int e = 2; e < 8; e += 2) {
        t0 = fma(a.v[e], b.v[e], t0);
        t1 = fma(a.v[e + 1], b.v[e + 1], t1);
    }
    return t0 + t1;
}

// Every thread accumulates its own partial dot products in shared memory,
// s_part[k * kT + tid]; at the end the block reduces them (fixed order) and
// hands the block sums to the last block.
__device__ void finish_dots(const double* s_part, int K, double* partials, unsigned* counter,
                            double* res, int bid, int nb) {
    __shared__ bool s_last;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < K; k += kT / 32) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kT / 32; ++q) t += s_part[k * kT + q * 32 + lane];
        t = warp_sum(t);
        if (lane == 0) partials[(size_t)bid * kMaxKrylov + k] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == nb - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int k = warp; k < K; k += kT / 32) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(partials + (size_t)b * kMaxKrylov + k);
        t = warp_sum(t);
        if (lane == 0) res[k] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// h[k] = V[k] . w for k < K
template <bool TAIL>
__device__ __forceinline__ void mdot_chunk(const double* __restrict__ V, int K, int64_t n,
                                           const double* __restrict__ w, int64_t base,
                                           double* s_part) {
    const int tid = threadIdx.x;
    const Slice ws = load_slice<TAIL>(w, base, n);
    const double* vk = V;
    int k = 0;
    for (; k + 2 <= K; k += 2, vk += 2 * n) {
        const Slice v0 = load_slice<TAIL>(vk, base, n);
        const Slice v1 = load_slice<TAIL>(vk + n, base, n);
        s_part[(k + 0) * kT + tid] += slice_dot(v0, ws);
        s_part[(k + 1) * kT + tid] += slice_dot(v1, ws);
    }
    if (k < K) s_part[k * kT + tid] += slice_dot(load_slice<TAIL>(vk, base, n), ws);
}

// block bid of nb (a plain launch: blockIdx.x of gridDim.x; a grouped one: the
// block's index within its instance's range)
__device__ void mdot_run(const double* __restrict__ V, int K, int64_t n, const double* __restrict__ w,
                         double* partials, unsigned* counter, double* h, int bid, int nb, double* s_part) {
    const int tid = threadIdx.x;
    for (int k = 0; k < K; ++k) s_part[k * kT + tid] = 0.0;
    const int64_t full = n / kChunk, nchunks = (n + kChunk - 1) / kChunk;
    for (int64_t ch = bid; ch < nchunks; ch += nb) {
        if (ch < full)
            mdot_chunk<false>(V, K, n, w, slice_base(ch), s_part);
        else
            mdot_chunk<true>(V, K, n, w, slice_base(ch), s_part);
    }
    finish_dots(s_part, K, partials, counter, h, bid, nb);
}

__global__ void __launch_bounds__(kT) k_mdot(const double* __restrict__ V, int K, int64_t n,
                                             const double* __restrict__ w, double* partials,
                                             unsigned* counter, double* h) {
    extern __shared__ double s_part[];          // [K][kT]
    mdot_run(V, K, n, w, partials, counter, h, blockIdx.x, gridDim.x, s_part);
}

// w <- w - sum_k V[k] h1[k] on one chunk; then (DOTS) s_part[k] += V[k] . w
template <bool TAIL, bool DOTS>
__device__ __forceinline__ Slice update_chunk(const double* __restrict__ V, int K, int64_t n,
                                              double* __restrict__ w, const double* sh,
                                              int64_t base, double* s_part) {
    const int tid = threadIdx.x;
    Slice ws = load_slice<TAIL>(w, base, n);
    const double* vk = V;
    int k = 0;
    for (; k + 2 <= K; k += 2, vk += 2 * n) {
        const Slice v0 = load_slice<TAIL>(vk, base, n);
        const Slice v1 = load_slice<TAIL>(vk + n, base, n);
        const double h0 = sh[k], h1 = sh[k + 1];
#pragma unroll
        for (int e = 0; e < 8; ++e) ws.v[e] = fma(-h1, v1.v[e], fma(-h0, v0.v[e], ws.v[e]));
    }
    if (k < K) {
        const Slice v0 = load_slice<TAIL>(vk, base, n);
        const double h0 = sh[k];
#pragma unroll
        for (int e = 0; e < 8; ++e) ws.v[e] = fma(-h0, v0.v[e], ws.v[e]);
    }
    store_slice<TAIL>(w, base, n, ws);
    if (DOTS) {
        vk = V;
        k = 0;
        for (; k + 2 <= K; k += 2, vk += 2 * n) {
            const Slice v0 = load_slice<TAIL>(vk, base, n);
            const Slice v1 = load_slice<TAIL>(vk + n, base, n);
            s_part[(k + 0) * kT + tid] += slice_dot(v0, ws);
            s_part[(k + 1) * kT + tid] += slice_dot(v1, ws);
        }
        if (k < K) s_part[k * kT + tid] += slice_dot(load_slice<TAIL>(vk, base, n), ws);
    }
    return ws;
}

// w <- w - sum_k V[k] h1[k]; then h2[k] = V[k] . w   (V re-read from cache)
__device__ void update_dot_run(const double* __restrict__ V, int K, int64_t n, double* __restrict__ w,
                               const double* __restrict__ h1, double* partials, unsigned* counter, double* h2,
                               int bid, int nb, double* s_part) {
    __shared__ double sh[kMaxKrylov];
    const int tid = threadIdx.x;
    for (int k = tid; k < K; k += blockDim.x) sh[k] = h1[k];
    for (int k = 0; k < K; ++k) s_part[k * kT + tid] = 0.0;
    __syncthreads();
    const int64_t full = n / kChunk, nchunks = (n + kChunk - 1) / kChunk;
    for (int64_t ch = bid; ch < nchunks; ch += nb) {
        if (ch < full)
            update_chunk<false, true>(V, K, n, w, sh, slice_base(ch), s_part);
        else
            update_chunk<true, true>(V, K, n, w, sh, slice_base(ch), s_part);
    }
    finish_dots(s_part, K, partials, counter, h2, bid, nb);
}

__global__ void __launch_bounds__(kT) k_update_dot(const double* __restrict__ V, int K, int64_t n,
                                                   double* __restrict__ w,
                                                   const double* __restrict__ h1,
                                                   double* partials, unsigned* counter,
                                                   double* h2) {
    extern __shared__ double s_part[];          // [K][kT]
    update_dot_run(V, K, n, w, h1, partials, counter, h2, blockIdx.x, gridDim.x, s_part);
}

// w <- w - sum_k V[k] h2[k]; out[K] = ||w||; out[k] = h1[k] + h2[k]
__device__ void update_norm_run(const double* __restrict__ V, int K, int64_t n, double* __restrict__ w,
                                const double* __restrict__ h1, const double* __restrict__ h2, double* partials,
                                unsigned* counter, double* out, int bid, int nb) {
    __shared__ double sh[kMaxKrylov];
    for (int k = threadIdx.x; k < K; k += blockDim.x) sh[k] = h2[k];
    __syncthreads();
    double acc[1] = {0.0};
    const int64_t full = n / kChunk, nchunks = (n + kChunk - 1) / kChunk;
    for (int64_t ch = bid; ch < nchunks; ch += nb) {
        Slice ws;
        if (ch < full)
            ws = update_chunk<false, false>(V, K, n, w, sh, slice_base(ch), nullptr);
        else
            ws = update_chunk<true, false>(V, K, n, w, sh, slice_base(ch), nullptr);
        acc[0] += slice_dot(ws, ws);
    }
    // out[K] = ||w||; block 0 also writes out[k] = h1[k] + h2[k]
    block_reduce_finish<1>(acc, 1, partials, counter, out + K, true, bid, nb);
    if (bid == 0)
        for (int k = threadIdx.x; k < K; k += blockDim.x) out[k] = h1[k] + h2[k];
}

__global__ void __launch_bounds__(kT) k_update_norm(const double* __restrict__ V, int K, int64_t n,
                                                    double* __restrict__ w,
                                                    const double* __restrict__ h1,
                                                    const double* __restrict__ h2,
                                                    double* partials, unsigned* counter,
                                                    double* out) {
    update_norm_run(V, K, n, w, h1, h2, partials, counter, out, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kT) k_norm(const double* __restrict__ x, int64_t n,
                                             double* partials, unsigned* counter, double* out) {
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc[0] = fma(x[i], x[i], acc[0]);
    block_reduce_finish<1>(acc, 1, partials, counter, out, true, blockIdx.x, gridDim.x);
}

__device__ void scale_run(const double* __restrict__ x, const double* __restrict__ s, int64_t n,
                          double* __restrict__ y, int bid, int nb) {
    const double v = s[0];
    const double inv = (v != 0.0) ? 1.0 / v : 1.0;
    for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x)
        y[i] = x[i] * inv;
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ s, int64_t n,
                        double* __restrict__ y) {
    scale_run(x, s, n, y, blockIdx.x, gridDim.x);
}

__global__ void k_combine_update(double* __restrict__ x, const float* __restrict__ Z, int K,
                                 int64_t n, const double* __restrict__ y) {
    __shared__ double sy[kMaxKrylov];
    for (int k = threadIdx.x; k < K; k += blockDim.x) sy[k] = y[k];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int k = 0; k < K; ++k) s = fma((double)Z[(size_t)k * n + i], sy[k], s);
        x[i] = s;
    }
}

// Grid for the kernels with K x kT doubles of dynamic shared memory: as many
// resident blocks per SM as the shared memory allows (at most 4).
int dot_blocks(rte_ctx* ctx, int64_t n, int K, const void* kern) {
    const size_t smem = (size_t)K * kT * sizeof(double);
    raise_smem_limit((const void*)kern, (size_t)((kMaxKrylov * kT * sizeof(double))));
    int per_sm = 0;
    check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem), "occupancy");
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    int64_t want = (n + kT - 1) / kT;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

int red_blocks(rte_ctx* ctx, int64_t n) {
    int64_t want = (n + kT - 1) / kT;
    int64_t cap = ctx->max_red_blocks;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

void launch_mdot(rte_ctx* ctx, const double* V, int k, const double* w, double* h) {
    const int g = dot_blocks(ctx, ctx->n, k, (const void*)k_mdot);
    ProfScope ps(ctx, K_MDOT, (double)(k + 1) * ctx->n * 8, 1, 2.0 * k * ctx->n);
    k_mdot<<<g, kT, (size_t)k * kT * sizeof(double), ctx->stream>>>(V, k, ctx->n, w, ctx->partials,
                                                                 ctx->counter, h);
    check(cudaGetLastError(), "k_mdot");
}

void launch_update_dot(rte_ctx* ctx, const double* V, int k, double* w, const double* h1,
                       double* h2) {
    const int g = dot_blocks(ctx, ctx->n, k, (const void*)k_update_dot);
    ProfScope ps(ctx, K_UPDATE_DOT, (double)(k + 2) * ctx->n * 8, 1, 4.0 * k * ctx->n);
    k_update_dot<<<g, kT, (size_t)k * kT * sizeof(double), ctx->stream>>>(V, k, ctx->n, w, h1,
                                                                       ctx->partials, ctx->counter,
                                                                       h2);
    check(cudaGetLastError(), "k_update_dot");
}

void launch_update_norm(rte_ctx* ctx, const double* V, int k, double* w, const double* h1,
                        const double* h2, double* out) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_UPDATE_NORM, (double)(k + 2) * ctx->n * 8, 1, (2.0 * k + 2.0) * ctx->n);
    k_update_norm<<<g, kT, 0, ctx->stream>>>(V, k, ctx->n, w, h1, h2, ctx->partials, ctx->counter,
                                             out);
    check(cudaGetLastError(), "k_update_norm");
}

void launch_norm(rte_ctx* ctx, const double* x, double* out) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_NORM, (double)ctx->n * 8);
    k_norm<<<g, kT, 0, ctx->stream>>>(x, ctx->n, ctx->partials, ctx->counter, out);
    check(cudaGetLastError(), "k_norm");
}

void launch_scale(rte_ctx* ctx, const double* x, const double* s, double* y) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_SCALE, (double)ctx->n * 16);
    k_scale<<<g, kT, 0, ctx->stream>>>(x, s, ctx->n, y);
    check(cudaGetLastError(), "k_scale");
}

void launch_combine_update(rte_ctx* ctx, double* x, const float* Z, int k, const double* y) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_XUPDATE, (double)ctx->n * (16 + 4 * k));
    k_combine_update<<<g, kT, 0, ctx->stream>>>(x, Z, k, ctx->n, y);
    check(cudaGetLastError(), "k_combine_update");
}

}  // namespace rte

// ---------------------------------------------------------------------------
// Allocation-free Gram-Schmidt step (rte_cgs2_noalloc).
//
// Same kernels as rte_cgs2, but the scratch they need (per-block partial
// sums, the two projection vectors and the last-block ticket) lives in one
// file-scope device array instead of context buffers, so the call allocates
// nothing.  Layout, in doubles:
//   [0, kNoAllocBlocks * kMaxKrylov)   per-block partial sums
//   next kMaxKrylov                    h1 (first projection)
//   next kMaxKrylov                    h2 (second projection)
//   next 32                            ticket counter (first 4 bytes)
// 640 blocks x 64 + 160 doubles = 328,960 bytes per device, held by every GPU
// that loads the library until the process exits.
// ---------------------------------------------------------------------------
namespace rte {
namespace {

constexpr int kNoAllocBlocks = 640;
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocBlocks * kMaxKrylov + 2 * kMaxKrylov + 32;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Host side: the array's name is only a host stand-in; its device address is
// looked up once per device with that device current and cached here.
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
    std::mutex mu;
    bool ready = false;          // set only once every set-up step succeeded
    double* ptr = nullptr;
    int num_sms = 0;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// Looks up the scratch array's device address and the launch limits of this
// device once; a failure (e.g. during a stream capture, or with a pending
// error) is returned and not cached, so a later call retries.
cudaError_t noalloc_setup(NoAllocDevice& d, int dev) {
    std::lock_guard<std::mutex> lock(d.mu);
    if (d.ready) return cudaSuccess;
    double* ptr = nullptr;
    int sms = 0;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mdot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kMaxKrylov * kT * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_update_dot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kMaxKrylov * kT * sizeof(double)));
    if (e != cudaSuccess) return e;
    d.ptr = ptr;
    d.num_sms = sms;
    d.ready = true;
    return cudaSuccess;
}

int noalloc_grid(int64_t n, int num_sms, int per_sm) {
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    int64_t want = (n + kT - 1) / kT;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (cap > kNoAllocBlocks) cap = kNoAllocBlocks;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace
}  // namespace rte

extern "C" RTE_API rte_status rte_cgs2_noalloc(const double* V_dev, int k, int64_t n,
                                               double* w_dev, double* h_dev, void* stream) {
    using namespace rte;
    if (!V_dev || !w_dev || !h_dev || n < 1) {
        set_error(nullptr, "rte_cgs2_noalloc: NULL pointer or n < 1");
        return RTE_EINVAL;
    }
    if (k < 1 || k > kMaxKrylov) {
        set_error(nullptr, "rte_cgs2_noalloc: k must be in [1, 64] (the static scratch holds 64 "
                           "projections per block)");
        return RTE_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error(nullptr, "rte_cgs2_noalloc: device ordinal above 63");
        return RTE_EINVAL;
    }
    NoAllocDevice& d = g_noalloc_dev[dev];
    e = noalloc_setup(d, dev);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "rte_cgs2_noalloc set-up");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* partials = d.ptr;
    double* h1 = partials + (size_t)kNoAllocBlocks * kMaxKrylov;
    double* h2 = h1 + kMaxKrylov;
    unsigned* counter = reinterpret_cast<unsigned*>(h2 + kMaxKrylov);
    const size_t smem = (size_t)k * kT * sizeof(double);
    int per_mdot = 0, per_ud = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_mdot, k_mdot, kT, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_ud, k_update_dot, kT, smem);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "occupancy");
    // the ticket must start at zero; the array keeps the previous call's bytes
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "cudaMemsetAsync");
    const int g1 = noalloc_grid(n, d.num_sms, per_mdot);
    const int g2 = noalloc_grid(n, d.num_sms, per_ud);
    const int g3 = noalloc_grid(n, d.num_sms, 4);
    k_mdot<<<g1, kT, smem, st>>>(V_dev, k, n, w_dev, partials, counter, h1);
    k_update_dot<<<g2, kT, smem, st>>>(V_dev, k, n, w_dev, h1, partials, counter, h2);
    k_update_norm<<<g3, kT, 0, st>>>(V_dev, k, n, w_dev, h1, h2, partials, counter, h_dev);
    k_scale<<<g3, kT, 0, st>>>(w_dev, h_dev + k, n, w_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(nullptr, e, "rte_cgs2_noalloc launch");
    return RTE_OK;
}

