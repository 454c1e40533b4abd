// Krylov kernels of flexible GMRES: multi-dot, fused Gram-Schmidt passes,
// norms, scaling, solution update, Givens/Hessenberg update and the
// triangular solve -- all FP64 on the device.
//
// Classical Gram-Schmidt with one reorthogonalisation is done in three passes
// over the basis V (k vectors of n doubles, vector j at V + j*n):
//   pass 1  h1 = V^T w
//   pass 2  w <- w - V h1,  h2 = V^T w        (fused: V read once)
//   pass 3  w <- w - V h2,  ||w||^2            (fused)
// Reductions are deterministic: every block writes its partial sums, the last
// block to finish (atomic ticket) adds them in block order with a fixed tree,
// so a result does not depend on scheduling -- an instance gives the same
// bits alone or beside others.
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
                                    bool sqrt_result) {
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
        partials[(size_t)blockIdx.x * KMAX + k] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nw = blockDim.x >> 5;
    for (int k = warp; k < K; k += nw) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partials + (size_t)b * KMAX + k);
        s = warp_sum(s);
        if (lane == 0) res[k] = sqrt_result ? sqrt(s) : s;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

template <int KMAX>
__global__ void __launch_bounds__(kT) k_mdot(const double* __restrict__ V, int K, int64_t n,
                                             const double* __restrict__ w, double* partials,
                                             unsigned* counter, double* h) {
    double acc[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) acc[k] = fma(V[(size_t)k * n + i], wi, acc[k]);
    }
    block_reduce_finish<KMAX>(acc, K, partials, counter, h, false);
}

template <int KMAX>
__global__ void __launch_bounds__(kT) k_update_dot(const double* __restrict__ V, int K, int64_t n,
                                                   double* __restrict__ w,
                                                   const double* __restrict__ h1,
                                                   double* partials, unsigned* counter,
                                                   double* h2) {
    __shared__ double sh[KMAX];
    for (int k = threadIdx.x; k < K; k += blockDim.x) sh[k] = h1[k];
    __syncthreads();
    double acc[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) s = fma(V[(size_t)k * n + i], sh[k], s);
        const double wi = w[i] - s;
        w[i] = wi;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) acc[k] = fma(V[(size_t)k * n + i], wi, acc[k]);
    }
    block_reduce_finish<KMAX>(acc, K, partials, counter, h2, false);
}

template <int KMAX>
__global__ void __launch_bounds__(kT) k_update_norm(const double* __restrict__ V, int K, int64_t n,
                                                    double* __restrict__ w,
                                                    const double* __restrict__ h1,
                                                    const double* __restrict__ h2,
                                                    double* partials, unsigned* counter,
                                                    double* out) {
    __shared__ double sh[KMAX];
    for (int k = threadIdx.x; k < K; k += blockDim.x) sh[k] = h2[k];
    __syncthreads();
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) s = fma(V[(size_t)k * n + i], sh[k], s);
        const double wi = w[i] - s;
        w[i] = wi;
        acc[0] = fma(wi, wi, acc[0]);
    }
    // out[K] = ||w||; the last block also writes out[k] = h1[k] + h2[k]
    block_reduce_finish<1>(acc, 1, partials, counter, out + K, true);
    if (blockIdx.x == 0) {
        // every block could do this; block 0 does it once (h1, h2 are final)
        for (int k = threadIdx.x; k < K; k += blockDim.x) out[k] = h1[k] + h2[k];
    }
}

__global__ void __launch_bounds__(kT) k_norm(const double* __restrict__ x, int64_t n,
                                             double* partials, unsigned* counter, double* out) {
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc[0] = fma(x[i], x[i], acc[0]);
    block_reduce_finish<1>(acc, 1, partials, counter, out, true);
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ s, int64_t n,
                        double* __restrict__ y) {
    const double v = s[0];
    const double inv = (v != 0.0) ? 1.0 / v : 1.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * inv;
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

int red_blocks(rte_ctx* ctx, int64_t n) {
    int64_t want = (n + kT - 1) / kT;
    int64_t cap = ctx->max_red_blocks;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

void launch_mdot(rte_ctx* ctx, const double* V, int k, const double* w, double* h) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_MDOT, (double)(k + 1) * ctx->n * 8);
#define RTE_MDOT(KM) \
    k_mdot<KM><<<g, kT, 0, ctx->stream>>>(V, k, ctx->n, w, ctx->partials, ctx->counter, h)
    if (k <= 8) RTE_MDOT(8); else if (k <= 16) RTE_MDOT(16); else if (k <= 32) RTE_MDOT(32);
    else RTE_MDOT(64);
#undef RTE_MDOT
    check(cudaGetLastError(), "k_mdot");
}

void launch_update_dot(rte_ctx* ctx, const double* V, int k, double* w, const double* h1,
                       double* h2) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_UPDATE_DOT, (double)(k + 2) * ctx->n * 8);
#define RTE_UD(KM)                                                                     \
    k_update_dot<KM><<<g, kT, 0, ctx->stream>>>(V, k, ctx->n, w, h1, ctx->partials, \
                                                ctx->counter, h2)
    if (k <= 8) RTE_UD(8); else if (k <= 16) RTE_UD(16); else if (k <= 32) RTE_UD(32);
    else RTE_UD(64);
#undef RTE_UD
    check(cudaGetLastError(), "k_update_dot");
}

void launch_update_norm(rte_ctx* ctx, const double* V, int k, double* w, const double* h1,
                        const double* h2, double* out) {
    const int g = red_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_UPDATE_NORM, (double)(k + 2) * ctx->n * 8);
#define RTE_UN(KM)                                                                         \
    k_update_norm<KM><<<g, kT, 0, ctx->stream>>>(V, k, ctx->n, w, h1, h2, ctx->partials, \
                                                 ctx->counter, out)
    if (k <= 8) RTE_UN(8); else if (k <= 16) RTE_UN(16); else if (k <= 32) RTE_UN(32);
    else RTE_UN(64);
#undef RTE_UN
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
