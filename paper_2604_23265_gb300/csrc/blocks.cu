// Per-cell diagonal blocks of A: build G_C, invert it, apply D_C = G_C^{-1}.
//
// G_C[row (f, j)][k] = L[m_row][k] * d_{k,f}(tau_C): the derivative of the row
// of cell C at face f (direction m_row entering C) with respect to its own
// coefficient k (Eq. 2DTFPS_continuity_cond / boundary_cond).  D_C is the
// block-Jacobi preconditioner of Sec. 4 and the map D of Eq. loss.
//
// Inversion: one CTA per cell, the 2M x 2M block in shared memory (row stride
// 2M+1 so column walks are conflict-free), in-place Gauss-Jordan with partial
// pivoting in FP32; row swaps are undone as column swaps at the end.  FP32 is
// enough here: the block only preconditions, and the flexible Krylov method
// absorbs its rounding.
//
// Storage: Dt[c][j][i] = D_C[i][j] (column-major per cell) so that the apply
// z_i = sum_j D_ij r_j streams each block once with 16-byte loads.
#include "rte_internal.h"

namespace rte {
namespace {

__global__ void __launch_bounds__(256) k_build_invert(int M, const int* __restrict__ mat,
                                                      const double* __restrict__ tau,
                                                      const double* __restrict__ xi,
                                                      const double* __restrict__ L,
                                                      const int* __restrict__ rowdir,
                                                      float* __restrict__ Dt,
                                                      int* __restrict__ singular) {
    extern __shared__ float sm[];
    const int n2 = 2 * M, M2 = M / 2, ld = n2 + 1;
    float* A = sm;                       // [n2][ld]
    float* fac = A + n2 * ld;            // [n2]
    float* half = fac + n2;              // [n2]
    int* perm = reinterpret_cast<int*>(half + n2);   // [n2]
    __shared__ int s_piv;
    __shared__ float s_pivval;
    const int c = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mc = mat[c];
    const double t = tau[c];
    for (int k = tid; k < n2; k += nt) half[k] = (float)exp(-0.5 * t * fabs(xi[(size_t)mc * n2 + k]));
    __syncthreads();
    const double* Lm = L + (size_t)mc * M * n2;
    for (int e = tid; e < n2 * n2; e += nt) {
        const int r = e / n2, k = e - r * n2;
        const int f = r / M2, fk = k / M2;
        const float d = (f == fk) ? 1.0f : ((f == (fk ^ 1)) ? half[k] * half[k] : half[k]);
        A[r * ld + k] = (float)Lm[(size_t)rowdir[r] * n2 + k] * d;
    }
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < n2; ++k) {
        if (tid < 32) {
            float best = -1.0f;
            int bi = k;
            for (int r = k + tid; r < n2; r += 32) {
                const float v = fabsf(A[r * ld + k]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) { s_piv = bi; s_pivval = A[bi * ld + k]; }
        }
        __syncthreads();
        const int p = s_piv;
        const float pv = s_pivval;
        if (!(fabsf(pv) > 0.0f) || !isfinite(pv)) bad = true;
        if (p != k) {
            for (int j = tid; j < n2; j += nt) {
                const float tmp = A[k * ld + j];
                A[k * ld + j] = A[p * ld + j];
                A[p * ld + j] = tmp;
            }
        }
        if (tid == 0) perm[k] = p;
        __syncthreads();
        const float inv = 1.0f / pv;
        for (int j = tid; j < n2; j += nt) {
            const float v = (j == k) ? 1.0f : A[k * ld + j];
            A[k * ld + j] = v * inv;
        }
        for (int i = tid; i < n2; i += nt) fac[i] = (i == k) ? 0.0f : A[i * ld + k];
        __syncthreads();
        for (int e = tid; e < n2 * n2; e += nt) {
            const int i = e / n2, j = e - i * n2;
            if (i == k) continue;
            const float base = (j == k) ? 0.0f : A[i * ld + j];
            A[i * ld + j] = fmaf(-fac[i], A[k * ld + j], base);
        }
        __syncthreads();
    }
    for (int k = n2 - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k) {
            for (int i = tid; i < n2; i += nt) {
                const float tmp = A[i * ld + k];
                A[i * ld + k] = A[i * ld + p];
                A[i * ld + p] = tmp;
            }
        }
        __syncthreads();
    }
    float* out = Dt + (size_t)c * n2 * n2;
    for (int e = tid; e < n2 * n2; e += nt) {
        const int j = e / n2, i = e - j * n2;
        out[e] = A[i * ld + j];
    }
    if (bad && tid == 0) atomicExch(singular, 1);
}

template <typename TIN>
__device__ __forceinline__ float load_in(const TIN* p, size_t i, float s) {
    return (float)((double)p[i] * (double)s);
}

// z_C = D_C r_C.  threads per cell G = 2M/4 (four rows each); block = 256
// threads = 256/G cells; r staged in shared memory.
template <typename TIN>
__global__ void __launch_bounds__(256) k_block_apply(int M, int N, const float* __restrict__ Dt,
                                                     const TIN* __restrict__ r,
                                                     const double* __restrict__ scale,
                                                     float* __restrict__ z) {
    extern __shared__ float sm[];
    const int n2 = 2 * M, G = n2 / 4;
    const int cells = blockDim.x / G;
    float* rs = sm;                    // [n2][cells]
    float* zs = sm + n2 * cells;       // [n2][cells]
    const int c0 = blockIdx.x * cells;
    const float s = scale ? (float)(1.0 / scale[0]) : 1.0f;
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int j = e / cells, cc = e - j * cells;
        const int c = c0 + cc;
        rs[e] = (c < N) ? load_in(r, (size_t)j * N + c, s) : 0.0f;
    }
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const float4* D4 = reinterpret_cast<const float4*>(Dt + (size_t)c * n2 * n2) + g;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
        for (int j = 0; j < n2; ++j) {
            const float4 d = __ldg(D4 + (size_t)j * G);
            const float rv = rs[j * cells + cc];
            acc.x = fmaf(d.x, rv, acc.x);
            acc.y = fmaf(d.y, rv, acc.y);
            acc.z = fmaf(d.z, rv, acc.z);
            acc.w = fmaf(d.w, rv, acc.w);
        }
        zs[(4 * g + 0) * cells + cc] = acc.x;
        zs[(4 * g + 1) * cells + cc] = acc.y;
        zs[(4 * g + 2) * cells + cc] = acc.z;
        zs[(4 * g + 3) * cells + cc] = acc.w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int i = e / cells, c2 = e - i * cells;
        if (c0 + c2 < N) z[(size_t)i * N + c0 + c2] = zs[e];
    }
}

// z_C = D_C^T r_C: output j = row j of Dt dotted with r.
template <typename TIN>
__global__ void __launch_bounds__(256) k_block_apply_t(int M, int N, const float* __restrict__ Dt,
                                                       const TIN* __restrict__ r,
                                                       const double* __restrict__ scale,
                                                       float* __restrict__ z) {
    extern __shared__ float sm[];
    const int n2 = 2 * M, G = n2 / 4;
    const int cells = blockDim.x / G;
    float* rs = sm;
    float* zs = sm + n2 * cells;
    const int c0 = blockIdx.x * cells;
    const float s = scale ? (float)(1.0 / scale[0]) : 1.0f;
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int j = e / cells, cc = e - j * cells;
        const int c = c0 + cc;
        rs[e] = (c < N) ? load_in(r, (size_t)j * N + c, s) : 0.0f;
    }
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const float* D = Dt + (size_t)c * n2 * n2;
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * g + t;
            const float4* row = reinterpret_cast<const float4*>(D + (size_t)j * n2);
            float acc = 0.f;
            for (int i4 = 0; i4 < G; ++i4) {
                const float4 d = __ldg(row + i4);
                acc = fmaf(d.x, rs[(4 * i4 + 0) * cells + cc], acc);
                acc = fmaf(d.y, rs[(4 * i4 + 1) * cells + cc], acc);
                acc = fmaf(d.z, rs[(4 * i4 + 2) * cells + cc], acc);
                acc = fmaf(d.w, rs[(4 * i4 + 3) * cells + cc], acc);
            }
            zs[j * cells + cc] = acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int i = e / cells, c2 = e - i * cells;
        if (c0 + c2 < N) z[(size_t)i * N + c0 + c2] = zs[e];
    }
}

}  // namespace

void launch_build_invert(rte_ctx* ctx, int* singular_dev) {
    const int M = ctx->M, n2 = 2 * M;
    const size_t smem = sizeof(float) * ((size_t)n2 * (n2 + 1) + 3 * n2);
    check(cudaFuncSetAttribute(k_build_invert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem), "build_invert smem");
    const int threads = n2 >= 64 ? 256 : 128;
    ProfScope ps(ctx, K_INVERT, (double)ctx->N * n2 * n2 * 4);
    k_build_invert<<<ctx->N, threads, smem, ctx->stream>>>(M, ctx->mat, ctx->tau, ctx->xi,
                                                           ctx->L64, ctx->rowdir, ctx->Dt,
                                                           singular_dev);
    check(cudaGetLastError(), "k_build_invert");
}

void launch_block_apply(rte_ctx* ctx, bool transpose, const void* r, bool r_is_double, float* z,
                        const double* scale_dev) {
    const int M = ctx->M, n2 = 2 * M, G = n2 / 4;
    const int threads = G >= 256 ? G : (256 / G) * G;
    const int cells = threads / G;
    const int blocks = (ctx->N + cells - 1) / cells;
    const size_t smem = sizeof(float) * 2 * n2 * cells;
    ProfScope ps(ctx, transpose ? K_BLOCK_T : K_BLOCK,
                 (double)ctx->N * n2 * n2 * 4 + (double)ctx->n * ((r_is_double ? 8 : 4) + 4));
    if (!transpose) {
        if (r_is_double) {
            check(cudaFuncSetAttribute(k_block_apply<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "ba");
            k_block_apply<double><<<blocks, threads, smem, ctx->stream>>>(
                M, ctx->N, ctx->Dt, (const double*)r, scale_dev, z);
        } else {
            check(cudaFuncSetAttribute(k_block_apply<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "ba");
            k_block_apply<float><<<blocks, threads, smem, ctx->stream>>>(
                M, ctx->N, ctx->Dt, (const float*)r, scale_dev, z);
        }
    } else {
        if (r_is_double) {
            check(cudaFuncSetAttribute(k_block_apply_t<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "bat");
            k_block_apply_t<double><<<blocks, threads, smem, ctx->stream>>>(
                M, ctx->N, ctx->Dt, (const double*)r, scale_dev, z);
        } else {
            check(cudaFuncSetAttribute(k_block_apply_t<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "bat");
            k_block_apply_t<float><<<blocks, threads, smem, ctx->stream>>>(
                M, ctx->N, ctx->Dt, (const float*)r, scale_dev, z);
        }
    }
    check(cudaGetLastError(), "k_block_apply");
}

}  // namespace rte
