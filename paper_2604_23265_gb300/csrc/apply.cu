// TFPS operator kernels: y = A x, x = A^T y, reconstruction and right-hand side.
//
// A (Eq. 2DTFPS_linear_sys) is applied matrix-free.  For every cell C the four
// face-midpoint traces of sum_k x_Ck chi_C^k (Eq. 2D_eigenfunc) are
//   T_W = L_x (dW o x_x) + L_y (h o x_y)    T_E = L_x (dE o x_x) + L_y (h o x_y)
//   T_S = L_x (h o x_x) + L_y (dS o x_y)    T_N = L_x (h o x_x) + L_y (dN o x_y)
// with decay factors 1 at the centred face, exp(-tau|xi|) at the opposite face
// and h = exp(-tau|xi|/2) at the perpendicular faces: six M x M products per
// cell.  Rows entering C through f take T_{C,f} (kernel 1, written straight
// into y); the other half of each trace is the outgoing half the neighbour
// across f needs, staged in a scratch buffer; kernel 2 subtracts the
// neighbour's outgoing trace (Eq. 2DTFPS_continuity_cond) -- boundary rows keep
// the trace alone (Eq. 2DTFPS_boundary_cond).
//
// Layout: x, y direction-major [2M][N]; one warp = 32 consecutive cells (lanes),
// warps of a block split the M directions into chunks of MB, so the scaled
// coefficients sit in shared memory ([6M][32]) and the basis rows are
// broadcast loads.
#include <type_traits>

#include "rte_internal.h"

namespace rte {
namespace {

constexpr int kCellsPerBlock = 32;

template <typename T>
__device__ __forceinline__ T dexp(T v);
template <>
__device__ __forceinline__ double dexp<double>(double v) { return exp(v); }
template <>
__device__ __forceinline__ float dexp<float>(float v) { return expf(v); }

struct OpArgs {
    int I, M, N;
    const int* mat;
    const double* tau;
    const double* xi;
    const int* rowinfo;
};

// Kernel 1: traces.  blockDim = 32 * (M / MB).
template <typename T, int MB>
__global__ void __launch_bounds__(256) k_traces(OpArgs a, const T* __restrict__ Lt,
                                                const T* __restrict__ x, T* __restrict__ y,
                                                T* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);        // [6][M][32]: W,E,P (x) then S,N,Q (y)
    const int M = a.M, N = a.N, M2 = M / 2;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int c = blockIdx.x * kCellsPerBlock + lane;
    const bool valid = c < N;
    const int mat = valid ? a.mat[c] : 0;
    const T tau = valid ? (T)a.tau[c] : (T)0;
    const double* xim = a.xi + (size_t)mat * 2 * M;

    // stage scaled coefficients
    for (int k = warp; k < 2 * M; k += nwarps) {
        T v = valid ? x[(size_t)k * N + c] : (T)0;
        T half = dexp<T>((T)(-0.5) * tau * (T)fabs(xim[k]));
        T full = half * half;
        int grp = k / M2;                          // 0 W, 1 E, 2 S, 3 N
        int kk = k % M;                            // index within x- or y-type
        T* base = s + (grp < 2 ? 0 : 3 * M * 32);
        T dfirst = (grp == 0 || grp == 2) ? (T)1 : full;   // at W (x) or S (y)
        T dsecond = (grp == 0 || grp == 2) ? full : (T)1;  // at E (x) or N (y)
        base[(0 * M + kk) * 32 + lane] = v * dfirst;
        base[(1 * M + kk) * 32 + lane] = v * dsecond;
        base[(2 * M + kk) * 32 + lane] = v * half;
    }
    __syncthreads();

    const T* LtM = Lt + (size_t)mat * 2 * M * M;
    for (int m0 = warp * MB; m0 < M; m0 += nwarps * MB) {
        T xw[MB], xe[MB], xp[MB], ys[MB], yn[MB], yp[MB];
#pragma unroll
        for (int i = 0; i < MB; ++i) xw[i] = xe[i] = xp[i] = ys[i] = yn[i] = yp[i] = (T)0;
        for (int k = 0; k < M; ++k) {
            const T sw = s[(0 * M + k) * 32 + lane];
            const T se = s[(1 * M + k) * 32 + lane];
            const T sp = s[(2 * M + k) * 32 + lane];
            const T ss = s[(3 * M + k) * 32 + lane];
            const T sn = s[(4 * M + k) * 32 + lane];
            const T sq = s[(5 * M + k) * 32 + lane];
            const T* lx = LtM + (size_t)k * M + m0;
            const T* ly = LtM + (size_t)(M + k) * M + m0;
#pragma unroll
            for (int i = 0; i < MB; ++i) {
                const T vx = __ldg(lx + i);
                const T vy = __ldg(ly + i);
                xw[i] = fma(vx, sw, xw[i]);
                xe[i] = fma(vx, se, xe[i]);
                xp[i] = fma(vx, sp, xp[i]);
                ys[i] = fma(vy, ss, ys[i]);
                yn[i] = fma(vy, sn, yn[i]);
                yp[i] = fma(vy, sq, yp[i]);
            }
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < MB; ++i) {
                const int m = m0 + i;
                const T tr[4] = {xw[i] + yp[i], xe[i] + yp[i], xp[i] + ys[i], xp[i] + yn[i]};
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const int info = a.rowinfo[f * M + m];
                    if (info >= 0)
                        y[(size_t)(f * M2 + info) * N + c] = tr[f];
                    else
                        out[(size_t)(f * M2 + (-info - 1)) * N + c] = tr[f];
                }
            }
        }
    }
}

// Kernel 1, single-material variant: the basis (Lt, 2M x M) is staged in
// shared memory once per block and read with 16-byte broadcast loads; each
// thread keeps a 6 x MB register tile (MB = 16 directions).
template <typename T, int MB>
__global__ void __launch_bounds__(256) k_traces_shl(OpArgs a, const T* __restrict__ Lt,
                                                    const T* __restrict__ x, T* __restrict__ y,
                                                    T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = a.M, N = a.N, M2 = M / 2;
    T* Ls = reinterpret_cast<T*>(smem_raw);        // [2M][M]
    T* s = Ls + 2 * M * M;                          // [6][M][32]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int c = blockIdx.x * kCellsPerBlock + lane;
    const bool valid = c < N;
    const T tau = valid ? (T)a.tau[c] : (T)0;
    const double* xim = a.xi;                       // material 0
    for (int e = threadIdx.x; e < 2 * M * M; e += blockDim.x) Ls[e] = Lt[e];
    for (int k = warp; k < 2 * M; k += nwarps) {
        T v = valid ? x[(size_t)k * N + c] : (T)0;
        T half = dexp<T>((T)(-0.5) * tau * (T)fabs(xim[k]));
        T full = half * half;
        int grp = k / M2;
        int kk = k % M;
        T* base = s + (grp < 2 ? 0 : 3 * M * 32);
        T dfirst = (grp == 0 || grp == 2) ? (T)1 : full;
        T dsecond = (grp == 0 || grp == 2) ? full : (T)1;
        base[(0 * M + kk) * 32 + lane] = v * dfirst;
        base[(1 * M + kk) * 32 + lane] = v * dsecond;
        base[(2 * M + kk) * 32 + lane] = v * half;
    }
    __syncthreads();
    constexpr int VW = 16 / sizeof(T);              // elements per 16-byte load
    using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    for (int m0 = warp * MB; m0 < M; m0 += nwarps * MB) {
        T xw[MB], xe[MB], xp[MB], ys[MB], yn[MB], yp[MB];
#pragma unroll
        for (int i = 0; i < MB; ++i) xw[i] = xe[i] = xp[i] = ys[i] = yn[i] = yp[i] = (T)0;
#pragma unroll 2
        for (int k = 0; k < M; ++k) {
            const T sw = s[(0 * M + k) * 32 + lane];
            const T se = s[(1 * M + k) * 32 + lane];
            const T sp = s[(2 * M + k) * 32 + lane];
            const T ss = s[(3 * M + k) * 32 + lane];
            const T sn = s[(4 * M + k) * 32 + lane];
            const T sq = s[(5 * M + k) * 32 + lane];
            const V16* lx4 = reinterpret_cast<const V16*>(Ls + (size_t)k * M + m0);
            const V16* ly4 = reinterpret_cast<const V16*>(Ls + (size_t)(M + k) * M + m0);
#pragma unroll
            for (int q = 0; q < MB / VW; ++q) {
                const V16 lxv = lx4[q];
                const V16 lyv = ly4[q];
                const T* lx = reinterpret_cast<const T*>(&lxv);
                const T* ly = reinterpret_cast<const T*>(&lyv);
#pragma unroll
                for (int t = 0; t < VW; ++t) {
                    const int i = q * VW + t;
                    xw[i] = fma(lx[t], sw, xw[i]);
                    xe[i] = fma(lx[t], se, xe[i]);
                    xp[i] = fma(lx[t], sp, xp[i]);
                    ys[i] = fma(ly[t], ss, ys[i]);
                    yn[i] = fma(ly[t], sn, yn[i]);
                    yp[i] = fma(ly[t], sq, yp[i]);
                }
            }
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < MB; ++i) {
                const int m = m0 + i;
                const T tr[4] = {xw[i] + yp[i], xe[i] + yp[i], xp[i] + ys[i], xp[i] + yn[i]};
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const int info = a.rowinfo[f * M + m];
                    if (info >= 0)
                        y[(size_t)(f * M2 + info) * N + c] = tr[f];
                    else
                        out[(size_t)(f * M2 + (-info - 1)) * N + c] = tr[f];
                }
            }
        }
    }
}

// Kernel 2: subtract the neighbour's outgoing trace; optionally r = b - A x.
template <typename T, typename TO>
__global__ void k_combine(int I, int M, const T* __restrict__ yown, const T* __restrict__ out,
                          const double* __restrict__ b, TO* __restrict__ y) {
    const int N = I * I;
    const int M2 = M / 2;
    const int64_t n = (int64_t)2 * M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / N);
        const int c = (int)(e - (int64_t)row * N);
        const int f = row / M2;
        const int j = row - f * M2;
        const int iy = c / I, ix = c - iy * I;
        int nb = -1;
        if (f == 0 && ix > 0) nb = c - 1;
        if (f == 1 && ix < I - 1) nb = c + 1;
        if (f == 2 && iy > 0) nb = c - I;
        if (f == 3 && iy < I - 1) nb = c + I;
        double v = (double)yown[e];
        if (nb >= 0) {
            const int of = f ^ 1;                    // opposite face
            v -= (double)out[(int64_t)(of * M2 + j) * N + nb];
        }
        if (b != nullptr) v = b[e] - v;
        y[e] = (TO)v;
    }
}

// Adjoint: x = A^T y.  Gather the trace cotangents U_f per cell, then apply
// the transposed basis: x_k = sum_f d_{k,f} (L^T U_f)_k.
template <typename T, int MB>
__global__ void __launch_bounds__(256) k_adjoint(OpArgs a, const T* __restrict__ L,
                                                 const T* __restrict__ y, T* __restrict__ x) {
    extern __shared__ unsigned char smem_raw[];
    T* u = reinterpret_cast<T*>(smem_raw);        // [4][M][32]
    const int M = a.M, N = a.N, M2 = M / 2, I = a.I;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int c = blockIdx.x * kCellsPerBlock + lane;
    const bool valid = c < N;
    const int iy = c / I, ix = c - iy * I;
    int nb[4] = {-1, -1, -1, -1};
    if (valid) {
        if (ix > 0) nb[0] = c - 1;
        if (ix < I - 1) nb[1] = c + 1;
        if (iy > 0) nb[2] = c - I;
        if (iy < I - 1) nb[3] = c + I;
    }
    for (int q = warp; q < 4 * M; q += nwarps) {
        const int f = q / M, m = q - f * M;
        const int info = a.rowinfo[f * M + m];
        T v = (T)0;
        if (valid) {
            if (info >= 0) {
                v = y[(size_t)(f * M2 + info) * N + c];
            } else if (nb[f] >= 0) {
                const int of = f ^ 1;
                v = -y[(size_t)(of * M2 + (-info - 1)) * N + nb[f]];
            }
        }
        u[(f * M + m) * 32 + lane] = v;
    }
    __syncthreads();
    const int mat = valid ? a.mat[c] : 0;
    const T tau = valid ? (T)a.tau[c] : (T)0;
    const double* xim = a.xi + (size_t)mat * 2 * M;
    const T* Lm = L + (size_t)mat * M * 2 * M;    // [M][2M]
    for (int k0 = warp * MB; k0 < M; k0 += nwarps * MB) {
        T aw[MB], ae[MB], ap[MB], bs[MB], bn[MB], bp[MB];
#pragma unroll
        for (int i = 0; i < MB; ++i) aw[i] = ae[i] = ap[i] = bs[i] = bn[i] = bp[i] = (T)0;
        for (int m = 0; m < M; ++m) {
            const T uw = u[(0 * M + m) * 32 + lane];
            const T ue = u[(1 * M + m) * 32 + lane];
            const T us = u[(2 * M + m) * 32 + lane];
            const T un = u[(3 * M + m) * 32 + lane];
            const T* lx = Lm + (size_t)m * 2 * M + k0;
            const T* ly = lx + M;
#pragma unroll
            for (int i = 0; i < MB; ++i) {
                const T vx = __ldg(lx + i);
                const T vy = __ldg(ly + i);
                aw[i] = fma(vx, uw, aw[i]);
                ae[i] = fma(vx, ue, ae[i]);
                ap[i] = fma(vx, us + un, ap[i]);
                bs[i] = fma(vy, us, bs[i]);
                bn[i] = fma(vy, un, bn[i]);
                bp[i] = fma(vy, uw + ue, bp[i]);
            }
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < MB; ++i) {
                const int kx = k0 + i;          // x-type slot (W if kx < M2 else E)
                const int ky = M + k0 + i;      // y-type slot (S if k0+i < M2 else N)
                const T hx = dexp<T>((T)(-0.5) * tau * (T)fabs(xim[kx]));
                const T hy = dexp<T>((T)(-0.5) * tau * (T)fabs(xim[ky]));
                const T fx = hx * hx, fy = hy * hy;
                const bool first = (k0 + i) < M2;
                x[(size_t)kx * N + c] = first ? (aw[i] + ae[i] * fx + ap[i] * hx)
                                              : (aw[i] * fx + ae[i] + ap[i] * hx);
                x[(size_t)ky * N + c] = first ? (bs[i] + bn[i] * fy + bp[i] * hy)
                                              : (bs[i] * fy + bn[i] + bp[i] * hy);
            }
        }
    }
}

// psi_m(centre) = sum_k L[m][k] x_k exp(-tau|xi_k|/2) + q/sigma_a  (Eq. 2DTFPS_sol)
template <int MB>
__global__ void __launch_bounds__(256) k_reconstruct(OpArgs a, const double* __restrict__ Lt,
                                                     const double* __restrict__ chis,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ psi) {
    extern __shared__ unsigned char smem_raw[];
    double* s = reinterpret_cast<double*>(smem_raw);   // [2M][32]
    const int M = a.M, N = a.N;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int c = blockIdx.x * kCellsPerBlock + lane;
    const bool valid = c < N;
    const int mat = valid ? a.mat[c] : 0;
    const double tau = valid ? a.tau[c] : 0.0;
    const double* xim = a.xi + (size_t)mat * 2 * M;
    for (int k = warp; k < 2 * M; k += nwarps) {
        const double v = valid ? x[(size_t)k * N + c] : 0.0;
        s[k * 32 + lane] = v * exp(-0.5 * tau * fabs(xim[k]));
    }
    __syncthreads();
    const double* LtM = Lt + (size_t)mat * 2 * M * M;
    for (int m0 = warp * MB; m0 < M; m0 += nwarps * MB) {
        double acc[MB];
#pragma unroll
        for (int i = 0; i < MB; ++i) acc[i] = 0.0;
        for (int k = 0; k < 2 * M; ++k) {
            const double sv = s[k * 32 + lane];
#pragma unroll
            for (int i = 0; i < MB; ++i) acc[i] = fma(__ldg(LtM + (size_t)k * M + m0 + i), sv, acc[i]);
        }
        if (valid) {
            const double p = chis[c];
#pragma unroll
            for (int i = 0; i < MB; ++i) psi[(size_t)(m0 + i) * N + c] = acc[i] + p;
        }
    }
}

// b of Eq. 2DTFPS_linear_sys: chis(nbr) - chis(C) inside, inflow - chis(C) on the boundary
__global__ void k_rhs(int I, int M, const int* __restrict__ rowdir, const double* __restrict__ chis,
                      const double* __restrict__ inflow, double* __restrict__ b) {
    const int N = I * I, M2 = M / 2;
    const int64_t n = (int64_t)2 * M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / N);
        const int c = (int)(e - (int64_t)row * N);
        const int f = row / M2;
        const int iy = c / I, ix = c - iy * I;
        int nb = -1, pos = 0;
        if (f == 0) { nb = ix > 0 ? c - 1 : -1; pos = iy; }
        if (f == 1) { nb = ix < I - 1 ? c + 1 : -1; pos = iy; }
        if (f == 2) { nb = iy > 0 ? c - I : -1; pos = ix; }
        if (f == 3) { nb = iy < I - 1 ? c + I : -1; pos = ix; }
        const int m = rowdir[row];
        b[e] = (nb >= 0 ? chis[nb] : inflow[((size_t)f * I + pos) * M + m]) - chis[c];
    }
}

// CoeffNet input channels per cell: log sigma_T, log sigma_a, log eps, log tau
__global__ void k_coef_inputs(int N, double h, const double* __restrict__ sT,
                              const double* __restrict__ sa, const double* __restrict__ eps,
                              float* __restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        out[c] = (float)log(sT[c]);
        out[N + c] = (float)log(sa[c]);
        out[2 * N + c] = (float)log(eps[c]);
        out[3 * N + c] = (float)log(sT[c] * h / eps[c]);
    }
}

OpArgs op_args(rte_ctx* ctx) {
    return OpArgs{ctx->I, ctx->M, ctx->N, ctx->mat, ctx->tau, ctx->xi, ctx->rowinfo};
}

int grid_stride_blocks(rte_ctx* ctx, int64_t n) {
    int64_t want = (n + 255) / 256;
    int64_t cap = (int64_t)ctx->num_sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename T>
void apply_impl(rte_ctx* ctx, const T* x, void* y, bool y_is_double, const double* b) {
    const int M = ctx->M;
    const int blocks = (ctx->N + kCellsPerBlock - 1) / kCellsPerBlock;
    T* own = reinterpret_cast<T*>(ctx->trace_out);                    // first half of scratch
    T* out = own + ctx->n;                                            // second half
    const T* Lt = std::is_same<T, double>::value ? (const T*)ctx->Lt64 : (const T*)ctx->Lt32;
    {
        ProfScope ps(ctx, K_TRACES, (double)ctx->n * sizeof(T), 1,
                     sizeof(T) == 8 ? 12.0 * ctx->M * ctx->M * ctx->N : 0.0);
        constexpr int MBS = sizeof(T) == 4 ? 16 : 8;
        const size_t smem_shl = sizeof(T) * (2 * (size_t)M * M + 6 * (size_t)M * 32);
        if (ctx->nmat == 1 && M % MBS == 0 && smem_shl <= 200 * 1024) {
            const int warps = M / MBS < 8 ? M / MBS : 8;
            auto kern = k_traces_shl<T, MBS>;
            raise_smem_limit((const void*)kern, (size_t)(smem_shl));
            kern<<<blocks, warps * 32, smem_shl, ctx->stream>>>(op_args(ctx), Lt, x, own, out);
        } else {
            const int MB = (M % 8 == 0) ? 8 : 4;
            const int warps = M / MB < 8 ? M / MB : 8;
            const size_t smem = sizeof(T) * 6 * M * 32;
            auto kern = (MB == 8) ? k_traces<T, 8> : k_traces<T, 4>;
            raise_smem_limit((const void*)kern, (size_t)(smem));
            kern<<<blocks, warps * 32, smem, ctx->stream>>>(op_args(ctx), Lt, x, own, out);
        }
        check(cudaGetLastError(), "k_traces");
    }
    const int g = grid_stride_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_COMBINE,
                 (double)ctx->n * ((y_is_double ? 8 : 4) + (b ? 8 : 0)));
    if (y_is_double)
        k_combine<T, double><<<g, 256, 0, ctx->stream>>>(ctx->I, M, own, out, b, (double*)y);
    else
        k_combine<T, float><<<g, 256, 0, ctx->stream>>>(ctx->I, M, own, out, b, (float*)y);
    check(cudaGetLastError(), "k_combine");
}

template <typename T>
void adjoint_impl(rte_ctx* ctx, const T* y, T* x) {
    const int M = ctx->M;
    const int MB = (M % 8 == 0) ? 8 : 4;
    const int warps = M / MB < 8 ? M / MB : 8;
    const int blocks = (ctx->N + kCellsPerBlock - 1) / kCellsPerBlock;
    const size_t smem = sizeof(T) * 4 * M * 32;
    const T* L = std::is_same<T, double>::value ? (const T*)ctx->L64 : (const T*)ctx->L32;
    auto kern = (MB == 8) ? k_adjoint<T, 8> : k_adjoint<T, 4>;
    raise_smem_limit((const void*)kern, (size_t)(smem));
    ProfScope ps(ctx, K_ADJOINT, 2.0 * ctx->n * sizeof(T));
    kern<<<blocks, warps * 32, smem, ctx->stream>>>(op_args(ctx), L, y, x);
    check(cudaGetLastError(), "k_adjoint");
}

}  // namespace

void launch_apply(rte_ctx* ctx, bool f64, const void* x, void* y, bool y_is_double,
                  const double* b) {
    if (f64)
        apply_impl<double>(ctx, (const double*)x, y, y_is_double, b);
    else
        apply_impl<float>(ctx, (const float*)x, y, y_is_double, b);
}

void launch_apply_adjoint(rte_ctx* ctx, bool f64, const void* y, void* x) {
    if (f64)
        adjoint_impl<double>(ctx, (const double*)y, (double*)x);
    else
        adjoint_impl<float>(ctx, (const float*)y, (float*)x);
}

void launch_reconstruct(rte_ctx* ctx, const double* x, double* psi) {
    const int M = ctx->M;
    const int MB = (M % 8 == 0) ? 8 : 4;
    const int warps = M / MB < 8 ? M / MB : 8;
    const int blocks = (ctx->N + kCellsPerBlock - 1) / kCellsPerBlock;
    const size_t smem = sizeof(double) * 2 * M * 32;
    auto kern = (MB == 8) ? k_reconstruct<8> : k_reconstruct<4>;
    raise_smem_limit((const void*)kern, (size_t)(smem));
    ProfScope ps(ctx, K_RECONSTRUCT, (double)ctx->n * 8 + (double)ctx->M * ctx->N * 8);
    kern<<<blocks, warps * 32, smem, ctx->stream>>>(op_args(ctx), ctx->Lt64, ctx->chis, x, psi);
    check(cudaGetLastError(), "k_reconstruct");
}

void launch_coef_inputs(rte_ctx* ctx, const double* sT, const double* sa, const double* eps) {
    k_coef_inputs<<<(ctx->N + 255) / 256, 256, 0, ctx->stream>>>(ctx->N, 1.0 / ctx->I, sT, sa, eps,
                                                                  ctx->coef_in);
    check(cudaGetLastError(), "k_coef_inputs");
}

void launch_rhs(rte_ctx* ctx) {
    const int g = grid_stride_blocks(ctx, ctx->n);
    ProfScope ps(ctx, K_RHS, (double)ctx->n * 8);
    k_rhs<<<g, 256, 0, ctx->stream>>>(ctx->I, ctx->M, ctx->rowdir, ctx->chis, ctx->inflow, ctx->b);
    check(cudaGetLastError(), "k_rhs");
}

}  // namespace rte
