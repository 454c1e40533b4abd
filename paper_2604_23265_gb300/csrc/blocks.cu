// Per-cell diagonal blocks of A: build G_C, invert it, apply D_C = G_C^{-1}.
//
// G_C[row (f, j)][k] = L[m_row][k] * d_{k,f}(tau_C): the derivative of the row
// of cell C at face f (direction m_row entering C) with respect to its own
// coefficient k (Eq. 2DTFPS_continuity_cond / boundary_cond).  D_C is the
// block-Jacobi preconditioner of Sec. 4 and the map D of Eq. loss.
//
// Inversion: one CTA per cell, the 2M x 2M block in shared memory (row stride
// 2M+1 so column walks are conflict-free), in-place Gauss-Jordan with partial
// pivoting in FP64; row swaps are undone as column swaps at the end.  FP64 is
// needed: in the diffusive limit the four slow basis functions of a cell are
// nearly parallel, cond(G_C) reaches 1e8, and D_C maps the Krylov correction
// back to the coefficients once per restart cycle.
//
// Storage: Dt[c][j][i] = D_C[i][j] (column-major per cell) so that the apply
// z_i = sum_j D_ij r_j streams each block once with 16-byte loads.
#include "df64.h"
#include "rte_internal.h"

namespace rte {
namespace {

// In-place Gauss-Jordan inversion with partial pivoting of the n2 x n2 block
// A (row stride ld) in shared memory by the whole CTA; fac, perm: n2 scratch
// each.  Row swaps are undone as column swaps.  Returns true (thread 0) when a
// pivot is zero or not finite.
__device__ bool gauss_jordan_inplace(double* A, int n2, int ld, double* fac, int* perm) {
    __shared__ int s_piv;
    __shared__ double s_pivval;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int R = nt >= n2 ? nt / n2 : 1;          // row classes per column
    bool bad = false;
    for (int k = 0; k < n2; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int r = k + tid; r < n2; r += 32) {
                const double v = fabs(A[r * ld + k]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) { s_piv = bi; s_pivval = A[bi * ld + k]; }
        }
        __syncthreads();
        const int p = s_piv;
        const double pv = s_pivval;
        if (!(fabs(pv) > 0.0) || !isfinite(pv)) bad = true;
        if (p != k) {
            for (int j = tid; j < n2; j += nt) {
                const double tmp = A[k * ld + j];
                A[k * ld + j] = A[p * ld + j];
                A[p * ld + j] = tmp;
            }
        }
        if (tid == 0) perm[k] = p;
        __syncthreads();
        const double inv = 1.0 / pv;
        for (int j = tid; j < n2; j += nt) {
            const double v = (j == k) ? 1.0 : A[k * ld + j];
            A[k * ld + j] = v * inv;
        }
        for (int i = tid; i < n2; i += nt) fac[i] = (i == k) ? 0.0 : A[i * ld + k];
        __syncthreads();
        // thread: column j, rows r0, r0 + R, ...; the pivot row's entry stays
        // in a register, a warp covers consecutive columns of one row
        for (int c0 = tid; c0 < R * n2; c0 += nt) {
            const int j = c0 % n2, r0 = c0 / n2;
            const double pk = A[k * ld + j];
            const bool jk = (j == k);
#pragma unroll 8
            for (int i = r0; i < n2; i += R) {
                if (i == k) continue;
                const double base = jk ? 0.0 : A[i * ld + j];
                A[i * ld + j] = fma(-fac[i], pk, base);
            }
        }
        __syncthreads();
    }
    for (int k = n2 - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k) {
            for (int i = tid; i < n2; i += nt) {
                const double tmp = A[i * ld + k];
                A[i * ld + k] = A[i * ld + p];
                A[i * ld + p] = tmp;
            }
        }
        __syncthreads();
    }
    return bad;
}

__global__ void __launch_bounds__(512) k_build_invert(int M, const int* __restrict__ mat,
                                                      const double* __restrict__ tau,
                                                      const double* __restrict__ xi,
                                                      const double* __restrict__ L,
                                                      const int* __restrict__ rowdir,
                                                      double* __restrict__ Dt,
                                                      int* __restrict__ singular) {
    extern __shared__ double smd[];
    const int n2 = 2 * M, M2 = M / 2, ld = n2 + 1;
    double* A = smd;                     // [n2][ld]
    double* fac = A + n2 * ld;           // [n2]
    double* half = fac + n2;             // [n2]
    int* perm = reinterpret_cast<int*>(half + n2);   // [n2]
    const int c = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mc = mat[c];
    const double t = tau[c];
    for (int k = tid; k < n2; k += nt) half[k] = exp(-0.5 * t * fabs(xi[(size_t)mc * n2 + k]));
    __syncthreads();
    const double* Lm = L + (size_t)mc * M * n2;
    for (int e = tid; e < n2 * n2; e += nt) {
        const int r = e / n2, k = e - r * n2;
        const int f = r / M2, fk = k / M2;
        const double d = (f == fk) ? 1.0 : ((f == (fk ^ 1)) ? half[k] * half[k] : half[k]);
        A[r * ld + k] = Lm[(size_t)rowdir[r] * n2 + k] * d;
    }
    __syncthreads();
    const bool bad = gauss_jordan_inplace(A, n2, ld, fac, perm);
    double* out = Dt + (size_t)c * n2 * n2;
    for (int e = tid; e < n2 * n2; e += nt) {
        const int j = e / n2, i = e - j * n2;
        out[e] = A[i * ld + j];
    }
    if (bad && tid == 0) atomicExch(singular, 1);
}

// Response matrix of every cell, R_C = T_out,C D_C: row (f, j) of T_out is the
// trace at face f, direction dirs[opp f][j] (leaving C), of every basis
// function -- so R_C maps the cell's incoming face data to its outgoing face
// data.  Computed in FP64 from the FP64 inverse, stored in FP32 as
// Rt[c][i][row] = R_C[row][i].  Its entries are bounded transfer
// coefficients (row sums of |R| near one), so FP32 keeps them accurate where
// D_C itself (entries up to ~1e5 in the diffusive limit) would not.
template <typename TR>
__global__ void __launch_bounds__(256) k_response(int M, const int* __restrict__ mat,
                                                  const double* __restrict__ tau,
                                                  const double* __restrict__ xi,
                                                  const double* __restrict__ L,
                                                  const int* __restrict__ rowdir,
                                                  const double* __restrict__ Dt,
                                                  TR* __restrict__ Rt) {
    extern __shared__ double smd[];
    const int n2 = 2 * M, M2 = M / 2, ld = n2 + 1;
    double* T = smd;                     // [n2][ld] outgoing traces
    double* half = T + n2 * ld;          // [n2]
    const int c = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mc = mat[c];
    const double t = tau[c];
    for (int k = tid; k < n2; k += nt) half[k] = exp(-0.5 * t * fabs(xi[(size_t)mc * n2 + k]));
    __syncthreads();
    const double* Lm = L + (size_t)mc * M * n2;
    for (int e = tid; e < n2 * n2; e += nt) {
        const int r = e / n2, k = e - r * n2;
        const int f = r / M2, fk = k / M2, j = r - f * M2;
        const int m = rowdir[(f ^ 1) * M2 + j];           // a direction leaving through f
        const double d = (f == fk) ? 1.0 : ((f == (fk ^ 1)) ? half[k] * half[k] : half[k]);
        T[r * ld + k] = Lm[(size_t)m * n2 + k] * d;
    }
    __syncthreads();
    const double* D = Dt + (size_t)c * n2 * n2;      // D[k][i] = Dt[i][k]
    TR* out = Rt + (size_t)c * n2 * n2;
    for (int e = tid; e < n2 * n2; e += nt) {
        const int i = e / n2, r = e - i * n2;
        const double* di = D + (size_t)i * n2;
        double acc = 0.0;
        for (int k = 0; k < n2; ++k) acc = fma(T[r * ld + k], __ldg(di + k), acc);
        out[e] = (TR)acc;
    }
}

// Blocks of a cell from tabulated nodes (set-up by interpolation in ln tau):
// for the cells of bin b (all interpolating between the nodes node0 ..
// node0 + 7), D_C = sum_p w_Cp D_p elementwise.  Block (b, y) holds the node
// values of elements 1024 y .. 1024 y + 1023 in registers and writes them for
// every cell of the bin.  bins[b] = (node0, first, end) positions in the cell
// list.  The sums are double-float (df64.h: the node values and the weights
// as float pairs, products by TwoProd, sums by TwoSum) on the FP32 pipe,
// about 2^-46 relative: far below the FP64 inversion's own rounding of the
// nodes, cond(G) 2^-52, and eight times faster than the FP64 pipe.
__global__ void __launch_bounds__(256) k_interp_D(int E, const int4* __restrict__ bins,
                                                  const int* __restrict__ cells, const double* __restrict__ wts,
                                                  const double* __restrict__ Dn, double* __restrict__ Dt) {
    const int4 bn = bins[blockIdx.x];
    const int e0 = (blockIdx.y * 256 + threadIdx.x) * 4;
    if (e0 >= E) return;                       // E = (2M)^2, a multiple of 4
    float dh[8][4], dl[8][4];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const double2* dp = reinterpret_cast<const double2*>(Dn + (size_t)(bn.x + p) * E + e0);
        const double2 d0 = __ldg(dp), d1 = __ldg(dp + 1);
        df::from_double(d0.x, dh[p][0], dl[p][0]);
        df::from_double(d0.y, dh[p][1], dl[p][1]);
        df::from_double(d1.x, dh[p][2], dl[p][2]);
        df::from_double(d1.y, dh[p][3], dl[p][3]);
    }
    for (int pos = bn.y; pos < bn.z; ++pos) {
        const int c = __ldg(cells + pos);
        float wh[8], wl[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) df::from_double(__ldg(wts + (size_t)pos * 8 + p), wh[p], wl[p]);
        double d[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float S = 0.f, C = 0.f;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                float pr, er;
                df::mul(dh[p][q], dl[p][q], wh[p], wl[p], pr, er);
                df::acc(S, C, pr, er);
            }
            d[q] = df::to_double(S, C);
        }
        double2* dd = reinterpret_cast<double2*>(Dt + (size_t)c * E + e0);
        dd[0] = make_double2(d[0], d[1]);
        dd[1] = make_double2(d[2], d[3]);
    }
}

// The per-cell response of tabulated blocks, R_C = sum_p w_Cp R_p (FP64,
// rounded to FP32 once), as k_interp_D.
__global__ void __launch_bounds__(256) k_interp_R(int E, const int4* __restrict__ bins,
                                                  const int* __restrict__ cells, const double* __restrict__ wts,
                                                  const double* __restrict__ Rn, float* __restrict__ Rt) {
    const int4 bn = bins[blockIdx.x];
    const int e0 = (blockIdx.y * 256 + threadIdx.x) * 4;
    if (e0 >= E) return;
    double rn[8][4];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const double2* rp = reinterpret_cast<const double2*>(Rn + (size_t)(bn.x + p) * E + e0);
        const double2 r0 = __ldg(rp), r1 = __ldg(rp + 1);
        rn[p][0] = r0.x; rn[p][1] = r0.y; rn[p][2] = r1.x; rn[p][3] = r1.y;
    }
    for (int pos = bn.y; pos < bn.z; ++pos) {
        const int c = __ldg(cells + pos);
        double w[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) w[p] = __ldg(wts + (size_t)pos * 8 + p);
        double r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            r[q] = w[0] * rn[0][q];
#pragma unroll
            for (int p = 1; p < 8; ++p) r[q] = fma(w[p], rn[p][q], r[q]);
        }
        *reinterpret_cast<float4*>(Rt + (size_t)c * E + e0) =
            make_float4((float)r[0], (float)r[1], (float)r[2], (float)r[3]);
    }
}

// z_C = X_C r_C for per-cell column-major matrices Xt[c][j][i] = X_C[i][j]
// (D or the response R).  Threads per cell G = 2M/4 (four rows each); block =
// 256 threads = 256/G cells; r staged in shared memory; accumulation in the
// matrix's precision.
template <typename TD, typename TIN, typename TOUT>
__device__ void block_apply_run(int M, int N, const TD* __restrict__ Xt, const TIN* __restrict__ r,
                                TOUT* __restrict__ z, int bid, unsigned char* smb) {
    TD* rs = reinterpret_cast<TD*>(smb);
    const int n2 = 2 * M, G = n2 / 4;
    const int cells = blockDim.x / G;
    TD* zs = rs + n2 * cells;
    const int c0 = bid * cells;
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int j = e / cells, cc = e - j * cells;
        const int c = c0 + cc;
        rs[e] = (c < N) ? (TD)r[(size_t)j * N + c] : (TD)0;
    }
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const TD* X = Xt + (size_t)c * n2 * n2 + 4 * g;
        TD a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 8
        for (int j = 0; j < n2; ++j) {
            const TD* p = X + (size_t)j * n2;
            TD d0, d1, d2, d3;
            if (sizeof(TD) == 4) {
                const float4 d = __ldg(reinterpret_cast<const float4*>(p));
                d0 = d.x; d1 = d.y; d2 = d.z; d3 = d.w;
            } else {
                const double2 u = __ldg(reinterpret_cast<const double2*>(p));
                const double2 v = __ldg(reinterpret_cast<const double2*>(p) + 1);
                d0 = u.x; d1 = u.y; d2 = v.x; d3 = v.y;
            }
            const TD rv = rs[j * cells + cc];
            a0 = fma(d0, rv, a0);
            a1 = fma(d1, rv, a1);
            a2 = fma(d2, rv, a2);
            a3 = fma(d3, rv, a3);
        }
        zs[(4 * g + 0) * cells + cc] = a0;
        zs[(4 * g + 1) * cells + cc] = a1;
        zs[(4 * g + 2) * cells + cc] = a2;
        zs[(4 * g + 3) * cells + cc] = a3;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int i = e / cells, c2 = e - i * cells;
        if (c0 + c2 < N) z[(size_t)i * N + c0 + c2] = (TOUT)zs[e];
    }
}

template <typename TD, typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) k_block_apply(int M, int N, const TD* __restrict__ Xt,
                                                     const TIN* __restrict__ r,
                                                     TOUT* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char smb[];
    block_apply_run<TD, TIN, TOUT>(M, N, Xt, r, z, blockIdx.x, smb);
}

// w = v - P o: subtract the outgoing data o of the neighbour across each face
// (o laid out like the rows: row (f, j) of cell C holds the value leaving C
// through f in direction dirs[opp f][j]).  With o = R v this is w = A D v.
template <typename TV, typename TO, typename TW>
__device__ void gather_run(int I, int M, const TV* __restrict__ v, const TO* __restrict__ o, TW* __restrict__ w,
                           int bid, int nb) {
    const int N = I * I, M2 = M / 2;
    const int64_t n = (int64_t)2 * M * N;
    for (int64_t e = (int64_t)bid * blockDim.x + threadIdx.x; e < n; e += (int64_t)nb * blockDim.x) {
        const int row = (int)(e / N);
        const int c = (int)(e - (int64_t)row * N);
        const int f = row / M2, j = row - f * M2;
        const int iy = c / I, ix = c - iy * I;
        int nb = -1;
        if (f == 0 && ix > 0) nb = c - 1;
        if (f == 1 && ix < I - 1) nb = c + 1;
        if (f == 2 && iy > 0) nb = c - I;
        if (f == 3 && iy < I - 1) nb = c + I;
        double val = (double)v[e];
        if (nb >= 0) val -= (double)o[(int64_t)((f ^ 1) * M2 + j) * N + nb];
        w[e] = (TW)val;
    }
}

template <typename TV, typename TO, typename TW>
__global__ void k_gather(int I, int M, const TV* __restrict__ v, const TO* __restrict__ o,
                         TW* __restrict__ w) {
    gather_run<TV, TO, TW>(I, M, v, o, w, blockIdx.x, gridDim.x);
}

// The same into a df64 w (planar hi / lo, df64.h): v is the FP32 vector vh
// (vl null) or the df64 vector (vh, vl); o is FP32.  v - o is formed exactly
// by TwoSum, so w carries v to 48 bits and the FP32 neighbour term exactly.
__device__ void gather_df_run(int I, int M, const float* __restrict__ vh, const float* __restrict__ vl,
                              const float* __restrict__ o, float* __restrict__ w, int bid, int nb) {
    const int N = I * I, M2 = M / 2;
    const int64_t n = (int64_t)2 * M * N;
    for (int64_t e = (int64_t)bid * blockDim.x + threadIdx.x; e < n; e += (int64_t)nb * blockDim.x) {
        const int row = (int)(e / N);
        const int c = (int)(e - (int64_t)row * N);
        const int f = row / M2, j = row - f * M2;
        const int iy = c / I, ix = c - iy * I;
        int nbr = -1;
        if (f == 0 && ix > 0) nbr = c - 1;
        if (f == 1 && ix < I - 1) nbr = c + 1;
        if (f == 2 && iy > 0) nbr = c - I;
        if (f == 3 && iy < I - 1) nbr = c + I;
        const float ov = nbr >= 0 ? o[(int64_t)((f ^ 1) * M2 + j) * N + nbr] : 0.f;
        float s, t, h, l;
        df::two_sum(vh[e], -ov, s, t);
        if (vl) t = __fadd_rn(t, vl[e]);
        df::two_sum(s, t, h, l);
        w[e] = h;
        w[n + e] = l;
    }
}

__global__ void k_gather_df(int I, int M, const float* __restrict__ vh, const float* __restrict__ vl,
                            const float* __restrict__ o, float* __restrict__ w) {
    gather_df_run(I, M, vh, vl, o, w, blockIdx.x, gridDim.x);
}

// q = P u: every row (f, j) of cell C takes the neighbour's row (opp f, j)
// across f (zero on the boundary).  P is its own transpose.
__global__ void k_permute(int I, int M, const float* __restrict__ u, float* __restrict__ q) {
    const int N = I * I, M2 = M / 2;
    const int64_t n = (int64_t)2 * M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / N);
        const int c = (int)(e - (int64_t)row * N);
        const int f = row / M2, j = row - f * M2;
        const int iy = c / I, ix = c - iy * I;
        int nb = -1;
        if (f == 0 && ix > 0) nb = c - 1;
        if (f == 1 && ix < I - 1) nb = c + 1;
        if (f == 2 && iy > 0) nb = c - I;
        if (f == 3 && iy < I - 1) nb = c + I;
        q[e] = nb >= 0 ? u[(int64_t)((f ^ 1) * M2 + j) * N + nb] : 0.f;
    }
}

// w = u - X_C^T q per cell with Xt[c][i][row] = X_C[row][i] (the transposed
// response, used by the gradient of the loss): w_i = u_i - sum_row Xt[i][row] q_row.
__global__ void __launch_bounds__(256) k_response_t(int M, int N, const float* __restrict__ Xt,
                                                    const float* __restrict__ u,
                                                    const float* __restrict__ q,
                                                    float* __restrict__ w) {
    extern __shared__ __align__(16) unsigned char smb[];
    float* qs = reinterpret_cast<float*>(smb);
    const int n2 = 2 * M, G = n2 / 4;
    const int cells = blockDim.x / G;
    float* zs = qs + n2 * cells;
    const int c0 = blockIdx.x * cells;
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int j = e / cells, cc = e - j * cells;
        const int c = c0 + cc;
        qs[e] = (c < N) ? q[(size_t)j * N + c] : 0.f;
    }
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const float* X = Xt + (size_t)c * n2 * n2;
        for (int t = 0; t < 4; ++t) {
            const int i = 4 * g + t;
            const float4* row = reinterpret_cast<const float4*>(X + (size_t)i * n2);
            float acc = 0.f;
            for (int r4 = 0; r4 < G; ++r4) {
                const float4 d = __ldg(row + r4);
                acc = fmaf(d.x, qs[(4 * r4 + 0) * cells + cc], acc);
                acc = fmaf(d.y, qs[(4 * r4 + 1) * cells + cc], acc);
                acc = fmaf(d.z, qs[(4 * r4 + 2) * cells + cc], acc);
                acc = fmaf(d.w, qs[(4 * r4 + 3) * cells + cc], acc);
            }
            zs[i * cells + cc] = acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int i = e / cells, c2 = e - i * cells;
        if (c0 + c2 < N) {
            const size_t idx = (size_t)i * N + c0 + c2;
            w[idx] = u[idx] - zs[e];
        }
    }
}

// z_C = D_C^T r_C: output j = row j of Dt dotted with r (FP64 accumulation).
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) k_block_apply_t(int M, int N, const double* __restrict__ Dt,
                                                       const TIN* __restrict__ r,
                                                       TOUT* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char smb[];
    double* rs = reinterpret_cast<double*>(smb);
    const int n2 = 2 * M, G = n2 / 4;
    const int cells = blockDim.x / G;
    double* zs = rs + n2 * cells;
    const int c0 = blockIdx.x * cells;
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int j = e / cells, cc = e - j * cells;
        const int c = c0 + cc;
        rs[e] = (c < N) ? (double)r[(size_t)j * N + c] : 0.0;
    }
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const double* D = Dt + (size_t)c * n2 * n2;
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * g + t;
            const double2* row = reinterpret_cast<const double2*>(D + (size_t)j * n2);
            double acc = 0.0;
            for (int i2 = 0; i2 < n2 / 2; ++i2) {
                const double2 d = __ldg(row + i2);
                acc = fma(d.x, rs[(2 * i2 + 0) * cells + cc], acc);
                acc = fma(d.y, rs[(2 * i2 + 1) * cells + cc], acc);
            }
            zs[j * cells + cc] = acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int i = e / cells, c2 = e - i * cells;
        if (c0 + c2 < N) z[(size_t)i * N + c0 + c2] = (TOUT)zs[e];
    }
}

}  // namespace

void launch_build_invert(rte_ctx* ctx, int* singular_dev) {
    const int M = ctx->M, n2 = 2 * M;
    const size_t smem = sizeof(double) * ((size_t)n2 * (n2 + 1) + 3 * n2);
    raise_smem_limit((const void*)k_build_invert, (size_t)(smem));
    // one CTA per SM fits (the block is 2M x (2M+1) doubles): 16 warps hide
    // the shared-memory and FP64 latencies of the elimination
    const int threads_inv = n2 >= 128 ? 512 : (n2 >= 64 ? 256 : 128);
    const int threads = n2 >= 64 ? 256 : 128;
    {
        ProfScope ps(ctx, K_INVERT, (double)ctx->N * n2 * n2 * 8);
        k_build_invert<<<ctx->N, threads_inv, smem, ctx->stream>>>(M, ctx->mat, ctx->tau, ctx->xi,
                                                               ctx->L64, ctx->rowdir, ctx->Dt,
                                                               singular_dev);
        check(cudaGetLastError(), "k_build_invert");
    }
    const size_t smem2 = sizeof(double) * ((size_t)n2 * (n2 + 1) + n2);
    raise_smem_limit((const void*)k_response<float>, (size_t)(smem2));
    ProfScope ps(ctx, K_RESPONSE, (double)ctx->N * n2 * n2 * 12);
    k_response<float><<<ctx->N, threads, smem2, ctx->stream>>>(M, ctx->mat, ctx->tau, ctx->xi, ctx->L64,
                                                               ctx->rowdir, ctx->Dt, ctx->Rt);
    check(cudaGetLastError(), "k_response");
}

void launch_tabulated_blocks(rte_ctx* ctx, const TabPlan& plan, int* singular_dev) {
    const int M = ctx->M, n2 = 2 * M, E = n2 * n2;
    const int J = (int)plan.node_tau.size();
    const cudaStream_t st = ctx->stream;
    // temporary tables: node materials and tau, the nodes' D (FP64); kept in
    // the context for the per-cell R on demand: the nodes' R (FP64), the cell
    // list, the weights and the bins
    std::vector<void*> tmp;
    auto alloc = [&](size_t bytes) {
        void* p = nullptr;
        check(cudaMallocAsync(&p, bytes, st), "cudaMallocAsync (tabulated blocks)");
        tmp.push_back(p);
        return p;
    };
    auto up = [&](void* dst, const void* src, size_t bytes) {
        check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "h2d (tabulated blocks)");
    };
    try {
        int* nmat = static_cast<int*>(alloc(J * sizeof(int)));
        double* ntau = static_cast<double*>(alloc(J * sizeof(double)));
        double* Dn = static_cast<double*>(alloc((size_t)J * E * sizeof(double)));
        double* Rn = static_cast<double*>(dev_alloc(ctx, (size_t)J * E * sizeof(double)));
        int* cells = static_cast<int*>(dev_alloc(ctx, plan.cells.size() * sizeof(int)));
        double* wts = static_cast<double*>(dev_alloc(ctx, plan.weights.size() * sizeof(double)));
        int4* bins = static_cast<int4*>(dev_alloc(ctx, plan.bins.size() * sizeof(int4)));
        ctx->tab_Rn = Rn;
        ctx->tab_cells = cells;
        ctx->tab_wts = wts;
        ctx->tab_bins = bins;
        ctx->tab_nbins = (int)plan.bins.size();
        ctx->rt_ready = false;
        up(nmat, plan.node_mat.data(), J * sizeof(int));
        up(ntau, plan.node_tau.data(), J * sizeof(double));
        up(cells, plan.cells.data(), plan.cells.size() * sizeof(int));
        up(wts, plan.weights.data(), plan.weights.size() * sizeof(double));
        up(bins, plan.bins.data(), plan.bins.size() * sizeof(int4));
        const size_t smem = sizeof(double) * ((size_t)n2 * (n2 + 1) + 3 * n2);
        raise_smem_limit((const void*)k_build_invert, smem);
        const int threads_inv = n2 >= 128 ? 512 : (n2 >= 64 ? 256 : 128);
        const int threads = n2 >= 64 ? 256 : 128;
        {
            ProfScope ps(ctx, K_INVERT, (double)J * E * 8);
            k_build_invert<<<J, threads_inv, smem, st>>>(M, nmat, ntau, ctx->xi, ctx->L64, ctx->rowdir, Dn,
                                                         singular_dev);
            check(cudaGetLastError(), "k_build_invert (nodes)");
        }
        {
            const size_t smem2 = sizeof(double) * ((size_t)n2 * (n2 + 1) + n2);
            raise_smem_limit((const void*)k_response<double>, smem2);
            ProfScope ps(ctx, K_RESPONSE, (double)J * E * 16);
            k_response<double><<<J, threads, smem2, st>>>(M, nmat, ntau, ctx->xi, ctx->L64, ctx->rowdir, Dn, Rn);
            check(cudaGetLastError(), "k_response (nodes)");
        }
        build_response_tc(ctx, plan, Rn);
        {
            ProfScope ps(ctx, K_RESPONSE, (double)ctx->N * E * 8);
            const dim3 grid((unsigned)plan.bins.size(), (unsigned)((E / 4 + 255) / 256));
            k_interp_D<<<grid, 256, 0, st>>>(E, bins, cells, wts, Dn, ctx->Dt);
            check(cudaGetLastError(), "k_interp_D");
        }
    } catch (...) {
        for (void* p : tmp) cudaFreeAsync(p, st);
        throw;
    }
    for (void* p : tmp) cudaFreeAsync(p, st);
}

void ensure_cell_response(rte_ctx* ctx) {
    if (ctx->rt_ready) return;
    if (!ctx->tab_Rn) throw StatusError{RTE_EINVAL, "per-cell response: no blocks"};
    const int n2 = 2 * ctx->M, E = n2 * n2;
    float* Rt = static_cast<float*>(dev_alloc(ctx, (size_t)ctx->N * E * sizeof(float)));
    {
        ProfScope ps(ctx, K_RESPONSE, (double)ctx->N * E * 4);
        const dim3 grid((unsigned)ctx->tab_nbins, (unsigned)((E / 4 + 255) / 256));
        k_interp_R<<<grid, 256, 0, ctx->stream>>>(E, ctx->tab_bins, ctx->tab_cells, ctx->tab_wts, ctx->tab_Rn, Rt);
        check(cudaGetLastError(), "k_interp_R");
    }
    ctx->Rt = Rt;
    ctx->rt_ready = true;
}

namespace {
template <typename TD, typename TIN, typename TOUT>
void block_apply_t(rte_ctx* ctx, const TD* X, const void* r, void* z, int kid, double bytes) {
    const int M = ctx->M, n2 = 2 * M, G = n2 / 4;
    const int threads = G >= 256 ? G : (256 / G) * G;
    const int cells = threads / G;
    const int blocks = (ctx->N + cells - 1) / cells;
    const size_t smem = sizeof(TD) * 2 * n2 * cells;
    auto kern = k_block_apply<TD, TIN, TOUT>;
    raise_smem_limit((const void*)kern, (size_t)(smem));
    ProfScope ps(ctx, kid, bytes);
    kern<<<blocks, threads, smem, ctx->stream>>>(M, ctx->N, X, (const TIN*)r, (TOUT*)z);
    check(cudaGetLastError(), "k_block_apply");
}
}  // namespace

void launch_block_apply(rte_ctx* ctx, bool transpose, const void* r, bool r_is_double, void* z,
                        bool z_is_double) {
    const int M = ctx->M, n2 = 2 * M, G = n2 / 4;
    const double bytes = (double)ctx->N * n2 * n2 * 8 +
                         (double)ctx->n * ((r_is_double ? 8 : 4) + (z_is_double ? 8 : 4));
    if (!transpose) {
        if (r_is_double && z_is_double)
            block_apply_t<double, double, double>(ctx, ctx->Dt, r, z, K_BLOCK, bytes);
        else if (r_is_double)
            block_apply_t<double, double, float>(ctx, ctx->Dt, r, z, K_BLOCK, bytes);
        else if (z_is_double)
            block_apply_t<double, float, double>(ctx, ctx->Dt, r, z, K_BLOCK, bytes);
        else
            block_apply_t<double, float, float>(ctx, ctx->Dt, r, z, K_BLOCK, bytes);
        return;
    }
    const int threads = G >= 256 ? G : (256 / G) * G;
    const int cells = threads / G;
    const int blocks = (ctx->N + cells - 1) / cells;
    const size_t smem = sizeof(double) * 2 * n2 * cells;
    ProfScope ps(ctx, K_BLOCK_T, bytes);
    if (r_is_double && z_is_double) {
        raise_smem_limit((const void*)k_block_apply_t<double, double>, smem);
        k_block_apply_t<double, double><<<blocks, threads, smem, ctx->stream>>>(
            M, ctx->N, ctx->Dt, (const double*)r, (double*)z);
    } else if (!r_is_double && !z_is_double) {
        raise_smem_limit((const void*)k_block_apply_t<float, float>, smem);
        k_block_apply_t<float, float><<<blocks, threads, smem, ctx->stream>>>(
            M, ctx->N, ctx->Dt, (const float*)r, (float*)z);
    } else {
        throw StatusError{RTE_EINVAL, "transposed block apply needs matching precisions"};
    }
    check(cudaGetLastError(), "k_block_apply_t");
}

void launch_response_apply_t(rte_ctx* ctx, const float* u, float* w, float* scratch) {
    ensure_cell_response(ctx);
    const int M = ctx->M, n2 = 2 * M, G = n2 / 4;
    int64_t want = (ctx->n + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
    const int g = (int)(want < cap ? want : cap);
    {
        ProfScope ps(ctx, K_GATHER, (double)ctx->n * 8);
        k_permute<<<g, 256, 0, ctx->stream>>>(ctx->I, M, u, scratch);
        check(cudaGetLastError(), "k_permute");
    }
    const int threads = G >= 256 ? G : (256 / G) * G;
    const int cells = threads / G;
    const int blocks = (ctx->N + cells - 1) / cells;
    const size_t smem = sizeof(float) * 2 * n2 * cells;
    raise_smem_limit((const void*)k_response_t, (size_t)(smem));
    ProfScope ps(ctx, K_RESPONSE_APPLY, (double)ctx->N * n2 * n2 * 4 + (double)ctx->n * 12);
    k_response_t<<<blocks, threads, smem, ctx->stream>>>(M, ctx->N, ctx->Rt, u, scratch, w);
    check(cudaGetLastError(), "k_response_t");
}

namespace {

__global__ void __launch_bounds__(256) k_block_apply_group(const GroupItem* __restrict__ items, int count) {
    extern __shared__ __align__(16) unsigned char smb[];
    const GroupItem& it = items[group_item_of<&GroupItem::b_ba>(items, count)];
    const int bid = blockIdx.x - it.b_ba;
    block_apply_run<float, float, float>(it.M, it.N, it.Rt, it.z, it.o, bid, smb);
}

__global__ void k_gather_group(const GroupItem* __restrict__ items, int count) {
    const GroupItem& it = items[group_item_of<&GroupItem::b_ga>(items, count)];
    const int bid = blockIdx.x - it.b_ga;
    gather_df_run(it.I, it.M, it.z, it.z_lo, it.o, it.w, bid, it.n_ga);
}
}  // namespace

// the block counts a lone response apply of this context uses (block_apply_t
// and launch_response_apply), so a grouped launch reproduces its arithmetic
void group_response_geometry(rte_ctx* ctx, int* n_ba, int* n_ga, size_t* smem_ba) {
    const int M = ctx->M, n2 = 2 * M, G = n2 / 4;
    const int threads = G >= 256 ? G : (256 / G) * G;
    if (threads != 256 && G < 256) {
        // grouped blocks have 256 threads: the cells per block must be the same
        if (256 / G != threads / G) throw StatusError{RTE_EINVAL, "grouped response apply: unsupported M"};
    }
    const int cells = threads / G;
    *n_ba = (ctx->N + cells - 1) / cells;
    *smem_ba = sizeof(float) * 2 * n2 * cells;
    int64_t want = (ctx->n + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
    *n_ga = (int)(want < cap ? want : cap);
}

void launch_group_response(const GroupItem* items_dev, int count, int blocks_ba, int blocks_ga, size_t smem_ba,
                           cudaStream_t st) {
    if (blocks_ba > 0) {
        raise_smem_limit((const void*)k_block_apply_group, (size_t)(smem_ba));
        k_block_apply_group<<<blocks_ba, 256, smem_ba, st>>>(items_dev, count);
    }
    if (blocks_ga > 0) k_gather_group<<<blocks_ga, 256, 0, st>>>(items_dev, count);
    check(cudaGetLastError(), "grouped response apply");
}

void launch_response_apply(rte_ctx* ctx, const void* v, bool v_is_double, void* w,
                           bool w_is_double) {
    const int M = ctx->M, n2 = 2 * M;
    float* o = reinterpret_cast<float*>(ctx->trace_out);
    const double bytes = (double)ctx->N * n2 * n2 * 4 + (double)ctx->n * ((v_is_double ? 8 : 4) + 4);
    if (response_tc_active(ctx)) {
        launch_response_tc(ctx, v, v_is_double);
        launch_gather_tiles(ctx, v, v_is_double, w, w_is_double);
        return;
    }
    ensure_cell_response(ctx);
    if (v_is_double)
        block_apply_t<float, double, float>(ctx, ctx->Rt, v, o, K_RESPONSE_APPLY, bytes);
    else
        block_apply_t<float, float, float>(ctx, ctx->Rt, v, o, K_RESPONSE_APPLY, bytes);
    int64_t want = (ctx->n + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
    const int g = (int)(want < cap ? want : cap);
    ProfScope ps(ctx, K_GATHER, (double)ctx->n * ((v_is_double ? 8 : 4) + (w_is_double ? 8 : 4)));
    if (v_is_double && w_is_double)
        k_gather<double, float, double><<<g, 256, 0, ctx->stream>>>(ctx->I, M, (const double*)v, o,
                                                                    (double*)w);
    else if (!v_is_double && !w_is_double)
        k_gather<float, float, float><<<g, 256, 0, ctx->stream>>>(ctx->I, M, (const float*)v, o,
                                                                  (float*)w);
    else if (!v_is_double && w_is_double)
        k_gather<float, float, double><<<g, 256, 0, ctx->stream>>>(ctx->I, M, (const float*)v, o,
                                                                   (double*)w);
    else
        k_gather<double, float, float><<<g, 256, 0, ctx->stream>>>(ctx->I, M, (const double*)v, o,
                                                                   (float*)w);
    check(cudaGetLastError(), "k_gather");
}

void launch_response_apply_df(rte_ctx* ctx, const float* z_hi, const float* z_lo, float* w) {
    const int M = ctx->M, n2 = 2 * M;
    float* o = reinterpret_cast<float*>(ctx->trace_out);
    const double bytes = (double)ctx->N * n2 * n2 * 4 + (double)ctx->n * 8;
    if (response_tc_active(ctx)) {
        launch_response_tc(ctx, z_hi, false);
        launch_gather_tiles_df(ctx, z_hi, z_lo, w);
        return;
    }
    ensure_cell_response(ctx);
    block_apply_t<float, float, float>(ctx, ctx->Rt, z_hi, o, K_RESPONSE_APPLY, bytes);
    int64_t want = (ctx->n + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
    const int g = (int)(want < cap ? want : cap);
    ProfScope ps(ctx, K_GATHER, (double)ctx->n * ((z_lo ? 8 : 4) + 4 + 8));
    k_gather_df<<<g, 256, 0, ctx->stream>>>(ctx->I, M, z_hi, z_lo, o, w);
    check(cudaGetLastError(), "k_gather_df");
}

}  // namespace rte
