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
// values of elements 1024 y .. 1024 y + 1023 in registers (df64, converted
// once) and writes them for every cell of the bin.  bins[b] = (node0, first,
// end) positions in the cell list; w16[pos] the position's weights as float
// pairs (8 hi, 8 lo).  The sums are double-float on the FP32 pipe, two
// elements a packed instruction (df64.h: TwoProd, TwoSum), about 2^-46
// relative: far below the FP64 inversion's own rounding of the nodes,
// cond(G) 2^-52.  The result stays df64 (hi and lo planes of the cell), so
// no FP64 instruction runs per element: on this GPU the FP64 pipe (and the
// conversions to and from double) is some 30 times narrower than FP32.
__global__ void __launch_bounds__(256) k_interp_D(int E, const int4* __restrict__ bins,
                                                  const int* __restrict__ cells, const float* __restrict__ w16,
                                                  const double* __restrict__ Dn, float* __restrict__ Dt) {
    using df::f2;
    const int4 bn = bins[blockIdx.x];
    const int e0 = (blockIdx.y * 256 + threadIdx.x) * 4;
    if (e0 >= E) return;                       // E = (2M)^2, a multiple of 4
    f2 ah[8][2], al[8][2];                     // node p, element pairs (e0, e0 + 1), (e0 + 2, e0 + 3)
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const double2* dp = reinterpret_cast<const double2*>(Dn + (size_t)(bn.x + p) * E + e0);
        const double2 d0 = __ldg(dp), d1 = __ldg(dp + 1);
        float h[4], l[4];
        df::from_double(d0.x, h[0], l[0]);
        df::from_double(d0.y, h[1], l[1]);
        df::from_double(d1.x, h[2], l[2]);
        df::from_double(d1.y, h[3], l[3]);
        ah[p][0] = df::pk(h[0], h[1]);
        al[p][0] = df::pk(l[0], l[1]);
        ah[p][1] = df::pk(h[2], h[3]);
        al[p][1] = df::pk(l[2], l[3]);
    }
    for (int pos = bn.y; pos < bn.z; ++pos) {
        const int c = __ldg(cells + pos);
        const float4* wp = reinterpret_cast<const float4*>(w16 + (size_t)pos * 16);
        const float4 h0 = __ldg(wp), h1 = __ldg(wp + 1), l0 = __ldg(wp + 2), l1 = __ldg(wp + 3);
        const float wh[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        const float wl[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
        f2 S[2] = {0ull, 0ull}, C[2] = {0ull, 0ull};
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const f2 bh = df::pk(wh[p], wh[p]), nbh = df::pk(-wh[p], -wh[p]), nbl = df::pk(-wl[p], -wl[p]);
            df::mac2(S[0], C[0], ah[p][0], al[p][0], nbh, nbl, bh);
            df::mac2(S[1], C[1], ah[p][1], al[p][1], nbh, nbl, bh);
        }
        df::renorm2(S[0], C[0]);
        df::renorm2(S[1], C[1]);
        float o[8];
        df::upk(S[0], o[0], o[1]);
        df::upk(S[1], o[2], o[3]);
        df::upk(C[0], o[4], o[5]);
        df::upk(C[1], o[6], o[7]);
        float* out = Dt + (size_t)c * 2 * E + e0;
        *reinterpret_cast<float4*>(out) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4*>(out + E) = make_float4(o[4], o[5], o[6], o[7]);
    }
}

// FP64 blocks [cells][E] (per-cell inversion) into the df64 planes of the
// same cells of Dt
__global__ void k_blocks_to_df(int64_t total, int E, const double* __restrict__ Dx, float* __restrict__ Dt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / E, i = e - c * E;
        float h, l;
        df::from_double(Dx[e], h, l);
        Dt[c * 2 * E + i] = h;
        Dt[c * 2 * E + E + i] = l;
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

// r (FP32 or FP64) of the block's cells into shared memory as df64 planes
// [2M][cells]
template <typename TIN>
__device__ __forceinline__ void stage_df(int n2, int N, int c0, int cells, const TIN* __restrict__ r, float* rh,
                                         float* rl) {
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int j = e / cells, cc = e - j * cells;
        const int c = c0 + cc;
        float h = 0.f, l = 0.f;
        if (c < N) {
            if (sizeof(TIN) == 8)
                df::from_double((double)r[(size_t)j * N + c], h, l);
            else
                h = (float)r[(size_t)j * N + c];
        }
        rh[e] = h;
        rl[e] = l;
    }
}

// z_C = D_C r_C with D_C as df64 planes (Dt[c][0][j][i] + Dt[c][1][j][i] =
// D_C[i][j]).  G = 2M/4 threads a cell, four consecutive rows i each, two per
// packed df64 accumulator; r staged in shared memory as df64.  The sums are
// df64 (TwoProd and TwoSum on the FP32 pipe, renormalised every 8 terms), as
// accurate as an FP64 sum of the 2M terms, and the kernel is bound by HBM,
// not by the FP64 pipe.
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) k_block_apply_df(int M, int N, const float* __restrict__ Dt,
                                                        const TIN* __restrict__ r, TOUT* __restrict__ z) {
    using df::f2;
    extern __shared__ __align__(16) unsigned char smb[];
    const int n2 = 2 * M, G = n2 / 4, E = n2 * n2;
    const int cells = blockDim.x / G;
    float* rh = reinterpret_cast<float*>(smb);
    float* rl = rh + n2 * cells;
    double* zs = reinterpret_cast<double*>(rl + n2 * cells);
    const int c0 = blockIdx.x * cells;
    stage_df<TIN>(n2, N, c0, cells, r, rh, rl);
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const float* Xh = Dt + (size_t)c * 2 * E + 4 * g;
        const float* Xl = Xh + E;
        f2 S0 = 0ull, C0 = 0ull, S1 = 0ull, C1 = 0ull;
        for (int j0 = 0; j0 < n2; j0 += 8) {
#pragma unroll
            for (int j = j0; j < j0 + 8; ++j) {
                const float4 dh = __ldg(reinterpret_cast<const float4*>(Xh + (size_t)j * n2));
                const float4 dl = __ldg(reinterpret_cast<const float4*>(Xl + (size_t)j * n2));
                const float vh = rh[j * cells + cc], vl = rl[j * cells + cc];
                const f2 bh = df::pk(vh, vh), nbh = df::pk(-vh, -vh), nbl = df::pk(-vl, -vl);
                df::mac2(S0, C0, df::pk(dh.x, dh.y), df::pk(dl.x, dl.y), nbh, nbl, bh);
                df::mac2(S1, C1, df::pk(dh.z, dh.w), df::pk(dl.z, dl.w), nbh, nbl, bh);
            }
            df::renorm2(S0, C0);
            df::renorm2(S1, C1);
        }
        float s[4], t[4];
        df::upk(S0, s[0], s[1]);
        df::upk(S1, s[2], s[3]);
        df::upk(C0, t[0], t[1]);
        df::upk(C1, t[2], t[3]);
#pragma unroll
        for (int q = 0; q < 4; ++q) zs[(4 * g + q) * cells + cc] = df::to_double(s[q], t[q]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * cells; e += blockDim.x) {
        const int i = e / cells, c2 = e - i * cells;
        if (c0 + c2 < N) z[(size_t)i * N + c0 + c2] = (TOUT)zs[e];
    }
}

// z_C = D_C^T r_C: output j = row j of the planes dotted with r (df64 sums,
// even and odd i in the two halves of a packed accumulator).
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) k_block_apply_t(int M, int N, const float* __restrict__ Dt,
                                                       const TIN* __restrict__ r, TOUT* __restrict__ z) {
    using df::f2;
    extern __shared__ __align__(16) unsigned char smb[];
    const int n2 = 2 * M, G = n2 / 4, E = n2 * n2;
    const int cells = blockDim.x / G;
    float* rh = reinterpret_cast<float*>(smb);
    float* rl = rh + n2 * cells;
    double* zs = reinterpret_cast<double*>(rl + n2 * cells);
    const int c0 = blockIdx.x * cells;
    stage_df<TIN>(n2, N, c0, cells, r, rh, rl);
    __syncthreads();
    const int cc = threadIdx.x / G, g = threadIdx.x - cc * G;
    const int c = c0 + cc;
    if (cc < cells && c < N) {
        const float* Xh = Dt + (size_t)c * 2 * E;
        for (int t = 0; t < 4; ++t) {
            const int j = 4 * g + t;
            const float2* rowh = reinterpret_cast<const float2*>(Xh + (size_t)j * n2);
            const float2* rowl = reinterpret_cast<const float2*>(Xh + E + (size_t)j * n2);
            f2 S = 0ull, C = 0ull;
            for (int i0 = 0; i0 < n2 / 2; i0 += 8) {
                for (int i2 = i0; i2 < i0 + 8 && i2 < n2 / 2; ++i2) {
                    const float2 dh = __ldg(rowh + i2), dl = __ldg(rowl + i2);
                    const float xh = rh[(2 * i2) * cells + cc], yh = rh[(2 * i2 + 1) * cells + cc];
                    const float xl = rl[(2 * i2) * cells + cc], yl = rl[(2 * i2 + 1) * cells + cc];
                    df::mac2(S, C, df::pk(dh.x, dh.y), df::pk(dl.x, dl.y), df::pk(-xh, -yh), df::pk(-xl, -yl),
                             df::pk(xh, yh));
                }
                df::renorm2(S, C);
            }
            float sx, sy, cx, cy, h, l;
            df::upk(S, sx, sy);
            df::upk(C, cx, cy);
            df::two_sum(sx, sy, h, l);
            l = __fadd_rn(l, __fadd_rn(cx, cy));
            zs[j * cells + cc] = df::to_double(h, l);
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
    const int M = ctx->M, n2 = 2 * M, E = n2 * n2, N = ctx->N;
    const size_t smem = sizeof(double) * ((size_t)n2 * (n2 + 1) + 3 * n2);
    raise_smem_limit((const void*)k_build_invert, (size_t)(smem));
    const size_t smem2 = sizeof(double) * ((size_t)n2 * (n2 + 1) + n2);
    raise_smem_limit((const void*)k_response<float>, (size_t)(smem2));
    // one CTA per SM fits (the block is 2M x (2M+1) doubles): 16 warps hide
    // the shared-memory and FP64 latencies of the elimination
    const int threads_inv = n2 >= 128 ? 512 : (n2 >= 64 ? 256 : 128);
    const int threads = n2 >= 64 ? 256 : 128;
    // batches of cells: the FP64 inverses of a batch feed the response
    // matrices, then are stored as df64 planes
    const int batch = N < 16384 ? N : 16384;
    double* Dx = nullptr;
    check(pool_malloc(reinterpret_cast<void**>(&Dx), (size_t)batch * E * sizeof(double), ctx->stream),
          "cudaMallocFromPoolAsync (inverses)");
    try {
        for (int c0 = 0; c0 < N; c0 += batch) {
            const int nc = N - c0 < batch ? N - c0 : batch;
            {
                ProfScope ps(ctx, K_INVERT, (double)nc * E * 8);
                k_build_invert<<<nc, threads_inv, smem, ctx->stream>>>(M, ctx->mat + c0, ctx->tau + c0, ctx->xi,
                                                                       ctx->L64, ctx->rowdir, Dx, singular_dev);
                check(cudaGetLastError(), "k_build_invert");
            }
            {
                ProfScope ps(ctx, K_RESPONSE, (double)nc * E * 12);
                k_response<float><<<nc, threads, smem2, ctx->stream>>>(M, ctx->mat + c0, ctx->tau + c0, ctx->xi,
                                                                       ctx->L64, ctx->rowdir, Dx,
                                                                       ctx->Rt + (size_t)c0 * E);
                check(cudaGetLastError(), "k_response");
            }
            const int64_t total = (int64_t)nc * E;
            const int g = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 16);
            k_blocks_to_df<<<g, 256, 0, ctx->stream>>>(total, E, Dx, ctx->Dt + (size_t)c0 * 2 * E);
            check(cudaGetLastError(), "k_blocks_to_df");
        }
    } catch (...) {
        cudaFreeAsync(Dx, ctx->stream);
        throw;
    }
    check(cudaFreeAsync(Dx, ctx->stream), "cudaFreeAsync (inverses)");
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
        check(pool_malloc(&p, bytes, st), "cudaMallocFromPoolAsync (tabulated blocks)");
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
        float* w16 = static_cast<float*>(dev_alloc(ctx, plan.weights.size() * 2 * sizeof(float)));
        int4* bins = static_cast<int4*>(dev_alloc(ctx, plan.bins.size() * sizeof(int4)));
        ctx->tab_Rn = Rn;
        ctx->tab_cells = cells;
        ctx->tab_wts = wts;
        ctx->tab_w16 = w16;
        ctx->tab_bins = bins;
        ctx->tab_nbins = (int)plan.bins.size();
        ctx->rt_ready = false;
        up(nmat, plan.node_mat.data(), J * sizeof(int));
        up(ntau, plan.node_tau.data(), J * sizeof(double));
        up(cells, plan.cells.data(), plan.cells.size() * sizeof(int));
        up(wts, plan.weights.data(), plan.weights.size() * sizeof(double));
        // the weights as float pairs (8 hi, then 8 lo a position)
        std::vector<float> w16h(plan.weights.size() * 2);
        for (size_t pos = 0; pos < plan.weights.size() / 8; ++pos)
            for (int p = 0; p < 8; ++p) {
                const double w = plan.weights[pos * 8 + p];
                const float hi = (float)w;
                w16h[pos * 16 + p] = hi;
                w16h[pos * 16 + 8 + p] = (float)(w - (double)hi);
            }
        up(w16, w16h.data(), w16h.size() * sizeof(float));
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
            k_interp_D<<<grid, 256, 0, st>>>(E, bins, cells, w16, Dn, ctx->Dt);
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
    const int threads = G >= 256 ? G : (256 / G) * G;
    const int cells = threads / G;
    const int blocks = (ctx->N + cells - 1) / cells;
    // r as df64 planes and z in FP64
    const size_t smem = (2 * sizeof(float) + sizeof(double)) * n2 * cells;
    auto run = [&](auto kern, auto rp, auto zp) {
        raise_smem_limit((const void*)kern, smem);
        kern<<<blocks, threads, smem, ctx->stream>>>(M, ctx->N, ctx->Dt, rp, zp);
    };
    {
        ProfScope ps(ctx, transpose ? K_BLOCK_T : K_BLOCK, bytes);
        const double* rd = static_cast<const double*>(r);
        const float* rf = static_cast<const float*>(r);
        double* zd = static_cast<double*>(z);
        float* zf = static_cast<float*>(z);
        if (!transpose) {
            if (r_is_double && z_is_double) run(k_block_apply_df<double, double>, rd, zd);
            else if (r_is_double) run(k_block_apply_df<double, float>, rd, zf);
            else if (z_is_double) run(k_block_apply_df<float, double>, rf, zd);
            else run(k_block_apply_df<float, float>, rf, zf);
        } else {
            if (r_is_double && z_is_double) run(k_block_apply_t<double, double>, rd, zd);
            else if (!r_is_double && !z_is_double) run(k_block_apply_t<float, float>, rf, zf);
            else throw StatusError{RTE_EINVAL, "transposed block apply needs matching precisions"};
        }
    }
    check(cudaGetLastError(), transpose ? "k_block_apply_t" : "k_block_apply_df");
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
