// ATFPS filter of the physics-informed loss (Sec. 2.3, Eqs. def_V_delta,
// 2DAdaptiveTFPS_continuity_cond / boundary_cond and loss_delta) on the device.
//
// Selection: basis function k of cell c is kept iff exp(-|xi_k| tau_c / 2) >
// delta (the lambda of Eq. def_V_delta read as xi).
//
// Interfaces, in this order: interior vertical faces (row-major over (iy, ix),
// C- left, C+ right), interior horizontal faces (C- below, C+ above), then per
// row iy the west and east boundary faces, then per column ix the south and
// north boundary faces.  For an interface the functions centred there (C- then
// C+, each group in ascending |xi|) are split into kept and dropped; the kept
// columns are orthonormalised (classical Gram-Schmidt applied twice, which
// gives the Q of a QR with positive R diagonal), the dropped columns follow,
// every column is scaled to max-norm one, and the first s rows of E^{-1}
// (s kept) are the interface's projections.  On a boundary face only the
// incoming direction components enter (M/2 rows).
//
// F maps a vector y indexed like the rows of A ([2M][N]) to the kept
// coordinates of every interface: on an interior interface the midpoint jump
// over all M directions is read off the rows -- the rows of C- entering
// through the shared face carry +jump, those of C+ carry -jump.  Every row of
// A belongs to exactly one interface, so F^T writes each row once.
//
// One CTA per interface builds E and its inverse (Gauss-Jordan with partial
// pivoting, FP64, in shared memory); the projections are stored as [m][k]
// (k fastest) so that F y reads them coalesced.
#include <cmath>
#include <algorithm>

#include "rte_internal.h"

namespace rte {

struct Atfps {
    double delta = 0.0;
    int nif = 0;                    // interfaces (every face of the grid)
    int64_t rows = 0;               // kept coordinates over all interfaces
    int64_t ndrop = 0;              // dropped functions over all interfaces
    size_t bytes = 0;
    std::vector<void*> allocs;
    unsigned char* mask = nullptr;  // [2M][N], 1 = kept
    int* desc = nullptr;            // [nif][8]: C-, C+ (-1 on a boundary), face of C-, face of C+, s, rows of E, r0, d0
    long long* off = nullptr;       // [nif] offset of the interface's kept projections
    double* proj = nullptr;         // kept projections, [m][k] per interface
    double* ekeep = nullptr;        // kept columns of E (unit max-norm), [m][k] per interface
    long long* loff = nullptr;      // [nif] offset of the interface's dropped projections
    double* lproj = nullptr;        // dropped projections, [m][d] per interface
    long long* kcol = nullptr;      // [rows] slot index k N + c of the function behind each kept row
    long long* dcol = nullptr;      // [ndrop] slot index of each dropped function
    double* dsc = nullptr;          // [ndrop] -1 / scale (C- or boundary cell) or +1 / scale (C+)
    int* singular = nullptr;        // set when an interface basis is numerically singular
    std::vector<unsigned char> mask_h;
    // compressed solve (built by the first atfps_solve after the set-up)
    double* bbar = nullptr;         // [2M][N] compressed right-hand side in slot layout (zero at dropped slots)
    double* scratch = nullptr;      // [2M][N] row-space scratch
    double* scratch2 = nullptr;     // [2M][N] row-space scratch
};

namespace {

constexpr int kBuildThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// E and the first s rows of its inverse for interface blockIdx.x.
// ord[(mat * 4 + group) * M2 + q]: slot of the q-th smallest |xi| of the group.
// dirs[f * M2 + j]: direction of incoming row j at face f.
__global__ void __launch_bounds__(kBuildThreads)
    k_atfps_build(const int* __restrict__ desc, const long long* __restrict__ off, const int* __restrict__ ord,
                  const int* __restrict__ dirs, const double* __restrict__ L64, const int* __restrict__ mat,
                  const unsigned char* __restrict__ mask, int M, int N, double pivot_tol,
                  double* __restrict__ proj, double* __restrict__ ekeep, const long long* __restrict__ loff,
                  double* __restrict__ lproj,
                  long long* __restrict__ kcol, long long* __restrict__ dcol, double* __restrict__ dsc,
                  int* __restrict__ singular) {
    extern __shared__ double sm[];
    __shared__ int col_cell[2 * 64], col_slot[2 * 64];
    __shared__ double col_scale[2 * 64];
    __shared__ double red[kBuildThreads / 32];
    __shared__ int s_piv;
    const int* d = desc + 8 * blockIdx.x;
    const int cm = d[0], cp = d[1], fm = d[2], fp = d[3], s = d[4], Mi = d[5], r0 = d[6], d0 = d[7];
    const int M2 = M / 2, n2 = 2 * M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* E = sm;                   // column-major: E[j * Mi + r]
    double* X = sm + Mi * Mi;         // inverse, row-major: X[r * Mi + c]
    double* h = X + Mi * Mi;          // [Mi] projection coefficients

    // columns: kept functions (C- then C+, ascending |xi|), then dropped ones
    if (tid == 0) {
        int nk = 0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int side = 0; side < 2; ++side) {
                const int c = side == 0 ? cm : cp;
                if (c < 0) continue;
                const int grp = side == 0 ? fm : fp;
                const int mt = mat[c];
                for (int q = 0; q < M2; ++q) {
                    const int k = ord[(mt * 4 + grp) * M2 + q];
                    const bool kept = mask[(size_t)k * N + c] != 0;
                    if (kept == (pass == 0)) {
                        col_cell[nk] = c;
                        col_slot[nk] = k;
                        ++nk;
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < Mi * Mi; e += blockDim.x) {
        const int j = e / Mi, r = e - j * Mi;
        const int dir = (cp < 0) ? dirs[fm * M2 + r] : r;
        E[e] = L64[((size_t)mat[col_cell[j]] * M + dir) * n2 + col_slot[j]];
    }
    __syncthreads();
    // orthonormalise the kept columns: for column j, twice h = Q^T e_j, e_j -= Q h
    for (int j = 0; j < s; ++j) {
        double* ej = E + j * Mi;
        for (int pass = 0; pass < 2; ++pass) {
            for (int p = warp; p < j; p += blockDim.x / 32) {
                double t = 0.0;
                for (int r = lane; r < Mi; r += 32) t = fma(E[p * Mi + r], ej[r], t);
                t = warp_sum(t);
                if (lane == 0) h[p] = t;
            }
            __syncthreads();
            for (int r = tid; r < Mi; r += blockDim.x) {
                double v = ej[r];
                for (int p = 0; p < j; ++p) v = fma(-h[p], E[p * Mi + r], v);
                ej[r] = v;
            }
            __syncthreads();
        }
        double t = 0.0;
        for (int r = tid; r < Mi; r += blockDim.x) t = fma(ej[r], ej[r], t);
        t = warp_sum(t);
        if (lane == 0) red[warp] = t;
        __syncthreads();
        double nrm = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) nrm += red[w];
        nrm = sqrt(nrm);
        for (int r = tid; r < Mi; r += blockDim.x) ej[r] = nrm > 0.0 ? ej[r] / nrm : 0.0;
        __syncthreads();
    }
    // every column to max-norm one
    for (int j = warp; j < Mi; j += blockDim.x / 32) {
        double mx = 0.0;
        for (int r = lane; r < Mi; r += 32) mx = fmax(mx, fabs(E[j * Mi + r]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        for (int r = lane; r < Mi; r += 32) E[j * Mi + r] = mx > 0.0 ? E[j * Mi + r] / mx : 0.0;
        if (lane == 0) col_scale[j] = mx;
    }
    __syncthreads();
    // the kept columns, [m][k], before the elimination overwrites E
    for (int e = tid; e < s * Mi; e += blockDim.x) {
        const int m = e / s, k = e - m * s;
        ekeep[off[blockIdx.x] + e] = E[k * Mi + m];
    }
    // Gauss-Jordan: E X = I with partial pivoting (A = E kept in place, row-swapped)
    for (int e = tid; e < Mi * Mi; e += blockDim.x) X[e] = (e / Mi == e % Mi) ? 1.0 : 0.0;
    __syncthreads();
    bool bad = false;
    for (int c = 0; c < Mi; ++c) {
        if (tid == 0) {
            int pr = c;
            double pv = fabs(E[c * Mi + c]);
            for (int r = c + 1; r < Mi; ++r) {
                const double v = fabs(E[c * Mi + r]);
                if (v > pv) { pv = v; pr = r; }
            }
            s_piv = pr;
            if (!(pv > pivot_tol)) bad = true;
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != c) {
            for (int j = tid; j < Mi; j += blockDim.x) {
                const double a = E[j * Mi + c];
                E[j * Mi + c] = E[j * Mi + pr];
                E[j * Mi + pr] = a;
                const double x = X[c * Mi + j];
                X[c * Mi + j] = X[pr * Mi + j];
                X[pr * Mi + j] = x;
            }
            __syncthreads();
        }
        const double piv = E[c * Mi + c];
        const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
        __syncthreads();
        for (int j = tid; j < Mi; j += blockDim.x) {
            E[j * Mi + c] *= inv;
            X[c * Mi + j] *= inv;
        }
        __syncthreads();
        // factors of column c, then eliminate it from every other row
        for (int r = tid; r < Mi; r += blockDim.x) h[r] = r == c ? 0.0 : E[c * Mi + r];
        __syncthreads();
        for (int e = tid; e < Mi * Mi; e += blockDim.x) {
            const int r = e / Mi, j = e - r * Mi;
            const double f = h[r];
            if (f == 0.0) continue;
            if (j > c) E[j * Mi + r] = fma(-f, E[j * Mi + c], E[j * Mi + r]);
            X[r * Mi + j] = fma(-f, X[c * Mi + j], X[r * Mi + j]);
        }
        for (int r = tid; r < Mi; r += blockDim.x)
            if (r != c) E[c * Mi + r] = 0.0;
        __syncthreads();
    }
    if (tid == 0 && bad) atomicExch(singular, 1);
    __syncthreads();
    // kept rows of the inverse, stored [m][k], and the functions behind them
    double* out = proj + off[blockIdx.x];
    for (int e = tid; e < s * Mi; e += blockDim.x) {
        const int m = e / s, k = e - m * s;
        out[e] = X[k * Mi + m];
    }
    for (int k = tid; k < s; k += blockDim.x) kcol[r0 + k] = (long long)col_slot[k] * N + col_cell[k];
    // dropped rows [m][d]; a dropped column is its function itself scaled to
    // max-norm one, so P^k l^k = scale
    const int nd = Mi - s;
    double* lout = lproj + loff[blockIdx.x];
    for (int e = tid; e < nd * Mi; e += blockDim.x) {
        const int m = e / nd, dd = e - m * nd;
        lout[e] = X[(s + dd) * Mi + m];
    }
    for (int dd = tid; dd < nd; dd += blockDim.x) {
        const int j = s + dd;
        dcol[d0 + dd] = (long long)col_slot[j] * N + col_cell[j];
        const double sc = col_scale[j] > 0.0 ? 1.0 / col_scale[j] : 0.0;
        dsc[d0 + dd] = col_cell[j] == cm ? -sc : sc;
    }
}

// row of A and sign of direction m of an interface (see the header comment)
__device__ __forceinline__ size_t iface_row(const int* d, const int* rowinfo, int m, int M, int N, double& sign) {
    const int cm = d[0], cp = d[1], fm = d[2], fp = d[3];
    const int M2 = M / 2;
    if (cp < 0) {
        sign = 1.0;
        return (size_t)(fm * M2 + m) * N + cm;
    }
    const int j = rowinfo[fm * M + m];
    if (j >= 0) {
        sign = 1.0;
        return (size_t)(fm * M2 + j) * N + cm;
    }
    sign = -1.0;
    return (size_t)(fp * M2 + rowinfo[fp * M + m]) * N + cp;
}

// out[r0 + k] = sum_m P[m][k] sign_m y[row_m]: one warp per interface.  With
// kcol the row goes to slot kcol[r0 + k] instead (slot layout [2M][N]), as
// bsub - value when bsub is given.
__global__ void k_atfps_apply(const int* __restrict__ desc, const long long* __restrict__ off,
                              const int* __restrict__ rowinfo, const double* __restrict__ proj, int nif, int M,
                              int N, const double* __restrict__ y, double* __restrict__ out,
                              const long long* __restrict__ kcol, const double* __restrict__ bsub) {
    __shared__ double yv[8][80];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + w;
    if (i >= nif) return;
    const int* d = desc + 8 * i;
    const int s = d[4], Mi = d[5], r0 = d[6];
    for (int m = lane; m < Mi; m += 32) {
        double sg;
        const size_t row = iface_row(d, rowinfo, m, M, N, sg);
        yv[w][m] = sg * y[row];
    }
    __syncwarp();
    const double* P = proj + off[i];
    for (int k = lane; k < s; k += 32) {
        double acc = 0.0;
        for (int m = 0; m < Mi; ++m) acc = fma(P[(size_t)m * s + k], yv[w][m], acc);
        if (kcol) {
            const long long q = kcol[r0 + k];
            out[q] = bsub ? bsub[q] - acc : acc;
        } else {
            out[r0 + k] = acc;
        }
    }
}

// Layer coefficients (Eqs. 2DAdaptive_TFPS_layer1 / layer2): w = b - A x of
// the smooth solution x holds, on the rows of an interface, -(jump); the
// dropped coordinate beta_d of the jump gives x[dcol] = dsc beta_d (the sign
// by the function's side).  One warp per interface.
__global__ void k_atfps_layers(const int* __restrict__ desc, const long long* __restrict__ loff,
                               const int* __restrict__ rowinfo, const double* __restrict__ lproj,
                               const long long* __restrict__ dcol, const double* __restrict__ dsc, int nif, int M,
                               int N, const double* __restrict__ w, double* __restrict__ x) {
    __shared__ double jv[8][80];
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + wp;
    if (i >= nif) return;
    const int* d = desc + 8 * i;
    const int s = d[4], Mi = d[5], d0 = d[7], nd = Mi - s;
    if (nd == 0) return;
    for (int m = lane; m < Mi; m += 32) {
        double sg;
        const size_t row = iface_row(d, rowinfo, m, M, N, sg);
        jv[wp][m] = -sg * w[row];
    }
    __syncwarp();
    const double* P = lproj + loff[i];
    for (int dd = lane; dd < nd; dd += 32) {
        double acc = 0.0;
        for (int m = 0; m < Mi; ++m) acc = fma(P[(size_t)m * nd + dd], jv[wp][m], acc);
        x[dcol[d0 + dd]] = dsc[d0 + dd] * acc;
    }
}

// Right inverse of F (F S = I): y[row_m] = sign_m sum_k E[m][k] r[kcol[r0 + k]]
// -- each compressed row (in slot layout) back to the rows of its interface
// as the kept basis column; every row of A is written once.  One warp per
// interface.
__global__ void k_atfps_S(const int* __restrict__ desc, const long long* __restrict__ off,
                          const int* __restrict__ rowinfo, const double* __restrict__ ekeep,
                          const long long* __restrict__ kcol, int nif, int M, int N, const double* __restrict__ r,
                          double* __restrict__ y) {
    __shared__ double rv[8][80];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + w;
    if (i >= nif) return;
    const int* d = desc + 8 * i;
    const int s = d[4], Mi = d[5], r0 = d[6];
    for (int k = lane; k < s; k += 32) rv[w][k] = r[kcol[r0 + k]];
    __syncwarp();
    const double* E = ekeep + off[i];
    for (int m = lane; m < Mi; m += 32) {
        double acc = 0.0;
        for (int k = 0; k < s; ++k) acc = fma(E[(size_t)m * s + k], rv[w][k], acc);
        double sg;
        const size_t row = iface_row(d, rowinfo, m, M, N, sg);
        y[row] = sg * acc;
    }
}

// y[row_m] = sign_m sum_k P[m][k] r[r0 + k]: one warp per interface (rows of
// interfaces without kept functions are left as they are; callers zero y)
__global__ void k_atfps_apply_t(const int* __restrict__ desc, const long long* __restrict__ off,
                                const int* __restrict__ rowinfo, const double* __restrict__ proj, int nif, int M,
                                int N, const double* __restrict__ r, double* __restrict__ y) {
    __shared__ double rv[8][64];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + w;
    if (i >= nif) return;
    const int* d = desc + 8 * i;
    const int s = d[4], Mi = d[5], r0 = d[6];
    for (int k = lane; k < s; k += 32) rv[w][k] = r[r0 + k];
    __syncwarp();
    const double* P = proj + off[i];
    for (int m = 0; m < Mi; ++m) {
        double acc = 0.0;
        for (int k = lane; k < s; k += 32) acc = fma(P[(size_t)m * s + k], rv[w][k], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            double sg;
            const size_t row = iface_row(d, rowinfo, m, M, N, sg);
            y[row] = sg * acc;
        }
    }
}

__global__ void k_mask_mul(double* __restrict__ x, const unsigned char* __restrict__ mask, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!mask[i]) x[i] = 0.0;
}

template <typename T>
T* atfps_alloc(rte_ctx* ctx, Atfps* a, size_t count) {
    void* p = nullptr;
    const size_t bytes = count * sizeof(T) + 16;
    check(pool_malloc(&p, bytes, ctx->stream), "cudaMallocFromPoolAsync (ATFPS)");
    a->allocs.push_back(p);
    a->bytes += bytes;
    ctx->device_bytes += bytes;
    check(cudaMemsetAsync(p, 0, bytes, ctx->stream), "memset (ATFPS)");
    return static_cast<T*>(p);
}

}  // namespace

void atfps_free(rte_ctx* ctx) {
    if (!ctx || !ctx->atfps) return;
    for (void* p : ctx->atfps->allocs) cudaFreeAsync(p, ctx->stream);
    ctx->device_bytes -= ctx->atfps->bytes;
    delete ctx->atfps;
    ctx->atfps = nullptr;
}

void atfps_setup(rte_ctx* ctx, double delta) {
    atfps_free(ctx);
    const int I = ctx->I, M = ctx->M, N = ctx->N, M2 = M / 2, n2 = 2 * M;
    if (M > 80) throw StatusError{RTE_EINVAL, "ATFPS filter: M <= 80"};
    Atfps* a = new Atfps();
    ctx->atfps = a;
    a->delta = delta;
    std::vector<double> tau(N);
    check(cudaMemcpyAsync(tau.data(), ctx->tau, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "d2h tau");
    std::vector<int> rowinfo(4 * M);
    check(cudaMemcpyAsync(rowinfo.data(), ctx->rowinfo, 4 * M * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
          "d2h rowinfo");
    check(cudaStreamSynchronize(ctx->stream), "sync");
    // selection (Eq. def_V_delta)
    a->mask_h.assign((size_t)n2 * N, 0);
    for (int c = 0; c < N; ++c) {
        const double* xi = &ctx->xi_h[(size_t)ctx->mat_h[c] * n2];
        for (int k = 0; k < n2; ++k)
            a->mask_h[(size_t)k * N + c] = std::exp(-0.5 * std::fabs(xi[k]) * tau[c]) > delta ? 1 : 0;
    }
    // slot order per (material, group): ascending |xi|, ties by slot
    std::vector<int> ord((size_t)ctx->nmat * 4 * M2);
    for (int mt = 0; mt < ctx->nmat; ++mt)
        for (int grp = 0; grp < 4; ++grp) {
            int* o = &ord[((size_t)mt * 4 + grp) * M2];
            for (int q = 0; q < M2; ++q) o[q] = grp * M2 + q;
            const double* xi = &ctx->xi_h[(size_t)mt * n2];
            std::stable_sort(o, o + M2, [&](int x, int y) { return std::fabs(xi[x]) < std::fabs(xi[y]); });
        }
    std::vector<int> dirs(4 * M2);
    for (int f = 0; f < 4; ++f)
        for (int m = 0; m < M; ++m)
            if (rowinfo[f * M + m] >= 0) dirs[f * M2 + rowinfo[f * M + m]] = m;
    // interfaces (order as in the header comment) and their kept counts
    std::vector<int> desc;
    std::vector<long long> off, loff;
    long long total = 0, ltotal = 0;
    int64_t rows = 0, ndrop = 0;
    auto kept_in = [&](int c, int grp) {
        int s = 0;
        for (int q = 0; q < M2; ++q) s += a->mask_h[(size_t)(grp * M2 + q) * N + c];
        return s;
    };
    auto add = [&](int cm, int cp, int fm, int fp) {
        const int s = kept_in(cm, fm) + (cp >= 0 ? kept_in(cp, fp) : 0);
        const int Mi = cp >= 0 ? M : M2;
        desc.insert(desc.end(), {cm, cp, fm, fp, s, Mi, (int)rows, (int)ndrop});
        off.push_back(total);
        loff.push_back(ltotal);
        total += (long long)s * Mi;
        ltotal += (long long)(Mi - s) * Mi;
        rows += s;
        ndrop += Mi - s;
    };
    for (int iy = 0; iy < I; ++iy)
        for (int ix = 0; ix + 1 < I; ++ix) add(iy * I + ix, iy * I + ix + 1, 1, 0);
    for (int iy = 0; iy + 1 < I; ++iy)
        for (int ix = 0; ix < I; ++ix) add(iy * I + ix, (iy + 1) * I + ix, 3, 2);
    for (int iy = 0; iy < I; ++iy) {
        add(iy * I, -1, 0, -1);
        add(iy * I + I - 1, -1, 1, -1);
    }
    for (int ix = 0; ix < I; ++ix) {
        add(ix, -1, 2, -1);
        add((I - 1) * I + ix, -1, 3, -1);
    }
    a->nif = (int)off.size();
    a->rows = rows;
    a->ndrop = ndrop;
    a->mask = atfps_alloc<unsigned char>(ctx, a, a->mask_h.size());
    check(cudaMemcpyAsync(a->mask, a->mask_h.data(), a->mask_h.size(), cudaMemcpyHostToDevice, ctx->stream), "h2d");
    a->singular = atfps_alloc<int>(ctx, a, 1);
    if (a->nif == 0) {
        check(cudaStreamSynchronize(ctx->stream), "sync");
        return;
    }
    a->desc = atfps_alloc<int>(ctx, a, desc.size());
    a->off = atfps_alloc<long long>(ctx, a, off.size());
    a->proj = atfps_alloc<double>(ctx, a, (size_t)total);
    a->ekeep = atfps_alloc<double>(ctx, a, (size_t)total);
    a->loff = atfps_alloc<long long>(ctx, a, loff.size());
    a->lproj = atfps_alloc<double>(ctx, a, (size_t)ltotal);
    a->kcol = atfps_alloc<long long>(ctx, a, (size_t)rows);
    a->dcol = atfps_alloc<long long>(ctx, a, (size_t)ndrop);
    a->dsc = atfps_alloc<double>(ctx, a, (size_t)ndrop);
    check(cudaMemcpyAsync(a->loff, loff.data(), loff.size() * sizeof(long long), cudaMemcpyHostToDevice,
                          ctx->stream), "h2d");
    int* d_ord = atfps_alloc<int>(ctx, a, ord.size());
    int* d_dirs = atfps_alloc<int>(ctx, a, dirs.size());
    check(cudaMemcpyAsync(a->desc, desc.data(), desc.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "h2d");
    check(cudaMemcpyAsync(a->off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream),
          "h2d");
    check(cudaMemcpyAsync(d_ord, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "h2d");
    check(cudaMemcpyAsync(d_dirs, dirs.data(), dirs.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
          "h2d");
    const size_t smem = (size_t)(2 * M * M + M) * sizeof(double);
    raise_smem_limit((const void*)k_atfps_build, (size_t)(smem));
    // a pivot below 1e-12 of the (unit max-norm) columns: cond(E) beyond ~1e12
    k_atfps_build<<<a->nif, kBuildThreads, smem, ctx->stream>>>(a->desc, a->off, d_ord, d_dirs, ctx->L64, ctx->mat,
                                                                a->mask, M, N, 1e-12, a->proj, a->ekeep, a->loff,
                                                                a->lproj,
                                                                a->kcol, a->dcol, a->dsc, a->singular);
    check(cudaGetLastError(), "k_atfps_build");
    int bad = 0;
    check(cudaMemcpyAsync(&bad, a->singular, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "d2h");
    check(cudaStreamSynchronize(ctx->stream), "sync");
    if (bad) {
        atfps_free(ctx);
        throw StatusError{RTE_ESINGULAR, "ATFPS interface basis is numerically singular"};
    }
}

void atfps_apply(rte_ctx* ctx, const double* y, double* out) {
    Atfps* a = ctx->atfps;
    if (!a) throw StatusError{RTE_EINVAL, "no ATFPS filter on this context (rte_atfps_setup)"};
    if (a->nif == 0) return;
    k_atfps_apply<<<(a->nif + 7) / 8, 256, 0, ctx->stream>>>(a->desc, a->off, ctx->rowinfo, a->proj, a->nif, ctx->M,
                                                             ctx->N, y, out, nullptr, nullptr);
    check(cudaGetLastError(), "k_atfps_apply");
}

void atfps_apply_t(rte_ctx* ctx, const double* r, double* y) {
    Atfps* a = ctx->atfps;
    if (!a) throw StatusError{RTE_EINVAL, "no ATFPS filter on this context (rte_atfps_setup)"};
    check(cudaMemsetAsync(y, 0, (size_t)ctx->n * sizeof(double), ctx->stream), "memset");
    if (a->nif == 0) return;
    k_atfps_apply_t<<<(a->nif + 7) / 8, 256, 0, ctx->stream>>>(a->desc, a->off, ctx->rowinfo, a->proj, a->nif,
                                                               ctx->M, ctx->N, r, y);
    check(cudaGetLastError(), "k_atfps_apply_t");
}

namespace {
Atfps* need_filter(rte_ctx* ctx) {
    if (!ctx->atfps) throw StatusError{RTE_EINVAL, "no ATFPS filter on this context (rte_atfps_setup)"};
    return ctx->atfps;
}

// b_bar and the scratch, once per filter
void comp_prepare(rte_ctx* ctx) {
    Atfps* a = need_filter(ctx);
    if (a->bbar) return;
    const int64_t n = ctx->n;
    a->scratch = atfps_alloc<double>(ctx, a, (size_t)n);
    a->scratch2 = atfps_alloc<double>(ctx, a, (size_t)n);
    a->bbar = atfps_alloc<double>(ctx, a, (size_t)n);
    k_atfps_apply<<<(a->nif + 7) / 8, 256, 0, ctx->stream>>>(a->desc, a->off, ctx->rowinfo, a->proj, a->nif, ctx->M,
                                                             ctx->N, ctx->b, a->bbar, a->kcol, nullptr);
    check(cudaGetLastError(), "k_atfps_apply");
}
}  // namespace

const double* atfps_comp_rhs(rte_ctx* ctx) {
    comp_prepare(ctx);
    return ctx->atfps->bbar;
}

void atfps_comp_precond(rte_ctx* ctx, const double* z, double* out) {
    Atfps* a = need_filter(ctx);
    comp_prepare(ctx);
    k_atfps_S<<<(a->nif + 7) / 8, 256, 0, ctx->stream>>>(a->desc, a->off, ctx->rowinfo, a->ekeep, a->kcol, a->nif,
                                                         ctx->M, ctx->N, z, a->scratch2);
    check(cudaGetLastError(), "k_atfps_S");
    launch_block_apply(ctx, false, a->scratch2, true, out, true);
    atfps_mask_mul(ctx, out);
}

void atfps_comp_apply(rte_ctx* ctx, const double* x, double* out, bool residual) {
    Atfps* a = need_filter(ctx);
    launch_apply(ctx, true, x, a->scratch, true, nullptr);
    check(cudaMemsetAsync(out, 0, (size_t)ctx->n * sizeof(double), ctx->stream), "memset");
    k_atfps_apply<<<(a->nif + 7) / 8, 256, 0, ctx->stream>>>(a->desc, a->off, ctx->rowinfo, a->proj, a->nif, ctx->M,
                                                             ctx->N, a->scratch, out, a->kcol,
                                                             residual ? a->bbar : nullptr);
    check(cudaGetLastError(), "k_atfps_apply");
}

void atfps_layers(rte_ctx* ctx, double* x) {
    Atfps* a = need_filter(ctx);
    comp_prepare(ctx);
    launch_apply(ctx, true, x, a->scratch, true, ctx->b);        // b - A x
    k_atfps_layers<<<(a->nif + 7) / 8, 256, 0, ctx->stream>>>(a->desc, a->loff, ctx->rowinfo, a->lproj, a->dcol,
                                                              a->dsc, a->nif, ctx->M, ctx->N, a->scratch, x);
    check(cudaGetLastError(), "k_atfps_layers");
}

void atfps_mask_mul(rte_ctx* ctx, double* x) {
    Atfps* a = ctx->atfps;
    if (!a) throw StatusError{RTE_EINVAL, "no ATFPS filter on this context (rte_atfps_setup)"};
    const int64_t n = ctx->n;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
    k_mask_mul<<<blocks, 256, 0, ctx->stream>>>(x, a->mask, n);
    check(cudaGetLastError(), "k_mask_mul");
}

int64_t atfps_rows(const rte_ctx* ctx) { return ctx->atfps ? ctx->atfps->rows : -1; }

}  // namespace rte

using namespace rte;

extern "C" {

RTE_API rte_status rte_atfps_setup(rte_ctx* ctx, double delta, int64_t* rows_out) {
    if (!ctx || !(delta >= 0.0) || !(delta < 1.0)) {
        set_error(ctx, "bad argument (0 <= delta < 1)");
        return RTE_EINVAL;
    }
    try {
        atfps_setup(ctx, delta);
        if (rows_out) *rows_out = ctx->atfps->rows;
    } catch (const CudaError& e) {
        return cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        set_error(ctx, "host allocation failed");
        return RTE_ENOMEM;
    }
    return RTE_OK;
}

RTE_API rte_status rte_atfps_mask(rte_ctx* ctx, unsigned char* mask_host) {
    if (!ctx || !mask_host) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    if (!ctx->atfps) { set_error(ctx, "no ATFPS filter on this context (rte_atfps_setup)"); return RTE_EINVAL; }
    std::copy(ctx->atfps->mask_h.begin(), ctx->atfps->mask_h.end(), mask_host);
    return RTE_OK;
}

RTE_API rte_status rte_atfps_apply(rte_ctx* ctx, const double* y_dev, double* out_dev) {
    if (!ctx || !y_dev || !out_dev) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    try {
        atfps_apply(ctx, y_dev, out_dev);
    } catch (const CudaError& e) {
        return cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        return e.code;
    }
    return RTE_OK;
}

RTE_API rte_status rte_atfps_apply_t(rte_ctx* ctx, const double* r_dev, double* y_dev) {
    if (!ctx || !r_dev || !y_dev) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    try {
        atfps_apply_t(ctx, r_dev, y_dev);
    } catch (const CudaError& e) {
        return cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        return e.code;
    }
    return RTE_OK;
}

}  // extern "C"
