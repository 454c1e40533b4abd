// Batched eigenbases of the local TFPS problem (Eq.
// discretization_2D_eigenfunc_constraint) on the device, for media with many
// materials (every distinct 1 - gamma = eps^2 sigma_a / sigma_T is one; with
// independent sigma_a and sigma_T fields every cell is its own).
//
// Per material and axis, (gamma K W - I) l = xi diag(d) l with d = c (axis 0)
// or s (axis 1) is the symmetric definite pencil diag(d) l = mu S l,
// S = I - gamma K W, mu = -1 / xi.  The pencil commutes with the reflection of
// the directions that leaves d unchanged, so it splits into the mirror-
// symmetric and antisymmetric halves (orthonormal columns (e_m +- e_m')/sqrt 2
// for the pairs m < m' = refl(m)); each half is reduced by the Cholesky factor
// S_P = R^T R to the symmetric eigenproblem of B = R^-T D_P R^-1 (D_P is
// diagonal: d is invariant under the reflection) and diagonalised by cyclic
// Jacobi rotations, h / 2 disjoint pairs per round in the round-robin order,
// with the threshold rule (an entry below 1e-18 of the geometric mean of its
// diagonal pair is not rotated) until a sweep rotates nothing or the
// off-diagonal square sum is below 1e-32 of the diagonal's.
//
// One CTA per (material, axis, half); a second kernel orders each axis's M
// modes by xi (ties: symmetric first) and scales every eigenvector by its first
// entry within 1e-8 of its largest magnitude (||l||_inf = 1), the order and
// normalisation of the host eigenbasis.  Loops are bounded (sweeps <= 50).
#include <cmath>

#include "rte_internal.h"

namespace rte {
namespace {

constexpr int kEigThreads = 64;
constexpr int kMaxSweeps = 50;

// one pencil: blockIdx.x = (mat * 2 + axis) * 2 + odd
__global__ void __launch_bounds__(kEigThreads)
    k_pencil(int M, int nmat, const double* __restrict__ omg, const double* __restrict__ K,
             const double* __restrict__ kwoff, const double* __restrict__ cdir, const double* __restrict__ sdir,
             const int* __restrict__ pairm, const int* __restrict__ refl, double* __restrict__ xi_out,
             double* __restrict__ l_out, int* __restrict__ bad) {
    extern __shared__ double sm[];
    const int h = M / 2;
    const int q = blockIdx.x;
    const int odd = q & 1, axis = (q >> 1) & 1, mat = q >> 2;
    if (mat >= nmat) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ld = h + 1;           // padded rows: column walks stay off one bank
    double* S = sm;                 // [h][ld], then B
    double* Ri = S + h * ld;        // [h][ld] R^-1 (upper)
    double* R = Ri + h * ld;        // [h][ld] Cholesky factor (upper)
    double* V = R + h * ld;         // [h][ld] rotations
    double* dp = V + h * ld;        // [h]
    double* cs = dp + h;            // [h/2] cosines
    double* sn = cs + h / 2;        // [h/2] sines
    __shared__ int arr[64];
    __shared__ int stop, rotated;
    const double w = omg[mat], gamma = 1.0 - w;
    const double sg = odd ? -1.0 : 1.0;
    const int* pm = pairm + axis * h;
    const int* rf = refl + axis * M;
    const double* d = axis == 0 ? cdir : sdir;
    auto Sx = [&](int i, int j) {       // S = (1 - gamma) I + gamma (I - K W)
        return i == j ? w + gamma * kwoff[i] : -gamma * K[(size_t)i * M + j] / M;
    };
    for (int e = tid; e < h * h; e += nt) {
        const int a = e / h, b = e - a * h;
        const int ma = pm[a], mb = pm[b], na = rf[ma], nb = rf[mb];
        const double v = 0.5 * (Sx(ma, mb) + sg * Sx(ma, nb) + sg * Sx(na, mb) + Sx(na, nb));
        S[a * ld + b] = v;
    }
    for (int a = tid; a < h; a += nt) dp[a] = d[pm[a]];
    __syncthreads();
    for (int e = tid; e < h * h; e += nt) {          // symmetrise
        const int a = e / h, b = e - a * h;
        if (a < b) {
            const double t = 0.5 * (S[a * ld + b] + S[b * ld + a]);
            S[a * ld + b] = t;
            S[b * ld + a] = t;
        }
    }
    for (int e = tid; e < h * ld; e += nt) R[e] = 0.0;
    __syncthreads();
    // Cholesky S = R^T R, column j of R: R[j][j], then R[j][i] for i > j
    for (int j = 0; j < h; ++j) {
        if (tid == 0) {
            double s = S[j * ld + j];
            for (int k = 0; k < j; ++k) s -= R[k * ld + j] * R[k * ld + j];
            if (!(s > 0.0)) {
                atomicExch(bad, 1);
                s = 1.0;
            }
            R[j * ld + j] = sqrt(s);
        }
        __syncthreads();
        const double rjj = R[j * ld + j];
        for (int i = j + 1 + tid; i < h; i += nt) {
            double t = S[j * ld + i];
            for (int k = 0; k < j; ++k) t -= R[k * ld + j] * R[k * ld + i];
            R[j * ld + i] = t / rjj;
        }
        __syncthreads();
    }
    // Ri = R^-1, one column per thread (back substitution)
    for (int col = tid; col < h; col += nt) {
        for (int i = h - 1; i >= 0; --i) Ri[i * ld + col] = 0.0;
        for (int i = col; i >= 0; --i) {
            double t = (i == col) ? 1.0 : 0.0;
            for (int k = i + 1; k <= col; ++k) t -= R[i * ld + k] * Ri[k * ld + col];
            Ri[i * ld + col] = t / R[i * ld + i];
        }
    }
    __syncthreads();
    // B = Ri^T diag(dp) Ri (overwrites S), V = I
    for (int e = tid; e < h * h; e += nt) {
        const int i = e / h, j = e - i * h;
        double t = 0.0;
        const int kk = i < j ? i : j;
        for (int k = 0; k <= kk; ++k) t += Ri[k * ld + i] * dp[k] * Ri[k * ld + j];
        S[i * ld + j] = t;
        V[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < h * h; e += nt) {
        const int a = e / h, b = e - a * h;
        if (a < b) {
            const double t = 0.5 * (S[a * ld + b] + S[b * ld + a]);
            S[a * ld + b] = t;
            S[b * ld + a] = t;
        }
    }
    for (int i = tid; i < h; i += nt) arr[i] = i;
    if (tid == 0) stop = 0;
    __syncthreads();
    const int np = h / 2;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        // convergence: off-diagonal and diagonal square sums
        if (tid == 0) {
            double off = 0.0, dg = 0.0;
            for (int p = 0; p < h; ++p) {
                dg += S[p * ld + p] * S[p * ld + p];
                for (int r = p + 1; r < h; ++r) off += S[p * ld + r] * S[p * ld + r];
            }
            stop = (off <= 1e-32 * dg || off == 0.0) ? 1 : 0;
            rotated = 0;
        }
        __syncthreads();
        if (stop) break;
        for (int round = 0; round < h - 1; ++round) {
            // angles of this round's disjoint pairs, from the current matrix
            for (int k = tid; k < np; k += nt) {
                const int p = arr[k], r = arr[h - 1 - k];
                const double apq = S[p * ld + r];
                double c = 1.0, s = 0.0;
                // threshold rule: entries at rounding level of their diagonal
                // pair are not rotated (a sweep without rotation ends the loop)
                if (fabs(apq) > 1e-18 * sqrt(fabs(S[p * ld + p] * S[r * ld + r]))) {
                    rotated = 1;
                    const double theta = (S[r * ld + r] - S[p * ld + p]) / (2.0 * apq);
                    const double t = fabs(theta) > 1e150
                                         ? 0.5 / theta
                                         : (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(t * t + 1.0);
                    s = t * c;
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // rows p, r of every pair
            for (int e = tid; e < np * h; e += nt) {
                const int k = e / h, col = e - k * h;
                const int p = arr[k], r = arr[h - 1 - k];
                const double c = cs[k], s = sn[k];
                const double apk = S[p * ld + col], ark = S[r * ld + col];
                S[p * ld + col] = c * apk - s * ark;
                S[r * ld + col] = s * apk + c * ark;
            }
            __syncthreads();
            // columns p, r of every pair, and of V
            for (int e = tid; e < np * h; e += nt) {
                const int k = e / h, row = e - k * h;
                const int p = arr[k], r = arr[h - 1 - k];
                const double c = cs[k], s = sn[k];
                const double akp = S[row * ld + p], akr = S[row * ld + r];
                S[row * ld + p] = c * akp - s * akr;
                S[row * ld + r] = s * akp + c * akr;
                const double vkp = V[row * ld + p], vkr = V[row * ld + r];
                V[row * ld + p] = c * vkp - s * vkr;
                V[row * ld + r] = s * vkp + c * vkr;
            }
            __syncthreads();
            // next round: position 0 stays, the others rotate by one
            if (tid == 0) {
                const int last = arr[h - 1];
                for (int i = h - 1; i > 1; --i) arr[i] = arr[i - 1];
                if (h > 1) arr[1] = last;
            }
            __syncthreads();
        }
        if (!rotated) break;
    }
    // xi = -1 / mu; mode k: l = P (Ri y_k)
    double* xo = xi_out + (size_t)q * h;
    double* lo = l_out + (size_t)q * h * M;
    const double r2 = sqrt(0.5);
    for (int k = tid; k < h; k += nt) xo[k] = -1.0 / S[k * ld + k];
    for (int e = tid; e < h * h; e += nt) {
        const int k = e / h, b = e - k * h;
        double t = 0.0;
        for (int j = b; j < h; ++j) t += Ri[b * ld + j] * V[j * ld + k];
        lo[(size_t)k * M + pm[b]] = r2 * t;
        lo[(size_t)k * M + rf[pm[b]]] = sg * r2 * t;
    }
}

// order and normalise one axis of one material: blockIdx.x = mat * 2 + axis
__global__ void k_basis_merge(int M, const double* __restrict__ xi_p, const double* __restrict__ l_p,
                              double* __restrict__ xi, double* __restrict__ L) {
    const int h = M / 2, n2 = 2 * M;
    const int mat = blockIdx.x >> 1, axis = blockIdx.x & 1;
    __shared__ int order[80];
    __shared__ double xv[80];
    const double* xs = xi_p + (size_t)(blockIdx.x * 2) * h;        // symmetric half, then antisymmetric
    const double* ls = l_p + (size_t)(blockIdx.x * 2) * h * M;
    for (int k = threadIdx.x; k < M; k += blockDim.x) xv[k] = xs[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        // stable insertion sort by (xi, antisymmetric after symmetric)
        for (int k = 0; k < M; ++k) order[k] = k;
        for (int i = 1; i < M; ++i) {
            const int a = order[i];
            int j = i - 1;
            while (j >= 0) {
                const int b = order[j];
                const bool after = xv[b] > xv[a] || (xv[b] == xv[a] && b >= h && a < h);
                if (!after) break;
                order[j + 1] = b;
                --j;
            }
            order[j + 1] = a;
        }
    }
    __syncthreads();
    for (int kk = threadIdx.x; kk < M; kk += blockDim.x) {
        const int k = order[kk];
        const double* l = ls + (size_t)k * M;
        double amax = 0.0;
        for (int i = 0; i < M; ++i) amax = fmax(amax, fabs(l[i]));
        int p = 0;
        while (p < M - 1 && fabs(l[p]) < (1.0 - 1e-8) * amax) ++p;
        const double lp = l[p];
        xi[(size_t)mat * n2 + axis * M + kk] = xv[k];
        for (int i = 0; i < M; ++i)
            L[((size_t)mat * M + i) * n2 + axis * M + kk] = (i == p) ? 1.0 : l[i] / lp;
    }
}

// the transposed and single-precision copies of the bases
__global__ void k_basis_copies(int M, int nmat, const double* __restrict__ L, double* __restrict__ Lt64,
                               float* __restrict__ Lt32, float* __restrict__ L32) {
    const int n2 = 2 * M;
    const int64_t n = (int64_t)nmat * M * n2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / ((int64_t)M * n2);
        const int rem = (int)(e - j * M * n2), m = rem / n2, k = rem - m * n2;
        const double v = L[e];
        L32[e] = (float)v;
        Lt64[(j * n2 + k) * M + m] = v;
        Lt32[(j * n2 + k) * M + m] = (float)v;
    }
}

}  // namespace

void device_eigenbases(rte_ctx* ctx, const std::vector<double>& omg, const std::vector<double>& K,
                       const std::vector<double>& cdir, const std::vector<double>& sdir, double* xi_dev,
                       double* L64_dev, double* Lt64_dev, float* Lt32_dev, float* L32_dev) {
    const int M = ctx->M, h = M / 2, nmat = (int)omg.size();
    if (M > 80 || M % 4) throw StatusError{RTE_EINVAL, "device eigenbases: M % 4 == 0, M <= 80"};
    std::vector<double> kwoff(M);
    for (int i = 0; i < M; ++i) {
        double s = 0.0;
        for (int j = 0; j < M; ++j)
            if (j != i) s += K[(size_t)i * M + j] / M;
        kwoff[i] = s;
    }
    std::vector<int> pairm(2 * h), refl(2 * M);
    for (int axis = 0; axis < 2; ++axis) {
        for (int m = 0; m < M; ++m)
            refl[axis * M + m] = axis == 0 ? M - 1 - m : (((M / 2 - 1 - m) % M) + M) % M;
        int col = 0;
        for (int m = 0; m < M; ++m)
            if (m < refl[axis * M + m]) pairm[axis * h + col++] = m;
    }
    const size_t pencils = (size_t)nmat * 4;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bytes = al(omg.size() * 8) + al(K.size() * 8) + 3 * al((size_t)M * 8) + al(pairm.size() * 4) +
                         al(refl.size() * 4) + al(pencils * h * 8) + al(pencils * h * M * 8) + al(4);
    char* buf = nullptr;
    check(pool_malloc(reinterpret_cast<void**>(&buf), bytes, ctx->stream), "cudaMallocFromPoolAsync (eigenbases)");
    struct Scratch {                    // released on every path out of here
        char* p;
        cudaStream_t st;
        ~Scratch() { cudaFreeAsync(p, st); }
    } scratch{buf, ctx->stream};
    auto take = [&](size_t b) {
        char* p = buf;
        buf += al(b);
        return p;
    };
    double* d_omg = reinterpret_cast<double*>(take(omg.size() * 8));
    double* d_K = reinterpret_cast<double*>(take(K.size() * 8));
    double* d_kw = reinterpret_cast<double*>(take(M * 8));
    double* d_c = reinterpret_cast<double*>(take(M * 8));
    double* d_s = reinterpret_cast<double*>(take(M * 8));
    int* d_pair = reinterpret_cast<int*>(take(pairm.size() * 4));
    int* d_refl = reinterpret_cast<int*>(take(refl.size() * 4));
    double* d_xp = reinterpret_cast<double*>(take(pencils * h * 8));
    double* d_lp = reinterpret_cast<double*>(take(pencils * h * M * 8));
    int* d_bad = reinterpret_cast<int*>(take(4));
    auto up = [&](void* dst, const void* src, size_t b) {
        check(cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, ctx->stream), "h2d (eigenbases)");
    };
    up(d_omg, omg.data(), omg.size() * 8);
    up(d_K, K.data(), K.size() * 8);
    up(d_kw, kwoff.data(), M * 8);
    up(d_c, cdir.data(), M * 8);
    up(d_s, sdir.data(), M * 8);
    up(d_pair, pairm.data(), pairm.size() * 4);
    up(d_refl, refl.data(), refl.size() * 4);
    check(cudaMemsetAsync(d_bad, 0, 4, ctx->stream), "memset");
    check(cudaMemsetAsync(d_lp, 0, pencils * h * M * 8, ctx->stream), "memset");
    const size_t smem = (size_t)(4 * h * (h + 1) + 2 * h) * sizeof(double);
    raise_smem_limit((const void*)k_pencil, smem);
    k_pencil<<<(unsigned)pencils, kEigThreads, smem, ctx->stream>>>(M, nmat, d_omg, d_K, d_kw, d_c, d_s, d_pair,
                                                                     d_refl, d_xp, d_lp, d_bad);
    check(cudaGetLastError(), "k_pencil");
    k_basis_merge<<<(unsigned)(nmat * 2), 128, 0, ctx->stream>>>(M, d_xp, d_lp, xi_dev, L64_dev);
    check(cudaGetLastError(), "k_basis_merge");
    const int64_t n = (int64_t)nmat * M * 2 * M;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16);
    k_basis_copies<<<blocks, 256, 0, ctx->stream>>>(M, nmat, L64_dev, Lt64_dev, Lt32_dev, L32_dev);
    check(cudaGetLastError(), "k_basis_copies");
    int bad = 0;
    check(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, ctx->stream), "d2h");
    check(cudaStreamSynchronize(ctx->stream), "sync (eigenbases)");
    if (bad) throw StatusError{RTE_ESINGULAR, "scattering operator not positive definite"};
}

}  // namespace rte
