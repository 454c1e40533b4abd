// Host set-up of one TFPS system (Sec. 2.1-2.2) and the plain entry points.
//
// The host computes, in FP64, the direction set, the normalised HG matrix
// (Eq. hg), and one eigenbasis per distinct scattering ratio (Eq.
// discretization_2D_eigenfunc_constraint) by a cyclic Jacobi eigen-solver of
// the symmetric-definite pencil diag(c) l = mu (I - gamma K W) l, xi = -1/mu.
// Everything proportional to the grid (b, the per-cell blocks and their
// inverses) is built on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "rte_internal.h"

namespace rte {

static thread_local std::string g_thread_error;

void set_error(rte_ctx* ctx, const std::string& msg) {
    g_thread_error = msg;
    if (ctx) ctx->err = msg;
}

rte_status cuda_status(rte_ctx* ctx, cudaError_t e, const char* where) {
    set_error(ctx, std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? RTE_ENOMEM : RTE_ECUDA;
}

namespace {
// The library's stream-ordered memory pool of each device.  Freed blocks stay
// mapped up to a quarter of the device memory, so a context set up after
// another one was destroyed (a serving loop, repeated solves) reuses the
// physical pages instead of mapping gigabytes again; rte_trim_memory returns
// them to the device.
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t library_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    uint64_t keep = (uint64_t)total_b / 4;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);       // not cached: the next allocation tries again
        return e;
    }
    g_pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}
}  // namespace

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = library_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes == 0 ? 16 : bytes, pool, st);
}

void* dev_alloc_raw(rte_ctx* ctx, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    // stream-ordered: a context's allocations and frees never synchronise
    // the device, so concurrent solves on other streams keep running
    cudaError_t e = pool_malloc(&p, bytes, ctx->stream);
    if (e != cudaSuccess) throw CudaError{e, "cudaMallocFromPoolAsync"};
    ctx->allocations.push_back(p);
    ctx->device_bytes += bytes;
    return p;
}

void* dev_alloc(rte_ctx* ctx, size_t bytes) {
    void* p = dev_alloc_raw(ctx, bytes);
    check(cudaMemsetAsync(p, 0, bytes == 0 ? 16 : bytes, ctx->stream), "cudaMemset");
    return p;
}

void raise_smem_limit(const void* kern, size_t bytes) {
    static std::mutex mu;
    static std::map<const void*, size_t> limit;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[kern];
    if (bytes <= cur) return;
    check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
          "cudaFuncSetAttribute (dynamic shared memory)");
    cur = bytes;
}

const char* const kKernelNames[K_COUNT] = {
    "traces", "combine", "adjoint", "reconstruct", "rhs", "build_invert", "block_apply",
    "block_apply_t", "mdot", "update_dot", "update_norm", "norm", "scale", "x_update",
    "givens", "backsub", "cycle_start", "f2d", "mgnet", "response_build", "response_apply",
    "gather", "response_tc", "tile_order", "fix_dot", "update_dot_norm"};

static cudaEvent_t prof_event(rte_ctx* ctx) {
    if (!ctx->prof.pool.empty()) {
        cudaEvent_t e = ctx->prof.pool.back();
        ctx->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    check(cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

ProfScope::ProfScope(rte_ctx* c, int k, double bytes, int launches, double flops64)
    : ctx(c), kid(k) {
    ctx->prof.launches[k] += launches;
    ctx->prof.bytes[k] += bytes;
    ctx->prof.flops[k] += flops64;
    if (ctx->prof.on) {
        b = prof_event(ctx);
        check(cudaEventRecord(b, ctx->stream), "cudaEventRecord");
    }
}

ProfScope::~ProfScope() {
    if (!b) return;
    cudaEvent_t e = nullptr;
    try {
        e = prof_event(ctx);
    } catch (...) {
        return;
    }
    cudaEventRecord(e, ctx->stream);
    ctx->prof.pending.push_back({kid, b, e});
}

void prof_resolve(rte_ctx* ctx) {
    // launches still running (queued ahead of the host) stay pending
    size_t keep = 0;
    for (auto& p : ctx->prof.pending) {
        if (cudaEventQuery(p.b) == cudaErrorNotReady) {
            ctx->prof.pending[keep++] = p;
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->prof.ms[p.kid] += ms;
        ctx->prof.pool.push_back(p.a);
        ctx->prof.pool.push_back(p.b);
    }
    ctx->prof.pending.erase(ctx->prof.pending.begin() + (std::ptrdiff_t)keep, ctx->prof.pending.end());
}

void prof_free(rte_ctx* ctx) {
    for (auto& p : ctx->prof.pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->prof.pool) cudaEventDestroy(e);
    ctx->prof.pending.clear();
    ctx->prof.pool.clear();
}

namespace {

// ---------------------------------------------------------------- linear algebra
// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (row-major,
// overwritten).  On return w holds the eigenvalues and the columns of V the
// orthonormal eigenvectors (V row-major).
void jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += A[(size_t)p * n + p] * A[(size_t)p * n + p];
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                double t;
                if (std::fabs(theta) > 1e150)
                    t = 0.5 / theta;
                else
                    t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Eigenpairs of the pencil diag(d) l = mu S l, S = I - gamma K W, restricted to
// the h orthonormal columns of P (M x h, row-major): xi = -1/mu and the
// eigenvectors l = P R^-1 y (unnormalised), from Cholesky S_P = R^T R of
// S_P = P^T S P and the symmetric eigenproblem of R^-T (P^T diag(d) P) R^-1.
void pencil(int M, int h, double omg, const std::vector<double>& K, const std::vector<double>& d,
            const std::vector<double>& P, std::vector<double>& xi, std::vector<double>& Lcols) {
    const double gamma = 1.0 - omg;
    // S = (1 - gamma) I + gamma (I - K W); the diagonal of I - KW is written as
    // the sum of the off-diagonal K W entries of its row.
    std::vector<double> S((size_t)M * M);
    for (int i = 0; i < M; ++i) {
        double offsum = 0.0;
        for (int j = 0; j < M; ++j) {
            if (j == i) continue;
            const double kw = K[(size_t)i * M + j] / M;
            offsum += kw;
            S[(size_t)i * M + j] = -gamma * kw;
        }
        S[(size_t)i * M + i] = omg + gamma * offsum;
    }
    // S_P = P^T S P, D_P = P^T diag(d) P
    std::vector<double> SP((size_t)M * h, 0.0), Sh((size_t)h * h, 0.0), Dh((size_t)h * h, 0.0);
    for (int i = 0; i < M; ++i)
        for (int b = 0; b < h; ++b) {
            double t = 0.0;
            for (int j = 0; j < M; ++j) t += S[(size_t)i * M + j] * P[(size_t)j * h + b];
            SP[(size_t)i * h + b] = t;
        }
    for (int a = 0; a < h; ++a)
        for (int b = 0; b < h; ++b) {
            double t = 0.0, u = 0.0;
            for (int i = 0; i < M; ++i) {
                t += P[(size_t)i * h + a] * SP[(size_t)i * h + b];
                u += P[(size_t)i * h + a] * d[i] * P[(size_t)i * h + b];
            }
            Sh[(size_t)a * h + b] = t;
            Dh[(size_t)a * h + b] = u;
        }
    for (int a = 0; a < h; ++a)
        for (int b = a + 1; b < h; ++b) {
            const double t = 0.5 * (Sh[(size_t)a * h + b] + Sh[(size_t)b * h + a]);
            Sh[(size_t)a * h + b] = Sh[(size_t)b * h + a] = t;
        }
    // Cholesky S_P = R^T R (R upper)
    std::vector<double> R((size_t)h * h, 0.0);
    for (int j = 0; j < h; ++j) {
        double sjj = Sh[(size_t)j * h + j];
        for (int k = 0; k < j; ++k) sjj -= R[(size_t)k * h + j] * R[(size_t)k * h + j];
        if (!(sjj > 0.0)) throw StatusError{RTE_ESINGULAR, "scattering operator not positive definite"};
        const double rjj = std::sqrt(sjj);
        R[(size_t)j * h + j] = rjj;
        for (int i = j + 1; i < h; ++i) {
            double t = Sh[(size_t)j * h + i];
            for (int k = 0; k < j; ++k) t -= R[(size_t)k * h + j] * R[(size_t)k * h + i];
            R[(size_t)j * h + i] = t / rjj;
        }
    }
    // Ri = R^-1 (upper triangular)
    std::vector<double> Ri((size_t)h * h, 0.0);
    for (int col = 0; col < h; ++col)
        for (int i = col; i >= 0; --i) {
            double t = (i == col) ? 1.0 : 0.0;
            for (int k = i + 1; k <= col; ++k) t -= R[(size_t)i * h + k] * Ri[(size_t)k * h + col];
            Ri[(size_t)i * h + col] = t / R[(size_t)i * h + i];
        }
    // B = Ri^T D_P Ri
    std::vector<double> T((size_t)h * h, 0.0), B((size_t)h * h, 0.0);
    for (int a = 0; a < h; ++a)
        for (int j = 0; j < h; ++j) {
            double t = 0.0;
            for (int k = 0; k <= j; ++k) t += Dh[(size_t)a * h + k] * Ri[(size_t)k * h + j];
            T[(size_t)a * h + j] = t;
        }
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) {
            double t = 0.0;
            for (int k = 0; k <= i; ++k) t += Ri[(size_t)k * h + i] * T[(size_t)k * h + j];
            B[(size_t)i * h + j] = t;
        }
    for (int i = 0; i < h; ++i)
        for (int j = i + 1; j < h; ++j) {
            const double t = 0.5 * (B[(size_t)i * h + j] + B[(size_t)j * h + i]);
            B[(size_t)i * h + j] = B[(size_t)j * h + i] = t;
        }
    std::vector<double> mu, Y;
    jacobi_eigh(h, B, mu, Y);
    xi.resize(h);
    Lcols.assign((size_t)h * M, 0.0);          // column-major: mode k at Lcols[k*M ..]
    std::vector<double> v(h);
    for (int k = 0; k < h; ++k) {
        xi[k] = -1.0 / mu[k];
        for (int i = 0; i < h; ++i) {
            double t = 0.0;
            for (int j = i; j < h; ++j) t += Ri[(size_t)i * h + j] * Y[(size_t)j * h + k];
            v[i] = t;
        }
        for (int m = 0; m < M; ++m) {
            double t = 0.0;
            for (int b = 0; b < h; ++b) t += P[(size_t)m * h + b] * v[b];
            Lcols[(size_t)k * M + m] = t;
        }
    }
}

// Eigenpairs of (gamma K W - I) l = xi diag(d) l for one value of 1 - gamma,
// d = c (axis 0) or s (axis 1).  The pencil commutes with the reflection of
// the directions that leaves d unchanged, so it is solved separately on the
// mirror-symmetric and antisymmetric halves; this fixes the basis uniquely
// where a symmetric and an antisymmetric mode nearly share xi.
// Returns xi ascending (ties: symmetric first) and L (row-major M x M, column
// k = eigenvector k) with ||l||_inf = 1 (to 1e-8): each vector is divided by
// its first entry within 1e-8 of the largest magnitude.
void eigenbasis(int M, double omg, const std::vector<double>& K, const std::vector<double>& d,
                int axis, std::vector<double>& xi, std::vector<double>& L) {
    const int h = M / 2;
    std::vector<int> refl(M);
    for (int m = 0; m < M; ++m) refl[m] = axis == 0 ? M - 1 - m : (((M / 2 - 1 - m) % M) + M) % M;
    std::vector<double> Ps((size_t)M * h, 0.0), Pa((size_t)M * h, 0.0);
    const double r2 = std::sqrt(0.5);
    int col = 0;
    for (int m = 0; m < M; ++m) {
        if (m < refl[m]) {
            Ps[(size_t)m * h + col] = r2;
            Ps[(size_t)refl[m] * h + col] = r2;
            Pa[(size_t)m * h + col] = r2;
            Pa[(size_t)refl[m] * h + col] = -r2;
            ++col;
        }
    }
    std::vector<double> xs, Ls, xa, La;
    pencil(M, h, omg, K, d, Ps, xs, Ls);
    pencil(M, h, omg, K, d, Pa, xa, La);
    std::vector<double> xv(M);
    std::vector<int> order(M);
    for (int k = 0; k < M; ++k) {
        xv[k] = k < h ? xs[k] : xa[k - h];
        order[k] = k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (xv[a] != xv[b]) return xv[a] < xv[b];
        return (a < h) && !(b < h);
    });
    xi.resize(M);
    L.assign((size_t)M * M, 0.0);
    for (int kk = 0; kk < M; ++kk) {
        const int k = order[kk];
        xi[kk] = xv[k];
        const double* l = (k < h) ? &Ls[(size_t)k * M] : &La[(size_t)(k - h) * M];
        double amax = 0.0;
        for (int i = 0; i < M; ++i) amax = std::max(amax, std::fabs(l[i]));
        // divide by the first entry within 1e-8 of the largest magnitude: that
        // entry becomes +1 and near-ties resolve the same way on any machine
        int p = 0;
        while (std::fabs(l[p]) < (1.0 - 1e-8) * amax) ++p;
        const double lp = l[p];
        for (int i = 0; i < M; ++i) L[(size_t)i * M + kk] = (i == p) ? 1.0 : l[i] / lp;
    }
}

// Normalised HG scattering matrix (Eq. hg): one scalar so that rows sum to M
// (sum_n kappa_mn w_n = 1 with w = 1/M).
std::vector<double> hg_matrix(int M, double g) {
    std::vector<double> K((size_t)M * M);
    double total = 0.0;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            const double th_i = 2.0 * M_PI * (i + 0.5) / M, th_j = 2.0 * M_PI * (j + 0.5) / M;
            const double mu = std::cos(th_i - th_j);
            const double v = (1.0 - g * g) / std::pow(1.0 + g * g - 2.0 * g * mu, 1.5);
            K[(size_t)i * M + j] = v;
            total += v / M;
        }
    const double rowmean = total / M;
    for (auto& v : K) v /= rowmean;
    return K;
}

template <typename T>
T* upload(rte_ctx* ctx, const std::vector<T>& h) {
    T* d = static_cast<T*>(dev_alloc(ctx, h.size() * sizeof(T)));
    check(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream),
          "upload");
    return d;
}

// Spacing of the interpolation nodes in ln tau and the smallest material
// (cells) the automatic mode tabulates.  At ds = 0.04 the 8-point Lagrange
// interpolation of D(tau) and R(tau) is exact to about 1e-11 of the blocks'
// size on well-conditioned media, below the rounding of an FP64 inversion
// once cond(G_C) exceeds about 1e5 and of the FP32 response matrices always.
constexpr double kTabStep = 0.04;
constexpr int kTabMinCells = 4096;

// Decides the set-up of the per-cell blocks and, when it tabulates, plans
// it: per material the nodes s = (base + i) ds over the range of its cells'
// ln tau (three nodes beyond each end), per cell the first node of its
// stencil and the Lagrange weights at t = ln(tau) / ds, cells binned by the
// stencil's first node.  Automatic mode: at least kTabMinCells cells and 16
// cells per node over all materials (a material of a few cells, e.g. one
// whose 1 - gamma rounds differently, costs only its eight nodes).
bool plan_tabulation(rte_ctx* ctx, const std::vector<double>& tau, TabPlan& plan) {
    const int N = ctx->N, nmat = ctx->nmat;
    if (ctx->block_mode == RTE_BLOCKS_EXACT) return false;
    std::vector<double> smin(nmat, 1e300), smax(nmat, -1e300), lt(N);
    for (int c = 0; c < N; ++c) {
        const int j = ctx->mat_h[c];
        const double sv = std::log(tau[c]);
        lt[c] = sv;
        smin[j] = std::min(smin[j], sv);
        smax[j] = std::max(smax[j], sv);
    }
    std::vector<long long> base(nmat), off(nmat + 1, 0);
    for (int j = 0; j < nmat; ++j) {
        base[j] = (long long)std::floor(smin[j] / kTabStep) - 3;
        const long long J = (long long)std::floor(smax[j] / kTabStep) - base[j] + 5;
        off[j + 1] = off[j] + J;
    }
    if (off[nmat] > 1 << 20) return false;
    if (ctx->block_mode == RTE_BLOCKS_AUTO && (N < kTabMinCells || off[nmat] * 16 > N)) return false;
    const int J = (int)off[nmat];
    plan.node_mat.resize(J);
    plan.node_tau.resize(J);
    for (int j = 0; j < nmat; ++j)
        for (long long i = off[j]; i < off[j + 1]; ++i) {
            plan.node_mat[i] = j;
            plan.node_tau[i] = std::exp((double)(base[j] + (i - off[j])) * kTabStep);
        }
    // stencil of every cell: nodes fl - 3 .. fl + 4 around t = ln(tau) / ds;
    // Lagrange weight m = prod_{q != m} (t - t_q) / prod_{q != m} (m - q),
    // the numerator from prefix and suffix products
    double inv_den[8];
    for (int m = 0; m < 8; ++m) {
        double d = 1.0;
        for (int q = 0; q < 8; ++q)
            if (q != m) d *= (double)(m - q);
        inv_den[m] = 1.0 / d;
    }
    std::vector<int> first(N);
    std::vector<double> w((size_t)N * 8);
    for (int c = 0; c < N; ++c) {
        const int j = ctx->mat_h[c];
        const double t = lt[c] / kTabStep;
        const long long fl = (long long)std::floor(t);
        first[c] = (int)(off[j] + (fl - 3 - base[j]));
        double dq[8], pre[8], suf[8];
        for (int q = 0; q < 8; ++q) dq[q] = t - (double)(fl - 3 + q);
        pre[0] = 1.0;
        for (int q = 1; q < 8; ++q) pre[q] = pre[q - 1] * dq[q - 1];
        suf[7] = 1.0;
        for (int q = 6; q >= 0; --q) suf[q] = suf[q + 1] * dq[q + 1];
        for (int m = 0; m < 8; ++m) w[(size_t)c * 8 + m] = pre[m] * suf[m] * inv_den[m];
    }
    // bins by first node (counting sort, cells in ascending order per bin)
    std::vector<int> nb(J + 1, 0);
    for (int c = 0; c < N; ++c) ++nb[first[c] + 1];
    for (int i = 0; i < J; ++i) nb[i + 1] += nb[i];
    plan.cells.assign(N, 0);
    plan.weights.assign((size_t)N * 8, 0.0);
    std::vector<int> fillp(nb.begin(), nb.end() - 1);
    for (int c = 0; c < N; ++c) {
        const int pos = fillp[first[c]]++;
        plan.cells[pos] = c;
        for (int m = 0; m < 8; ++m) plan.weights[(size_t)pos * 8 + m] = w[(size_t)c * 8 + m];
    }
    for (int i = 0; i < J; ++i)
        if (nb[i + 1] > nb[i]) plan.bins.push_back(make_int4(i, nb[i], nb[i + 1], 0));
    return true;
}

void build(rte_ctx* ctx, const double* sigma_T, const double* sigma_a, const double* q,
           const double* eps, int eps_is_scalar, const double* inflow) {
    NvtxRange range("rte_setup");
    const int I = ctx->I, M = ctx->M, N = ctx->N, M2 = M / 2;
    const double h = 1.0 / I;
    int dev = 0;
    check(cudaGetDevice(&dev), "cudaGetDevice");
    check(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev), "attr");
    // directions and HG matrix
    std::vector<double> cdir(M), sdir(M);
    for (int m = 0; m < M; ++m) {
        const double th = 2.0 * M_PI * (m + 0.5) / M;
        cdir[m] = std::cos(th);
        sdir[m] = std::sin(th);
    }
    const std::vector<double> K = hg_matrix(M, ctx->g);
    // cell data and materials (one per distinct 1 - gamma)
    std::vector<double> tau(N), chis(N), omg(N);
    for (int c = 0; c < N; ++c) {
        const double e = eps_is_scalar ? eps[0] : eps[c];
        if (!(sigma_T[c] > 0.0) || !(sigma_a[c] > 0.0) || !(e > 0.0) || !(q[c] >= 0.0) ||
            !std::isfinite(sigma_T[c]) || !std::isfinite(sigma_a[c]) || !std::isfinite(q[c]) ||
            !std::isfinite(e))
            throw StatusError{RTE_EINVAL, "sigma_T, sigma_a, eps must be positive and finite, q >= 0"};
        tau[c] = sigma_T[c] / e * h;
        chis[c] = q[c] / sigma_a[c];
        omg[c] = e * e * sigma_a[c] / sigma_T[c];
        if (!(omg[c] < 1.0 + 1e-15))
            throw StatusError{RTE_EINVAL, "eps^2 sigma_a must not exceed sigma_T (negative scattering)"};
    }
    // the distinct values of 1 - gamma, ascending; a material's id is its rank
    std::vector<double> mvals(omg);
    std::sort(mvals.begin(), mvals.end());
    mvals.erase(std::unique(mvals.begin(), mvals.end()), mvals.end());
    ctx->nmat = (int)mvals.size();
    ctx->mat_h.resize(N);
    for (int c = 0, last = 0; c < N; ++c) {
        // cells of one material come in runs: the last id is tried first
        if (mvals[last] != omg[c])
            last = (int)(std::lower_bound(mvals.begin(), mvals.end(), omg[c]) - mvals.begin());
        ctx->mat_h[c] = last;
    }
    const int n2 = 2 * M;
    // many materials (1 - gamma varying from cell to cell): the eigenbases are
    // computed on the device, batched; a few: on the host
    const bool dev_eig = ctx->nmat > kHostEigenMaterials;
    ctx->xi_h.assign((size_t)ctx->nmat * n2, 0.0);
    if (!dev_eig) ctx->L_h.assign((size_t)ctx->nmat * M * n2, 0.0);
    // a few materials: the eigenproblems (material, axis) are independent and
    // run on host threads
    std::vector<std::vector<double>> exs, els;
    if (!dev_eig) {
        const int nt = 2 * ctx->nmat;
        std::vector<double> omv(ctx->nmat);
        for (int j = 0; j < ctx->nmat; ++j) omv[j] = std::min(mvals[j], 1.0);
        exs.resize(nt);
        els.resize(nt);
        std::vector<std::exception_ptr> errs(nt);
        std::atomic<int> next{0};
        auto work = [&]() {
            for (int t; (t = next.fetch_add(1)) < nt;) {
                try {
                    eigenbasis(M, omv[t / 2], K, t % 2 == 0 ? cdir : sdir, t % 2, exs[t], els[t]);
                } catch (...) {
                    errs[t] = std::current_exception();
                }
            }
        };
        const unsigned hw = std::thread::hardware_concurrency();
        const int nthreads = std::min<int>(nt, hw > 1 ? (int)hw : 1);
        std::vector<std::thread> pool;
        for (int w = 1; w < nthreads; ++w) pool.emplace_back(work);
        work();
        for (auto& th : pool) th.join();
        for (auto& e : errs)
            if (e) std::rethrow_exception(e);
    }
    for (int j = 0; j < ctx->nmat; ++j) {
        if (dev_eig) break;
        const std::vector<double>&xx = exs[2 * j], &Lx = els[2 * j], &xy = exs[2 * j + 1], &Ly = els[2 * j + 1];
        for (int k = 0; k < M2; ++k) {
            if (!(xx[k] < 0 && xx[M2 + k] > 0 && xy[k] < 0 && xy[M2 + k] > 0))
                throw StatusError{RTE_ESINGULAR, "eigenvalue inertia is not M/2 negative, M/2 positive"};
        }
        for (int k = 0; k < M; ++k) {
            ctx->xi_h[(size_t)j * n2 + k] = xx[k];
            ctx->xi_h[(size_t)j * n2 + M + k] = xy[k];
        }
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < M; ++k) {
                ctx->L_h[((size_t)j * M + m) * n2 + k] = Lx[(size_t)m * M + k];
                ctx->L_h[((size_t)j * M + m) * n2 + M + k] = Ly[(size_t)m * M + k];
            }
    }
    // row tables
    std::vector<int> dirs[4];
    for (int m = 0; m < M; ++m) {
        if (cdir[m] > 0) dirs[0].push_back(m); else dirs[1].push_back(m);
        if (sdir[m] > 0) dirs[2].push_back(m); else dirs[3].push_back(m);
    }
    for (int f = 0; f < 4; ++f)
        if ((int)dirs[f].size() != M2) throw StatusError{RTE_EINVAL, "direction set not symmetric"};
    std::vector<int> rowinfo(4 * M), rowdir(n2);
    for (int f = 0; f < 4; ++f) {
        for (int j = 0; j < M2; ++j) {
            rowinfo[f * M + dirs[f][j]] = j;
            rowinfo[f * M + dirs[f ^ 1][j]] = -(j + 1);
            rowdir[f * M2 + j] = dirs[f][j];
        }
    }
    std::vector<double> infl((size_t)4 * I * M, 0.0);
    if (inflow) std::memcpy(infl.data(), inflow, infl.size() * sizeof(double));
    ctx->mat = upload(ctx, ctx->mat_h);
    ctx->tau = upload(ctx, tau);
    ctx->chis = upload(ctx, chis);
    if (dev_eig) {
        const size_t nb = (size_t)ctx->nmat * M * n2;
        ctx->xi = static_cast<double*>(dev_alloc(ctx, ctx->xi_h.size() * sizeof(double)));
        ctx->L64 = static_cast<double*>(dev_alloc(ctx, nb * sizeof(double)));
        ctx->Lt64 = static_cast<double*>(dev_alloc(ctx, nb * sizeof(double)));
        ctx->Lt32 = static_cast<float*>(dev_alloc(ctx, nb * sizeof(float)));
        ctx->L32 = static_cast<float*>(dev_alloc(ctx, nb * sizeof(float)));
        std::vector<double> omv(ctx->nmat);
        for (int j = 0; j < ctx->nmat; ++j) omv[j] = std::min(mvals[j], 1.0);
        device_eigenbases(ctx, omv, K, cdir, sdir, ctx->xi, ctx->L64, ctx->Lt64, ctx->Lt32, ctx->L32);
        check(cudaMemcpyAsync(ctx->xi_h.data(), ctx->xi, ctx->xi_h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                              ctx->stream), "d2h xi");
        check(cudaStreamSynchronize(ctx->stream), "sync");
        for (int j = 0; j < ctx->nmat; ++j)
            for (int k = 0; k < M2; ++k) {
                const double* x = &ctx->xi_h[(size_t)j * n2];
                if (!(x[k] < 0 && x[M2 + k] > 0 && x[M + k] < 0 && x[M + M2 + k] > 0))
                    throw StatusError{RTE_ESINGULAR, "eigenvalue inertia is not M/2 negative, M/2 positive"};
            }
    } else {
        std::vector<double> Lt64((size_t)ctx->nmat * n2 * M);
        std::vector<float> Lt32(Lt64.size()), L32(ctx->L_h.size());
        for (int j = 0; j < ctx->nmat; ++j)
            for (int m = 0; m < M; ++m)
                for (int k = 0; k < n2; ++k) {
                    const double v = ctx->L_h[((size_t)j * M + m) * n2 + k];
                    Lt64[((size_t)j * n2 + k) * M + m] = v;
                    Lt32[((size_t)j * n2 + k) * M + m] = (float)v;
                    L32[((size_t)j * M + m) * n2 + k] = (float)v;
                }
        ctx->xi = upload(ctx, ctx->xi_h);
        ctx->L64 = upload(ctx, ctx->L_h);
        ctx->L32 = upload(ctx, L32);
        ctx->Lt64 = upload(ctx, Lt64);
        ctx->Lt32 = upload(ctx, Lt32);
    }
    ctx->rowinfo = upload(ctx, rowinfo);
    ctx->rowdir = upload(ctx, rowdir);
    ctx->inflow = upload(ctx, infl);
    // vectors and scratch
    ctx->b = static_cast<double*>(dev_alloc(ctx, ctx->n * sizeof(double)));
    ctx->trace_out = static_cast<double*>(dev_alloc(ctx, 2 * ctx->n * sizeof(double)));
    ctx->max_red_blocks = ctx->num_sms * 4;
    ctx->partials = static_cast<double*>(
        dev_alloc(ctx, (size_t)ctx->max_red_blocks * (kMaxKrylov + 1) * sizeof(double)));
    ctx->counter = static_cast<unsigned*>(dev_alloc(ctx, 64));
    ctx->scal = static_cast<double*>(dev_alloc(ctx, kScal * sizeof(double)));
    // every element of D is written by the set-up kernels
    ctx->Dt = static_cast<float*>(dev_alloc_raw(ctx, (size_t)N * 2 * n2 * n2 * sizeof(float)));
    launch_rhs(ctx);
    {
        std::vector<double> eh(N);
        for (int c = 0; c < N; ++c) eh[c] = eps_is_scalar ? eps[0] : eps[c];
        std::vector<double> sTh(sigma_T, sigma_T + N), sah(sigma_a, sigma_a + N);
        double* dsT = upload(ctx, sTh);
        double* dsa = upload(ctx, sah);
        double* de = upload(ctx, eh);
        ctx->coef_in = static_cast<float*>(dev_alloc(ctx, (size_t)4 * N * sizeof(float)));
        launch_coef_inputs(ctx, dsT, dsa, de);
    }
    int* sing = reinterpret_cast<int*>(ctx->scal + kScal - 1);
    TabPlan plan;
    if (plan_tabulation(ctx, tau, plan)) {
        ctx->tab_nodes = (int)plan.node_tau.size();
        launch_tabulated_blocks(ctx, plan, sing);
    } else {
        ctx->Rt = static_cast<float*>(dev_alloc(ctx, (size_t)N * n2 * n2 * sizeof(float)));
        ctx->rt_ready = true;
        launch_build_invert(ctx, sing);
    }
    int sing_h = 0;
    check(cudaMemcpyAsync(&sing_h, sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "d2h");
    check(cudaStreamSynchronize(ctx->stream), "setup sync");
    if (sing_h) throw StatusError{RTE_ESINGULAR, "a per-cell block has a zero pivot"};
}

}  // namespace
}  // namespace rte

using namespace rte;

#define RTE_GUARD_BEGIN try {
#define RTE_GUARD_END(ctx)                                                      \
    }                                                                           \
    catch (const CudaError& e) { return cuda_status(ctx, e.code, e.where); }   \
    catch (const StatusError& e) { set_error(ctx, e.msg); return e.code; }     \
    catch (const std::bad_alloc&) { set_error(ctx, "host allocation failed"); return RTE_ENOMEM; } \
    catch (...) { set_error(ctx, "unexpected exception"); return RTE_EINVAL; }

extern "C" {

RTE_API const char* rte_last_error(const rte_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    return g_thread_error.c_str();
}

RTE_API rte_status rte_setup(const rte_grid* grid, const rte_quadrature* quad,
                             const double* sigma_T, const double* sigma_a, const double* q,
                             const double* eps, int eps_is_scalar, double g,
                             const double* inflow, void* stream, rte_ctx** out) {
    return rte_setup_ex(grid, quad, sigma_T, sigma_a, q, eps, eps_is_scalar, g, inflow, stream, RTE_BLOCKS_AUTO,
                        out);
}

RTE_API rte_status rte_setup_ex(const rte_grid* grid, const rte_quadrature* quad,
                                const double* sigma_T, const double* sigma_a, const double* q,
                                const double* eps, int eps_is_scalar, double g,
                                const double* inflow, void* stream, int block_mode, rte_ctx** out) {
    if (!out) { set_error(nullptr, "out is NULL"); return RTE_EINVAL; }
    if (block_mode != RTE_BLOCKS_AUTO && block_mode != RTE_BLOCKS_EXACT && block_mode != RTE_BLOCKS_TABULATED) {
        set_error(nullptr, "unknown block_mode");
        return RTE_EINVAL;
    }
    *out = nullptr;
    if (!grid || !quad || !sigma_T || !sigma_a || !q || !eps) {
        set_error(nullptr, "NULL argument");
        return RTE_EINVAL;
    }
    if (grid->I < 1 || grid->I > 8192 || quad->M < 4 || quad->M % 4 != 0 || quad->M > 80) {
        set_error(nullptr, "need I in [1, 8192] and M a multiple of 4 in [4, 80]");
        return RTE_EINVAL;
    }
    if (!(std::fabs(g) < 1.0)) { set_error(nullptr, "need |g| < 1"); return RTE_EINVAL; }
    rte_ctx* ctx = new (std::nothrow) rte_ctx();
    if (!ctx) { set_error(nullptr, "host allocation failed"); return RTE_ENOMEM; }
    ctx->I = grid->I;
    ctx->M = quad->M;
    ctx->N = grid->I * grid->I;
    ctx->n = (int64_t)2 * ctx->M * ctx->N;
    ctx->g = g;
    ctx->block_mode = block_mode;
    ctx->stream = static_cast<cudaStream_t>(stream);
    static std::atomic<uint64_t> next_uid{1};
    ctx->uid = next_uid.fetch_add(1);
    rte_status st = RTE_OK;
    try {
        build(ctx, sigma_T, sigma_a, q, eps, eps_is_scalar, inflow);
    } catch (const CudaError& e) {
        st = cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        st = e.code;
    } catch (const std::bad_alloc&) {
        set_error(ctx, "host allocation failed");
        st = RTE_ENOMEM;
    }
    if (st != RTE_OK) {
        rte_destroy(ctx);
        return st;
    }
    *out = ctx;
    return RTE_OK;
}

RTE_API rte_status rte_block_setup_info(const rte_ctx* ctx, int* tabulated_nodes) {
    if (!ctx || !tabulated_nodes) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    *tabulated_nodes = ctx->tab_nodes;
    return RTE_OK;
}

RTE_API rte_status rte_set_response_path(rte_ctx* ctx, int path) {
    if (!ctx) { set_error(nullptr, "NULL context"); return RTE_EINVAL; }
    if (path != RTE_RESPONSE_AUTO && path != RTE_RESPONSE_PER_CELL) {
        set_error(ctx, "unknown response path");
        return RTE_EINVAL;
    }
    ctx->response_path = path;
    return RTE_OK;
}

RTE_API int rte_response_on_tensor_cores(const rte_ctx* ctx) {
    if (!ctx) return -1;
    return response_tc_active(ctx) ? 1 : 0;
}

RTE_API rte_status rte_info(const rte_ctx* ctx, rte_ctx_info* info) {
    if (!ctx || !info) { set_error(nullptr, "NULL argument"); return RTE_EINVAL; }
    info->I = ctx->I;
    info->M = ctx->M;
    info->N = ctx->N;
    info->nmat = ctx->nmat;
    info->n = ctx->n;
    info->device_bytes = ctx->device_bytes;
    return RTE_OK;
}

RTE_API rte_status rte_rhs(rte_ctx* ctx, double* b_dev) {
    if (!ctx || !b_dev) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    check(cudaMemcpyAsync(b_dev, ctx->b, ctx->n * sizeof(double), cudaMemcpyDeviceToDevice,
                          ctx->stream), "rhs copy");
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_apply(rte_ctx* ctx, int precision, const void* x_dev, void* y_dev) {
    if (!ctx || !x_dev || !y_dev || x_dev == y_dev) { set_error(ctx, "bad argument"); return RTE_EINVAL; }
    if (precision != RTE_F64 && precision != RTE_F32) { set_error(ctx, "bad precision"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    launch_apply(ctx, precision == RTE_F64, x_dev, y_dev, precision == RTE_F64, nullptr);
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_apply_adjoint(rte_ctx* ctx, int precision, const void* y_dev, void* x_dev) {
    if (!ctx || !x_dev || !y_dev || x_dev == y_dev) { set_error(ctx, "bad argument"); return RTE_EINVAL; }
    if (precision != RTE_F64 && precision != RTE_F32) { set_error(ctx, "bad precision"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    launch_apply_adjoint(ctx, precision == RTE_F64, y_dev, x_dev);
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_block_apply(rte_ctx* ctx, int transpose, const float* r_dev, float* z_dev) {
    if (!ctx || !r_dev || !z_dev || (const void*)r_dev == (const void*)z_dev) {
        set_error(ctx, "bad argument");
        return RTE_EINVAL;
    }
    RTE_GUARD_BEGIN
    launch_block_apply(ctx, transpose != 0, r_dev, false, z_dev, false);
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_reconstruct(rte_ctx* ctx, const double* x_dev, double* psi_dev) {
    if (!ctx || !x_dev || !psi_dev) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    launch_reconstruct(ctx, x_dev, psi_dev);
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_export_basis(const rte_ctx* ctx, double* xi, double* L, int* mat_id) {
    if (!ctx) { set_error(nullptr, "NULL ctx"); return RTE_EINVAL; }
    if (xi) std::memcpy(xi, ctx->xi_h.data(), ctx->xi_h.size() * sizeof(double));
    if (L && !ctx->L_h.empty()) {
        std::memcpy(L, ctx->L_h.data(), ctx->L_h.size() * sizeof(double));
    } else if (L) {                      // bases computed on the device
        const size_t nb = (size_t)ctx->nmat * ctx->M * 2 * ctx->M;
        if (cudaMemcpy(L, ctx->L64, nb * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error(nullptr, "cudaMemcpy (bases)");
            return RTE_ECUDA;
        }
    }
    if (mat_id) std::memcpy(mat_id, ctx->mat_h.data(), ctx->mat_h.size() * sizeof(int));
    return RTE_OK;
}

RTE_API rte_status rte_export_blocks(rte_ctx* ctx, double* D_host, float* R_host) {
    if (!ctx || (!D_host && !R_host)) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    const size_t n2 = 2 * (size_t)ctx->M, per = n2 * n2;
    if (D_host) {
        std::vector<float> tmp(2 * per * ctx->N);
        check(cudaMemcpyAsync(tmp.data(), ctx->Dt, tmp.size() * sizeof(float),
                              cudaMemcpyDeviceToHost, ctx->stream), "export blocks");
        check(cudaStreamSynchronize(ctx->stream), "export sync");
        for (int c = 0; c < ctx->N; ++c) {
            const float* hi = tmp.data() + 2 * c * per;
            const float* lo = hi + per;
            for (size_t j = 0; j < n2; ++j)
                for (size_t i = 0; i < n2; ++i)
                    D_host[c * per + i * n2 + j] = (double)hi[j * n2 + i] + (double)lo[j * n2 + i];
        }
    }
    if (R_host) {
        ensure_cell_response(ctx);
        std::vector<float> tmp(per * ctx->N);
        check(cudaMemcpyAsync(tmp.data(), ctx->Rt, tmp.size() * sizeof(float),
                              cudaMemcpyDeviceToHost, ctx->stream), "export response");
        check(cudaStreamSynchronize(ctx->stream), "export sync");
        for (int c = 0; c < ctx->N; ++c)
            for (size_t i = 0; i < n2; ++i)
                for (size_t r = 0; r < n2; ++r) R_host[c * per + r * n2 + i] = tmp[c * per + i * n2 + r];
    }
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_response_apply(rte_ctx* ctx, const double* v_dev, double* w_dev) {
    if (!ctx || !v_dev || !w_dev || v_dev == w_dev) { set_error(ctx, "bad argument"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    launch_response_apply(ctx, v_dev, true, w_dev, true);
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_cgs2(rte_ctx* ctx, const double* V_dev, int k, double* w_dev, double* h_dev) {
    if (!ctx || !V_dev || !w_dev || !h_dev || k < 1 || k > kMaxKrylov) {
        set_error(ctx, "bad argument (need 1 <= k <= 64)");
        return RTE_EINVAL;
    }
    RTE_GUARD_BEGIN
    double* h1 = ctx->scal;                 // [64] first projection
    double* h2 = ctx->scal + kMaxKrylov;    // [64] second projection
    launch_mdot(ctx, V_dev, k, w_dev, h1);
    launch_update_dot(ctx, V_dev, k, w_dev, h1, h2);
    launch_update_norm(ctx, V_dev, k, w_dev, h1, h2, h_dev);  // h1 + h2, then ||w||
    launch_scale(ctx, w_dev, h_dev + k, w_dev);
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_cgs2_df64(rte_ctx* ctx, const float* V_dev, int k, float* w_dev, double* h_dev) {
    if (!ctx || !V_dev || !w_dev || !h_dev || k < 1 || k > kMaxKrylov) {
        set_error(ctx, "bad argument (need 1 <= k <= 64)");
        return RTE_EINVAL;
    }
    RTE_GUARD_BEGIN
    double* h1 = ctx->scal;                 // [64] first projection
    double* h2 = ctx->scal + kMaxKrylov;    // [64] second projection
    launch_orthogonalise_df(ctx, V_dev, k, w_dev, h1, h2, h_dev);
    launch_scale_df(ctx, w_dev, h_dev + k, w_dev);
    if (const char* why = device_wait_expired()) throw StatusError{RTE_ETIMEOUT, why};
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API rte_status rte_eigenbasis(int M, double g, double one_minus_gamma, int axis, double* xi,
                                  double* L) {
    if (M < 4 || M % 4 != 0 || M > 112 || !(std::fabs(g) < 1.0) || !(one_minus_gamma > 0.0) ||
        !(one_minus_gamma <= 1.0) || (axis != 0 && axis != 1) || !xi || !L) {
        set_error(nullptr, "bad argument");
        return RTE_EINVAL;
    }
    RTE_GUARD_BEGIN
    std::vector<double> d(M), x, Lv;
    for (int m = 0; m < M; ++m) {
        const double th = 2.0 * M_PI * (m + 0.5) / M;
        d[m] = axis == 0 ? std::cos(th) : std::sin(th);
    }
    eigenbasis(M, one_minus_gamma, hg_matrix(M, g), d, axis, x, Lv);
    std::memcpy(xi, x.data(), M * sizeof(double));
    std::memcpy(L, Lv.data(), (size_t)M * M * sizeof(double));
    return RTE_OK;
    RTE_GUARD_END(nullptr)
}

RTE_API rte_status rte_profile(rte_ctx* ctx, int enable) {
    if (!ctx) { set_error(nullptr, "NULL ctx"); return RTE_EINVAL; }
    RTE_GUARD_BEGIN
    check(cudaStreamSynchronize(ctx->stream), "profile sync");
    prof_resolve(ctx);
    for (int k = 0; k < K_COUNT; ++k) {
        ctx->prof.ms[k] = 0.0;
        ctx->prof.bytes[k] = 0.0;
        ctx->prof.flops[k] = 0.0;
        ctx->prof.launches[k] = 0;
    }
    ctx->prof.on = enable != 0;
    return RTE_OK;
    RTE_GUARD_END(ctx)
}

RTE_API int rte_profile_read(rte_ctx* ctx, rte_kernel_stat* out, int max) {
    if (!ctx) return -1;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return -1;
    prof_resolve(ctx);
    int n = 0;
    for (int k = 0; k < K_COUNT && n < max; ++k) {
        if (!out) break;
        out[n].name = kKernelNames[k];
        out[n].launches = ctx->prof.launches[k];
        out[n].ms = ctx->prof.ms[k];
        out[n].bytes = ctx->prof.bytes[k];
        out[n].flops = ctx->prof.flops[k];
        ++n;
    }
    return out ? n : K_COUNT;
}

RTE_API rte_status rte_trim_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& kv : g_pools) {
        const cudaError_t e = cudaMemPoolTrimTo(kv.second, 0);
        if (e != cudaSuccess) return cuda_status(nullptr, e, "cudaMemPoolTrimTo");
    }
    return RTE_OK;
}

RTE_API void rte_destroy(rte_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_workspace(ctx);
    atfps_free(ctx);
    prof_free(ctx);
    for (void* p : ctx->allocations) cudaFreeAsync(p, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
}

}  // extern "C"
