// rte_solve: flexible GMRES(restart) for A alpha = b, right-preconditioned by
// block Jacobi, and optionally by the MgNet V-cycle on top.
//
// The Krylov iteration works in face-flux space on B = A D (D = blockdiag
// G_C^{-1}, block Jacobi, Sec. 4): B v = v - P R v with the per-cell response
// matrices R_C = T_out D_C in FP32.  R is a bounded transfer map, so FP32
// keeps B accurate, whereas alpha = D y itself cancels heavily in the
// diffusive limit and needs FP64.  Per Arnoldi step j:
//   z_j = Net(v_j)  (MgNet, in face-flux space)  or  z_j = v_j
//   w   = B z_j                                   FP32 products, FP64 vectors
//   CGS2: h = V^T w twice, w /= ||w|| -> v_{j+1}  (FP64)
//   Givens update of the Hessenberg column         (FP64, one thread)
// The host reads only the residual estimate after each step.  At the end of a
// cycle y = H^{-1} g, dy = Z y, alpha += D dy (FP64), and the true residual
// r = b - A alpha is recomputed in FP64: it alone decides convergence
// (iterative refinement around the FP32 inner operator).  With
// inner_precision = RTE_F64 the inner operator is instead A (D z) with the
// FP64 trace kernel.
#include <chrono>
#include <cmath>

#include "rte_internal.h"
#include "mgnet_internal.h"

namespace rte {

struct Workspace {
    int m = 0;
    double* V = nullptr;      // [(m+1)][n]
    float* Z = nullptr;       // [m][n]
    double* w = nullptr;      // [n]
    double* tmp = nullptr;    // [n] FP64 copy of z for FP64 inner applies
    double* H = nullptr;      // [(m+1) * m] column-major, ld = m+1
    double* cs = nullptr;     // [m]
    double* sn = nullptr;     // [m]
    double* g = nullptr;      // [m+1]
    double* y = nullptr;      // [m]
    double* h1 = nullptr;     // [m+1]
    double* h2 = nullptr;     // [m+1]
    double* hcol = nullptr;   // [m+2]
    double* est = nullptr;    // [4] device status: est, beta, bnorm
    double* est_host = nullptr;   // pinned [4]
    std::vector<void*> allocs;
    size_t bytes = 0;
};

void free_workspace(rte_ctx* ctx) {
    if (!ctx || !ctx->ws) return;
    for (void* p : ctx->ws->allocs) cudaFreeAsync(p, ctx->stream);
    if (ctx->ws->est_host) cudaFreeHost(ctx->ws->est_host);
    ctx->device_bytes -= ctx->ws->bytes;
    delete ctx->ws;
    ctx->ws = nullptr;
}

namespace {

template <typename T>
T* ws_alloc(rte_ctx* ctx, Workspace* ws, size_t count) {
    void* p = nullptr;
    const size_t bytes = count * sizeof(T) + 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) throw CudaError{e, "cudaMallocAsync (solve workspace)"};
    ws->allocs.push_back(p);
    ws->bytes += bytes;
    ctx->device_bytes += bytes;
    check(cudaMemsetAsync(p, 0, bytes, ctx->stream), "memset workspace");
    return static_cast<T*>(p);
}

Workspace* get_workspace(rte_ctx* ctx, int m) {
    if (ctx->ws && ctx->ws->m == m) return ctx->ws;
    free_workspace(ctx);
    Workspace* ws = new Workspace();
    ctx->ws = ws;
    ws->m = m;
    const size_t n = (size_t)ctx->n;
    ws->V = ws_alloc<double>(ctx, ws, (size_t)(m + 1) * n);
    ws->Z = ws_alloc<float>(ctx, ws, (size_t)m * n);    // MgNet outputs (flexible GMRES)
    ws->w = ws_alloc<double>(ctx, ws, n);
    ws->tmp = ws_alloc<double>(ctx, ws, n);
    ws->H = ws_alloc<double>(ctx, ws, (size_t)(m + 1) * m);
    ws->cs = ws_alloc<double>(ctx, ws, m);
    ws->sn = ws_alloc<double>(ctx, ws, m);
    ws->g = ws_alloc<double>(ctx, ws, m + 1);
    ws->y = ws_alloc<double>(ctx, ws, m);
    ws->h1 = ws_alloc<double>(ctx, ws, m + 1);
    ws->h2 = ws_alloc<double>(ctx, ws, m + 1);
    ws->hcol = ws_alloc<double>(ctx, ws, m + 2);
    ws->est = ws_alloc<double>(ctx, ws, 4);
    check(cudaMallocHost(&ws->est_host, 4 * sizeof(double)), "cudaMallocHost");
    return ws;
}

// Orthogonalises w against V[0..K) (orthonormal) by classical Gram-Schmidt
// with one reorthogonalisation in three passes over V, leaving
// ws->hcol = [h1 + h2, ||w||] and the projected (unnormalised) vector in w.
// On the diffusive workloads the second projection is needed at almost every
// step (the first removes more than half of w's squared length at 98% of the
// steps), so it is always done.
void orthogonalise(rte_ctx* ctx, Workspace* ws, const double* V, int K) {
    launch_mdot(ctx, V, K, ws->w, ws->h1);
    launch_update_dot(ctx, V, K, ws->w, ws->h1, ws->h2);
    launch_update_norm(ctx, V, K, ws->w, ws->h1, ws->h2, ws->hcol);
}

// Start of a cycle: g = (beta, 0, ...), H = 0.
__global__ void k_cycle_start(int m, const double* __restrict__ beta, double* H, double* g) {
    for (int i = threadIdx.x; i < (m + 1) * m; i += blockDim.x) H[i] = 0.0;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta[0] : 0.0;
}

// Hessenberg column j: apply the previous rotations, make a new one, update g.
__global__ void k_givens(int j, int m, const double* __restrict__ hcol, double* H, double* cs,
                         double* sn, double* g, double* est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* col = H + (size_t)j * (m + 1);
    for (int i = 0; i <= j + 1; ++i) col[i] = hcol[i];
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    double c = 1.0, s = 0.0;
    if (b != 0.0) {
        const double r = hypot(a, b);
        c = a / r;
        s = b / r;
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = c * a + s * b;
    col[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    est[0] = fabs(g[j + 1]);
    est[1] = hcol[j + 1];         // ||w|| before normalisation (breakdown test)
}

// y = H(0:k,0:k)^{-1} g(0:k)  (upper triangular)
__global__ void k_backsub(int k, int m, const double* __restrict__ H, const double* __restrict__ g,
                          double* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
        y[i] = s / H[(size_t)i * (m + 1) + i];
    }
}

__global__ void k_f2d(const float* __restrict__ x, int64_t n, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// out = sum_k Z[k] y[k]   (Z float or double)
template <typename TZ>
__global__ void k_lincomb(const TZ* __restrict__ Z, int K, int64_t n, const double* __restrict__ y,
                          double* __restrict__ out) {
    __shared__ double sy[kMaxKrylov];
    for (int k = threadIdx.x; k < K; k += blockDim.x) sy[k] = y[k];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s = fma((double)Z[(size_t)k * n + i], sy[k], s);
        out[i] = s;
    }
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

__global__ void k_isfinite_f(const float* __restrict__ x, int64_t n, int* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) { *flag = 1; return; }
}

double read_scalar(rte_ctx* ctx, Workspace* ws, const double* dev) {
    check(cudaMemcpyAsync(ws->est_host, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
          "d2h scalar");
    check(cudaStreamSynchronize(ctx->stream), "sync");
    return ws->est_host[0];
}

}  // namespace
}  // namespace rte

using namespace rte;

extern "C" {

RTE_API void rte_solve_opts_default(rte_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-8;
    o->restart = 50;
    o->max_iter = 20000;
    o->inner_precision = RTE_F32;
    o->use_x0 = 0;
    o->stall_ratio = 0.9;
    o->timeout_ms = 0.0;
    o->cancel = nullptr;
}

RTE_API rte_status rte_arnoldi_basis(rte_ctx* ctx, int k, double* V_dev) {
    if (!ctx || !V_dev || k < 1 || k > kMaxKrylov) { set_error(ctx, "bad argument (1 <= k <= 64)"); return RTE_EINVAL; }
    try {
        Workspace* ws = get_workspace(ctx, ctx->ws ? ctx->ws->m : kMaxKrylov);
        if (ws->m < k) ws = get_workspace(ctx, kMaxKrylov);
        const int64_t n = ctx->n;
        launch_norm(ctx, ctx->b, ws->est + 3);
        launch_scale(ctx, ctx->b, ws->est + 3, V_dev);
        for (int j = 0; j + 1 < k; ++j) {
            launch_response_apply(ctx, V_dev + (size_t)j * n, true, ws->w, true);
            const int K = j + 1;
            orthogonalise(ctx, ws, V_dev, K);
            launch_scale(ctx, ws->w, ws->hcol + K, V_dev + (size_t)(j + 1) * n);
        }
        check(cudaStreamSynchronize(ctx->stream), "sync");
    } catch (const CudaError& e) {
        return cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        return e.code;
    }
    return RTE_OK;
}

RTE_API rte_status rte_solve(rte_ctx* ctx, mgnet* pc, const rte_solve_opts* opts_in,
                             double* x_dev, rte_solve_info* info) {
    if (!ctx || !x_dev) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    rte_solve_opts opts;
    if (opts_in) opts = *opts_in; else rte_solve_opts_default(&opts);
    if (opts.restart < 1 || opts.restart > kMaxKrylov || !(opts.tol > 0.0) || opts.max_iter < 0 ||
        (opts.inner_precision != RTE_F32 && opts.inner_precision != RTE_F64)) {
        set_error(ctx, "bad solve options (restart in [1, 64], tol > 0)");
        return RTE_EINVAL;
    }
    rte_solve_info inf{};
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed_ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    rte_status status = RTE_OK;
    try {
        if (pc) mgnet_prepare(pc, ctx);
        const int m = opts.restart;
        Workspace* ws = get_workspace(ctx, m);
        const int64_t n = ctx->n;
        const int gblk = ctx->num_sms * 4;
        if (!opts.use_x0) check(cudaMemsetAsync(x_dev, 0, n * sizeof(double), ctx->stream), "zero x");
        launch_norm(ctx, ctx->b, ws->est + 2);
        const double bnorm = read_scalar(ctx, ws, ws->est + 2);
        if (bnorm == 0.0) {
            check(cudaMemsetAsync(x_dev, 0, n * sizeof(double), ctx->stream), "zero x");
            inf.converged = 1;
            inf.relres = 0.0;
            inf.seconds = elapsed_ms() * 1e-3;
            if (info) *info = inf;
            return RTE_OK;
        }
        bool use_net = (pc != nullptr);
        double prev_res = -1.0;
        bool first = true;
        while (true) {
            // true residual in FP64
            if (first && !opts.use_x0)
                check(cudaMemcpyAsync(ws->w, ctx->b, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                      ctx->stream), "r = b");
            else
                launch_apply(ctx, true, x_dev, ws->w, true, ctx->b);
            first = false;
            launch_norm(ctx, ws->w, ws->est + 3);
            const double beta = read_scalar(ctx, ws, ws->est + 3);
            inf.relres = beta / bnorm;
            if (!std::isfinite(beta)) {
                set_error(ctx, "non-finite residual");
                status = RTE_ESTALL;
                break;
            }
            if (use_net && prev_res > 0.0 && inf.relres > opts.stall_ratio * prev_res) {
                use_net = false;          // the learned preconditioner stalled
                inf.fell_back = 1;
            }
            prev_res = inf.relres;
            if (inf.relres <= opts.tol) { inf.converged = 1; break; }
            if (inf.iterations >= opts.max_iter) { status = RTE_ENOTCONV; break; }
            if (opts.timeout_ms > 0 && elapsed_ms() > opts.timeout_ms) { status = RTE_ETIMEOUT; break; }
            if (opts.cancel && *opts.cancel) {
                set_error(ctx, "cancelled");
                status = RTE_ECANCELLED;
                break;
            }
            launch_scale(ctx, ws->w, ws->est + 3, ws->V);
            {
                ProfScope ps(ctx, K_CYCLE, 0.0);
                k_cycle_start<<<1, 256, 0, ctx->stream>>>(m, ws->est + 3, ws->H, ws->g);
                check(cudaGetLastError(), "k_cycle_start");
            }
            const bool cycle_net = use_net;
            int k = 0;
            for (int j = 0; j < m; ++j) {
                const double* vj = ws->V + (size_t)j * n;
                const void* zj = vj;
                bool z_double = true;
                if (cycle_net) {
                    float* zf = ws->Z + (size_t)j * n;
                    mgnet_precondition(pc, ctx, vj, zf);
                    zj = zf;
                    z_double = false;
                }
                if (opts.inner_precision == RTE_F32) {
                    launch_response_apply(ctx, zj, z_double, ws->w, true);
                } else {
                    launch_block_apply(ctx, false, zj, z_double, ws->tmp, true);
                    launch_apply(ctx, true, ws->tmp, ws->w, true, nullptr);
                }
                const int K = j + 1;
                orthogonalise(ctx, ws, ws->V, K);
                launch_scale(ctx, ws->w, ws->hcol + K, ws->V + (size_t)(j + 1) * n);
                {
                    ProfScope ps(ctx, K_GIVENS, 0.0);
                    k_givens<<<1, 32, 0, ctx->stream>>>(j, m, ws->hcol, ws->H, ws->cs, ws->sn,
                                                         ws->g, ws->est);
                    check(cudaGetLastError(), "k_givens");
                }
                check(cudaMemcpyAsync(ws->est_host, ws->est, 2 * sizeof(double),
                                      cudaMemcpyDeviceToHost, ctx->stream), "d2h est");
                check(cudaStreamSynchronize(ctx->stream), "step sync");
                prof_resolve(ctx);
                ++inf.iterations;
                k = j + 1;
                const double est = ws->est_host[0], wn = ws->est_host[1];
                if (!std::isfinite(est)) {
                    if (use_net) { use_net = false; inf.fell_back = 1; }
                    k = j;           // drop the bad column
                    break;
                }
                if (est / bnorm <= opts.tol || wn == 0.0 || inf.iterations >= opts.max_iter) break;
                if (opts.timeout_ms > 0 && elapsed_ms() > opts.timeout_ms) break;
                if (opts.cancel && *opts.cancel) break;
            }
            if (k > 0) {
                {
                    ProfScope ps(ctx, K_BACKSUB, 0.0);
                    k_backsub<<<1, 32, 0, ctx->stream>>>(k, m, ws->H, ws->g, ws->y);
                    check(cudaGetLastError(), "k_backsub");
                }
                {
                    ProfScope ps(ctx, K_XUPDATE, (double)n * (8 + (cycle_net ? 4 : 8) * k));
                    if (cycle_net)
                        k_lincomb<float><<<gblk, 256, 0, ctx->stream>>>(ws->Z, k, n, ws->y, ws->tmp);
                    else
                        k_lincomb<double><<<gblk, 256, 0, ctx->stream>>>(ws->V, k, n, ws->y, ws->tmp);
                    check(cudaGetLastError(), "k_lincomb");
                }
                launch_block_apply(ctx, false, ws->tmp, true, ws->w, true);   // D dy
                {
                    ProfScope ps(ctx, K_XUPDATE, (double)n * 24);
                    k_axpy<<<gblk, 256, 0, ctx->stream>>>(x_dev, ws->w, n);
                    check(cudaGetLastError(), "k_axpy");
                }
            }
            ++inf.cycles;
        }
    } catch (const CudaError& e) {
        status = cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        status = e.code;
    } catch (const std::bad_alloc&) {
        set_error(ctx, "host allocation failed");
        status = RTE_ENOMEM;
    }
    inf.seconds = elapsed_ms() * 1e-3;
    if (info) *info = inf;
    return status;
}

}  // extern "C"
