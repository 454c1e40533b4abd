// rte_solve: flexible GMRES(restart) for A alpha = b, right-preconditioned by
// block Jacobi, and optionally by the MgNet V-cycle on top.
//
// The Krylov iteration works in face-flux space on B = A D (D = blockdiag
// G_C^{-1}, block Jacobi, Sec. 4): B v = v - P R v with the per-cell response
// matrices R_C = T_out D_C in FP32.  R is a bounded transfer map, so FP32
// keeps B accurate, whereas alpha = D y itself cancels heavily in the
// diffusive limit and needs FP64.  Per Arnoldi step j:
//   z_j = Net(v_j)  (MgNet, in face-flux space)  or  z_j = v_j
//   w   = B z_j                                   FP32 products, df64 w
//   CGS2: h = V^T w twice, w /= ||w|| -> v_{j+1}  (df64 vectors, FP64 h)
//   Givens update of the Hessenberg column         (FP64, one thread)
// The Krylov vectors V and w are df64 (df64.h: a float pair, 48 significant
// bits): the Gram-Schmidt passes then stream at the memory bound on the FP32
// pipe, where FP64 vectors would be bound by this GPU's narrow FP64 pipe.
// The host reads only the residual estimate after each step.  At the end of a
// cycle y = H^{-1} g, dy = Z y, alpha += D dy (FP64), and the true residual
// r = b - A alpha is recomputed in FP64: it alone decides convergence
// (iterative refinement around the FP32 inner operator).  With
// inner_precision = RTE_F64 the inner operator is instead A (D z) with the
// FP64 trace kernel.
#include <chrono>
#include <cmath>

#include "df64.h"
#include "rte_internal.h"
#include "mgnet_internal.h"

namespace rte {

struct Workspace {
    int m = 0;
    float* V = nullptr;       // [(m+1)][2][n] df64 Krylov basis (hi plane, lo plane)
    float* Z = nullptr;       // [m][n] network outputs (flexible GMRES)
    float* w = nullptr;       // [2][n] df64 vector being orthogonalised
    double* w64 = nullptr;    // [n] FP64 residual / FP64 operator output
    double* tmp = nullptr;    // [n] FP64 scratch (D z, Z y)
    double* tmp2 = nullptr;   // [n] FP64 copy of a df64 Krylov vector
    double* H = nullptr;      // [(m+1) * m] column-major, ld = m+1
    double* cs = nullptr;     // [m]
    double* sn = nullptr;     // [m]
    double* g = nullptr;      // [m+1]
    double* y = nullptr;      // [m]
    double* h1 = nullptr;     // [m+1]
    double* h2 = nullptr;     // [m+1]
    double* hcol = nullptr;   // [m+2]
    // deferred Gram-Schmidt: betas[i] = beta_{i-1} (betas[0] = 1), the
    // coefficients that fix the next row (the last step's h2), and
    // U[(j) (m+1) + i] = h2_{j-1}[i] / beta_{j-1} for the V-based update
    double* betas = nullptr;  // [m+1]
    double* cfix = nullptr;   // [m+1]
    double* U = nullptr;      // [(m+1) (m+1)]
    double* est = nullptr;    // [4] device status: est, beta, bnorm
    double* est_host = nullptr;   // pinned [4]
    cudaEvent_t est_ready = nullptr;   // the step's estimate has reached est_host
    std::vector<void*> allocs;
    size_t bytes = 0;
};

void free_workspace(rte_ctx* ctx) {
    if (!ctx || !ctx->ws) return;
    for (void* p : ctx->ws->allocs) cudaFreeAsync(p, ctx->stream);
    if (ctx->ws->est_host) cudaFreeHost(ctx->ws->est_host);
    if (ctx->ws->est_ready) cudaEventDestroy(ctx->ws->est_ready);
    ctx->device_bytes -= ctx->ws->bytes;
    delete ctx->ws;
    ctx->ws = nullptr;
}

namespace {

template <typename T>
T* ws_alloc(rte_ctx* ctx, Workspace* ws, size_t count) {
    void* p = nullptr;
    const size_t bytes = count * sizeof(T) + 16;
    cudaError_t e = pool_malloc(&p, bytes, ctx->stream);
    if (e != cudaSuccess) throw CudaError{e, "cudaMallocFromPoolAsync (solve workspace)"};
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
    ws->V = ws_alloc<float>(ctx, ws, (size_t)(m + 1) * 2 * n);
    ws->Z = ws_alloc<float>(ctx, ws, (size_t)m * n);    // MgNet outputs (flexible GMRES)
    ws->w = ws_alloc<float>(ctx, ws, 2 * n);
    ws->w64 = ws_alloc<double>(ctx, ws, n);
    ws->tmp = ws_alloc<double>(ctx, ws, n);
    ws->tmp2 = ws_alloc<double>(ctx, ws, n);
    ws->H = ws_alloc<double>(ctx, ws, (size_t)(m + 1) * m);
    ws->cs = ws_alloc<double>(ctx, ws, m);
    ws->sn = ws_alloc<double>(ctx, ws, m);
    ws->g = ws_alloc<double>(ctx, ws, m + 1);
    ws->y = ws_alloc<double>(ctx, ws, m);
    ws->h1 = ws_alloc<double>(ctx, ws, m + 1);
    ws->h2 = ws_alloc<double>(ctx, ws, m + 1);
    ws->hcol = ws_alloc<double>(ctx, ws, m + 2);
    ws->betas = ws_alloc<double>(ctx, ws, m + 1);
    ws->cfix = ws_alloc<double>(ctx, ws, m + 1);
    ws->U = ws_alloc<double>(ctx, ws, (size_t)(m + 1) * (m + 1));
    ws->est = ws_alloc<double>(ctx, ws, 4);
    check(cudaMallocHost(&ws->est_host, 4 * sizeof(double)), "cudaMallocHost");
    check(cudaEventCreateWithFlags(&ws->est_ready, cudaEventDisableTiming), "cudaEventCreate");
    return ws;
}

// FP64 Arnoldi orthogonalisation of the double vector w against V[0..K)
// (rte_arnoldi_basis): classical Gram-Schmidt with one reorthogonalisation in
// three passes, leaving ws->hcol = [h1 + h2, ||w||] and the projected
// (unnormalised) vector in w.
void orthogonalise64(rte_ctx* ctx, Workspace* ws, const double* V, int K, double* w) {
    launch_mdot(ctx, V, K, w, ws->h1);
    launch_update_dot(ctx, V, K, w, ws->h1, ws->h2);
    launch_update_norm(ctx, V, K, w, ws->h1, ws->h2, ws->hcol);
}

// Start of a cycle: g = (beta, 0, ...), H = 0, betas[0] = 1 (v_0 is final).
__global__ void k_cycle_start(int m, const double* __restrict__ beta, double* H, double* g, double* betas) {
    for (int i = threadIdx.x; i < (m + 1) * m; i += blockDim.x) H[i] = 0.0;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta[0] : 0.0;
    if (threadIdx.x == 0) betas[0] = 1.0;
}

// Hessenberg column j: apply the previous rotations, make a new one, update g.
__device__ void givens_run(int j, int m, const double* __restrict__ hcol, double* H, double* cs, double* sn,
                           double* g, double* est) {
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

__global__ void k_givens(int j, int m, const double* __restrict__ hcol, double* H, double* cs,
                         double* sn, double* g, double* est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    givens_run(j, m, hcol, H, cs, sn, g, est);
}

// Column j of the deferred Gram-Schmidt (launch_cgs2_deferred_df): the step
// orthogonalised w = B z_j with z_j = M(u_j), u_j = beta_{j-1} v_j + V c, so
// the flexible-GMRES column of zhat_j = z_j / beta_{j-1} is
//   (h1 + h2, beta_j) / beta_{j-1},  beta_j^2 = ||w'||^2 - ||h2||^2
// (Pythagoras: h2 is the small second projection).  Keeps beta_j and h2 to
// fix row j + 1 in the next step, and h2 / beta_j as column j + 1 of U; then
// the Givens update of column j.  One warp: the lanes stage the column and
// the previous rotations in shared memory, lane 0 applies the rotations.
__device__ void column_run(int j, int m, const double* __restrict__ h1, const double* __restrict__ h2nu,
                           double* betas, double* cfix, double* U, double* hcol, double* H, double* cs,
                           double* sn, double* g, double* est) {
    __shared__ double col[kMaxKrylov + 2], scs[kMaxKrylov], ssn[kMaxKrylov];
    __shared__ double s_bj;
    const int lane = threadIdx.x & 31, K = j + 1;
    const double bprev = betas[j];
    double part = 0.0;
    for (int i = lane; i < K; i += 32) {
        const double b2 = h2nu[i];
        part += b2 * b2;
        const double c = (h1[i] + b2) / bprev;
        hcol[i] = c;
        col[i] = c;
        cfix[i] = b2;
    }
    for (int i = lane; i < j; i += 32) {
        scs[i] = cs[i];
        ssn[i] = sn[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) {
        const double d = h2nu[K] - part;
        const double bj = d > 0.0 ? sqrt(d) : (d <= 0.0 ? 0.0 : d);     // a NaN step stays NaN
        s_bj = bj;
        betas[j + 1] = bj;
        hcol[K] = bj / bprev;
        col[K] = bj / bprev;
    }
    __syncwarp();
    const double bj = s_bj;
    for (int i = lane; i < K; i += 32) U[(size_t)(j + 1) * (m + 1) + i] = bj > 0.0 ? h2nu[i] / bj : 0.0;
    if (lane == 0) {
        for (int i = 0; i < j; ++i) {
            const double t = scs[i] * col[i] + ssn[i] * col[i + 1];
            col[i + 1] = -ssn[i] * col[i] + scs[i] * col[i + 1];
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
        est[1] = bj / bprev;          // the new vector's length before normalisation (breakdown test)
    }
    __syncwarp();
    double* Hc = H + (size_t)j * (m + 1);
    for (int i = lane; i <= K; i += 32) Hc[i] = col[i];
}

__global__ void k_column_givens(int j, int m, const double* __restrict__ h1, const double* __restrict__ h2nu,
                                double* betas, double* cfix, double* U, double* hcol, double* H, double* cs,
                                double* sn, double* g, double* est) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    column_run(j, m, h1, h2nu, betas, cfix, U, hcol, H, cs, sn, g, est);
}

// The update's coefficients for the stored vectors of a deferred cycle of k
// columns: the network outputs z_j take y_j / beta_{j-1}; the final Krylov
// vectors v_i take y_i + sum_{j > i} U[j][i] y_j (zhat_j = v_j + V U[j]).
// tmp: k doubles of scratch.
__global__ void k_deferred_y(int k, int m, bool net, const double* __restrict__ betas,
                             const double* __restrict__ U, double* y, double* tmp) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (net) {
        for (int i = 0; i < k; ++i) y[i] /= betas[i];
        return;
    }
    for (int i = 0; i < k; ++i) {
        double s = y[i];
        for (int j = i + 1; j < k; ++j) s += U[(size_t)j * (m + 1) + i] * y[j];
        tmp[i] = s;
    }
    for (int i = 0; i < k; ++i) y[i] = tmp[i];
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

// out = sum_k Z[k] y[k] for the FP32 network outputs Z: the products of z and
// the df64 y_k exact to about 2^-47 (TwoProd), summed in df64 (TwoSum), two
// elements a packed instruction and renormalised every 8 terms -- the
// accuracy of an FP64 sum of the K terms, with the kernel bound by HBM rather
// than by the FP64 pipe.  n = 2 M N is even.
__global__ void __launch_bounds__(256) k_lincomb_z(const float* __restrict__ Z, int K, int64_t n,
                                                   const double* __restrict__ y, double* __restrict__ out) {
    using df::f2;
    __shared__ f2 sb[kMaxKrylov][3];           // (h, h), (-h, -h), (-l, -l) of y_k = h + l
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float h, l;
        df::from_double(y[k], h, l);
        sb[k][0] = df::pk(h, h);
        sb[k][1] = df::pk(-h, -h);
        sb[k][2] = df::pk(-l, -l);
    }
    __syncthreads();
    const int64_t np = n / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        f2 S = 0ull, C = 0ull;
        int k = 0;
        for (; k + 8 <= K; k += 8) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 z = __ldg(reinterpret_cast<const float2*>(Z + (size_t)(k + q) * n) + i);
                df::mac2(S, C, df::pk(z.x, z.y), 0ull, sb[k + q][1], sb[k + q][2], sb[k + q][0]);
            }
            df::renorm2(S, C);
        }
        for (; k < K; ++k) {
            const float2 z = __ldg(reinterpret_cast<const float2*>(Z + (size_t)k * n) + i);
            df::mac2(S, C, df::pk(z.x, z.y), 0ull, sb[k][1], sb[k][2], sb[k][0]);
        }
        df::renorm2(S, C);
        float sx, sy, cx, cy;
        df::upk(S, sx, sy);
        df::upk(C, cx, cy);
        reinterpret_cast<double2*>(out)[i] = make_double2(df::to_double(sx, cx), df::to_double(sy, cy));
    }
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

double read_scalar(rte_ctx* ctx, Workspace* ws, const double* dev) {
    check(cudaMemcpyAsync(ws->est_host, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
          "d2h scalar");
    check(cudaStreamSynchronize(ctx->stream), "sync");
    return ws->est_host[0];
}

// Hessenberg column j: apply the previous rotations, make a new one, update
// g; one block per item of a grouped Arnoldi step.
__global__ void k_givens_group(const GroupItem* __restrict__ items) {
    if (threadIdx.x >= 32) return;
    const GroupItem& it = items[blockIdx.x];
    column_run(it.j, it.m, it.h1, it.h2, it.betas, const_cast<double*>(it.cfix), it.U, it.hcol, it.H, it.cs, it.sn,
               it.g, it.est);
    if (threadIdx.x == 0) {
        it.est_out[0] = it.est[0];
        it.est_out[1] = it.est[1];
    }
}

// One flexible-GMRES solve as a sequence of phases, so that several solves can
// advance in lockstep with their Arnoldi steps in shared launches
// (rte_solve_group); rte_solve runs the same phases for one solve.
struct Solver {
    rte_ctx* ctx = nullptr;
    mgnet* pc = nullptr;
    rte_solve_opts opts{};
    double* x = nullptr;
    rte_solve_info inf{};
    rte_status status = RTE_OK;
    Workspace* ws = nullptr;
    int m = 0, gblk = 0;
    int64_t n = 0;
    double bnorm = 0.0, prev_res = -1.0;
    bool use_net = false, first = true, cycle_net = false;
    // compressed ATFPS system (Eq. 2DAdaptiveTFPS_linear_sys) in slot layout:
    // operator A_bar (mask o D S), right-hand side b_bar, FP64 throughout, no network
    bool comp = false;
    const double* rhs = nullptr;
    int j = 0, k = 0;                 // Arnoldi step in the cycle; columns for the cycle end
    const float* zj = nullptr;        // z_j: the network output, or the hi plane of v_j
    const float* zj_lo = nullptr;     // lo plane of v_j when z_j = v_j (block Jacobi)
    int phase = 0;                    // grouped runs: 0 cycle start next, 1 stepping, 2 done
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double elapsed_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }

    // workspace, initial guess, ||b||; false when there is nothing to solve
    bool start() {
        if (pc) mgnet_prepare(pc, ctx);
        m = opts.restart;
        ws = get_workspace(ctx, m);
        n = ctx->n;
        gblk = ctx->num_sms * 4;
        if (!opts.use_x0) check(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->stream), "zero x");
        rhs = ctx->b;
        if (comp) rhs = atfps_comp_rhs(ctx);
        launch_norm(ctx, rhs, ws->est + 2);
        bnorm = read_scalar(ctx, ws, ws->est + 2);
        if (bnorm == 0.0) {
            check(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->stream), "zero x");
            inf.converged = 1;
            inf.relres = 0.0;
            return false;
        }
        use_net = (pc != nullptr);
        return true;
    }

    float* vec(int k) const { return ws->V + (size_t)2 * k * n; }

    // true residual in FP64 and the decisions on it; false when the solve ends
    bool cycle_begin() {
        NvtxRange range("restart cycle: true residual");
        if (first && !opts.use_x0)
            check(cudaMemcpyAsync(ws->w64, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream),
                  "r = b");
        else if (comp)
            atfps_comp_apply(ctx, x, ws->w64, true);
        else
            launch_apply(ctx, true, x, ws->w64, true, ctx->b);
        first = false;
        launch_norm(ctx, ws->w64, ws->est + 3);
        const double beta = read_scalar(ctx, ws, ws->est + 3);
        inf.relres = beta / bnorm;
        if (inf.history_len < 32) inf.history[inf.history_len++] = inf.relres;
        if (!std::isfinite(beta)) {
            set_error(ctx, "non-finite residual");
            status = RTE_ESTALL;
            return false;
        }
        if (use_net && prev_res > 0.0 && inf.relres > opts.stall_ratio * prev_res) {
            use_net = false;          // the learned preconditioner stalled
            inf.fell_back = 1;
        }
        prev_res = inf.relres;
        if (inf.relres <= opts.tol) { inf.converged = 1; return false; }
        if (inf.iterations >= opts.max_iter) { status = RTE_ENOTCONV; return false; }
        if (opts.timeout_ms > 0 && elapsed_ms() > opts.timeout_ms) { status = RTE_ETIMEOUT; return false; }
        if (opts.cancel && *opts.cancel) {
            set_error(ctx, "cancelled");
            status = RTE_ECANCELLED;
            return false;
        }
        launch_split_df(ctx, ws->w64, ws->est + 3, vec(0));        // v_0 = r / beta
        {
            ProfScope ps(ctx, K_CYCLE, 0.0);
            k_cycle_start<<<1, 256, 0, ctx->stream>>>(m, ws->est + 3, ws->H, ws->g, ws->betas);
            check(cudaGetLastError(), "k_cycle_start");
        }
        cycle_net = use_net;
        j = 0;
        k = 0;
        return true;
    }

    // z_j: the network's output, or v_j itself (block Jacobi is inside B)
    void precondition() {
        zj = vec(j);
        zj_lo = vec(j) + n;
        if (cycle_net) {
            float* zf = ws->Z + (size_t)j * n;
            mgnet_precondition_f(pc, ctx, vec(j), zf);
            zj = zf;
            zj_lo = nullptr;
        }
    }

    // z_j as a double vector in ws->tmp2 (FP64 inner operators)
    const double* zj_double() {
        if (zj_lo) {
            launch_compose_df(ctx, zj, ws->tmp2);
            return ws->tmp2;
        }
        return nullptr;
    }

    // the preconditioner and operator of step j + 1, queued before the host
    // reads step j's residual estimate so that the device does not idle
    // while the host decides; when the cycle ends at step j instead, the
    // work is discarded (it wrote only Z[j + 1] and scratch vectors that the
    // cycle end and the next cycle overwrite)
    void queue_next_step() {
        ++j;
        precondition();
        inner_apply();
        --j;
    }

    // w = B z_j
    void inner_apply() {
        if (comp) {
            atfps_comp_precond(ctx, zj_double(), ws->tmp);
            atfps_comp_apply(ctx, ws->tmp, ws->w64, false);
            launch_split_df(ctx, ws->w64, nullptr, ws->w);
        } else if (opts.inner_precision == RTE_F32) {
            launch_response_apply_df(ctx, zj, zj_lo, ws->w);
        } else {
            if (zj_lo)
                launch_block_apply(ctx, false, zj_double(), true, ws->tmp, true);
            else
                launch_block_apply(ctx, false, zj, false, ws->tmp, true);
            launch_apply(ctx, true, ws->tmp, ws->w64, true, nullptr);
            launch_split_df(ctx, ws->w64, nullptr, ws->w);
        }
    }

    // deferred CGS2 (v_j fixed, u_{j+1} = w' into row j + 1), the column, Givens
    void orthogonalise_step() {
        NvtxRange range("Gram-Schmidt and Givens");
        launch_cgs2_deferred_df(ctx, ws->V, j, ws->w, ws->cfix, ws->betas + j, ws->h1, ws->h2);
        ProfScope ps(ctx, K_GIVENS, 0.0);
        k_column_givens<<<1, 32, 0, ctx->stream>>>(j, m, ws->h1, ws->h2, ws->betas, ws->cfix, ws->U, ws->hcol,
                                                   ws->H, ws->cs, ws->sn, ws->g, ws->est);
        check(cudaGetLastError(), "k_column_givens");
    }

    // after the step's residual estimate est and ||w|| wn were read: false
    // when the cycle ends
    bool after_step(double est, double wn) {
        ++inf.iterations;
        k = j + 1;
        if (!std::isfinite(est)) {
            if (use_net) { use_net = false; inf.fell_back = 1; }
            k = j;           // drop the bad column
            return false;
        }
        if (est / bnorm <= opts.tol || wn == 0.0 || inf.iterations >= opts.max_iter) return false;
        if (opts.timeout_ms > 0 && elapsed_ms() > opts.timeout_ms) return false;
        if (opts.cancel && *opts.cancel) return false;
        return ++j < m;
    }

    // y = H^{-1} g, dy = Z y (or V y), alpha += D dy
    void cycle_end() {
        if (k > 0) {
            {
                ProfScope ps(ctx, K_BACKSUB, 0.0);
                k_backsub<<<1, 32, 0, ctx->stream>>>(k, m, ws->H, ws->g, ws->y);
                check(cudaGetLastError(), "k_backsub");
                k_deferred_y<<<1, 32, 0, ctx->stream>>>(k, m, cycle_net, ws->betas, ws->U, ws->y, ws->h1);
                check(cudaGetLastError(), "k_deferred_y");
            }
            if (cycle_net) {
                ProfScope ps(ctx, K_XUPDATE, (double)n * (8 + 4 * k));
                k_lincomb_z<<<gblk, 256, 0, ctx->stream>>>(ws->Z, k, n, ws->y, ws->tmp);
                check(cudaGetLastError(), "k_lincomb_z");
            } else {
                launch_lincomb_df(ctx, ws->V, k, ws->y, ws->tmp);
            }
            if (comp)
                atfps_comp_precond(ctx, ws->tmp, ws->w64);                   // mask o D S dy
            else
                launch_block_apply(ctx, false, ws->tmp, true, ws->w64, true);   // D dy
            ProfScope ps(ctx, K_XUPDATE, (double)n * 24);
            k_axpy<<<gblk, 256, 0, ctx->stream>>>(x, ws->w64, n);
            check(cudaGetLastError(), "k_axpy");
        }
        ++inf.cycles;
    }
};

// Lockstep rounds over a set of solves on one stream: the cycle starts of the
// solves that need one, then one Arnoldi step of every stepping solve in
// shared launches, one read of all residual estimates, and the per-solve
// decisions (cycle ends included).
struct GroupRunner {
    enum { kCycle = 0, kStep = 1, kDone = 2 };
    cudaStream_t st = nullptr;
    int cap = 0;
    GroupItem* items_h = nullptr;
    GroupItem* items_d = nullptr;
    void* maps_h = nullptr;        // tensor maps of the items' Gram-Schmidt passes
    void* maps_d = nullptr;
    double* est_h = nullptr;
    double* est_d = nullptr;

    GroupRunner(cudaStream_t s, int capacity) : st(s), cap(capacity) {
        check(cudaMallocHost(&items_h, cap * sizeof(GroupItem)), "cudaMallocHost");
        check(cudaMallocHost(&maps_h, cap * group_gs_maps_bytes()), "cudaMallocHost");
        check(cudaMallocHost(&est_h, 2 * cap * sizeof(double)), "cudaMallocHost");
        check(pool_malloc(reinterpret_cast<void**>(&items_d), cap * sizeof(GroupItem), st), "cudaMallocFromPoolAsync");
        check(pool_malloc(&maps_d, cap * group_gs_maps_bytes(), st), "cudaMallocFromPoolAsync");
        check(pool_malloc(reinterpret_cast<void**>(&est_d), 2 * cap * sizeof(double), st), "cudaMallocFromPoolAsync");
    }
    ~GroupRunner() {
        if (items_d) cudaFreeAsync(items_d, st);
        if (maps_d) cudaFreeAsync(maps_d, st);
        if (est_d) cudaFreeAsync(est_d, st);
        cudaStreamSynchronize(st);
        if (items_h) cudaFreeHost(items_h);
        if (maps_h) cudaFreeHost(maps_h);
        if (est_h) cudaFreeHost(est_h);
    }

    // one round; solves whose phase becomes kDone are finished
    void round(const std::vector<Solver*>& set) {
        for (Solver* s : set)
            if (s->phase == kCycle) s->phase = s->cycle_begin() ? kStep : kDone;
        std::vector<Solver*> live;
        for (Solver* s : set)
            if (s->phase == kStep) live.push_back(s);
        if (live.empty()) return;
        if ((int)live.size() > cap) throw StatusError{RTE_EINVAL, "group larger than its capacity"};
        // preconditioners: solves sharing a network and a grid size run its
        // layers once for all of them
        std::vector<bool> taken(live.size(), false);
        for (size_t q = 0; q < live.size(); ++q) {
            if (taken[q]) continue;
            Solver& s = *live[q];
            if (!s.cycle_net) {
                s.precondition();
                continue;
            }
            std::vector<Solver*> same;
            for (size_t r = q; r < live.size(); ++r)
                if (!taken[r] && live[r]->cycle_net && live[r]->pc == s.pc && live[r]->ctx->I == s.ctx->I) {
                    same.push_back(live[r]);
                    taken[r] = true;
                }
            if (same.size() == 1) {
                s.precondition();
                continue;
            }
            std::vector<rte_ctx*> cs;
            std::vector<const float*> vs;
            std::vector<float*> zs;
            for (Solver* t : same) {
                cs.push_back(t->ctx);
                vs.push_back(t->vec(t->j));
                zs.push_back(t->ws->Z + (size_t)t->j * t->n);
                t->zj = zs.back();
                t->zj_lo = nullptr;
            }
            mgnet_precondition_batch_f(s.pc, cs.data(), vs.data(), zs.data(), (int)same.size());
        }
        int ba = 0, ga = 0, gt = 0, md = 0, ud = 0, kmax = 1;
        size_t smem_ba = 0;
        bool f32 = true;
        for (size_t q = 0; q < live.size(); ++q) {
            Solver& s = *live[q];
            GroupItem& it = items_h[q];
            rte_ctx* c = s.ctx;
            const int K = s.j + 1;
            int nba = 0, nga = 0, nmd = 0, nud = 0;
            size_t sm = 0;
            int ngt = 0;
            group_response_geometry(c, &nba, &nga, &sm);
            const bool tc = response_tc_active(c);
            if (tc) {                      // R z on the tensor cores (launched per item), tile-ordered gather
                nba = nga = 0;
                ngt = tile_gather_blocks(c);
            }
            group_ortho_geometry_df(c, K, &nmd, &nud);
            f32 = f32 && s.opts.inner_precision == RTE_F32;
            if (!tc) ensure_cell_response(c);
            it.Rt = c->Rt;
            it.z = s.zj;
            it.z_lo = s.zj_lo;
            it.o = reinterpret_cast<float*>(c->trace_out);
            it.pos_of = tc ? c->tc_pos_of : nullptr;
            it.I = c->I;
            it.M = c->M;
            it.N = c->N;
            it.n = c->n;
            it.V = s.ws->V;
            it.w = s.ws->w;
            it.h1 = s.ws->h1;
            it.h2 = s.ws->h2;
            it.hcol = s.ws->hcol;
            it.cfix = s.ws->cfix;
            it.betas = s.ws->betas;
            it.U = s.ws->U;
            it.partials = c->partials;
            it.counter = c->counter;
            it.K = K;
            it.j = s.j;
            it.m = s.m;
            it.H = s.ws->H;
            it.cs = s.ws->cs;
            it.sn = s.ws->sn;
            it.g = s.ws->g;
            it.est = s.ws->est;
            it.est_out = est_d + 2 * q;
            it.b_ba = ba; it.n_ba = nba; ba += nba;
            it.b_ga = ga; it.n_ga = nga; ga += nga;
            it.b_gt = gt; it.n_gt = ngt; gt += ngt;
            it.b_md = md; it.n_md = nmd; md += nmd;
            it.b_ud = ud; it.n_ud = nud; ud += nud;
            kmax = K > kmax ? K : kmax;
            smem_ba = sm > smem_ba ? sm : smem_ba;
        }
        const int nl = (int)live.size();
        check(cudaMemcpyAsync(items_d, items_h, nl * sizeof(GroupItem), cudaMemcpyHostToDevice, st), "h2d items");
        encode_group_gs_maps(items_h, nl, maps_h);
        check(cudaMemcpyAsync(maps_d, maps_h, nl * group_gs_maps_bytes(), cudaMemcpyHostToDevice, st), "h2d maps");
        if (f32) {
            for (int q = 0; q < nl; ++q)
                if (items_h[q].pos_of) launch_response_tc_on(live[q]->ctx, items_h[q].z, false, st);
            launch_group_response(items_d, nl, ba, ga, smem_ba, st);
            launch_group_gather_tiles(items_d, nl, gt, st);
        } else {
            for (Solver* s : live) s->inner_apply();
        }
        launch_group_orthogonalise_df(items_d, maps_d, nl, md, ud, kmax, st);
        k_givens_group<<<nl, 32, 0, st>>>(items_d);
        check(cudaGetLastError(), "k_givens_group");
        check(cudaMemcpyAsync(est_h, est_d, 2 * nl * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h est");
        check(cudaStreamSynchronize(st), "group step sync");
        for (int q = 0; q < nl; ++q) {
            Solver& s = *live[q];
            prof_resolve(s.ctx);
            if (!s.after_step(est_h[2 * q], est_h[2 * q + 1])) {
                s.cycle_end();
                s.phase = kCycle;
            }
        }
    }
};

bool valid_opts(const rte_solve_opts& o) {
    return o.restart >= 1 && o.restart <= kMaxKrylov && o.tol > 0.0 && o.max_iter >= 0 &&
           (o.inner_precision == RTE_F32 || o.inner_precision == RTE_F64);
}

}  // namespace

struct GroupSolve : Solver {};
struct GroupRounds : GroupRunner {
    using GroupRunner::GroupRunner;
};

GroupSolve* group_solve_new(rte_ctx* ctx, mgnet* pc, const rte_solve_opts& opts, double* x) {
    GroupSolve* g = new GroupSolve();
    g->ctx = ctx;
    g->pc = pc;
    g->opts = opts;
    g->x = x;
    try {
        g->phase = g->start() ? GroupRunner::kCycle : GroupRunner::kDone;
    } catch (...) {
        delete g;
        throw;
    }
    return g;
}

bool group_solve_done(const GroupSolve* g) { return g->phase == GroupRunner::kDone; }

void group_solve_result(const GroupSolve* g, rte_solve_info* info, rte_status* status) {
    if (info) {
        *info = g->inf;
        info->seconds = g->elapsed_ms() * 1e-3;
    }
    if (status) *status = g->status;
}

void group_solve_free(GroupSolve* g) { delete g; }

GroupRounds* group_rounds_new(cudaStream_t st, int capacity) { return new GroupRounds(st, capacity); }

void group_rounds_step(GroupRounds* r, GroupSolve* const* set, int count) {
    std::vector<Solver*> v(set, set + count);
    r->round(v);
}

void group_rounds_free(GroupRounds* r) { delete r; }

namespace {
rte_status run_solve(rte_ctx* ctx, mgnet* pc, const rte_solve_opts* opts_in, double* x_dev, rte_solve_info* info,
                     bool comp, bool layers) {
    if (!ctx || !x_dev) { set_error(ctx, "NULL argument"); return RTE_EINVAL; }
    NvtxRange range(comp ? "rte_atfps_solve" : "rte_solve");
    Solver S;
    S.ctx = ctx;
    S.pc = pc;
    S.x = x_dev;
    S.comp = comp;
    if (opts_in) S.opts = *opts_in; else rte_solve_opts_default(&S.opts);
    if (!valid_opts(S.opts)) {
        set_error(ctx, "bad solve options (restart in [1, 64], tol > 0)");
        return RTE_EINVAL;
    }
    try {
        if (comp && !ctx->atfps) throw StatusError{RTE_EINVAL, "no ATFPS filter on this context (rte_atfps_setup)"};
        if (S.start()) {
            while (S.cycle_begin()) {
                S.precondition();
                S.inner_apply();
                for (;;) {
                    S.orthogonalise_step();
                    check(cudaMemcpyAsync(S.ws->est_host, S.ws->est, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                          ctx->stream), "d2h est");
                    check(cudaEventRecord(S.ws->est_ready, ctx->stream), "event record");
                    if (S.j + 1 < S.m) S.queue_next_step();
                    check(cudaEventSynchronize(S.ws->est_ready), "step sync");
                    prof_resolve(ctx);
                    if (!S.after_step(S.ws->est_host[0], S.ws->est_host[1])) break;
                }
                S.cycle_end();
            }
        }
        if (const char* why = device_wait_expired()) {
            set_error(ctx, why);
            S.status = RTE_ETIMEOUT;
        }
        if (comp && layers && (S.status == RTE_OK || S.status == RTE_ENOTCONV)) {
            atfps_layers(ctx, x_dev);
            check(cudaStreamSynchronize(ctx->stream), "sync");
        }
    } catch (const CudaError& e) {
        S.status = cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        S.status = e.code;
    } catch (const std::bad_alloc&) {
        set_error(ctx, "host allocation failed");
        S.status = RTE_ENOMEM;
    }
    S.inf.seconds = S.elapsed_ms() * 1e-3;
    if (info) *info = S.inf;
    return S.status;
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
            launch_response_apply(ctx, V_dev + (size_t)j * n, true, ws->w64, true);
            const int K = j + 1;
            orthogonalise64(ctx, ws, V_dev, K, ws->w64);
            launch_scale(ctx, ws->w64, ws->hcol + K, V_dev + (size_t)(j + 1) * n);
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


RTE_API rte_status rte_arnoldi_basis_df64(rte_ctx* ctx, int k, float* V_dev) {
    if (!ctx || !V_dev || k < 1 || k > kMaxKrylov) { set_error(ctx, "bad argument (1 <= k <= 64)"); return RTE_EINVAL; }
    try {
        Workspace* ws = get_workspace(ctx, ctx->ws ? ctx->ws->m : kMaxKrylov);
        if (ws->m < k) ws = get_workspace(ctx, kMaxKrylov);
        const int64_t n = ctx->n;
        launch_norm(ctx, ctx->b, ws->est + 3);
        launch_split_df(ctx, ctx->b, ws->est + 3, V_dev);
        for (int j = 0; j + 1 < k; ++j) {
            float* vj = V_dev + (size_t)2 * j * n;
            launch_response_apply_df(ctx, vj, vj + n, ws->w);
            launch_orthogonalise_df(ctx, V_dev, j + 1, ws->w, ws->h1, ws->h2, ws->hcol);
            launch_scale_df(ctx, ws->w, ws->hcol + j + 1, V_dev + (size_t)2 * (j + 1) * n);
        }
        check(cudaStreamSynchronize(ctx->stream), "sync");
        if (const char* why = device_wait_expired()) throw StatusError{RTE_ETIMEOUT, why};
    } catch (const CudaError& e) {
        return cuda_status(ctx, e.code, e.where);
    } catch (const StatusError& e) {
        set_error(ctx, e.msg);
        return e.code;
    }
    return RTE_OK;
}

RTE_API rte_status rte_solve(rte_ctx* ctx, mgnet* pc, const rte_solve_opts* opts_in, double* x_dev,
                             rte_solve_info* info) {
    return rte::run_solve(ctx, pc, opts_in, x_dev, info, false, false);
}

RTE_API rte_status rte_atfps_solve(rte_ctx* ctx, const rte_solve_opts* opts, int layers, double* x_dev,
                                   rte_solve_info* info) {
    return rte::run_solve(ctx, nullptr, opts, x_dev, info, true, layers != 0);
}

RTE_API rte_status rte_solve_group(rte_ctx* const* ctxs, mgnet* const* pcs, int count,
                                   const rte_solve_opts* opts_in, double* const* x_dev,
                                   rte_solve_info* infos, rte_status* statuses) {
    if (!ctxs || !x_dev || count < 1 || count > 1024) {
        set_error(nullptr, "bad argument (1 <= count <= 1024)");
        return RTE_EINVAL;
    }
    rte_solve_opts opts;
    if (opts_in) opts = *opts_in; else rte_solve_opts_default(&opts);
    if (!valid_opts(opts)) {
        set_error(nullptr, "bad solve options (restart in [1, 64], tol > 0)");
        return RTE_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i] || !x_dev[i]) { set_error(nullptr, "NULL context or solution"); return RTE_EINVAL; }
        if (ctxs[i]->stream != ctxs[0]->stream) {
            set_error(nullptr, "the contexts of a group must share one stream");
            return RTE_EINVAL;
        }
        for (int q = 0; q < i; ++q)
            if (ctxs[q] == ctxs[i]) { set_error(nullptr, "a context appears twice in the group"); return RTE_EINVAL; }
    }
    cudaStream_t st = ctxs[0]->stream;
    std::vector<Solver> S(count);
    rte_status fatal = RTE_OK;
    std::string fatal_msg;
    try {
        GroupRunner runner(st, count);
        std::vector<Solver*> set;
        for (int i = 0; i < count; ++i) {
            S[i].ctx = ctxs[i];
            S[i].pc = pcs ? pcs[i] : nullptr;
            S[i].x = x_dev[i];
            S[i].opts = opts;
            S[i].phase = S[i].start() ? GroupRunner::kCycle : GroupRunner::kDone;
            set.push_back(&S[i]);
        }
        while (true) {
            bool any = false;
            for (Solver* s : set) any = any || s->phase != GroupRunner::kDone;
            if (!any) break;
            runner.round(set);
        }
        if (const char* why = device_wait_expired()) {
            fatal = RTE_ETIMEOUT;
            fatal_msg = why;
        }
    } catch (const CudaError& e) {
        fatal = cuda_status(nullptr, e.code, e.where);
        fatal_msg = rte_last_error(nullptr);
    } catch (const StatusError& e) {
        fatal = e.code;
        fatal_msg = e.msg;
    } catch (const std::bad_alloc&) {
        fatal = RTE_ENOMEM;
        fatal_msg = "host allocation failed";
    }
    for (int i = 0; i < count; ++i) {
        S[i].inf.seconds = S[i].elapsed_ms() * 1e-3;
        if (fatal != RTE_OK) S[i].status = fatal;
        if (infos) infos[i] = S[i].inf;
        if (statuses) statuses[i] = S[i].status;
    }
    if (fatal != RTE_OK) {
        set_error(nullptr, fatal_msg);
        return fatal;
    }
    return RTE_OK;
}

}  // extern "C"
