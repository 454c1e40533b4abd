// Internal declarations shared by the translation units of librte.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rte.h"

namespace rte {

constexpr int kMaxKrylov = 64;      // largest restart (vectors orthogonalised against)
constexpr int kRedThreads = 256;    // block size of the reduction kernels
constexpr int kScal = 256;          // small device scalars per context
constexpr int kHostEigenMaterials = 16;   // more materials: eigenbases on the device

struct Workspace;                   // Krylov buffers of rte_solve (solve.cu)
struct Atfps;                       // ATFPS loss filter of a context (atfps.cu)

// Kernel classes counted (always) and timed (when profiling is on).
enum KernelId {
    K_TRACES, K_COMBINE, K_ADJOINT, K_RECONSTRUCT, K_RHS, K_INVERT, K_BLOCK, K_BLOCK_T,
    K_MDOT, K_UPDATE_DOT, K_UPDATE_NORM, K_NORM, K_SCALE, K_XUPDATE, K_GIVENS, K_BACKSUB,
    K_CYCLE, K_F2D, K_MGNET, K_RESPONSE, K_RESPONSE_APPLY, K_GATHER, K_RESPONSE_TC, K_TILE_ORDER,
    K_FIX_DOT, K_UPDATE_DOT_NORM, K_COUNT
};
extern const char* const kKernelNames[K_COUNT];

struct Profiler {
    bool on = false;
    struct Pending {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;
    double ms[K_COUNT] = {};
    double bytes[K_COUNT] = {};
    double flops[K_COUNT] = {};          // FP64 flops of the FP64-bound kernels; FP32 for the network;
                                         // issued BF16 tensor flops for response_tc
    long long launches[K_COUNT] = {};
};

}  // namespace rte

struct rte_ctx {
    int I = 0, M = 0, N = 0, nmat = 0;
    int64_t n = 0;
    double g = 0.0;
    cudaStream_t stream = nullptr;
    std::string err;
    int num_sms = 0;
    uint64_t uid = 0;                // unique per context (cache key for network features)

    // host copies of the set-up tables
    std::vector<double> xi_h;        // [nmat][2M]
    std::vector<double> L_h;         // [nmat][M][2M]
    std::vector<int> mat_h;          // [N]

    // device tables
    int* mat = nullptr;              // [N] material of each cell
    double* tau = nullptr;           // [N] sigma_T_eff * h
    double* chis = nullptr;          // [N] particular solution q / sigma_a
    double* xi = nullptr;            // [nmat][2M]
    double* Lt64 = nullptr;          // [nmat][2M][M]  Lt[k][m] = L[m][k]
    float* Lt32 = nullptr;
    double* L64 = nullptr;           // [nmat][M][2M]
    float* L32 = nullptr;
    int* rowinfo = nullptr;          // [4][M]: j >= 0 incoming row j of face f, -(j+1) outgoing
    int* rowdir = nullptr;           // [2M] direction of each row slot
    double* inflow = nullptr;        // [4][I][M]
    float* coef_in = nullptr;        // [4][N] CoeffNet inputs: log sigma_T, log sigma_a, log eps, log tau
    double* b = nullptr;             // [n]
    float* Dt = nullptr;             // [N][2][2M][2M] df64 planes per cell, hi then lo:
                                     // Dt[c][0][j][i] + Dt[c][1][j][i] = D_c[i][j]
    float* Rt = nullptr;             // [N][2M][2M], Rt[c][i][row] = R_c[row][i] (FP32); built on
                                     // first use when the blocks are tabulated (ensure_cell_response)
    bool rt_ready = false;
    // tabulated blocks, kept for the per-cell R_C built on demand: the nodes'
    // FP64 R, the bins, the cell list and the FP64 weights
    double* tab_Rn = nullptr;
    int4* tab_bins = nullptr;
    int* tab_cells = nullptr;
    double* tab_wts = nullptr;
    float* tab_w16 = nullptr;        // [N][16] the weights as float pairs: 8 hi, then 8 lo
    int tab_nbins = 0;

    // scratch
    double* trace_out = nullptr;     // n elements (float or double) of outgoing traces
    double* partials = nullptr;      // reduction partial sums
    unsigned* counter = nullptr;     // last-block counter of the reductions
    double* scal = nullptr;          // [kScal] small device scalars (projections, flags)
    int max_red_blocks = 0;

    size_t device_bytes = 0;
    int block_mode = 0;              // RTE_BLOCKS_AUTO / EXACT / TABULATED requested at set-up
    int tab_nodes = 0;               // nodes of the tabulated set-up (0: per-cell inversion)
    // response apply on the tensor cores from the node tables (response_tc.cu)
    uint16_t* tc_nodes = nullptr;    // BF16 parts of the nodes' R, staged layout
    int4* tc_tiles = nullptr;        // (first position, cells, first node, nodes)
    int* tc_pos_of = nullptr;        // [N] position of each cell in the list ordered by stencil
    int* tc_first = nullptr;         // [N] first stencil node per position
    float* tc_w16 = nullptr;         // [N][16] Lagrange weights per position (tab_w16)
    int tc_ntiles = 0;               // 0: no node tables
    double tc_mma_flops = 0.0;       // issued tensor flops per apply
    double tc_bytes = 0.0;           // algorithmic bytes per apply
    int response_path = 0;           // RTE_RESPONSE_AUTO / RTE_RESPONSE_PER_CELL
    rte::Workspace* ws = nullptr;
    rte::Atfps* atfps = nullptr;
    rte::Profiler prof;
    std::vector<void*> allocations;
};

namespace rte {

// error helpers ------------------------------------------------------------
void set_error(rte_ctx* ctx, const std::string& msg);
rte_status cuda_status(rte_ctx* ctx, cudaError_t e, const char* where);
// stream-ordered allocation from the library's memory pool of the current
// device (freed with cudaFreeAsync)
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
void* dev_alloc(rte_ctx* ctx, size_t bytes);      // tracked, zeroed; throws on failure
void* dev_alloc_raw(rte_ctx* ctx, size_t bytes);  // tracked, not zeroed (the caller writes all of it)
void free_workspace(rte_ctx* ctx);                 // releases the rte_solve buffers

struct CudaError {
    cudaError_t code;
    const char* where;
};
struct StatusError {
    rte_status code;
    std::string msg;
};
inline void check(cudaError_t e, const char* where) {
    if (e != cudaSuccess) throw CudaError{e, where};
}

// Raises a kernel's dynamic shared memory limit to at least `bytes`, never
// lowering it: concurrent callers (server threads, contexts of different M)
// cannot shrink the limit under another thread's pending launch.
void raise_smem_limit(const void* kern, size_t bytes);

// NVTX range for the phases of a call (visible to profilers; no cost without one)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// profiling (setup.cu): wrap every launch of the library.
// Counts the launch and its algorithmic bytes; with profiling on, brackets the
// launch with events on the context's stream (resolved at sync points).
struct ProfScope {
    rte_ctx* ctx;
    int kid;
    cudaEvent_t b = nullptr;
    ProfScope(rte_ctx* c, int k, double bytes, int launches = 1, double flops64 = 0.0);
    ~ProfScope();
};
void prof_resolve(rte_ctx* ctx);      // after a stream synchronisation
void prof_free(rte_ctx* ctx);

// operator kernels (apply.cu) ---------------------------------------------
// y = A x (precision of T); if b != nullptr the output is b - A x.
void launch_apply(rte_ctx* ctx, bool f64, const void* x, void* y, bool y_is_double,
                  const double* b);
void launch_apply_adjoint(rte_ctx* ctx, bool f64, const void* y, void* x);
void launch_reconstruct(rte_ctx* ctx, const double* x, double* psi);
void launch_rhs(rte_ctx* ctx);
void launch_coef_inputs(rte_ctx* ctx, const double* sT, const double* sa, const double* eps);

// grouped launches (rte_solve_group) ----------------------------------------
// One instance of a grouped Arnoldi step: its vectors, reduction scratch and,
// for every kernel of the step, the range of blocks it owns in the grouped
// launch -- the same block count as its own launch would use, so the
// instance's arithmetic (reduction order included) is that of a lone solve.
struct GroupItem {
    // inner operator w = z - P R z, o = R z scratch; z is the FP32 network
    // output, or the df64 Krylov vector v_j (block Jacobi: hi plane z, lo plane z_lo)
    const float* Rt;
    const float* z;
    const float* z_lo;
    float* o;
    int I, M, N;
    int64_t n;
    // deferred CGS2 step (launch_cgs2_deferred_df): row K - 1 of V fixed with
    // the coefficients cfix and betas[K - 1], h1 = V^T w, w' = w - V h1 into
    // row K, h2 = V^T w' and ||w'||^2 (h2[K])
    const float* V;
    float* w;
    double* h1;
    double* h2;
    double* hcol;
    const double* cfix;
    double* betas;
    double* U;
    double* partials;
    unsigned* counter;
    int K;
    // Givens on column j of the (m+1) x m Hessenberg matrix
    int j, m;
    double* H;
    double* cs;
    double* sn;
    double* g;
    double* est;             // the instance's own status (est, ||w||)
    double* est_out;         // and a copy in the group's array
    // tensor-core response (o in tile order, null: per cell)
    const int* pos_of;
    // block ranges: [b_x, b_x + n_x) of the grouped launch of kernel x
    int b_ba, n_ba, b_ga, n_ga, b_gt, n_gt, b_md, n_md, b_ud, n_ud;
};

// the item of a grouped launch that block blockIdx.x belongs to: the last
// item whose first block (field START) is at most blockIdx.x
template <int GroupItem::*START>
__device__ inline int group_item_of(const GroupItem* items, int count) {
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        int i = 0;
        while (i + 1 < count && items[i + 1].*START <= (int)blockIdx.x) ++i;
        s_item = i;
    }
    __syncthreads();
    return s_item;
}
// the tile-ordered gathers of the items on the tensor-core path (one launch)
void launch_group_gather_tiles(const GroupItem* items_dev, int count, int blocks, cudaStream_t st);
// w = z - P R z for every item (two grouped launches)
void launch_group_response(const GroupItem* items_dev, int count, int blocks_ba, int blocks_ga,
                           size_t smem_ba, cudaStream_t st);
// block counts and shared memory of one item's response apply / gather
void group_response_geometry(rte_ctx* ctx, int* n_ba, int* n_ga, size_t* smem_ba);
// the deferred CGS2 step (two df64 passes) for every item; maps_dev holds
// the items' tensor maps (encode_group_gs_maps of the same items,
// group_gs_maps_bytes each, 64-byte aligned, copied to the device before)
void launch_group_orthogonalise_df(const GroupItem* items_dev, const void* maps_dev, int count, int blocks_md,
                                   int blocks_ud, int kmax, cudaStream_t st);
size_t group_gs_maps_bytes();
void encode_group_gs_maps(const GroupItem* items_host, int count, void* maps_host);
// block counts of one item's two Gram-Schmidt passes (as launch_cgs2_deferred_df)
void group_ortho_geometry_df(rte_ctx* ctx, int K, int* n_md, int* n_ud);

// lockstep groups of solves (solve.cu), for the grouped server: a solve
// (started on creation: workspace, initial guess, ||b||) and rounds over a set
// of solves on one stream (cycle starts, then one Arnoldi step of every
// stepping solve in shared launches).  Errors throw CudaError / StatusError.
struct GroupSolve;
struct GroupRounds;
GroupSolve* group_solve_new(rte_ctx* ctx, mgnet* pc, const rte_solve_opts& opts, double* x);
bool group_solve_done(const GroupSolve* g);
void group_solve_result(const GroupSolve* g, rte_solve_info* info, rte_status* status);
void group_solve_free(GroupSolve* g);
GroupRounds* group_rounds_new(cudaStream_t st, int capacity);
void group_rounds_step(GroupRounds* r, GroupSolve* const* set, int count);
void group_rounds_free(GroupRounds* r);

// ATFPS loss filter (atfps.cu) -----------------------------------------------
void atfps_setup(rte_ctx* ctx, double delta);
void atfps_free(rte_ctx* ctx);
// out [rows] = F y, y [n] indexed like the rows of A
void atfps_apply(rte_ctx* ctx, const double* y, double* out);
// y [n] = F^T r
void atfps_apply_t(rte_ctx* ctx, const double* r, double* y);
// x [n] (TFPS coefficients, [2M][N]) *= selection mask
void atfps_mask_mul(rte_ctx* ctx, double* x);
int64_t atfps_rows(const rte_ctx* ctx);   // -1 without a filter
// Eigenbases of many materials on the device (eigen.cu): xi [nmat][2M], L64
// [nmat][M][2M] and its copies Lt64 [nmat][2M][M], Lt32, L32, from the
// materials' 1 - gamma, the HG matrix K [M][M] and the direction cosines.
void device_eigenbases(rte_ctx* ctx, const std::vector<double>& omg, const std::vector<double>& K,
                       const std::vector<double>& cdir, const std::vector<double>& sdir, double* xi_dev,
                       double* L64_dev, double* Lt64_dev, float* Lt32_dev, float* L32_dev);

// Compressed ATFPS system (Eq. 2DAdaptiveTFPS_linear_sys) in slot layout
// [2M][N] (a kept row at the slot of its function, zero at dropped slots):
// b_bar; out = A_bar x or b_bar - A_bar x (FP64); the preconditioner
// out = mask o D S z (S the right inverse of F: each compressed row as its
// kept interface basis column); the layer coefficients of Eqs.
// 2DAdaptive_TFPS_layer1 / layer2 written into x's dropped slots.
const double* atfps_comp_rhs(rte_ctx* ctx);
void atfps_comp_apply(rte_ctx* ctx, const double* x, double* out, bool residual);
void atfps_comp_precond(rte_ctx* ctx, const double* z, double* out);
void atfps_layers(rte_ctx* ctx, double* x);

// block kernels (blocks.cu) ------------------------------------------------
// builds G_C for every cell, inverts it in FP64 into ctx->Dt (stored as df64)
// and forms the response matrices ctx->Rt (FP32); *singular_dev set to 1 on a
// zero pivot.
void launch_build_invert(rte_ctx* ctx, int* singular_dev);
// Set-up by interpolation in ln tau (few materials, many cells): nodes of
// each material at tau = exp(s ds) on a uniform grid of s covering the
// cells' range; every cell's D_C and R_C are the 8-point Lagrange
// combination of the nodes around its ln tau.  Cells are binned by their
// first node so that one bin shares its node values.
struct TabPlan {
    std::vector<int> node_mat;       // [J] material of each node
    std::vector<double> node_tau;    // [J] its tau
    std::vector<int> cells;          // [N] cells ordered by bin
    std::vector<double> weights;     // [N][8] Lagrange weights, in the order of cells
    std::vector<int4> bins;          // (first node, first position, end position) in cells
};
void launch_tabulated_blocks(rte_ctx* ctx, const TabPlan& plan, int* singular_dev);
// the per-cell FP32 R_C (ctx->Rt) of a tabulated context, built on first use
// (the tensor-core response apply does not need it)
void ensure_cell_response(rte_ctx* ctx);

// response apply from the node tables on the tensor cores (response_tc.cu)
bool response_tc_supported(int M);                     // 2M in {32, 64, 128}
// node tables (BF16 parts of the nodes' R, FP64 Rn[J][j][i]), tiles, weights
void build_response_tc(rte_ctx* ctx, const TabPlan& plan, const double* Rn);
bool response_tc_active(const rte_ctx* ctx);
// o = R z (z float or double, direction-major) into response_tc_output(ctx):
// FP32 rows in the order of the cell list, [N][2M]; on ctx's stream
void launch_response_tc(rte_ctx* ctx, const void* z, bool z_is_double);
// the same on stream st, not profiled (grouped solves)
void launch_response_tc_on(rte_ctx* ctx, const void* z, bool z_is_double, cudaStream_t st);
float* response_tc_output(rte_ctx* ctx);
// w = v - P o with o = response_tc_output(ctx): df64 w as launch_response_apply_df,
// or float/double w as launch_response_apply
void launch_gather_tiles_df(rte_ctx* ctx, const float* vh, const float* vl, float* w);
void launch_gather_tiles(rte_ctx* ctx, const void* v, bool v_is_double, void* w, bool w_is_double);
int tile_gather_blocks(const rte_ctx* ctx);            // blocks of one tile-ordered gather
// 1 if a bounded wait of the tensor-core response apply ran out (reset clears), -1 on error
int response_tc_timeout_flag(bool reset);

// z = D r (or D^T r), FP64 accumulation; float or double in and out
void launch_block_apply(rte_ctx* ctx, bool transpose, const void* r, bool r_is_double, void* z,
                        bool z_is_double);
// w = A D v = v - P R v (the block-Jacobi preconditioned operator in face-flux
// space, R in FP32); v, w float or double; uses trace_out as scratch
void launch_response_apply(rte_ctx* ctx, const void* v, bool v_is_double, void* w,
                           bool w_is_double);
// w = (A D)^T u = u - R^T P u (float; scratch holds n floats)
void launch_response_apply_t(rte_ctx* ctx, const float* u, float* w, float* scratch);

// krylov kernels (krylov.cu) -----------------------------------------------
// h[0..k) = V^T w (deterministic, last-block reduction into h)
void launch_mdot(rte_ctx* ctx, const double* V, int k, const double* w, double* h);
// w <- w - V h1 ; h2 = V^T w
void launch_update_dot(rte_ctx* ctx, const double* V, int k, double* w, const double* h1,
                       double* h2);
// w <- w - V h2 ; out[0..k) = h1 + h2 ; out[k] = ||w||
void launch_update_norm(rte_ctx* ctx, const double* V, int k, double* w, const double* h1,
                        const double* h2, double* out);
// out[0] = ||x||
void launch_norm(rte_ctx* ctx, const double* x, double* out);

// df64 Krylov vectors (df64.h; krylov_df.cu): planar hi [n] then lo [n]
// floats, vector k of a basis at V + 2 k n.
// CGS2 of w against V[0..K) in three HBM-bound passes: h1, h2 and
// hcol = [h1 + h2, ||w||], w left orthogonalised (not normalised)
void launch_orthogonalise_df(rte_ctx* ctx, const float* V, int K, float* w, double* h1, double* h2,
                             double* hcol);
// v = w / s[0] (v = w if s[0] == 0)
void launch_scale_df(rte_ctx* ctx, const float* w, const double* s, float* v);
// out = x / s[0] (s may be null), double -> df64
void launch_split_df(rte_ctx* ctx, const double* x, const double* s, float* out);
// df64 -> double
void launch_compose_df(rte_ctx* ctx, const float* x, double* out);
// out = sum_k V_k y_k, df64 basis, double out
void launch_lincomb_df(rte_ctx* ctx, const float* V, int K, const double* y, double* out);
// w (df64) = z - P R z for z the FP32 vector z_hi (z_lo null) or the df64
// vector (z_hi, z_lo); R z in FP32 from z_hi
void launch_response_apply_df(rte_ctx* ctx, const float* z_hi, const float* z_lo, float* w);
// One Arnoldi step's Gram-Schmidt in the deferred form, two HBM passes: row
// j of V holds u_j, the previous step's w' (for j = 0, v_0 itself with
// c = 0 and beta = 1); pass 1 fixes it, v_j = (u_j - V[0..j) c) / beta_j[0],
// in place and forms h1 = V[0..j]^T w; pass 2 writes w' = w - V[0..j] h1 into
// row j + 1 and forms h2 = V[0..j]^T w' (h2nu[0..j]) and ||w'||^2
// (h2nu[j + 1]).  The step's Hessenberg column is (h1 + h2, beta_{j+1}) with
// beta_{j+1}^2 = ||w'||^2 - ||h2||^2; h2 and beta_{j+1} fix row j + 1 in the
// next step.
void launch_cgs2_deferred_df(rte_ctx* ctx, float* V, int j, const float* w, const double* c,
                             const double* beta_j, double* h1, double* h2nu);
// 1 if a bounded wait of a df64 Gram-Schmidt pass ran out (reset clears), -1 on error
int krylov_timeout_flag(bool reset);
// reads and clears the device flags of the bounded waits (Gram-Schmidt passes,
// tensor-core response apply): the message of the first that ran out, or null
inline const char* device_wait_expired() {
    const int a = krylov_timeout_flag(true), b = response_tc_timeout_flag(true);
    if (a == 1) return "a bounded wait of a Gram-Schmidt pass ran out";
    if (b == 1) return "a bounded wait of the tensor-core response apply ran out";
    return nullptr;
}
// y = x * (1 / s[0]) unless s[0] == 0 (then y = x)
void launch_scale(rte_ctx* ctx, const double* x, const double* s, double* y);
// x += sum_k Z[k] y[k]  (Z float, k vectors)
void launch_combine_update(rte_ctx* ctx, double* x, const float* Z, int k, const double* y);

}  // namespace rte
