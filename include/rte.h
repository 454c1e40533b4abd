/*
 * rte.h -- C ABI of the GB300 radiative-transfer solver library (librte.so).
 *
 * The library solves the discrete-ordinates / tailored-finite-point (TFPS)
 * system  A alpha = b  of the steady radiative transfer equation in x-y
 * geometry (Song, Zhang, Liu, "A filtered MgNet solver for radiative transfer
 * equations", Sec. 2.1-2.2, Eqs. RTE, hg, DORTE_2d, 2DTFPS_continuity_cond,
 * 2DTFPS_boundary_cond, 2DTFPS_linear_sys) with flexible GMRES preconditioned
 * by block Jacobi or by a learned MgNet V-cycle (Sec. 3, Sec. 4).
 *
 * Contents: context set-up and the operator (rte_setup, rte_apply,
 * rte_apply_adjoint, rte_block_apply, rte_reconstruct, ...); the solve
 * (rte_solve) and grouped solves in shared launches (rte_solve_group); the
 * ATFPS filter and the compressed solve with layer reconstruction (rte_atfps_*,
 * Sec. 2.3); the learned preconditioner (mgnet_*: forward, training on either
 * loss, checkpoints, fault injection); the continuous-batching server
 * (rte_server_*); per-kernel accounting (rte_profile*).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid: unit square, I x I cells, h = 1/I; cell index c = iy*I + ix covers
 *   [ix h, (ix+1) h] x [iy h, (iy+1) h].  N = I*I.
 * Directions: M (a positive multiple of 4) uniform on the circle,
 *   theta_m = 2 pi (m + 1/2) / M, weights 1/M.  (The paper's direction count
 *   is 4M in its own notation; M here is the total.)
 * Unknowns: n = 2 M N.  Every vector (x, b, r, z) is direction-major,
 *   element [k * N + c] for slot k in 0..2M-1 and cell c.
 *   Slots of a cell: [W-centred M/2 | E-centred M/2 | S-centred M/2 |
 *   N-centred M/2] basis functions (x-type with xi<0, x-type xi>0, y-type
 *   xi<0, y-type xi>0, each ascending in xi).
 *   Rows of a cell: [W-face incoming (c_m>0) | E-face incoming (c_m<0) |
 *   S-face incoming (s_m>0) | N-face incoming (s_m<0)], directions ascending.
 * Angular flux output psi: [M][N] at cell centres.
 *
 * Ownership: host arrays are read during the call only.  Device arrays are
 * owned by the caller, must hold the stated number of elements, and are used
 * on the context's stream; the call returns before the work finishes unless
 * stated otherwise.  The context owns every internal buffer.
 * Errors: every call returns an rte_status and never aborts; rte_last_error()
 * gives a message.  A context is not thread-safe; distinct contexts are
 * independent.  Device pointers must be 16-byte aligned.
 */
#ifndef RTE_H_
#define RTE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTE_API __attribute__((visibility("default")))

typedef enum rte_status {
    RTE_OK = 0,
    RTE_EINVAL = 1,      /* invalid argument */
    RTE_ENOMEM = 2,      /* device or host allocation failed */
    RTE_ECUDA = 3,       /* CUDA runtime error */
    RTE_ENOTCONV = 4,    /* iteration limit reached before the tolerance */
    RTE_ESTALL = 5,      /* the solver stalled */
    RTE_ETIMEOUT = 6,    /* a time limit or a bounded device wait ran out */
    RTE_ESINGULAR = 7,   /* a per-cell block could not be inverted */
    RTE_ECANCELLED = 8,  /* the request was cancelled */
    RTE_ENOTSUP = 9      /* unsupported configuration */
} rte_status;

typedef enum rte_precision {
    RTE_F64 = 0,   /* double in, double out, FP64 arithmetic */
    RTE_F32 = 1    /* float in, float out, FP32 arithmetic */
} rte_precision;

typedef struct rte_ctx rte_ctx;
typedef struct mgnet mgnet;

typedef struct rte_grid { int I; } rte_grid;                 /* Sec. 2.2: I x I cells, h = 1/I */
typedef struct rte_quadrature { int M; } rte_quadrature;     /* Sec. 2.1: M uniform directions */

typedef struct rte_ctx_info {
    int I, M, N;          /* cells per side, directions, cells */
    int nmat;             /* distinct scattering ratios (one eigenbasis each) */
    int64_t n;            /* unknowns, 2 M N */
    size_t device_bytes;  /* bytes the context holds on the device */
} rte_ctx_info;

/* ---------------------------------------------------------------------------
 * rte_setup -- build the TFPS system for one medium (Sec. 2.2).
 *
 * sigma_T, sigma_a, q : host [N] cell averages (Sec. 2.2); sigma_T > 0,
 *   sigma_a > 0 (the paper assumes a non-zero absorption), q >= 0.
 * eps : host pointer; one value if eps_is_scalar, else [N] per cell
 *   (Eq. RTE diffusive scaling: sigma_T/eps, sigma_T/eps - eps sigma_a, eps q).
 * g : Henyey-Greenstein anisotropy, |g| < 1 (Eq. hg).
 * inflow : host [4][I][M] (side W,E,S,N; face along the side, iy for W/E and
 *   ix for S/N; direction) or NULL for zero inflow; only incoming directions
 *   are read (Eq. boundary_condition_2d).
 * stream : cudaStream_t (NULL = legacy default stream) on which every later
 *   call of this context runs.
 * On success *out owns: the eigenbases (one per distinct 1 - gamma, computed
 * on the host in FP64), the per-cell optical thickness, b, the per-cell
 * inverse diagonal blocks D_C = G_C^{-1} (FP64, Gauss-Jordan on the device)
 * and the response matrices R_C (FP32).  M <= 80.
 * Synchronous.  Errors: EINVAL (bad sizes or values), ENOMEM, ECUDA,
 * ESINGULAR (a block has a zero pivot).
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_setup(const rte_grid* grid, const rte_quadrature* quad,
                             const double* sigma_T, const double* sigma_a, const double* q,
                             const double* eps, int eps_is_scalar, double g,
                             const double* inflow, void* stream, rte_ctx** out);

/* ---------------------------------------------------------------------------
 * rte_setup_ex -- rte_setup with a choice of how the per-cell blocks are built
 * (no counterpart in the paper: an implementation choice).  The diagonal
 * block G_C of a cell depends on the cell only through its material (1 -
 * gamma) and its optical thickness tau_C.  block_mode:
 *   RTE_BLOCKS_EXACT: every D_C = G_C^{-1} by FP64 Gauss-Jordan and
 *     R_C = T_out,C D_C, cell by cell (the set-up cost grows with N (2M)^3);
 *   RTE_BLOCKS_TABULATED: D and R of every material at nodes tau =
 *     exp(0.04 i) covering its cells' range of ln tau (FP64), and each cell's
 *     blocks as the 8-point Lagrange interpolation in ln tau of the nodes
 *     around it (FP64; R rounded to FP32 once).  The interpolation error is
 *     about 1e-11 of the blocks' size on well-conditioned media and below the
 *     FP64 inversion's own rounding (cond(G_C) u) once cond(G_C) exceeds about
 *     1e5.  The solver's true FP64 residual uses the exact per-cell traces
 *     either way, so the solution meets the same tolerance;
 *   RTE_BLOCKS_AUTO (rte_setup): tabulated when the medium has at least 4096
 *     cells and at least 16 cells per node over all materials, else exact.
 * EINVAL for another value; otherwise as rte_setup.
 * ------------------------------------------------------------------------- */
typedef enum rte_block_mode {
    RTE_BLOCKS_AUTO = 0,
    RTE_BLOCKS_EXACT = 1,
    RTE_BLOCKS_TABULATED = 2
} rte_block_mode;

RTE_API rte_status rte_setup_ex(const rte_grid* grid, const rte_quadrature* quad,
                                const double* sigma_T, const double* sigma_a, const double* q,
                                const double* eps, int eps_is_scalar, double g,
                                const double* inflow, void* stream, int block_mode, rte_ctx** out);

/* Number of interpolation nodes the context's blocks were built from (0 when
 * every block was inverted cell by cell). */
RTE_API rte_status rte_block_setup_info(const rte_ctx* ctx, int* tabulated_nodes);

/* ---------------------------------------------------------------------------
 * rte_set_response_path -- how the inner operator B = A D = I - P R (Sec. 4,
 * block-Jacobi right preconditioning in face-flux space) applies the response
 * matrices R_C (no counterpart in the paper: an implementation choice):
 *   RTE_RESPONSE_AUTO (default): on the tensor cores from the node tables when
 *     the blocks are tabulated and 2M is 32, 64 or 128.  With R_C =
 *     sum_p w_Cp R_p over the cell's eight stencil nodes, o_C = sum_q w_Cq
 *     (R_q z_C) is a dense contraction per tile of cells sharing nodes; the
 *     operands are split into three BF16 parts each (six products, FP32
 *     accumulation), so the result keeps FP32 accuracy.  Otherwise per cell;
 *   RTE_RESPONSE_PER_CELL: every o_C = R_C z_C from the per-cell FP32 R_C
 *     (streamed from device memory, FP32 arithmetic).
 * Applies to rte_response_apply, rte_solve, rte_solve_group and the
 * network's training loss.  EINVAL for another value.
 * rte_response_on_tensor_cores returns 1 when the context's response apply
 * runs on the tensor cores, 0 when per cell, -1 for a NULL context.
 * ------------------------------------------------------------------------- */
typedef enum rte_response_path {
    RTE_RESPONSE_AUTO = 0,
    RTE_RESPONSE_PER_CELL = 1
} rte_response_path;

RTE_API rte_status rte_set_response_path(rte_ctx* ctx, int path);
RTE_API int rte_response_on_tensor_cores(const rte_ctx* ctx);

/* Frees the context's device memory (stream-ordered on its stream).  The
 * blocks return to the library's memory pool of the device, which keeps up
 * to a quarter of the device memory mapped for the next context; see
 * rte_trim_memory. */
RTE_API void rte_destroy(rte_ctx* ctx);

/* Returns every unused block of the library's memory pools to the devices
 * (cudaMemPoolTrimTo(pool, 0)); blocks still held by live contexts stay.
 * RTE_ECUDA on a CUDA error. */
RTE_API rte_status rte_trim_memory(void);

/* Message of the last error of ctx (or of the calling thread if ctx is NULL). */
RTE_API const char* rte_last_error(const rte_ctx* ctx);

RTE_API rte_status rte_info(const rte_ctx* ctx, rte_ctx_info* info);

/* b of Eq. 2DTFPS_linear_sys into b_dev [n] (double). */
RTE_API rte_status rte_rhs(rte_ctx* ctx, double* b_dev);

/* ---------------------------------------------------------------------------
 * rte_apply -- y = A x, the TFPS operator (Eq. 2DTFPS_linear_sys): for every
 * cell C, face f and direction m entering C through f, the trace of
 * sum_k x_Ck chi_C^k at the midpoint of f minus the neighbour's trace there
 * (Eq. 2DTFPS_continuity_cond), or the trace alone on the boundary
 * (Eq. 2DTFPS_boundary_cond).
 * precision RTE_F64: x_dev, y_dev double [n]; RTE_F32: float [n].
 * x_dev and y_dev must not overlap.  Asynchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_apply(rte_ctx* ctx, int precision, const void* x_dev, void* y_dev);

/* x = A^T y (the transpose of rte_apply), same layout and precision rules. */
RTE_API rte_status rte_apply_adjoint(rte_ctx* ctx, int precision, const void* y_dev, void* x_dev);

/* ---------------------------------------------------------------------------
 * rte_block_apply -- z_C = D_C r_C (transpose = 0) or D_C^T r_C (1) for every
 * cell, D_C = G_C^{-1} the inverse of the cell's diagonal block of A: the
 * block-Jacobi preconditioner of Sec. 4 and the map D of Eq. loss (D inverted
 * in FP64 and stored as double-float pairs, 48 significant bits; the sums in
 * double-float, as accurate as FP64 sums).  r_dev, z_dev: float [n], must not
 * overlap.  Asynchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_block_apply(rte_ctx* ctx, int transpose, const float* r_dev, float* z_dev);

/* psi at cell centres, psi_dev double [M][N] (Eq. 2DTFPS_sol). Asynchronous. */
RTE_API rte_status rte_reconstruct(rte_ctx* ctx, const double* x_dev, double* psi_dev);

/* ---------------------------------------------------------------------------
 * rte_export_basis -- copy the host-side eigenbases (Eq.
 * discretization_2D_eigenfunc_constraint) out: xi [nmat][2M] (slot order),
 * L [nmat][M][2M] (row = direction, column = slot), mat_id [N].  Any pointer
 * may be NULL.  Synchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_export_basis(const rte_ctx* ctx, double* xi, double* L, int* mat_id);

/* ---------------------------------------------------------------------------
 * rte_eigenbasis -- host-only FP64 eigenpairs of the local TFPS problem
 * (Eq. discretization_2D_eigenfunc_constraint) for M uniform directions, HG
 * anisotropy g (Eq. hg) and 1 - gamma = eps^2 sigma_a / sigma_T in (0, 1]:
 * axis 0 solves (gamma K W - I) l = xi C l (xi_y = 0), axis 1 the S version.
 * xi [M] ascending, L [M][M] row-major (row = direction, column = mode),
 * each column divided by its first entry within 1e-8 of its largest
 * magnitude.  The same routine rte_setup uses.  Needs no GPU.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_eigenbasis(int M, double g, double one_minus_gamma, int axis, double* xi,
                                  double* L);

/* Copy the per-cell matrices out (host, row-major, either pointer may be NULL):
 * D [N][2M][2M] double, D_C = G_C^{-1} (rows = slots, columns = rows of A;
 * the stored double-float value, 48 significant bits);
 * R [N][2M][2M] float, the response R_C = T_out,C D_C whose row (f, j) is
 * the value leaving C through face f in direction dirs[opp f][j] for unit
 * incoming data.  Synchronous. */
RTE_API rte_status rte_export_blocks(rte_ctx* ctx, double* D_host, float* R_host);

/* ---------------------------------------------------------------------------
 * rte_response_apply -- w = A D v for v in the row space (face-flux space):
 * every cell's own rows give v back (G_C D_C = I) and each row loses the
 * neighbour's outgoing value, w = v - P R v, with R the FP32 response
 * matrices (FP32 accuracy: per cell, or on the tensor cores from the node
 * tables, rte_set_response_path; v and w double [n]).  This is the operator the
 * Krylov iteration of rte_solve works on (block-Jacobi right
 * preconditioning, Sec. 4).  v and w must not overlap.  Asynchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_response_apply(rte_ctx* ctx, const double* v_dev, double* w_dev);

/* ---------------------------------------------------------------------------
 * Krylov building block (Arnoldi step of flexible GMRES): orthogonalise w
 * against the k orthonormal columns V[0..k-1] (V_dev: k x n doubles, vector j
 * at V_dev + j*n) by classical Gram-Schmidt with one reorthogonalisation,
 * w <- w - V (V^T w) twice; h_dev[0..k-1] receives the summed projections and
 * h_dev[k] = ||w|| after orthogonalisation; w is then scaled to unit norm
 * unless that norm is zero.  1 <= k <= 64 (EINVAL otherwise).  Asynchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_cgs2(rte_ctx* ctx, const double* V_dev, int k, double* w_dev, double* h_dev);

/* ---------------------------------------------------------------------------
 * rte_cgs2_df64 -- the Gram-Schmidt step of rte_cgs2 on df64 vectors, the
 * arithmetic rte_solve uses for its Arnoldi process (Sec. 4, GMRES).  A df64
 * vector of n elements is two float planes, hi [n] then lo [n], holding the
 * value hi + lo with |lo| <= ulp(hi) (48 significant bits; a double x is
 * stored as hi = (float)x, lo = (float)(x - hi)).  V_dev: k df64 vectors,
 * vector j at V_dev + 2 j n (orthonormal); w_dev: one df64 vector,
 * orthogonalised in place by two classical Gram-Schmidt passes with df64
 * products and sums on the FP32 pipe, then scaled to unit norm unless that
 * norm is zero; h_dev (double [k + 1]): the summed projections and the norm.
 * 1 <= k <= 64 (EINVAL otherwise); n = the context's unknowns; all pointers
 * 16-byte aligned.  ETIMEOUT if a bounded wait inside a pass ran out (the
 * outputs are then NaN).  Asynchronous except for that check, which
 * synchronises with the device.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_cgs2_df64(rte_ctx* ctx, const float* V_dev, int k, float* w_dev, double* h_dev);

/* rte_arnoldi_basis_df64 -- rte_arnoldi_basis with the df64 arithmetic of
 * rte_solve: k (1..64) Arnoldi vectors of A D started from b / ||b||, written
 * as df64 vectors (vector j at V_dev + 2 j n, float [k][2][n]).  Synchronous. */
RTE_API rte_status rte_arnoldi_basis_df64(rte_ctx* ctx, int k, float* V_dev);

/* ---------------------------------------------------------------------------
 * rte_cgs2_noalloc -- the Gram-Schmidt step of rte_cgs2 without a context and
 * without any device allocation.  No counterpart in the paper: it exists for
 * callers that cannot let a library allocate device memory -- an application
 * that owns the whole device-memory budget through its own pool, or a
 * latency-critical loop where cudaMalloc (which may synchronise the device,
 * and may fail) is not allowed.
 *
 * Same arithmetic as rte_cgs2: V_dev holds k orthonormal vectors of n doubles
 * (vector j at V_dev + j*n), w_dev is orthogonalised in place (two classical
 * Gram-Schmidt passes) and scaled to unit norm unless that norm is zero;
 * h_dev[0..k-1] receives the summed projections, h_dev[k] the norm.  All
 * three are caller-owned device buffers; stream is a cudaStream_t (NULL =
 * legacy default stream).  Asynchronous.
 *
 * Scratch: one file-scope device array of 328,960 bytes (partial sums of up to
 * 640 blocks x 64 projections, the two projection vectors, a ticket counter),
 * present on every GPU that loads the library until the process exits.
 * Limits: 1 <= k <= 64 (EINVAL otherwise), n >= 1, device ordinal < 64.
 * The first successful call on a device looks up the array's device address
 * (with that device current) and caches it; make that first call before any
 * stream capture.  A look-up that fails is not cached: the next call tries
 * again.  Every call on a device shares the array and the ticket is cleared
 * at the start of each call, so calls that overlap on the GPU (other streams
 * or threads) race: serialise them.  Calls nothing that allocates.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_cgs2_noalloc(const double* V_dev, int k, int64_t n, double* w_dev,
                                    double* h_dev, void* stream);

/* ---------------------------------------------------------------------------
 * rte_arnoldi_basis -- k (1..64) steps of the Arnoldi process on the
 * block-Jacobi preconditioned operator A D (face-flux space, CGS2) started
 * from b / ||b||; V_dev receives the k orthonormal vectors (double, vector j
 * at V_dev + j*n).  The vectors the classical iteration works with: one
 * source of training inputs for the learned preconditioner.  Synchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_arnoldi_basis(rte_ctx* ctx, int k, double* V_dev);

/* ---------------------------------------------------------------------------
 * ATFPS filter of the loss (Sec. 2.3; Eqs. def_V_delta,
 * 2DAdaptiveTFPS_continuity_cond, 2DAdaptiveTFPS_boundary_cond, loss_delta).
 *
 * rte_atfps_setup builds, on the device, the selection (basis function k of
 * cell c kept iff exp(-|xi_k| tau_c / 2) > delta) and for every interface the
 * projections onto its kept coordinates: the kept functions centred at the
 * interface (lower/left cell first, each group in ascending |xi|) are
 * orthonormalised (QR with positive R diagonal), the dropped ones follow,
 * every column is scaled to max-norm one, and the first s rows of the inverse
 * of that basis are kept.  Interior interfaces use the midpoint jump over all
 * M directions; boundary faces the M/2 incoming components.  Interfaces are
 * ordered: interior vertical (row-major), interior horizontal, per row the
 * west and east boundary faces, per column the south and north ones.
 * delta in [0, 1).  rows_out (may be NULL): number of kept coordinates R.
 * ESINGULAR if an interface basis is numerically singular (pivot below 1e-12
 * of its unit max-norm columns).  Replaces a previous filter.  Synchronous.
 *
 * rte_atfps_mask: host uint8 [2M][N] copy of the selection (1 = kept).
 * rte_atfps_apply: out = F y, y double [n] indexed like the rows of A, out
 * double [R] (device).  rte_atfps_apply_t: y = F^T r (device).  EINVAL
 * without a filter.  Asynchronous on the context's stream.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_atfps_setup(rte_ctx* ctx, double delta, int64_t* rows_out);
RTE_API rte_status rte_atfps_mask(rte_ctx* ctx, unsigned char* mask_host);
RTE_API rte_status rte_atfps_apply(rte_ctx* ctx, const double* y_dev, double* out_dev);
RTE_API rte_status rte_atfps_apply_t(rte_ctx* ctx, const double* r_dev, double* y_dev);

/* ---------------------------------------------------------------------------
 * rte_solve -- solve A x = b for this context's b by right-preconditioned
 * flexible GMRES(restart): Arnoldi on df64 vectors (48 significant bits, see
 * rte_cgs2_df64) with classical Gram-Schmidt plus reorthogonalisation,
 * Givens/Hessenberg least squares in FP64 on the device,
 * inner operator applies in opts->inner_precision, and the true residual
 * ||b - A x|| / ||b|| recomputed in FP64 at the end of every cycle decides
 * convergence.  pc: NULL = block Jacobi (Sec. 4); else the MgNet
 * preconditioner z = D Net(r) (Sec. 3), replaced by block Jacobi for the
 * remaining cycles when a cycle reduces the true residual by less than
 * opts->stall_ratio or produces a non-finite value.
 * x_dev: double [n]; the initial guess if opts->use_x0, else zeroed.
 * Synchronous.  Returns RTE_OK when converged, RTE_ENOTCONV when max_iter is
 * reached (x holds the last iterate), RTE_ETIMEOUT when timeout_ms elapses.
 * ------------------------------------------------------------------------- */
typedef struct rte_solve_opts {
    double tol;            /* relative residual target (default 1e-8) */
    int restart;           /* Krylov dimension per cycle (default 50, <= 64) */
    int max_iter;          /* total Arnoldi steps (default 20000) */
    int inner_precision;   /* RTE_F32 (default) or RTE_F64 for the inner applies */
    int use_x0;            /* 1: x_dev holds the initial guess */
    double stall_ratio;    /* MgNet fallback threshold per cycle (default 0.9) */
    double timeout_ms;     /* wall-clock limit, <= 0 for none */
    const volatile int* cancel;   /* host flag read after every step (NULL: none);
                                     non-zero ends the solve with RTE_ECANCELLED */
} rte_solve_opts;

typedef struct rte_solve_info {
    int iterations;        /* Arnoldi steps taken */
    int cycles;            /* restart cycles */
    int converged;         /* 1 if the true residual <= tol */
    int fell_back;         /* 1 if MgNet was replaced by block Jacobi */
    double relres;         /* final true relative residual (FP64) */
    double seconds;        /* wall time of the call */
    int history_len;       /* entries of history */
    double history[32];    /* true relative residual at the start of each restart cycle
                              (the first 32; the last entry is the final one) */
} rte_solve_info;

RTE_API void rte_solve_opts_default(rte_solve_opts* opts);
RTE_API rte_status rte_solve(rte_ctx* ctx, mgnet* pc, const rte_solve_opts* opts,
                             double* x_dev, rte_solve_info* info);

/* ---------------------------------------------------------------------------
 * rte_atfps_solve -- the compressed ATFPS solve with layer reconstruction
 * (Sec. 2.3.3-2.3.4): the kept coefficients solve the compressed system of
 * Eq. 2DAdaptiveTFPS_linear_sys, A_bar alpha_bar = b_bar (its rows the kept
 * projections of every interface jump, Eqs. 2DAdaptiveTFPS_continuity_cond /
 * boundary_cond, i.e. A_bar = F A restricted to the kept columns, b_bar = F b),
 * by flexible GMRES right-preconditioned by mask o D S (FP64 throughout):
 * S takes each compressed row back onto the rows of its interface as its kept
 * basis column (F S = I) and D is the block-Jacobi inverse of the full system,
 * so that with nothing dropped A_bar mask o D S = F (A D) F^{-1}, the block-
 * Jacobi operator of the full system up to similarity; then,
 * with layers != 0, every dropped coefficient from the dropped projection of
 * its interface's jump of that smooth solution (Eqs. 2DAdaptive_TFPS_layer1 /
 * layer2), else zero.  Requires rte_atfps_setup (EINVAL otherwise).
 * x_dev: double [2M][N] (device), the full coefficient vector on return (the
 * layout of rte_solve; rte_reconstruct gives the angular flux).  opts as for
 * rte_solve except that inner_precision and stall_ratio are not used; the
 * reported relres is ||b_bar - A_bar alpha_bar|| / ||b_bar|| (b_bar and the
 * residual in slot layout).  Synchronous. */
RTE_API rte_status rte_atfps_solve(rte_ctx* ctx, const rte_solve_opts* opts, int layers, double* x_dev,
                                   rte_solve_info* info);

/* ---------------------------------------------------------------------------
 * rte_solve_group -- count (1..1024) solves of rte_solve advancing in
 * lockstep: in every round each live solve takes one Arnoldi step, and the
 * steps of all of them run as shared launches (inner operator w = B z and its
 * neighbour gather, the three Gram-Schmidt passes, the scaling to v_{j+1},
 * the Givens updates: six launches per round for the whole group, whatever
 * the grids and direction counts), with one device-to-host read of all
 * residual estimates.  Preconditioners (MgNet) and the cycle starts and ends
 * run per solve.  Every solve keeps the block partition of its lone launches,
 * so its result is bit-identical to rte_solve's.  ctxs: distinct contexts on
 * one stream (EINVAL otherwise); pcs: NULL or one network (or NULL) per
 * solve, on the same stream; x_dev[i]: double [n_i].  infos, statuses
 * (may be NULL): per solve, as rte_solve would return them.  Returns RTE_OK
 * unless the group itself failed (a CUDA error, an allocation), in which case
 * every status carries that error.  Synchronous.
 * ------------------------------------------------------------------------- */
RTE_API rte_status rte_solve_group(rte_ctx* const* ctxs, mgnet* const* pcs, int count,
                                   const rte_solve_opts* opts, double* const* x_dev,
                                   rte_solve_info* infos, rte_status* statuses);

/* ---------------------------------------------------------------------------
 * MgNet preconditioner (Sec. 3): CoeffNet + MgNet V-cycle in face-flux space.
 *
 * Network: CoeffNet levels l = 0..levels-1 (conv 3x3, stride 2 after level 0,
 * batch normalisation, ReLU; widths min(cc 2^l, ccmax)) on the per-cell
 * inputs log sigma_T, log sigma_a, log eps, log tau, with 1x1 heads
 * a_l = 1 + head, ainv_l = 1 + head of MgNet width min(c0 2^l, cmax);
 * MgNet: lift 1x1 (2M -> c0), smoothing u <- u + (B_l * act(f - (A_l * u) o a_l)) o ainv_l
 * (act = identity when act == 0, the default reading of Sec. 3.3; ReLU when 1),
 * restriction conv 3x3 stride 2, prolongation transposed conv 4x4 stride 2,
 * one pre- and one post-smoothing step per level (two on the coarsest),
 * projection 1x1 (c0 -> 2M) added to the input: psi_d = x + proj(u_0).
 * Requirements: cc <= c0, ccmax <= cmax, I divisible by 2^(levels-1).
 * Parameters are one float32 vector in this order, per level l:
 * coef{l}.w [Cc_l][Cin][3][3], coef{l}.gamma, coef{l}.beta, a{l}.w [C_l][Cc_l],
 * a{l}.b, ainv{l}.w, ainv{l}.b; then lift.w [C_0][2M]; A{l}.w, B{l}.w
 * [C_l][C_l][3][3] for every l; R{l}.w [C_{l+1}][C_l][3][3] and P{l}.w
 * [C_{l+1}][C_l][4][4] for l < levels-1; proj.w [2M][C_0].
 * FP32 weights and activations.  A network and a context must share M.
 * ------------------------------------------------------------------------- */
typedef struct mgnet_config {
    int M, levels, c0, cmax, cc, ccmax;
    int act;          /* 0: linear smoothers, 1: ReLU */
} mgnet_config;

/* stream: the network's initial CUDA stream (NULL: the legacy default
 * stream).  A call with a context runs on the context's stream and the
 * network keeps that stream for its calls without one (set/get params, save,
 * load, clone), so such a stream must outlive those calls; mgnet_destroy
 * waits for the whole device and uses no stream. */
RTE_API rte_status mgnet_create(const mgnet_config* cfg, void* stream, mgnet** out);
RTE_API void mgnet_destroy(mgnet* net);
RTE_API int64_t mgnet_param_count(const mgnet* net);
/* The configuration the network was created with.  EINVAL for NULL. */
RTE_API rte_status mgnet_get_config(const mgnet* net, mgnet_config* cfg);

/* Host-side fault injection (no counterpart in the paper): with
 * MGNET_FAULT_NAN every output of the preconditioner (mgnet_precond and the
 * solves using the network) is overwritten with NaN, as a failing network
 * would produce; the solver detects the non-finite step and falls back to
 * block Jacobi.  No device fault is raised.  EINVAL for another kind. */
typedef enum mgnet_fault { MGNET_FAULT_NONE = 0, MGNET_FAULT_NAN = 1 } mgnet_fault;
RTE_API rte_status mgnet_inject_fault(mgnet* net, int kind);

/* Arithmetic of the V-cycle convolutions when the network preconditions
 * (mgnet_precond, mgnet_apply, rte_solve); training always uses FP32.
 *   MGNET_BF16: tcgen05 tensor cores, BF16 operands (weights and gathered
 *               activations rounded to nearest even), FP32 accumulation and
 *               FP32 epilogue / storage (default);
 *   MGNET_FP32: FP32 FMA on the CUDA cores.
 * The CoeffNet features are FP32 in both.  EINVAL for another value. */
typedef enum mgnet_precision { MGNET_FP32 = 0, MGNET_BF16 = 1 } mgnet_precision;
RTE_API rte_status mgnet_set_precision(mgnet* net, int precision);
RTE_API int mgnet_get_precision(const mgnet* net);

/* Loss of mgnet_train_step / mgnet_loss_grad:
 *   MGNET_LOSS_PLAIN: Eq. loss in face-flux space, ||x - A D psi_d|| / ||x|| (default);
 *   MGNET_LOSS_FILTERED: Eq. loss_delta, ||F (A (mask o D psi_d) - x)|| / ||x||
 *     with the context's ATFPS filter (rte_atfps_setup; EINVAL at the step
 *     without one), A applied in FP64.
 * EINVAL for another value. */
typedef enum mgnet_loss { MGNET_LOSS_PLAIN = 0, MGNET_LOSS_FILTERED = 1 } mgnet_loss;
RTE_API rte_status mgnet_set_loss(mgnet* net, int kind);
RTE_API int mgnet_get_loss(const mgnet* net);

/* 1 if a bounded wait inside a tensor-core network kernel expired since the
 * last reset (that launch wrote NaN outputs), else 0; reset != 0 clears the
 * flag.  Synchronises with the device.  Returns -1 if the flag cannot be read. */
RTE_API int mgnet_kernel_status(int reset);
/* Host float32 [count] in the order above; set also resets the Adam state. */
RTE_API rte_status mgnet_set_params(mgnet* net, const float* host, int64_t count);
RTE_API rte_status mgnet_get_params(mgnet* net, float* host, int64_t count);

/* z = rms(r) Net(r / rms(r)) in face-flux space (the preconditioner rte_solve
 * applies before B = A D); r double [n], z float [n], device.  Asynchronous. */
RTE_API rte_status mgnet_precond(mgnet* net, rte_ctx* ctx, const double* r_dev, float* z_dev);

/* z = D rms(r) Net(r / rms(r)): the learned preconditioner mapped to the TFPS
 * coefficients (D of Eq. loss); r, z double [n], device.  Asynchronous. */
RTE_API rte_status mgnet_apply(mgnet* net, rte_ctx* ctx, const double* r_dev, double* z_dev);

/* ---------------------------------------------------------------------------
 * mgnet_train_step -- one Adam step (lr, beta 0.9/0.999, eps 1e-8) on the
 * unfiltered physics-informed loss of Eq. loss for a batch of right-hand
 * sides of one medium: mean_b ||x_b - A D psi_d,b|| / ||x_b||, x_b = r_b / rms(r_b).
 * r_dev: host array of batch (1..16) device pointers, double [n] each.
 * loss_out: the batch loss before the step.  Synchronous.
 * mgnet_loss_grad: same loss and the gradient (host float32 [count], may be
 * NULL) without updating the weights.
 * ------------------------------------------------------------------------- */
RTE_API rte_status mgnet_train_step(mgnet* net, rte_ctx* ctx, const double* const* r_dev, int batch,
                                    double lr, double* loss_out);
RTE_API rte_status mgnet_loss_grad(mgnet* net, rte_ctx* ctx, const double* const* r_dev, int batch,
                                   double* loss_out, float* grad_host);

/* Checkpoint to / from a file: "MGNET003", seven int32 (M, levels, c0, cmax,
 * cc, ccmax, act), int64 count, int64 Adam step, then count float32 weights,
 * count float32 Adam first moments, count float32 second moments, and a uint32
 * checksum (the step plus every 32-bit word, modulo 2^32).  Load checks the
 * configuration and checksum (EINVAL on mismatch) and restores weights, moments
 * and step, so training resumes where it stopped; it also reads the older
 * weights-only "MGNET002" layout (no step, no moments; the Adam state is reset). */
RTE_API rte_status mgnet_save(mgnet* net, const char* path);
/* A new network with the same configuration and weights (its own caches and
 * workspace, so copies can serve different streams at once). */
RTE_API rte_status mgnet_clone(const mgnet* src, void* stream, mgnet** out);
RTE_API rte_status mgnet_load(mgnet* net, const char* path);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of solve requests (no counterpart in the
 * paper).  rte_server_create starts `slots` worker threads, each with its own
 * CUDA stream (and its own copy of each network).  Submitted
 * requests (host arrays, copied at submission) wait in FIFO order and are
 * admitted as soon as a slot is free and their estimated device footprint
 * fits in max_device_bytes together with the requests already running; the
 * admitted solves overlap on the GPU and each releases its slot and bytes the
 * moment it finishes.  A request runs rte_setup, rte_solve and
 * rte_reconstruct; results are the same bits as a lone solve.  With use_net
 * the solve is preconditioned by the server's network for the request's M
 * whose depth fits its grid (I divisible by 2^(levels-1)); a request no
 * network fits, or without use_net, uses block Jacobi
 * (rte_result.used_net tells which).  rte_server_create_multi takes up to 16
 * networks (host array of count handles, read during the call; each is
 * copied, so the caller keeps ownership), at most one per M (EINVAL
 * otherwise); rte_server_create is the same with one network or none (NULL).
 * Errors are per request (rte_result.status): a malformed medium gives
 * EINVAL, a cancelled one ECANCELLED; submit rejects a request that can never
 * fit (ENOMEM) or is malformed (EINVAL).  inject_alloc_failure_id makes that
 * request fail with ENOMEM at admission (host-side fault injection, -1: off).
 * rte_server_wait blocks until the request is done (or timeout_ms > 0
 * elapses: ETIMEOUT, request kept) and copies psi [M][N] (cell centres) to
 * psi_host if not NULL; a finished request is forgotten after its wait.
 * Thread-safe: any thread may submit, wait or cancel.
 *
 * grouped = 1: the admitted requests (up to `slots`, same footprint rule) run
 * as one lockstep group on one stream: two threads set requests up, and one
 * thread advances every running solve by one Arnoldi step per round with the
 * steps of all of them in shared launches (as rte_solve_group); a request set
 * up while others run joins at the next round, a finished one leaves at once
 * (its bytes and slot go to the next waiting request).  Results are the same
 * bits as a lone solve.  grouped = 0 (default): one stream per slot.
 * ------------------------------------------------------------------------- */
typedef struct rte_server rte_server;
typedef struct rte_server_config {
    size_t max_device_bytes;
    int slots;
    int64_t inject_alloc_failure_id;
    int grouped;
} rte_server_config;
typedef struct rte_request {
    int I, M;
    const double *sigma_T, *sigma_a, *q, *eps;
    int eps_is_scalar;
    double g;
    const double* inflow;      /* [4][I][M] or NULL */
    double tol;                /* <= 0: 1e-8 */
    int max_iter, restart;     /* <= 0: defaults */
    int use_net;
} rte_request;
typedef struct rte_result {
    int status;                /* rte_status of the request */
    rte_solve_info info;
    double latency_s;          /* submission to completion */
    double queue_s;            /* submission to admission */
    size_t footprint;          /* estimated device bytes */
    int used_net;              /* 1: a network preconditioned the solve, 0: block Jacobi */
} rte_result;
typedef struct rte_server_stats_t {
    int64_t queued, completed;
    int active;
    size_t bytes_in_use;
} rte_server_stats_t;

RTE_API void rte_server_config_default(rte_server_config* cfg);
RTE_API rte_status rte_server_create(const rte_server_config* cfg, mgnet* net, rte_server** out);
RTE_API rte_status rte_server_create_multi(const rte_server_config* cfg, mgnet* const* nets, int count,
                                           rte_server** out);
RTE_API rte_status rte_server_submit(rte_server* s, const rte_request* req, int64_t* id_out);
RTE_API rte_status rte_server_wait(rte_server* s, int64_t id, double timeout_ms, rte_result* res,
                                   double* psi_host);
RTE_API rte_status rte_server_cancel(rte_server* s, int64_t id);
RTE_API rte_status rte_server_stats(rte_server* s, rte_server_stats_t* stats);
RTE_API void rte_server_destroy(rte_server* s);

/* ---------------------------------------------------------------------------
 * Per-kernel accounting (no counterpart in the paper: instrumentation).
 * Every kernel launch of a context is counted with its algorithmic bytes (the
 * bytes its operation must move: inputs read once, outputs written once).
 * rte_profile(ctx, 1) clears the counters and also brackets every launch with
 * CUDA events on the context's stream; rte_profile(ctx, 0) clears and stops
 * the timing.  rte_profile_read fills up to max entries (one per kernel
 * class, in a fixed order) and returns how many it wrote, or the number of
 * classes if out is NULL, or -1 on error.  Both synchronise the stream.
 * ------------------------------------------------------------------------- */
typedef struct rte_kernel_stat {
    const char* name;      /* kernel class (static string) */
    long long launches;    /* launches since the last rte_profile call */
    double ms;             /* summed event time (0 unless timing is on) */
    double bytes;          /* summed algorithmic bytes */
    double flops;          /* summed arithmetic flops: FP64 for the Gram-Schmidt passes and
                              the FP64 operator, FP32 for the network ("mgnet") */
} rte_kernel_stat;

RTE_API rte_status rte_profile(rte_ctx* ctx, int enable);

/* Measured FP64 FMA throughput of the current device in GFLOP/s (2 flops per
 * FMA), from a short event-timed kernel on stream: the denominator of the
 * roofline of kernels bound by FP64 arithmetic.  No counterpart in the paper. */
RTE_API rte_status rte_fp64_fma_rate(void* stream, double* gflops);
/* The same for FP32 FMA (CUDA cores): the roofline of the network's FP32
 * convolutions. */
RTE_API rte_status rte_fp32_fma_rate(void* stream, double* gflops);
RTE_API int rte_profile_read(rte_ctx* ctx, rte_kernel_stat* out, int max);

#ifdef __cplusplus
}
#endif
#endif /* RTE_H_ */
