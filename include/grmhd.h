/*
 * grmhd.h -- C ABI of the GB300 (sm_103a) implementation of one implicit-explicit
 * Runge-Kutta stage of resistive (general-relativistic) MHD on a uniform Cartesian
 * grid with a fixed background metric, after arXiv 2110.03732 (Cheong et al.).
 *
 * Problem statement (what the calls take):
 *   - grid: uniform Cartesian, 1-3 active directions, Sec. 5 boundary kinds
 *   - 3+1 metric (Sec. 2.1): lapse alpha, zero shift, spatial metric
 *     gamma_ij = psi^4 delta_ij (conformally flat, reference metric Cartesian)
 *   - state (Sec. 2.1): densitised cell-centred conserved variables
 *     q = psi^6 (D, S_1, S_2, S_3, tau, E^1, E^2, E^3) and staggered face fields
 *     q_B^d = psi^6 B^d on the lower d-face of each cell (Sec. 3.2)
 *   - primitives (Sec. 2.4/2.6): rho, u^i = W v^i (contravariant), p, E^i
 *   - resistivity eta (Sec. 2.2, xi = 0), per cell or uniform
 *   - IMEX tableau (Sec. 2.3), diagonally implicit with a_ii > 0; IMEX-SSP2(2,2,2)
 *     is provided by grmhd_tableau_ssp2
 *   - ideal-gas equation of state p = (Gamma - 1) rho eps (Sec. 2.4)
 *
 * Layout: every array is a padded grid of N0 * N1 * N2 doubles, x fastest, with
 * N_d = n_d + 4 in an active direction (two ghost cells per side) and N_d = 1 in an
 * inactive one.  Face arrays hold the value on the lower face of each cell; edge
 * arrays (vector potential) hold the value on the edge that is lower in both
 * transverse directions.  Directions become active in the order x, y, z.
 *
 * Ownership: the caller owns every buffer (device memory unless stated).  The
 * library allocates no device memory: grmhd_scratch_bytes says how much scratch the
 * caller must pass to grmhd_bind.  Pointers must stay valid while bound.
 *
 * Streams: all work is ordered on the stream passed in.  Only grmhd_compute_dt and
 * grmhd_diagnostics synchronise that stream (they return host scalars).
 *
 * Errors: every call returns a grmhd_status; negative values are errors, positive
 * values warnings.  grmhd_last_error() gives a message for the calling thread.  A
 * context is not thread-safe; use one per thread/stream.
 */
#ifndef GRMHD_H
#define GRMHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* grmhd_stream_t; /* same type as cudaStream_t */
typedef struct grmhd_ctx_s grmhd_ctx;

typedef enum {
    GRMHD_OK = 0,
    GRMHD_WARN_C2P_FAILED = 1, /* some cells' Newton solves did not converge (see diagnostics) */
    GRMHD_ERR_ARG = -1,        /* invalid argument (message in grmhd_last_error) */
    GRMHD_ERR_CUDA = -2,       /* a CUDA call failed */
    GRMHD_ERR_SCRATCH = -3,    /* scratch buffer too small or misaligned */
    GRMHD_ERR_TIMEOUT = -4,    /* a bounded device-side wait ran out (persistent batched launch) */
    GRMHD_ERR_STATE = -5       /* call out of order (e.g. step before bind) */
} grmhd_status;

enum { GRMHD_BC_PERIODIC = 0, GRMHD_BC_OUTFLOW = 1, GRMHD_BC_FIXED = 2 };
enum { GRMHD_PREC_FP64 = 0, GRMHD_PREC_MIXED = 1 };
/* Divergence-free handling of B (Sec. 3): staggered face fields with upwind
 * constrained transport (Sec. 3.2), or cell-centred fields with GLM hyperbolic
 * cleaning (Sec. 3.1). */
enum { GRMHD_DIVB_CT = 0, GRMHD_DIVB_GLM = 1 };
/* Edge EMF of the CT update: the resistive UCT of Sec. 3.2 (reconstructed electric
 * field), or the ideal-limit HLL UCT of App. A (Ehat = -vhat x q_B from HLL-weighted
 * transverse transport velocities stored at the faces and q_B, both reconstructed to
 * the edges).  The ideal EMF is valid where the stiff implicit solve drives E to
 * -v x B (eta -> 0). */
enum { GRMHD_EMF_RESISTIVE = 0, GRMHD_EMF_IDEAL = 1 };
/* Reconstruction of every face and edge state: the MC limiter (the default of Sec. 5)
 * or PPM (named in Sec. 5 for the star runs; Colella & Woodward's interface
 * interpolation with the MC slope and their monotonicity limits, reaching one cell
 * past the two ghost layers, where periodic wraps, outflow takes the boundary cell
 * and fixed the outermost stored ghost). */
enum { GRMHD_REC_MC = 0, GRMHD_REC_PPM = 1 };

/* Uniform Cartesian grid (Sec. 5 test set-ups).  bc: per direction; FIXED keeps the
 * ghost values that init wrote (Sec. 5, "values at the outer boundaries are kept
 * fixed").  lo/hi give the physical extent (finite, lo < hi in every active
 * direction); dx = (hi - lo)/n. */
typedef struct {
    int ndim;      /* 1, 2 or 3 active directions */
    int n[3];      /* interior cells; ignored (taken as 1) for inactive directions */
    double lo[3];
    double hi[3];
    int bc[3];
} grmhd_grid;

/* IMEX Butcher pair (Sec. 2.3): explicit At (strictly lower), implicit A (lower,
 * a_ii > 0), weights wt, w; row-major s x s in the first s*s entries. */
typedef struct {
    int s; /* 1..4 stages */
    double At[16];
    double A[16];
    double wt[4];
    double w[4];
} grmhd_tableau;

typedef struct {
    double gamma_eos;  /* ideal-gas Gamma (> 1) */
    double cfl;        /* Courant number for grmhd_compute_dt */
    double newton_tol; /* Newton residual tolerance, relative to the momentum terms of
                          f_i (Sec. 2.4); 0 -> 1e-13 (FP64) or 1e-10
                          (mixed, whose FP32 fluxes err near 1e-7).  The FP64 path
                          accepts a root by its FP64 residual; the mixed path by its
                          double-word residual (~1e-14 of the momentum scale) and so
                          needs newton_tol >= 1e-11 (else GRMHD_ERR_ARG) */
    int newton_kmax;   /* Newton iteration cap; 0 -> 50 */
    int precision;     /* GRMHD_PREC_FP64: every step in FP64.  GRMHD_PREC_MIXED: MC
                          reconstruction, HLL fluxes, the edge EMF and the non-stiff
                          sources in FP32, the flux divergence in double-word
                          arithmetic from the FP32 fluxes; the implicit solve /
                          con2prim (its root accepted by a double-word residual, its
                          outputs FP64), CT face update and stage combination stay FP64
                          (div B stays at FP64 round-off because each FP32 edge EMF is
                          shared by the faces around it) */
    double rho_atm;    /* atmosphere (not in the paper): a cell with D < 10 rho_atm, or
                          whose solve fails, is set to rest at (rho_atm, p_atm) with E
                          kept; 0 disables it (failures then keep their primitives) */
    double p_atm;
    int divb;          /* GRMHD_DIVB_CT (0, default) or GRMHD_DIVB_GLM.  GLM (Sec. 3.1):
                          the three "bface" arrays of every call hold cell-centred
                          q_B^i = psi^6 B^i instead of face values, and a fourth field
                          q_Phi = psi^6 Phi (grmhd_bind_phi) is evolved with
                          (f_Phi)^i = alpha q_B^i, s_Phi = -alpha kappa_b q_Phi
                          + q_B^i d_i alpha and s_B^i = -psi^6 alpha gamma^{ij} d_j Phi.
                          FP64 only; not accepted by the batched executor */
    double kappa_b;    /* GLM damping kappa_B >= 0 (Sec. 3.1); unused by CT */
    int emf;           /* GRMHD_EMF_RESISTIVE (0, default) or GRMHD_EMF_IDEAL (App. A):
                          CT, FP64, no FIXED boundary; not accepted by the batched
                          executor */
    int rec;           /* GRMHD_REC_MC (0, default) or GRMHD_REC_PPM: CT with the resistive
                          EMF (FP64, or mixed with FP32 reconstruction) or GLM (FP64); not
                          accepted by the batched executor */
} grmhd_params;

/* IMEX-SSP2(2,2,2) of Sec. 2.3 (Pareschi & Russo), gamma = 1 - 1/sqrt(2). */
grmhd_status grmhd_tableau_ssp2(grmhd_tableau* out);

/* Bytes of device scratch the caller must provide for this grid and tableau
 * (256-byte aligned base). */
grmhd_status grmhd_scratch_bytes(const grmhd_grid* grid, const grmhd_tableau* tab, size_t* bytes);

/* Create a context on the current CUDA device.  No device memory is allocated. */
grmhd_status grmhd_create(const grmhd_grid* grid, const grmhd_params* par, const grmhd_tableau* tab,
                          grmhd_ctx** out);
grmhd_status grmhd_destroy(grmhd_ctx* ctx);

/* Bind the caller's state and scratch.  q: 8 padded cell arrays (D, S_1..3, tau,
 * E^1..3, densitised); bface: 3 padded face arrays (q_B^x, q_B^y, q_B^z); scratch:
 * at least grmhd_scratch_bytes bytes, 256-byte aligned. */
grmhd_status grmhd_bind(grmhd_ctx* ctx, double* const* q, double* const* bface, void* scratch, size_t scratch_bytes);

/* GLM only (Sec. 3.1): bind the caller's q_Phi = psi^6 Phi, one padded cell array
 * (device), evolved in place with the bound state.  Required before
 * grmhd_init_from_prims and grmhd_stage on a GLM context; GRMHD_ERR_STATE on a CT
 * context. */
grmhd_status grmhd_bind_phi(grmhd_ctx* ctx, double* q_phi);

/* Fixed background metric (Sec. 2.1): alpha and psi as padded cell arrays read at
 * every padded cell (ghosts included, no boundary condition applied); NULL = flat
 * (alpha = psi = 1).  The shift is zero. */
grmhd_status grmhd_set_metric(grmhd_ctx* ctx, const double* alpha, const double* psi);

/* Resistivity (Sec. 2.2): eta_cc a padded cell array, or NULL for the uniform eta. */
grmhd_status grmhd_set_eta(grmhd_ctx* ctx, const double* eta_cc, double eta_uniform);

/* Mean-field dynamo (Sec. 2.2, Ohm's law e = xi b + eta j): uniform xi, 0 by
 * default.  The implicit solve then uses the full A_k(W) of Sec. 2.4.  A strong
 * dynamo can give the implicit system more than one physical root; the solve starts
 * from the previous stage's velocity and so follows the root continuous in time. */
grmhd_status grmhd_set_dynamo(grmhd_ctx* ctx, double xi);

/* Initial state (Sec. 4 + Sec. 2.1): if A_edge is not NULL the face fields become
 * the discrete curl q_B^i = eta^{ijk} d_j A_k of the three padded edge arrays (faces
 * whose stencil leaves the array are zero); otherwise the bound face arrays are used
 * as they are.  Then q = prim2con(prim, cell-averaged B) at every padded cell, and
 * prim (8 padded arrays, ghosts included: they are the FIXED boundary values) is
 * kept as the Newton starting point.
 * GLM context: A_edge, if given, is a potential at cell centres (read on the whole
 * padded grid) and the interior cell fields become its central-difference curl
 * (Sec. 4, cell-centred case; ghost values of q_B are left as bound); q uses the
 * cell fields directly.  prim then holds 9 pointers: the 8 above and the primitive
 * Phi (a padded cell array, or NULL for Phi = 0), and the bound q_Phi becomes
 * psi^6 Phi at every padded cell (Sec. 3.1). */
grmhd_status grmhd_init_from_prims(grmhd_ctx* ctx, const double* const* prim, const double* const* A_edge,
                                   grmhd_stream_t stream);

/* Delta t = cfl / max_cells sum_d alpha sqrt(gamma^dd) / dx_d (Sec. 2.5, speed of
 * light).  Synchronises the stream. */
grmhd_status grmhd_compute_dt(grmhd_ctx* ctx, double* dt, grmhd_stream_t stream);

/* One IMEX stage i (0-based) of Sec. 2.3: the implicit E + velocity solve of
 * Sec. 2.4 for the stage state, then the explicit operator (MC + HLL fluxes,
 * sources, UCT edge EMF and CT face update, Secs. 2.1, 3.2) folded into the later
 * stages' bases and the final combination; the last stage writes q^{n+1} into the
 * bound state.  Stages of one step must run in order 0..s-1 with the same dt. */
grmhd_status grmhd_stage(grmhd_ctx* ctx, int i, double dt, grmhd_stream_t stream);

/* All stages of one step: q^n -> q^{n+1}. */
grmhd_status grmhd_step(grmhd_ctx* ctx, double dt, grmhd_stream_t stream);

/* Primitives of the bound state with E held fixed (Sec. 2.6) into prim_out
 * (8 padded arrays; interior written, ghosts copied from the context). */
grmhd_status grmhd_get_prims(grmhd_ctx* ctx, double* const* prim_out, grmhd_stream_t stream);

/* Implicit solve (Sec. 2.4) on caller buffers over the interior: q (8, in/out: q_E
 * replaced by the solution), bface (3), prim (8, in: Newton start, out: solution),
 * R (3, out: (q_E - q_E,in)/a_dt).  a_dt = a_ii dt; a_dt <= 0 holds E fixed. */
grmhd_status grmhd_implicit(grmhd_ctx* ctx, double a_dt, double* const* q, const double* const* bface,
                            double* const* prim, double* const* R, grmhd_stream_t stream);

/* Explicit operator on caller buffers: prim (8 padded, ghosts = FIXED values) and
 * bface (3) -> L (11 padded: 8 cell-centred rates on the interior, 3 face rates on
 * the faces that the step updates).  CT contexts only. */
grmhd_status grmhd_explicit_L(grmhd_ctx* ctx, const double* const* prim, const double* const* bface,
                              double* const* L, grmhd_stream_t stream);

/* GLM explicit operator (Sec. 3.1) on caller buffers: prim (8), cell-centred q_B (3)
 * and q_Phi (padded, ghosts = FIXED values) -> L (12 padded arrays, interior: the 8
 * cell-centred rates, then q_B^1..3 and q_Phi).  GLM contexts only. */
grmhd_status grmhd_explicit_L_glm(grmhd_ctx* ctx, const double* const* prim, const double* const* qB,
                                  const double* q_phi, double* const* L, grmhd_stream_t stream);

/* Diagnostics of the bound state: divb = {mean |div q_B|, rms, max} over interior
 * cells (Sec. 3.2; on a GLM context the central-difference divergence of the cell
 * fields), totals = volume sums of the 8 cell-centred q, nfail = Newton failures
 * since create.  Synchronises the stream. */
grmhd_status grmhd_diagnostics(grmhd_ctx* ctx, double* divb, double* totals, long long* nfail,
                               grmhd_stream_t stream);

/* Elliptic divergence cleaning (Sec. 3.3): solve lap(Phi) = div q_B and set
 * q_B <- q_B - grad(Phi) on the bound field arrays, in place.  The paper applies it
 * after every step and once after the initial data (Sec. 4); call it at those points.
 * Operators (Cartesian reference metric): on a CT context the staggered div (face
 * differences) and face gradient, whose composition is the compact Laplacian, so the
 * cleaned field is divergence-free to the solver's accuracy; on a GLM context central
 * differences with the same compact Laplacian (an approximate projection).  Periodic
 * directions wrap; in the others Phi has zero normal gradient, so the boundary faces
 * are kept and the mean divergence (their net flux) stays.
 * Solver: `cycles` multigrid V(2,2) cycles (red-black Gauss-Seidel, cell-average
 * restriction, linear interpolation, conjugate gradients on the coarsest level), each
 * reducing the error about tenfold; launches only, deterministic, no synchronisation.
 * scratch: caller-owned device memory of grmhd_clean_scratch_bytes bytes, 256-byte
 * aligned.  Grids whose coarsest level (every active extent halved while all are even
 * and >= 4) exceeds 4096 cells are rejected with GRMHD_ERR_ARG. */
grmhd_status grmhd_clean_scratch_bytes(const grmhd_grid* grid, size_t* bytes);
grmhd_status grmhd_clean_divb(grmhd_ctx* ctx, int cycles, void* scratch, size_t scratch_bytes,
                              grmhd_stream_t stream);

/* Kernels launched by this context since create (host-side count). */
long long grmhd_launch_count(const grmhd_ctx* ctx);

/* Checkpoint / resume (not in the paper).  The state q^n and the face fields belong to
 * the caller, who saves them.  Beside them the context keeps the starting point of the
 * implicit solve (Sec. 2.4): the last stage primitives and, per stage, the last root
 * and its change over the previous step (FP32), all in its scratch.  The root of every
 * later solve does not depend on them beyond the Newton tolerance, but a bitwise
 * resume needs them: grmhd_start_bytes gives their size, grmhd_save_start copies them
 * to dst and grmhd_load_start back from src (device or host memory, stream-ordered
 * copies; dst / src at least start_bytes long, 8-byte aligned).  A blob loads only
 * into a context of the same grid, tableau and divergence scheme (the size is
 * checked).  The Newton failure count is not part of it. */
grmhd_status grmhd_start_bytes(const grmhd_ctx* ctx, size_t* bytes);
grmhd_status grmhd_save_start(grmhd_ctx* ctx, void* dst, size_t bytes, grmhd_stream_t stream);
grmhd_status grmhd_load_start(grmhd_ctx* ctx, const void* src, size_t bytes, grmhd_stream_t stream);

/* Optional per-kernel timing (not part of the paper's method: measurement only).
 * When enabled, CUDA events are recorded on the launching stream around every
 * stage kernel (at most 64 launches between two grmhd_kernel_times calls; later
 * ones go untimed).  grmhd_kernel_times waits for the recorded events and returns
 * the cumulative milliseconds and launch counts per kind: [0] implicit solve,
 * [1] face fluxes, [2] edge EMFs, [3] update.  With the resistive edge EMF (CT) the
 * fluxes of every direction and the edge EMFs run in one stencil launch per stage,
 * counted under [1]; [2] then stays empty.  grmhd_set_timing(ctx, 0) stops the
 * recording; what was recorded stays readable, and enabling again restarts the
 * totals from zero.  grmhd_kernel_times fails with GRMHD_ERR_STATE if timing was
 * never enabled. */
grmhd_status grmhd_set_timing(grmhd_ctx* ctx, int enable);
grmhd_status grmhd_kernel_times(grmhd_ctx* ctx, double* ms, long long* launches);

/* Launch overlap (not part of the paper's method: scheduling only).  When enabled,
 * grmhd_stage / grmhd_step launch their kernels with programmatic dependent launch: a
 * kernel may be scheduled as soon as every block of the one before it on the stream
 * has finished, ahead of that grid's completion and memory flush.  It waits on the
 * device until that grid has completed and its writes are visible before it reads or
 * writes anything.  Results are bitwise those of plain launches.  Ignored while
 * per-kernel timing is on (the events between the launches serialise them).  Off by
 * default for a context made by grmhd_create. */
grmhd_status grmhd_set_launch_overlap(grmhd_ctx* ctx, int enable);

/* FP64 fused multiply-add rate of the current device in TFLOP/s (measurement only,
 * not part of the paper's method): a register-only kernel of independent FMA chains,
 * the best of five launches timed with CUDA events on `stream` (synchronises it).  It
 * measures the denominator that FP64-bound kernels are compared with and changes no
 * device setting.  GRMHD_ERR_CUDA without a device. */
grmhd_status grmhd_fp64_fma_rate(double* tflops, grmhd_stream_t stream);

/* The library's own device arithmetic helpers, evaluated elementwise (testing only,
 * not part of the paper's method), so that they can be held to their definitions.
 * Per element, `in` holds 1, 2 or 3 doubles (the arity below, interleaved) and `out`
 * receives 1 or 2; a double-word result is written as hi, lo (each a binary32 value
 * widened exactly).
 *   RSQRT_GE1   1/sqrt(x) for 1 <= x < 2^127 (FP32 estimate + one step of order 3)
 *   RCP_POS     1/x for x > 0 of moderate size (likewise)
 *   D2F         binary64 -> binary32 on the integer pipe (round half away from zero;
 *               below the normal binary32 range a signed zero, above it infinity)
 *   F2D         binary32 -> binary64 on the integer pipe of the binary32 nearest x
 *               (exact; binary32 subnormals become a signed zero)
 *   DW_SPLIT    the double-word hi + lo of x (2 out)
 *   DW_ADD, DW_MUL   double-word sum / product of a, b (2 in, 2 out)
 *   DW_RCP, DW_SQRT  double-word 1/x and sqrt(x) (1 in, 2 out)
 *   QUARTER, TWICE   x/4 and 2x by an exponent move (exact in the normal range)
 *   MINMOD3     minmod(a, b, c) decided on the bit patterns (3 in); MINMOD3_F32 the
 *               same in binary32 of the nearest binary32 inputs
 *   PROD_SIGN   sign of a b decided on the bit patterns: 1, -1, or 0 (2 in)
 *   PPM_LIMIT   the limited parabola edges (aL, aR) of the cell a0 (3 in: a0, aL, aR;
 *               2 out)
 *   TESTS       finite(x) + 2 (x > 0, finite) + 4 (|x| < 1e10 by its high word)
 * Asynchronous on `stream`.  GRMHD_ERR_ARG for an unknown op, n < 0, or NULL arrays
 * with n > 0; n = 0 launches nothing. */
typedef enum {
    GRMHD_NUM_RSQRT_GE1 = 0,
    GRMHD_NUM_RCP_POS = 1,
    GRMHD_NUM_D2F = 2,
    GRMHD_NUM_F2D = 3,
    GRMHD_NUM_DW_SPLIT = 4,
    GRMHD_NUM_DW_ADD = 5,
    GRMHD_NUM_DW_MUL = 6,
    GRMHD_NUM_DW_RCP = 7,
    GRMHD_NUM_DW_SQRT = 8,
    GRMHD_NUM_QUARTER = 9,
    GRMHD_NUM_TWICE = 10,
    GRMHD_NUM_MINMOD3 = 11,
    GRMHD_NUM_MINMOD3_F32 = 12,
    GRMHD_NUM_PROD_SIGN = 13,
    GRMHD_NUM_PPM_LIMIT = 14,
    GRMHD_NUM_TESTS = 15,
    GRMHD_NUM_COUNT = 16
} grmhd_numeric_op;
grmhd_status grmhd_numerics_eval(int op, const double* in, double* out, long long n, grmhd_stream_t stream);

/* Index-bounds violations (diagnostic build only; not part of the paper's method).
 * The library is also built as a checked copy (compiled with GRMHD_CHECK_BOUNDS, in
 * _build_checked/): there every array index its kernels form from a grid position
 * or a stride offset is checked against the padded array; one outside it is counted
 * and the access redirected to element 0, so the kernel runs on without touching
 * memory outside its arrays (its results are then wrong, which the count reports).
 * This call synchronises the device and returns the count since the last reset in
 * *count (reset != 0 clears it).  In the normal build *count is -1 (no checks). */
grmhd_status grmhd_bounds_violations(long long* count, int reset);

/* Message of the last error on the calling thread ("" if none). */
const char* grmhd_last_error(void);

/* ------------------------------------------------------------------------
 * Batched execution (not in the paper: throughput for many independent problems).
 * A batch advances n bound contexts together -- uneven grid sizes, 1-D/2-D/3-D,
 * flat or fixed-metric, any resistivity -- issuing one launch per kernel kind and
 * stage for all of them.  Each problem runs exactly the per-cell arithmetic it runs
 * alone (same kernels' item bodies, no cross-problem reduction), so its results are
 * bitwise those of grmhd_step on that context.  All contexts must share the tableau
 * and the precision, and use constrained transport (GRMHD_DIVB_CT).  The batch reads the contexts' state, scratch, metric and eta
 * at the time of grmhd_batch_create; re-create it after re-binding a context.
 * ------------------------------------------------------------------------ */
typedef struct grmhd_batch_s grmhd_batch;

/* Device scratch (256-byte aligned) for a batch of these contexts: the per-problem,
 * per-stage descriptor table and the work lists. */
grmhd_status grmhd_batch_scratch_bytes(grmhd_ctx* const* ctxs, int n, size_t* bytes);
/* Build the batch (uploads its work lists; synchronises the legacy default stream). */
grmhd_status grmhd_batch_create(grmhd_ctx* const* ctxs, int n, void* scratch, size_t scratch_bytes,
                                grmhd_batch** out);
/* Per-problem time steps (host array of n); uploads the descriptors of problems
 * whose dt changed (synchronises the stream when it does). */
grmhd_status grmhd_batch_set_dt(grmhd_batch* b, const double* dt, grmhd_stream_t stream);
/* One IMEX step of every problem with its current dt (launches only: can be
 * captured in a CUDA graph once the dts are set). */
grmhd_status grmhd_batch_step(grmhd_batch* b, grmhd_stream_t stream);
/* Autotuner: times stage-0 kernels (which write only scratch) for each candidate
 * (threads per block, items per work chunk) per kernel kind and keeps the fastest.
 * The Newton starting points it overwrites are saved to host memory and restored,
 * so later results are unchanged.  reps: timed repetitions per candidate.
 * Synchronises the stream. */
grmhd_status grmhd_batch_autotune(grmhd_batch* b, int reps, grmhd_stream_t stream);
/* Chosen launch shape per kernel kind (8 entries: implicit, flux x/y/z, emf x/y/z,
 * update). */
grmhd_status grmhd_batch_config(const grmhd_batch* b, int* threads, int* items);

/* Persistent launch: nsteps IMEX steps of every problem in ONE cooperative launch
 * (blocks co-resident, at most the device holds).  Per stage it runs the phases of
 * grmhd_batch_step -- the implicit solves; the face fluxes and edge EMFs; the update
 * (after the FIXED-boundary face copy at the start of each step) -- over the same work
 * lists and per-item bodies, with a grid-wide barrier between phases.  A problem's
 * results are bitwise the same alone and in any batch, and for any split of its steps
 * into launches; against grmhd_batch_step they agree to round-off (the compiler may
 * contract the bodies inlined into this one kernel differently).  Every barrier wait
 * is bounded: a
 * block that waits longer than the batch's wait limit (grmhd_batch_set_wait_limit,
 * 1 s by default) sets the batch's error flag, and all blocks then leave the kernel;
 * the problems' states are then partly advanced and must be restored by the caller.
 * synchronize != 0: the call waits for the launch and returns GRMHD_ERR_TIMEOUT if a
 * wait ran out; synchronize == 0: launches only (a memset and a kernel: capturable in
 * a CUDA graph), and grmhd_batch_persistent_status reports later.  Uses the dts of the
 * last grmhd_batch_set_dt for every step.  GRMHD_ERR_CUDA if the device cannot make a
 * cooperative launch. */
grmhd_status grmhd_batch_step_persistent(grmhd_batch* b, int nsteps, int synchronize, grmhd_stream_t stream);
/* Limit of each grid-barrier wait of the persistent launch, in seconds (0..60). */
grmhd_status grmhd_batch_set_wait_limit(grmhd_batch* b, double seconds);
/* Synchronises the stream; GRMHD_ERR_TIMEOUT if a wait of the last persistent launch
 * ran out, GRMHD_OK otherwise. */
grmhd_status grmhd_batch_persistent_status(grmhd_batch* b, grmhd_stream_t stream);
grmhd_status grmhd_batch_destroy(grmhd_batch* b);

/* div B norms of caller-owned face fields without allocating anything.  The paper
 * has no counterpart to this call: it exists for callers that cannot allocate
 * device memory where they want the check (for example a host whose device memory
 * is all owned by its own pool or arena, or a loop that must not allocate after
 * start-up) and so cannot provide the scratch that grmhd_bind needs.
 *
 * grid: as for grmhd_create (finite lo < hi in every active direction); bface: 3
 * padded face arrays (device, q_B^x, q_B^y, q_B^z, read-only; the array of an
 * inactive direction is never read and may be NULL); out: 3 device doubles written
 * with {mean |div q_B|, rms, max |div q_B|} over interior cells, the same quantities
 * as grmhd_diagnostics.  Runs on `stream`; does not synchronise.
 *
 * Scratch: a fixed array inside the library (8192 rows x 3 doubles = 192 KiB) that
 * every GPU loading the library holds until the process exits; grids with more than
 * 8192 * 256 = 2,097,152 interior cells are rejected with GRMHD_ERR_ARG.  Each call
 * rewrites every row it reads, so nothing needs clearing between calls, but all
 * calls share the array: calls that overlap on the GPU (on different streams, or
 * from different threads) race and must be ordered by the caller.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The address
 * is kept until the process exits: after a reset of that device (cudaDeviceReset)
 * it is stale, so a process that resets a device must not call this entry point on
 * it again.  It calls no allocation routine. */
grmhd_status grmhd_divb_noalloc(const grmhd_grid* grid, const double* const* bface, double* out,
                                grmhd_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GRMHD_H */
