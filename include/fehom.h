/*
 * fehom.h -- C ABI of the GB300 (sm_103a) FFT-preconditioned matrix-free finite-element
 * homogenisation solver.
 *
 * The library solves the periodic cell problem of small-strain elasticity (Sec. 2, Eq. weak_form)
 * or scalar conduction (App. A, Eq. weak_form_scalar) discretised on a regular grid of one-node
 * stencils (Sec. 3, Fig. 3): K u = b with K = D^T W C D and b = -D^T W C e (Sec. 3.1,
 * Eq. lin_system, one Newton step from u = 0, which is exact for linear materials).  It uses
 * preconditioned CG with the reference-material preconditioner K_ref = D^T W C_ref D (Sec. 4.1,
 * Eq. Kref), applied in Fourier space as a per-wavevector block (pseudo-)inverse (Sec. 4.2,
 * Eq. M_inverse; Sec. 5.3, Eq. block_inversion) whose blocks are built matrix-free by
 * Algorithm 2 (Sec. 5.2).
 *
 * Conventions shared by every call:
 *   - Unit cell [0, l_x] x [0, l_y] (x [0, l_z]); n[a] nodes (= pixels/voxels) per axis; node
 *     (i, j, k) at (i h_x, j h_y, k h_z), h_a = l_a / n[a]; voxel (i, j, k) has the corner nodes
 *     (i + a, j + b, k + c) mod n.  Flat node index i + n_x (j + n_y k) (x fastest).
 *   - Fields are component-blocked ("SoA"): entry comp * N + node, N = n_x n_y n_z, the ordering
 *     u = [u_1; u_2; ...] of Eq. Du_mat.  c = 1 DOF per node for FEHOM_SCALAR, c = d for
 *     FEHOM_ELASTIC.
 *   - Flux / stress / gradient / strain vectors have m entries: m = d for FEHOM_SCALAR; Mandel
 *     form (Eq. mandel_grad) for FEHOM_ELASTIC with m = 3, order (11, 22, 12) in 2-D and m = 6,
 *     order (11, 22, 33, 23, 13, 12) in 3-D, sqrt(2) on shear strains.
 *   - Material matrices are m x m, row-major, symmetric positive definite.
 *   - Supported sizes: every n[a] is 2^k or 3 * 2^k with 2 <= n[a] <= 1024; n_x even.
 *   - Device pointers are CUDA device (or managed) addresses on the context's device; the caller
 *     owns every buffer it passes; the context owns everything it allocates.
 *   - No call aborts or throws: each returns a status; fehom_last_error() describes the last
 *     failure of a context.  A failed CUDA call returns FEHOM_E_CUDA and leaves the context
 *     unusable for further solves (destroy it).
 */
#ifndef FEHOM_H
#define FEHOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fehom_ctx fehom_ctx; /* opaque, owned by the library */

typedef enum {
  FEHOM_OK = 0,
  FEHOM_E_INVALID = 1,          /* bad argument (NULL, non-finite or non-SPD moduli, bad enum) */
  FEHOM_E_UNSUPPORTED_SIZE = 2, /* grid size outside 2^k / 3*2^k, odd n_x, or too large */
  FEHOM_E_OOM = 3,              /* device allocation failed */
  FEHOM_E_CUDA = 4,             /* a CUDA runtime call failed */
  FEHOM_E_NOT_CONVERGED = 5,    /* max_iter reached; outputs and info are still written */
  FEHOM_E_BREAKDOWN = 6,        /* PCG breakdown: non-positive or non-finite curvature */
  FEHOM_E_STATE = 7             /* call order violated (solve before precond_build, ...) */
} fehom_status;

typedef enum {
  FEHOM_P1TRI2_2D = 1, /* two linear triangles per pixel, split along (0,0)-(1,1), 1 QP each (Fig. 3 b) */
  FEHOM_HEX8_3D = 2,   /* trilinear hexahedron, 2x2x2 Gauss points (3-D analogue of Fig. 3 a) */
  FEHOM_Q1_2D = 3,     /* bilinear quadrilateral, 2x2 Gauss points (Fig. 3 a) */
  FEHOM_P1TRI4_2D = 4  /* two-node stencil (Fig. 3 c, N_n = 2): a corner node and a pixel-centre node per
                          pixel, four linear triangles (edge, centre) with one point each, w = V_p/4;
                          FEHOM_SCALAR only.  Fields have c = 2 blocks of N values: corner nodes
                          (node i + n_x j), then pixel centres (pixel i + n_x j).  The Fourier blocks are
                          Hermitian 2 x 2 (fehom_get_symbol_inverse: entries 00, 11, Re 01, Im 01); the
                          constant over both node types is the single null mode, removed from fields */
} fehom_elem;

typedef enum { FEHOM_SCALAR = 1, FEHOM_ELASTIC = 2 } fehom_physics;

typedef enum {
  FEHOM_FP64 = 0,  /* every step in FP64 */
  FEHOM_MIXED = 1  /* FP32 stiffness apply, FFT and vectors inside an FP64 iterative-refinement loop;
                      FP64 dots, alpha/beta, true residual and volume averages */
} fehom_precision;

typedef struct {
  int precision;     /* fehom_precision (default FEHOM_FP64) */
  int max_iter;      /* PCG iteration cap per load (default 10000); mixed: cap on inner iterations in total */
  double inner_tol;  /* mixed only: relative K_ref^-1-norm reduction per inner FP32 solve (default 1e-3) */
  void* stream;      /* cudaStream_t for every launch and copy; NULL = a blocking stream the context creates */
  int use_graph;     /* 1 (default): replay PCG iterations from a captured CUDA graph; 0: plain launches */
  int profile;       /* 1: record CUDA events around every kernel of the PCG iterations (see fehom_kernel_times) */
  int autotune;      /* 1 (default): on the first solve of a batch size, time the FFT passes' launch plans
                        (x-line pairs per CTA, columns per CTA) on the context's buffers and keep the fastest.
                        The chosen plans (and the stencil tuner's) are kept for the process: a later context
                        with the same device, element, grid, field blocks, batch size, precision and
                        restricting options takes them without timing again */
  int x0_scaling;    /* 1 (default): a warm start x0 (mean removed) is replaced, per load, by gamma x0 with
                        gamma = <b, x0> / <x0, K x0> (0 when <x0, K x0> = 0): the multiple of x0 closest to
                        the solution in the energy norm, never farther from it than the zero guess */
  int fft_xy;        /* FP32 register-split FFT passes: the fused x-y passes (3-D fields with n x n planes,
                        n = 32, 64, 96 or 128) and the last-axis pass (nz = 32, 64, 96, 128 or 256; c = 1 or
                        3): -1 (default) the tuner decides for
                        each (the generic passes when autotune = 0), 0 never, 1 always when supported */
  int residual_df;   /* mixed only: 1 (default) the refinement residual is updated as r -= K d for each FP32
                        correction d, with K d evaluated in double-float arithmetic (pairs of floats, about
                        48 significant bits, on the FP32 pipe) where supported (FEHOM_HEX8_3D elasticity with
                        isotropic phases on cubic voxels; see fehom_residual_update); 0 always recomputes
                        b - K x with the FP64 stiffness */
  int stencil_rows;  /* FEHOM_HEX8_3D PCG stiffness apply: node rows per tile (tiles are 32 x rows nodes), 8 or
                        16 (FP32: node planes staged by cp.async copies); 0 (default) the stencil tuner times
                        both heights, and for FP32 both node-plane stagings (cp.async copies or one Tensor
                        Memory Accelerator box per plane), on the first solve of a batch size and keeps the
                        fastest (with autotune = 0: 16 rows for FP64, 8 for FP32, cp.async); see
                        fehom_stencil_plan */
} fehom_options;

/* Kernel classes of one PCG iteration, for fehom_kernel_times. */
enum {
  FEHOM_K_STIFFNESS = 0, /* K p and <p, K p> (Sec. 5.1) */
  FEHOM_K_FFT_X_FWD = 1, /* r -= alpha K p, forward FFT along x */
  FEHOM_K_FFT_Y_FWD = 2, /* forward FFT along y (3-D only) */
  FEHOM_K_FFT_LAST = 3,  /* last axis: forward FFT, block solve (Sec. 5.3), <r, z>, inverse FFT */
  FEHOM_K_FFT_Y_INV = 4, /* inverse FFT along y (3-D only) */
  FEHOM_K_FFT_X_INV = 5, /* inverse FFT along x, x += alpha p, p = z + beta p */
  FEHOM_K_COUNT = 6
};

typedef struct {
  int iterations;          /* PCG iterations (mixed: inner FP32 iterations summed over refinements) */
  int refinements;         /* mixed: outer FP64 refinement steps (FP64: 0) */
  int converged;           /* 1 if sqrt(<r, K_ref^+ r>) <= tol * sqrt(<b, K_ref^+ b>) in FP64 */
  double rel_residual_M;   /* final sqrt(<r, K_ref^+ r> / <b, K_ref^+ b>), r the recursive (FP64) or true (mixed) residual */
  double rel_residual_2;   /* final true ||b - K u||_2 / ||b||_2, computed in FP64 */
  double solve_ms;         /* device time of this load's share of the solve (the batch time for batched loads) */
} fehom_solve_info;

/* Default options (precision FP64, max_iter 10000, inner_tol 1e-3, default stream, graphs on). */
void fehom_default_options(fehom_options* opt);

/*
 * fehom_setup -- create a context for one periodic cell (Sec. 3, Fig. 3; Sec. 4.1, Eq. Kref).
 *   out            receives the new context (set to NULL on failure).
 *   elem, physics  fehom_elem / fehom_physics; FEHOM_HEX8_3D needs n[2] > 1, the 2-D elements n[2] == 1.
 *   n              nodes per axis (x, y, z), see the size rule above.
 *   cell           cell edge lengths l_x, l_y, l_z (host, 3 doubles), or NULL for the unit cell.
 *   phase_ids      N uint8 phase ids, one per pixel/voxel, x fastest (host or device, per ids_on_device);
 *                  copied, the caller may free it after the call.  Every id must be < n_phases.
 *   n_phases       1..256.
 *   phase_moduli   host, n_phases x m x m doubles: the material matrix C of each phase (Sec. 3.1; the
 *                  conductivity matrix of App. A for FEHOM_SCALAR).  Copied.
 *   ref_material   host m x m C_ref, or NULL for the volume mean C_mean = (1/|Y|) sum_Q C(x_Q) w_Q
 *                  (Sec. 6.2).  Copied.
 *   opt            NULL for the defaults.
 * Allocates the device work buffers of one load; fehom_solve grows them for more loads.
 * Errors: FEHOM_E_INVALID, FEHOM_E_UNSUPPORTED_SIZE, FEHOM_E_OOM, FEHOM_E_CUDA.
 */
fehom_status fehom_setup(fehom_ctx** out, int elem, int physics, const int64_t n[3], const double* cell,
                         const uint8_t* phase_ids, int ids_on_device, int n_phases,
                         const double* phase_moduli, const double* ref_material, const fehom_options* opt);

/*
 * fehom_precond_build -- Algorithm 2 (Sec. 5.2) and the block (pseudo-)inversion of Sec. 5.3.
 * For each DOF type beta it applies K_ref (the stiffness kernel with the uniform material C_ref)
 * to the unit impulse at node 0, forward-FFTs the c result components into the diagonals of the
 * Fourier blocks K_hat[alpha, beta](k), checks that the blocks are real symmetric, inverts them per
 * wavevector and stores the Moore-Penrose pseudo-inverse of the k = 0 block (the zero matrix for
 * one-node stencils).  The table is kept in FP64 (and FP32 for the mixed path), half spectrum.
 * Errors: FEHOM_E_STATE (no setup), FEHOM_E_INVALID (a block that is not real symmetric positive
 * definite away from k = 0), FEHOM_E_OOM, FEHOM_E_CUDA.
 */
fehom_status fehom_precond_build(fehom_ctx* ctx);

/*
 * fehom_solve -- solve the cell problem for n_loads macroscopic gradients / strains e_l
 * (Eq. lin_system with u_(0) = 0 and Eq. prec_lin_system_FFT), all loads as one batch.
 *   loads          host, n_loads x m doubles (row l = e_l).
 *   tol            PCG stop: sqrt(<r, K_ref^+ r>) <= tol * sqrt(<b, K_ref^+ b>) (Sec. 6, termination
 *                  criteria, normalised by b).  0 < tol < 1.
 *   x0             NULL (zero initial guess) or a device array of n_loads x c x N FP64 initial guesses;
 *                  their mean per component is removed before use.
 *   fluct_out      NULL, or n_loads x c x N FP64 fluctuation fields u~ (mean zero per component),
 *                  host or device per fluct_on_device.
 *   mean_flux_out  NULL or host n_loads x m: <sigma>_l = (1/|Y|) sum_Q w_Q C_Q (e_l + (D u~_l)_Q).
 *   c_eff_out      NULL or host m x m: C_eff = S E^-1 (S, E: mean fluxes and loads as columns), written
 *                  only when n_loads == m and E is invertible (the unit loads give C_eff[:, l] = <sigma>_l).
 *   info           NULL or host array of n_loads fehom_solve_info.
 * Errors: FEHOM_E_STATE (before fehom_precond_build), FEHOM_E_INVALID, FEHOM_E_NOT_CONVERGED
 * (outputs written), FEHOM_E_BREAKDOWN, FEHOM_E_OOM, FEHOM_E_CUDA.
 */
fehom_status fehom_solve(fehom_ctx* ctx, int n_loads, const double* loads, double tol, const double* x0,
                         double* fluct_out, int fluct_on_device, double* mean_flux_out, double* c_eff_out,
                         fehom_solve_info* info);

/* ---------------------------------------------------------------------------------------------
 * Batches: many cells (contexts, possibly of different grid sizes and materials) solved together
 * for the same loads.  The PCG iterations of all contexts are captured into one CUDA graph with one
 * branch per context and replayed until every load of every context is finished (the stopping test
 * and iteration bookkeeping stay per context and load, in device memory); the set-up and refinement
 * steps of each context run on that context's own stream.  Contexts must share one device and one
 * precision, have passed fehom_precond_build, and should have their own streams (NULL stream option)
 * so that their branches can run concurrently.  A context must not be used elsewhere while a batch
 * that holds it is solving.
 * ------------------------------------------------------------------------------------------- */
typedef struct fehom_batch fehom_batch; /* opaque, owned by the library; the contexts stay the caller's */

/* Create a batch over n_ctx contexts (the array is copied; the contexts are not). */
fehom_status fehom_batch_create(fehom_batch** out, int n_ctx, fehom_ctx* const* ctxs);

/* Solve every context of the batch for the n_loads loads (host, n_loads x m, the same for all).
 * Outputs per context c, host arrays or NULL: mean_flux_out[c][n_loads][m], c_eff_out[c][m][m] (when
 * n_loads == m), info[c][n_loads] (solve_ms = the whole batch).  Fields stay in each context
 * (fluctuation fields are not returned by this call).  Returns the worst status over the contexts. */
fehom_status fehom_solve_batch(fehom_batch* b, int n_loads, const double* loads, double tol, double* mean_flux_out,
                               double* c_eff_out, fehom_solve_info* info);

void fehom_batch_destroy(fehom_batch* b);
const char* fehom_batch_last_error(const fehom_batch* b);

/* Release every device and host resource of the context (NULL is ignored). */
void fehom_destroy(fehom_ctx* ctx);

/* Text of the context's last error ("" if none); owned by the context, valid until the next call.  With
 * ctx == NULL: the message of the last failed fehom_setup on the calling thread. */
const char* fehom_last_error(const fehom_ctx* ctx);

/* Device time spent in each kernel class of the PCG iterations since setup, recorded with CUDA
 * events on the context's stream when opt.profile == 1 (iterations after a load has finished are
 * not counted).  precision selects the FP64 kernels or the FP32 kernels of the mixed path.
 * ms[FEHOM_K_COUNT]: total milliseconds; count[FEHOM_K_COUNT]: launches timed. */
fehom_status fehom_kernel_times(const fehom_ctx* ctx, int precision, double* ms, int64_t* count);

/* PCG coefficients alpha_j, beta_j (j = 0 .. count-1) of the last PCG run of a load (FP64 solve; the
 * last inner FP32 run of a mixed solve), up to `capacity` and at most 2048; with them the CG-Lanczos
 * tridiagonal matrix T (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_j,j+1 = sqrt(beta_j)/alpha_j)
 * gives Ritz values of K_ref^+ K (Sec. 4.3).  Host arrays. */
fehom_status fehom_pcg_coefficients(fehom_ctx* ctx, int load, int capacity, double* alpha, double* beta, int* count);

/* Element-by-element eigenvalue bounds of K_ref^+ K (Sec. 4.3).  For each node I the lower (upper)
 * bound is the smallest (largest) extreme generalized eigenvalue of (C_e, C_ref) over the voxels e that
 * contain the node; counted once per DOF of the node and sorted, they bound the eigenvalues of the
 * preconditioned operator one by one.  Returned as ascending (value, count) lists: lo_values /
 * lo_counts (n_lo entries) and hi_values / hi_counts (n_hi entries), host arrays of at least
 * n_phases entries; the counts add up to c N.  Needs fehom_setup. */
fehom_status fehom_eig_bounds(fehom_ctx* ctx, double* lo_values, int64_t* lo_counts, int* n_lo, double* hi_values,
                              int64_t* hi_counts, int* n_hi);

/* Launch plan of the FFT passes in use for a precision (FEHOM_FP64 / FEHOM_MIXED): x-line pairs per
 * CTA, columns per CTA of the y pass and of the last-axis pass (0 = built-in choice, not tuned yet),
 * the device milliseconds of the chosen plans measured by the tuner (ms[3]: x passes, y passes,
 * last-axis pass; may be NULL), and the register-split FP32 passes in use as a bit mask (*xy_fused,
 * may be NULL): bit 0 = fused x-y passes (n x n planes, n = 32, 64, 96 or 128; then ms[0] times them and
 * ms[1] = 0), bit 1 = register-split last-axis pass (nz = 32, 64, 96, 128 or 256). */
fehom_status fehom_fft_plan(const fehom_ctx* ctx, int precision, int* pairs, int* tc_y, int* tc_last, double* ms,
                            int* xy_fused);

/* Stencil plan of the PCG stiffness apply of one precision (FEHOM_HEX8_3D): *rows = the node rows per
   tile in use (8 or 16); *staging = the FP32 node-plane staging in use (0 cp.async copies, 3 one Tensor
   Memory Accelerator box per plane); ms[4] = the tuner's timings of one apply with 8 and 16 rows with
   cp.async staging, then with TMA staging (0 if not timed, -1 if the candidate failed to launch).  Any
   output may be NULL. */
fehom_status fehom_stencil_plan(const fehom_ctx* ctx, int precision, int* rows, int* staging, double* ms);

/* Replaces the reference material (Sec. 4.1, Eq. Kref; m x m, host, symmetric positive definite) of
 * the context, e.g. when the tangent of a nonlinear problem changes (the reassembly of Sec. 5 before
 * Algorithm 2).  Call fehom_precond_build before the next solve (FEHOM_E_STATE otherwise). */
fehom_status fehom_set_reference(fehom_ctx* ctx, const double* C_ref);

/* Newton's method of Algorithm 1 for a nonlinear conductivity (FEHOM_SCALAR on FEHOM_HEX8_3D):
 * the nonlinear system D^T W q(e + D u) = 0 (Sec. 3) with the per-phase law
 *     q(g) = k_p s^((n_p - 1) / 2) g,  s = 1 + |g|^2 / g0^2,
 * k_p from the context's (isotropic) phase conductivities, n_p = power_n[p] > 0 (n_p = 1: linear).
 * Each Newton step evaluates flux and tangent at the 2 x 2 x 2 Gauss points (FP64), sets the reference
 * material to the volume mean of the tangent and rebuilds the preconditioner (Algorithm 2), solves
 * K_t delta = -R with PCG to the relative K_ref^-1-norm tolerance tol_cg, updates u and stops when
 * ||D delta|| <= eta_nw ||D u|| (Sec. 6, termination criteria), after at most max_newton (<= 32) steps.
 * e: host, 3 entries.  fluct_out: NULL, or N doubles (device when fluct_on_device, else host) that
 * receive the mean-zero fluctuation.  mean_flux_out: host, 3 entries, or NULL.  info: host, filled.
 * Leaves the context's reference material at the last tangent mean.  FEHOM_E_NOT_CONVERGED when the
 * Newton test did not pass within max_newton steps (outputs are still written). */
typedef struct {
  int newton_iterations;  /* Newton steps taken */
  int pcg_iterations;     /* PCG iterations over all steps */
  int converged;          /* 1 when the Newton test passed */
  int n_hist;             /* entries of the histories below */
  double residual[32];    /* ||R(u_k)||_2 at the start of step k */
  double increment[32];   /* ||D delta_k|| / ||D u_{k+1}|| of step k */
  int pcg_per_step[32];   /* PCG iterations of step k */
} fehom_newton_info;
fehom_status fehom_newton_solve(fehom_ctx* ctx, const double* e, const double* power_n, double g0, double tol_cg,
                                double eta_nw, int max_newton, double* fluct_out, int fluct_on_device,
                                double* mean_flux_out, fehom_newton_info* info);

/* Energy form of the effective tensor of the last fehom_solve whose n_loads == m loads were linearly
 * independent and which asked for C_eff: with fields x_l, right-hand sides b_l and true residuals
 * r_l = b_l - K x_l, the energies sum_Q w_Q (e_i + D x_i)^T C (e_j + D x_j) = e_i^T C_eff e_j |Y|
 * (the Hill-Mandel form of the homogenised energy, Sec. 2 with the quadrature of Sec. 3) are
 * |Y| e_i^T <C> e_j - x_j . b_i - x_i . r_j, symmetrised; the result is stationary at the solution,
 * so its error is second order in the solve error (the volume-averaged stress of fehom_solve is
 * first order).  FP64, reduced on the device in a fixed order.  c_eff: host, m x m row-major.
 * FEHOM_E_STATE when no such solve has run. */
fehom_status fehom_effective_energy(const fehom_ctx* ctx, double* c_eff);

/* Number of kernel launches the context has issued since setup (kernels replayed from a CUDA graph
 * are counted once per replay). */
fehom_status fehom_launch_count(const fehom_ctx* ctx, int64_t* count);

/* Grid facts of a context: c (DOF per node), m (flux components), N (nodes), nxh (n_x / 2 + 1). */
fehom_status fehom_query(const fehom_ctx* ctx, int* c, int* m, int64_t* N, int64_t* nxh);

/* ---------------------------------------------------------------------------------------------
 * Operator-level entry points: single steps of the solve, exposed so that each can be checked on
 * its own.  All arrays are device arrays of the context's device; `precision` selects FP64
 * (double arrays) or FEHOM_MIXED (float arrays).  They run on the context's stream and return
 * after the work is complete.
 * ------------------------------------------------------------------------------------------- */

/* y = K x = D^T W C D x, matrix-free (Sec. 5.1, the gradient as a short convolution and the
 * weighted divergence D^T W).  x, y: c x N.  Needs fehom_setup. */
fehom_status fehom_apply_stiffness(fehom_ctx* ctx, const void* x, void* y, int precision);

/* b = -D^T W C e for one macroscopic gradient / strain e (host, m doubles); b: c x N FP64. */
fehom_status fehom_rhs(fehom_ctx* ctx, const double* e, double* b);

/* Refinement residual in double-float arithmetic (the step of the mixed solve, option residual_df):
   r_out = r_in - K d for one load, d an FP32 field (device, c x N, the layout of fehom_apply_stiffness),
   r_in / r_out FP64 fields (device; r_out may equal r_in).  K d is evaluated with the FP64 kernel's
   element (face form, closed-form isotropic duals, Sec. 5.1 operator K = D^T W C D) on pairs of floats
   hi + lo: the first butterfly stage of d is exact, later sums and products round once in double-float
   (relative error of order 2^-44 of the operands' magnitudes); r_out = r_in - (hi + lo) is formed in
   FP64.  sums_out (host, 1 + m doubles, or NULL): ||r_out||^2, then the volume-averaged stress of the
   field d alone (Mandel, no macroscopic strain; the change of <sigma> that adding d to the fluctuation
   makes).  FEHOM_E_UNSUPPORTED_SIZE unless the context is FEHOM_HEX8_3D elasticity with isotropic phases
   on cubic voxels. */
fehom_status fehom_residual_update(fehom_ctx* ctx, const float* d, const double* r_in, double* r_out,
                                   double* sums_out);

/* The right-hand side of fehom_rhs (b = -D^T W C e, Sec. 3.1 Eq. lin_system) in double-float arithmetic,
   as the mixed solve forms it when residual_df is on: the per-phase prestress w S P^T C e is split into
   float pairs on the host and the element's transposed operations run on pairs of floats; b (device,
   c x N doubles) = hi + lo.  Same support and errors as fehom_residual_update. */
fehom_status fehom_rhs_df(fehom_ctx* ctx, const double* e, double* b);

/* z = K_ref^+ r = F^-1 K_hat^+ F r (Eq. M_inverse); r, z: c x N.  Needs fehom_precond_build. */
fehom_status fehom_apply_precond(fehom_ctx* ctx, const void* r, void* z, int precision);

/* The two halves of one PCG iteration as the solve runs them (Sec. 4.1, PCG of Saad's Alg. 9.1 in the
 * symmetric form, with the operator K = D^T W C D of Sec. 5.1 and the preconditioner K_ref^+ of
 * Eq. M_inverse / Sec. 5.3), for n_loads loads at once (1 <= n_loads <= 64), exposed so that the fused
 * kernels of the iteration can be checked one by one.  Fields are device arrays of n_loads x c x N
 * values of the precision's type (double for FEHOM_FP64, float for FEHOM_MIXED), load-major; the
 * scalars are host arrays of n_loads doubles.  The calls use scratch PCG states of the context, not the
 * solve's, and return after the work is complete.
 *
 * fehom_pcg_apply_stiffness -- the stiffness launch of an iteration: ap = K p, with <p, K p> reduced in
 * the same launch (FP64 kernels in FP64; FP32 kernels with compensated FP32 products, then FP64) and
 * alpha = rz / <p, K p> formed on the device.
 *   rz       <r, z> of each load (the numerator of alpha).
 *   rows     FEHOM_HEX8_3D: node rows per tile, 8 or 16 (0 = the context's plan); ignored otherwise.
 *   staging  FEHOM_HEX8_3D FP32 node-plane staging: 0 = the context's plan (the stencil tuner's pick, else
 *            cp.async copies); 1 = 4-byte cp.async copies of every entry; 2 = 16-byte cp.async row copies
 *            (n_x a multiple of 32, rows 16-byte aligned); 3 = one Tensor Memory Accelerator box per plane,
 *            issued by one thread, with mbarrier completion (same condition).  A staging that does not apply
 *            to the context returns FEHOM_E_UNSUPPORTED_SIZE.
 *   pAp, alpha  NULL or host outputs.
 * Errors: FEHOM_E_INVALID, FEHOM_E_BREAKDOWN (<p, K p> not positive and finite for some load; outputs
 * still written), FEHOM_E_CUDA. */
fehom_status fehom_pcg_apply_stiffness(fehom_ctx* ctx, int precision, int n_loads, const void* p, void* ap,
                                       const double* rz, int rows, int staging, double* pAp, double* alpha);

/* fehom_pcg_precond_step -- the preconditioner passes of an iteration with their fused vector updates:
 *   alpha != NULL:  r -= alpha Ap;  z = K_ref^+ r;  rz_new = <r, z>;  beta = rz_new / rz;
 *                   x += alpha p;  p = z + beta p            (r, x, p updated in place; ap read)
 *   alpha == NULL:  the first apply of PCG:  z = K_ref^+ r;  rz_new = <r, z>;  p = z   (ap, x, rz unused)
 * <r, z> is the Parseval sum over the half spectrum, formed in the last-axis pass.  The FFT launch plan is
 * the context's (option fft_xy, or the tuner's choice after a solve).  rz_new, beta: NULL or host outputs.
 * Errors: FEHOM_E_STATE (before fehom_precond_build), FEHOM_E_INVALID, FEHOM_E_BREAKDOWN (non-finite
 * <r, z>), FEHOM_E_OOM, FEHOM_E_CUDA. */
fehom_status fehom_pcg_precond_step(fehom_ctx* ctx, int precision, int n_loads, void* r, const void* ap, void* x,
                                    void* p, const double* alpha, const double* rz, double* rz_new, double* beta);

/* Copy the FP64 inverse symbol table to the host: out[e * Nh + (kz * n_y + ky) * nxh + kx] for the
 * packed symmetric entries e of K_hat^+(k) (c = 1: (00); c = 2: (00, 11, 01); c = 3: (00, 11, 22,
 * 12, 02, 01)), half spectrum kx = 0..n_x/2, Nh = nxh n_y n_z.  The stored values include the
 * inverse-DFT factor 1/N.  out holds c(c+1)/2 * Nh doubles.  Needs fehom_precond_build. */
fehom_status fehom_get_symbol_inverse(fehom_ctx* ctx, double* out);

/* <sigma> = (1/|Y|) sum_Q w_Q C_Q (e + (D u)_Q) for a device FP64 field u (c x N) and host load e. */
fehom_status fehom_mean_flux(fehom_ctx* ctx, const double* e, const double* u, double* out);

/*
 * fehom_mean_flux_noalloc -- the same volume average as fehom_mean_flux, for callers that must not
 * allocate device memory during the call: code running while a memory budget or pool may not grow,
 * or in places where cudaMalloc is not allowed.  (The paper has no counterpart; it is an interface
 * convenience of this library.)  fehom_mean_flux allocates its load table and partial sums on first
 * use; this call allocates nothing.  Its scratch is a fixed array of 8192 doubles (64 KiB) inside the
 * library, which every GPU that loads the library keeps until the process exits.  It holds the
 * per-CTA partial sums, their totals and the per-phase load table, so it serves grids up to about
 * 256^3 voxels in 3-D; larger grids are rejected with FEHOM_E_UNSUPPORTED_SIZE and a message giving
 * the space they would need.  The first call on a device looks up the array's device address.  The call
 * copies the load table from host memory and waits for the stream, so it never runs on a stream that is
 * being captured into a CUDA graph: it returns FEHOM_E_STATE there.  All calls share the one array and it
 * keeps the last call's contents (each call overwrites every entry it reads, so nothing needs
 * clearing): calls that overlap on the GPU, from several threads or streams, race and must be
 * serialised by the caller.  Arguments as for fehom_mean_flux; the context is only read.
 */
fehom_status fehom_mean_flux_noalloc(fehom_ctx* ctx, const double* e, const double* u, double* out);

#ifdef __cplusplus
}
#endif

#endif /* FEHOM_H */
