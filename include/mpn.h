/*
 * mpn.h — C ABI of the batched NeuRLP-PDE least-squares solver (sm_103a).
 *
 * The solver computes, for a batch of independent PDE instances on a regular
 * (t, x[, y]) grid, the least-squares solution z* = argmin ||A z - d||_2 of the
 * constraint system of Section 3 of "Mechanistic PDE Networks" (Eqs. 3-8):
 *   equation rows        sum_v c_{v,i} z_{v,i} = b_i              (Eq. 3)
 *   Dirichlet rows       u_i = omega_i,  i in the boundary set    (Eq. 4)
 *   derivative rows      s^k z_{m,i} = finite difference of u     (Eq. 5)
 *   Taylor smoothness    u_i +- s u'_i + s^2/2 u''_i = u_{next/prev}(Eqs. 6-7)
 * through its normal equations A^T A z = A^T d (Eq. 9), and the adjoint
 * solve A^T A d_z = g_z of the backward saddle-point system (Eq. 11) with the
 * parameter gradients that follow it.
 *
 * Unknowns per grid point (V = 1 + 2D for D grid dimensions, time first):
 *   v = 0: u,  v = 1 + 2d: first derivative along d,  v = 2 + 2d: second.
 * Layouts (all row-major, last grid dimension fastest, N = n_t n_x [n_y]):
 *   z, g_z, dz       [B][V][N]  float
 *   fields, dfields  [F][B][N]  float   coefficient fields
 *   scalars,dscalars [V][B]     float   per-instance coefficients (read for
 *                                       v with field_of[v] < 0)
 *   rhs, drhs        [B][N]     float   b of the equation rows
 *   omega, domega    [B][N]     float   Dirichlet values; read (and written)
 *                                       only on boundary points
 *   u0               [B][N]     float   optional warm start for u
 * The coefficient of unknown v at point i of instance b is
 *   fields[field_of[v]][b][i] if field_of[v] >= 0, else scalars[v][b].
 *
 * Boundary set: the t = 0 face, both faces of every non-periodic spatial
 * dimension, and the t = t_f face when final_time_rows is set.
 * Derivative rows sit at every point; non-periodic edges use second-order
 * one-sided three-point forms (the paper says one-sided differences are used
 * at the grid edges without giving their order).
 *
 * Ownership: every array argument is caller-owned DEVICE memory unless marked
 * host.  The problem object owns its workspace (allocated by mpn_create).
 * Calls are asynchronous on `stream` (a cudaStream_t) except that each
 * refinement sweep reads a few per-instance scalars back to the host, so a
 * solve call returns after its work is complete.
 *
 * Diagnostics: with the environment variable MPN_TRACE set, every refinement
 * sweep prints its inner iterations, correction size, residual and predicted
 * error to stderr.
 *
 * Errors: every call returns an mpn_status.  Nothing aborts or hangs: PCG
 * and refinement counts are capped; a non-finite value or a growing residual
 * is reported, and stats are filled in either way.
 */
#ifndef MPN_H
#define MPN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPN_OK = 0,
  MPN_ERR_INVALID_ARG = 1,   /* bad descriptor, null pointer, bad size */
  MPN_ERR_UNSUPPORTED = 2,   /* valid for the method, not for this solver */
  MPN_ERR_NOT_CONVERGED = 3, /* max_refine reached above tolerance */
  MPN_ERR_NONFINITE = 4,     /* NaN/Inf in inputs or iterates */
  MPN_ERR_DIVERGED = 5,      /* refinement correction grew */
  MPN_ERR_CUDA = 6,          /* a CUDA call failed (see mpn_last_cuda_error) */
  MPN_ERR_NO_MEMORY = 7
} mpn_status;

typedef struct mpn_desc {
  int ndim;               /* D = 2 (t, x) or 3 (t, x, y) */
  int n[3];               /* grid points per dimension, time first; n[2] = 1 if D = 2 */
  double step[3];         /* uniform steps s_t, s_x, s_y */
  int periodic[3];        /* periodic[0] must be 0 */
  int stencil;            /* derivative rows: 3 (supported) or 5 (MPN_ERR_UNSUPPORTED) */
  int final_time_rows;    /* 1: Dirichlet rows also on t = t_f */
  int batch;              /* B independent instances */
  int nfields;            /* F coefficient fields */
  int field_of[7];        /* per unknown: field index, or -1 for a per-instance scalar */
  double tol;             /* stop when the predicted relative error of u is <= tol */
  int max_refine;         /* cap on FP64 refinement sweeps */
  int inner_iters;        /* FP32 PCG iterations per refinement sweep */
  int cheb_degree;        /* Chebyshev-Jacobi smoothing steps, pre and post */
  int coarse_min;         /* spatial dims are halved while the half is >= this */
  int max_coarse;         /* largest coarsest-level system (unknowns per instance) */
  int fused_coarse;       /* 1: the coarse levels whose data fit in one thread-block cluster's shared
                             memory per instance run as one kernel per V-cycle; 0: one kernel per
                             operator pass at every level (same arithmetic) */
  int fused_step;         /* 1: on levels with float4 rows (D = 3, n_y % 4 == 0, n_y >= 8,
                             n_x % 4 == 0) both operator passes of a smoothing step, residual or apply
                             run as one kernel through shared memory, on tiles of whole y rows where
                             n_y <= 128 (n_t % 4 == 0) and of 64-point y segments where n_y > 128
                             (n_y % 64 == 0, n_t % 8 == 0); 2: the same with y segments wherever
                             they apply (n_y >= 128); 3 (default): as 1, and on levels with periodic
                             x and y, n_x % 16 == 0, n_y % 64 == 0, n_t % 8 == 0, uniform steps and
                             a coefficient layout whose fields are c_x and c_y (transport) or c_0
                             and c_xx = c_yy (reaction-diffusion), whose 16 x 64 columns number at
                             least half the SMs over the batch, every step but PCG's direction
                             update marches along t through shared memory (one CTA per column and
                             chunk of time planes); 4: the same on every such level whatever its
                             size; 0: two kernels (same arithmetic) */
  int krylov;             /* inner FP32 solver of each refinement sweep: MPN_KRYLOV_CG (conjugate
                             gradients) or MPN_KRYLOV_FGMRES (flexible GMRES(m), m = the sweep's
                             iteration count, with the same V-cycle as right preconditioner, the
                             solver of Section 3.1) */
  int coarsen_time;       /* 1: the multigrid hierarchy halves the first (time) axis too, for problems
                             that are elliptic in it (no first time derivative, e.g. Laplace's
                             equation with the first axis as a space axis); 0 (default): time is
                             kept on every level, as a central first time derivative requires */
  int direct;             /* 1: batched direct path for small problems: no hierarchy, the whole reduced
                             system is factorised (banded Cholesky, explicit inverse) once per forward
                             solve and every refinement sweep applies the inverse (at most 4096 grid
                             points per instance); 0 (default): multigrid-preconditioned Krylov */
  int variable_steps;     /* 1: every interval of every axis has a step of its own, per instance
                             (Section 2, "discretization"; learnable), given by mpn_set_steps before
                             the first solve; step[] is then unused.  The derivative rows take the
                             three-point forms of the quadratic through their points (central inside
                             and on periodic axes with sbar = (h_{i-1} + h_i) / 2, one-sided at the
                             ends of open axes with sbar = the adjacent interval); the Taylor rows
                             use the interval to the neighbour.  Runs the general two-pass kernels
                             on every level (no fused step, no fused coarse end).  0 (default):
                             uniform steps step[] */
  double bc_alpha[3];     /* boundary rows on both faces of spatial axis d (d = 1, 2; entry 0 unused): */
  double bc_beta[3];      /* alpha_d u + beta_d du/dx_d = omega (Section 2: Dirichlet, Neumann or
                             mixed conditions).  Dirichlet (1, 0) is the default; any other pair on an
                             open axis makes the problem run the general two-pass kernels on every
                             level.  A point on several faces has the row of the first face in the
                             order t = 0, t = t_f, then the spatial axes in order (time faces are
                             Dirichlet).  alpha and beta must be finite and not both zero. */
  int adj_inner_iters;    /* FP32 PCG iterations per refinement sweep of the adjoint solve (its
                             right-hand side, the loss gradient, is rougher than the forward data and
                             may contract per sweep at another rate); 0 (default): inner_iters */
} mpn_desc;

enum { MPN_KRYLOV_CG = 0, MPN_KRYLOV_FGMRES = 1 };

typedef struct mpn_stats {
  int sweeps;             /* FP64 refinement sweeps done */
  int pcg_iters;          /* FP32 PCG iterations done (all sweeps) */
  double rel_residual;    /* max over instances: ||r|| / ||rhs|| of the reduced normal equations (FP64),
                             taken at the start of the last sweep, before its correction */
  double rel_update;      /* max over instances: last ||delta u|| / ||u|| */
  double pred_error;      /* max over instances: predicted relative error of u */
} mpn_stats;

typedef struct mpn_problem mpn_problem;

/* Fills *desc with defaults (tol 1e-7, max_refine 12, inner_iters 5,
 * cheb_degree 5, coarse_min 4, max_coarse 2048, stencil 3, fused_coarse 1, fused_step 3, krylov CG, coarsen_time 0, direct 0,
 * variable_steps 0, Dirichlet boundary rows: bc_alpha 1, bc_beta 0; adj_inner_iters 0). */
int mpn_default_desc(mpn_desc* desc);

/* Validates the descriptor, builds the grid hierarchy (spatial halving, time
 * kept) and allocates the workspace on the current device.  *out receives the
 * problem.  Errors: INVALID_ARG, UNSUPPORTED (five-point rows, a batch above
 * 65535 instances, a hierarchy whose coarsest system is too large), NO_MEMORY,
 * CUDA. */
int mpn_create(const mpn_desc* desc, mpn_problem** out);

/* Bytes of device workspace owned by the problem. */
size_t mpn_workspace_bytes(const mpn_problem* p);

/* Number of multigrid levels and their grid shapes (host array [levels][3]). */
int mpn_levels(const mpn_problem* p, int* nlevels, int* shapes /* host, 3 * 16 ints */);

/* First multigrid level of the fused coarse end of the V-cycle (that level
 * and all coarser ones run as one kernel launch per V-cycle), or -1 when
 * every level runs pass by pass (fused_coarse = 0, fewer than two levels
 * fit, or the thread-block cluster cannot be resident).  Host-side query. */
int mpn_fused_level(const mpn_problem* p);

/* Forward pass (Eqs. 9-10): writes z* [B][V][N] and, if z64 is non-null, the
 * FP64 solution [B][V][N] (double).  u0 is an optional warm start.  stats is
 * a host pointer (nullable). */
int mpn_forward(mpn_problem* p, const float* fields, const float* scalars,
                const float* rhs, const float* omega, const float* u0,
                float* z, double* z64, mpn_stats* stats, void* stream);

/* Backward pass (Eq. 11 and the gradients after it): given g_z = dl/dz*
 * [B][V][N], solves A^T A d_z = g_z and writes dl/dfields [F][B][N],
 * dl/dscalars [V][B] (entries of field-backed v are written as 0),
 * dl/drhs [B][N] and dl/domega [B][N] (zero off the boundary set).
 * dz (nullable) receives d_z [B][V][N] and dz64 (nullable) the same in FP64
 * (double), as the refinement holds it.  The duals lambda* and d_lambda are formed in
 * FP64 from the FP64 forward solution the problem keeps.
 * flags bit 0 (MPN_REUSE_SETUP): the data are those of the last mpn_forward
 * on this problem, so its multigrid setup and FP64 solution are reused;
 * without it, if no forward was done, or if fields, scalars, rhs or omega are
 * not the buffers that last forward read, the forward solve is recomputed
 * first.  (A caller that may have changed the contents of the same buffers,
 * or run another forward in between, compares mpn_generation before and
 * after.)  z (the caller's FP32 forward output) may be null; it is not read. */
#define MPN_REUSE_SETUP 1
int mpn_adjoint(mpn_problem* p, const float* fields, const float* scalars,
                const float* rhs, const float* omega, const float* z,
                const float* g_z, float* dfields, float* dscalars, float* drhs,
                float* domega, float* dz, double* dz64, int flags, mpn_stats* stats, void* stream);

/* Per-interval steps of a variable_steps problem (Section 2, "discretization"):
 * steps (device, float) holds, axis by axis (time first), [B][m_d] with
 * m_d = n_d - 1 intervals on an open axis (h_k = x_{k+1} - x_k) and n_d on a
 * periodic one (the last closes the period); sum over d of B m_d floats.  The
 * problem copies them (the caller may reuse the buffer on return) and the
 * next solve builds its hierarchy from them: a coarsened periodic axis sums
 * pairs of intervals, a coarsened open axis places its points at the fine
 * fractional indices and interpolates their coordinates.  Synchronises
 * `stream`.  Errors: INVALID_ARG (null, not a variable_steps problem, a step
 * that is not a positive finite number; the problem keeps no steps then). */
int mpn_set_steps(mpn_problem* p, const float* steps, void* stream);

/* dl/dsteps for a variable_steps problem, in the layout of mpn_set_steps,
 * from the FP64 forward solution z64 and the FP64 adjoint solution dz64
 * ([B][V][N] double each, as mpn_forward and mpn_adjoint write them for the
 * steps last set): the gradient formula after Eq. 11 through the entries of A
 * that depend on the steps.  With lambda = d - A z and d_lambda = -A d_z,
 *   dl/dh_k = -sum over the derivative and Taylor rows r of d(f_r g_r)/dh_k,
 *   f = A z, g = A d_z  (z, d_z held fixed),
 * computed exactly (forward-mode derivatives of each row's entries), one CTA
 * per (instance, axis, interval) summing in a fixed order.  Asynchronous on
 * `stream`.  Errors: INVALID_ARG. */
int mpn_step_grads(mpn_problem* p, const double* z64, const double* dz64, float* dsteps, void* stream);

/* Number of forward solves completed on this problem (the adjoint's own
 * recomputations included); -1 for a null problem.  Host-side query. */
long long mpn_generation(const mpn_problem* p);

/* Host-side fault injection for tests of the error path: the next solve on
 * this problem sets, by a memset on its stream before the first refinement
 * sweep, the device error word that a kernel's bounded wait sets when it
 * gives up, so that solve returns MPN_ERR_CUDA the way a real give-up would.
 * No kernel waits, traps or faults; the problem stays usable (every solve
 * starts with the word cleared). */
int mpn_inject_wait_failure(mpn_problem* p);

/* Bounds-checked build (the library compiled with -DMPN_DEBUG, built as
 * libmpn_debug.so): the index helpers of the stencil, transfer, FP64 and
 * two-pass operator kernels check every neighbour and point index they form;
 * an index out of range is replaced by an in-range one (no fault, no trap)
 * and the first one's code is recorded in a device word of the problem:
 * 1 neighbour (general forms), 2 neighbour (+-1 forms), 3 point, 4 float4
 * group, 5 float4 time neighbour of a 1-D + t level.  Synchronises the
 * device, writes the recorded code (0: none) to *code and clears it.  The
 * fused tile and marching kernels form their indices themselves and are not
 * covered.  Release builds: *code = 0 and MPN_ERR_UNSUPPORTED.  Not in the
 * paper (a replacement for a sanitizer run). */
int mpn_debug_take(mpn_problem* p, int* code);

/* dl/dz of l = mean over (b, i) of (u - target)^2, written into g_z [B][V][N]
 * (zero on the derivative unknowns): the loss used by the benchmarks. */
int mpn_mse_grad(mpn_problem* p, const float* z, const float* target, float* g_z,
                 void* stream);

/* Diagnostic: q = S u for the reduced normal operator S on the finest grid
 * (the Schur complement of A^T A onto the u unknowns, FP32), with the
 * multigrid setup of the given coefficients.  u, q: [B][N], 16-byte aligned
 * (the operator kernels move float4 groups; an unaligned one returns
 * MPN_ERR_INVALID_ARG). */
int mpn_apply_reduced(mpn_problem* p, const float* fields, const float* scalars,
                      const float* u, float* q, void* stream);

/* Live timing of the finest-level Chebyshev smoothing step (the solver's
 * dominant kernel work): CUDA events around one such step per V-cycle on the
 * solve stream.  Reads the totals accumulated since the last reset (time in
 * ms, launches, algorithmic bytes per launch = 4 (6 + F) N B where the level
 * runs the fused step: the iterate, the previous iterate, r, Dinv, rho and
 * the F fields read once, the new iterate written; 4 (7 + F) N B on the
 * two-pass kernels: e, d, r, Dinv, rho and the fields read, e and d written)
 * and the number of kernels
 * this problem launched; then, if enable >= 0, switches timing on (1) or off
 * (0) and resets the totals.  Outputs are host pointers (nullable). */
int mpn_profile(mpn_problem* p, int enable, double* ms_total, long long* launches, double* bytes,
                long long* kernels);

/* Allocation-free variant of mpn_apply_reduced.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory
 * (device memory owned by another allocator, or paths where the failure or
 * implicit synchronisation of cudaMalloc/cudaFree is unacceptable).  It takes
 * the descriptor instead of a problem object and allocates nothing: the
 * intermediate of the two-pass apply lives in a fixed device array of
 * MPN_NOALLOC_MAX_POINTS floats (16 MB, held by every GPU that loads the
 * library until exit), and the point weights are computed inline.
 *   desc     host; grid, batch, coefficient layout (solver fields unused)
 *   fields   device [F][B][N], scalars device [V][B], u device [B][N]
 *   q        device [B][N] output, q = S u
 * B * N above MPN_NOALLOC_MAX_POINTS, B above 65535, per-interval steps
 * (variable_steps) or a Neumann / mixed boundary row (bc_alpha, bc_beta other
 * than 1, 0 on an open axis) returns MPN_ERR_UNSUPPORTED.  Every call looks up the array's device address on
 * the current device (a host-side query that allocates nothing); the first
 * call on a device also loads the library's device code there, so make it
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU race.
 * Asynchronous on `stream`. */
#define MPN_NOALLOC_MAX_POINTS 4194304
int mpn_apply_reduced_noalloc(const mpn_desc* desc, const float* fields, const float* scalars,
                              const float* u, float* q, void* stream);

/* ------------------------------------------------------------------------
 * Learned warm start: a 3x3x3 convolutional network on the (t, x, y) grid
 * that predicts u from the coefficient fields and the right-hand side; its
 * prediction is passed as u0 to mpn_forward, and the solver iterates it to
 * the same tolerance as a cold start.  The paper has no such network; the
 * layer operations below are its inference and training kernels.
 * Activations are channels-last BF16 [B][N][C]; weights BF16 [27][Cout][Cin]
 * with tap = (dt+1)*9 + (dx+1)*3 + (dy+1); biases FP32 [Cout]; all device
 * memory owned by the caller.  Supported (Cin, Cout): (16, 32), (32, 32),
 * (32, 16).  Time is zero-padded; x, y wrap when periodic, else zero-padded.
 * Array arguments of the convolutions (activations, weights, outputs,
 * scratch) must be 16-byte aligned (they move in 16-byte pieces); an
 * unaligned one returns MPN_ERR_INVALID_ARG before any launch.
 * ------------------------------------------------------------------------ */
typedef struct mpn_conv_desc {
  int n[3];          /* n_t, n_x, n_y */
  int periodic[3];   /* periodic[0] must be 0 */
  int batch;
  int cin, cout;     /* padded channel counts */
} mpn_conv_desc;

#define MPN_CONV_RELU 1   /* y = max(., 0) */
#define MPN_CONV_F32 2    /* FP32 output (else BF16) */
#define MPN_CONV_BIAS 4   /* add bias */
#define MPN_CONV_MMA_SYNC 8   /* run the legacy warp-level tensor-core kernel (mma.sync) instead of tcgen05 */
#define MPN_WGRAD_CHUNK 65536   /* points per partial sum of the weight gradient */
#define MPN_MSE_BLOCKS 64

/* y = act(conv(x, W) + b): BF16 implicit GEMM on the 5th-generation tensor cores, FP32 accumulation
 * in tensor memory: per tile of 128 points and per 3x3x3 tap, tcgen05.mma of M = 128, N = cout,
 * K = 16 on the gathered input tile and the tap's weights, both staged in shared memory
 * (MPN_CONV_MMA_SYNC: the warp-level mma.sync m16n8k16 kernel instead).  Not in the paper: the
 * learned warm start (a 3D-conv network predicting the solution). */
int mpn_conv3d_forward(const mpn_conv_desc* d, const void* x, const void* w, const float* bias, void* y,
                       int flags, void* stream);
/* *flag = 1 if a tcgen05 convolution launched since the last call had a bounded wait for its
 * pipeline give up (its output is then undefined), else 0; clears the word.  Synchronous (waits
 * for the device).  Not in the paper: error reporting of the warm-start kernels. */
int mpn_conv_take_error(int* flag);
/* g_in [B][N][cin] FP32 = transposed convolution of g_out [B][N][cout] (BF16) with W, on the
 * tcgen05 kernel of mpn_conv3d_forward; wt_scratch: 27*cin*cout BF16 (flipped, transposed W).
 * Requires cin = 32. */
int mpn_conv3d_backward_data(const mpn_conv_desc* d, const void* g_out, const void* w, void* wt_scratch,
                             float* g_in, void* stream);
/* Bytes of FP32 scratch mpn_conv3d_backward_weights needs. */
size_t mpn_conv3d_wgrad_scratch_bytes(const mpn_conv_desc* d);
/* dW [27][cout][cin] = sum_p g_out[p][co] x[nbr(p, tap)][ci], db [cout] = sum_p g_out[p][co]:
 * per tap a GEMM over the points on the tensor cores (mma.sync m16n8k16 bf16, FP32 accumulation)
 * for every chunk of MPN_WGRAD_CHUNK points, then the chunks summed in a fixed order (deterministic). */
int mpn_conv3d_backward_weights(const mpn_conv_desc* d, const void* g_out, const void* x, float* scratch,
                                float* dw, float* db, void* stream);
/* out (BF16) = g * (y > 0) elementwise (y BF16, nullable: no mask), n elements. */
int mpn_relu_mask(long long n, const float* g, const void* y, void* out, void* stream);
/* Adam on FP32 master weights w with moments m, v (step >= 1); w_bf16 (nullable) gets the BF16 copy. */
int mpn_adam_step(long long n, float* w, const float* g, float* m, float* v, float lr, float beta1, float beta2,
                  float eps, int step, void* w_bf16, void* stream);
/* x0 [B][N][16] BF16 = (fields[0..F), rhs, running sum over time planes 0..t of rhs at the same
 * (x, y)) * scale[c], channels zero-padded; F <= 14. */
int mpn_pack_inputs(const mpn_conv_desc* d, int nfields, const float* fields, const float* rhs, const float* scale,
                    void* x0, void* stream);
/* MSE of channel 0 of y [B][N][16] (FP32) against target [B][N]: g (same shape as y) and
 * per-block partial sums of squares loss_part [B][MPN_MSE_BLOCKS]. */
int mpn_mse_u(const mpn_conv_desc* d, const float* y, const float* target, float* g, float* loss_part, void* stream);
/* u0 [B][N] = scale * y[., ., 0]. */
int mpn_unpack_u(const mpn_conv_desc* d, const float* y, float scale, float* u0, void* stream);

void mpn_destroy(mpn_problem* p);
const char* mpn_strerror(int status);
const char* mpn_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MPN_H */
