/*
 * ys.h -- C ABI of the GB300 Yin-Yang shell solver.
 *
 * The library advances the Navier-Stokes-Boussinesq system in a spherical
 * shell R1 <= r <= R2 (Sec. 1, Eq. eq_ns / eq_heat_convec of "A direction
 * splitting scheme for Navier-Stokes-Boussinesq system in spherical shell
 * geometries", arXiv:1905.02300) on two overset Yin/Yang latitude-longitude
 * patches (Sec. 2), with the second-order artificial-compressibility scheme
 * with bootstrapping (Sec. 3.3, Eq. ac1 / ac2), direction splitting of every
 * implicit operator into 1-D tridiagonal line solves (Sec. 3.2, Sec. 4), the
 * splitting-error reduction iteration (Sec. 4, Eq. er) and additive or
 * multiplicative Schwarz coupling of the patches (Sec. 4, Algorithm).
 *
 * Everything runs on one CUDA device in hand-written kernels.  There is no
 * CPU fallback: if no device is usable every call that needs one returns
 * YS_ECUDA.
 *
 * Field layout (host buffers, FP64, caller-owned; the library copies in/out).
 * Both patches are stored back to back, patch 0 (Yin) first, phi fastest:
 *   T, p : [2][Nr  ][Nth  ][Nph  ]  cell centres
 *   ur   : [2][Nr+1][Nth  ][Nph  ]  r-faces, wall faces included
 *   uth  : [2][Nr  ][Nth+1][Nph  ]  theta-faces, patch-edge faces included
 *   uph  : [2][Nr  ][Nth  ][Nph+1]  phi-faces, patch-edge faces included
 * Velocity components are in each patch's local spherical basis.  Patch-edge
 * faces, wall faces and the outermost ring of pressure cells are boundary
 * values: the library recomputes them from the other patch (Schwarz
 * exchange) and the wall data whenever fields are set, and returns them.
 *
 * Geometry: each patch covers theta in [pi/4 - d, 3pi/4 + d],
 * phi in [-3pi/4 - d, 3pi/4 + d] of its own frame with d = overlap * h_theta,
 * h_theta = (pi/2)/(Nth - 2 overlap), h_phi = (3pi/2 + 2d)/Nph; radially
 * uniform h_r = (R2 - R1)/Nr by default, or the half points of
 * ys_params.r_half (a non-uniform radial grid).  The Yang frame is the Yin
 * frame composed with M(x, y, z) = (-x, z, y) (Sec. 2).
 *
 * Threading: a context is not thread-safe; distinct contexts may be used
 * from distinct threads.
 */
#ifndef YS_H
#define YS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define YS_OK 0
#define YS_EINVAL 1     /* invalid argument or grid too coarse for the exchange */
#define YS_ENOMEM 2     /* device or host allocation failed */
#define YS_ECUDA 3      /* CUDA error (no device, launch failure, ...) */
#define YS_EDIVERGED 4  /* NaN/Inf increment norms, or Schwarz increments that grew more than
                           10^3-fold in one iteration past the step's first increment: the
                           state holds the diverged values */
#define YS_ETIMEOUT 5   /* a served request passed its deadline */
#define YS_EAGAIN 6     /* result not ready yet */
#define YS_EBUSY 7      /* admission refused: queue full */
#define YS_ECANCELED 8  /* a served request was cancelled */

/* precision */
#define YS_FP64 0       /* every field and operation in FP64 */
#define YS_MIXED 1      /* FP32 sweeps and stencils; FP64 pressure, norms, coefficients */

/* Schwarz variants (Sec. 4) */
#define YS_ADDITIVE 0       /* both patches from the previous iterate (default) */
#define YS_MULTIPLICATIVE 1 /* Yin, then Yang with Yin's newest data (Algorithm) */

/* number of per-field Schwarz increment norms reported by ys_get_norms:
 * T, u1_r, u1_th, u1_ph, p1, u2_r, u2_th, u2_ph, p2 */
#define YS_NFIELDS 9

typedef struct ys_ctx ys_ctx;

typedef struct {
  double R1, R2;        /* shell radii, 0 < R1 < R2 */
  double Pr, Ra;        /* Prandtl and Rayleigh numbers (Sec. 1) */
  double dt;            /* time step > 0 */
  int Nr, Nth, Nph;     /* cells per patch; Nth > 2 overlap + 4, Nph >= Nth */
  double chi;           /* AC parameter chi = O(1) of Eq. ac1 (default 1) */
  int overlap;          /* overlap d in theta cells (default 2) */
  int precision;        /* YS_FP64 (default) or YS_MIXED */
  int schwarz_mode;     /* YS_ADDITIVE (default) or YS_MULTIPLICATIVE */
  double schwarz_tol;   /* stop the Schwarz iteration once the largest l2
                           increment norm is below this; 0 = always run
                           n_schwarz iterations (default 0) */
  double T_inner, T_outer; /* Dirichlet wall temperatures (default 0, 0) */
  int step7;            /* 1 = interpolate the pressure ring from the other
                           patch after each pressure update (Algorithm step 7,
                           default); 0 = off */
  int step4;            /* 1 = mass-flux correction of the interpolated boundary
                           velocity after every exchange (Algorithm step 4: the
                           minimiser of its functional J, which the paper finds
                           by conjugate gradients and which has the closed form
                           v = u - alpha (w.u + c) / (1 + alpha w.w) w); 0 = off
                           (default, as for the paper's results) */
  double step4_eps;     /* epsilon << 1 of J (default 1e-8) */
  double step4_tol;     /* correct only when |net boundary flux| >= tol (default 1e-13) */
  /* temperature wall conditions a T + b dT/dn = T_inner (r = R1) and
     = T_outer (r = R2), n the outward normal (Sec. 1: Dirichlet, Neumann or
     Robin walls); a, b >= 0, a + b > 0; default a = 1, b = 0 (Dirichlet).  The
     mixed form keeps its conductive-profile deviation variables only for
     Dirichlet walls. */
  double Tbc_inner_a, Tbc_inner_b, Tbc_outer_a, Tbc_outer_b;
  /* non-uniform radial grid (Sec. 4: centred differences on a non-uniform
     grid): NULL = uniform (default), else 2 Nr + 1 strictly increasing radii of
     the radial half points, faces at even and cell centres at odd positions,
     r_half[0] = R1 and r_half[2 Nr] = R2 (to 1e-12 (R2 - R1)).  A half-cell
     difference divides by the distance of its two points, a whole-cell
     centred difference by twice the local spacing (the cell width at a
     centre, the centre distance at a face); averages of radial neighbours stay
     arithmetic means (the stretched-coordinate form, second order for smooth
     stretchings).  ys_create_ex copies the array; ys_submit and
     ys_factor_solve_static take uniform grids only (YS_EINVAL otherwise). */
  const double *r_half;
} ys_params;

/* Fill *p with defaults (all sizes zero, chi = 1, overlap = 2, FP64,
 * additive, tol 0, walls 0 (Dirichlet), step7 on, step4 off with eps 1e-8,
 * tol 1e-13). */
void ys_default_params(ys_params *p);

/* Create a context for one shell with default parameters.  Validates the
 * arguments (YS_EINVAL: R1 <= 0, R2 <= R1, dt <= 0, N* < 8, Nph < Nth, chi <= 0,
 * or a grid so coarse that an exchange donor stencil leaves the donor
 * patch's interior), builds the metric and exchange tables and allocates all
 * device state (YS_ENOMEM, YS_ECUDA).  Fields start at zero, t = 0.
 * *out receives the context (NULL on error). */
int ys_create(double R1, double R2, double Pr, double Ra, int Nr, int Nth, int Nph,
              double dt, ys_ctx **out);
int ys_create_ex(const ys_params *p, ys_ctx **out);

/* Set time level `level` (0 = n, 1 = n-1) from host buffers in the layout
 * above.  Sets u1 = u2 = u and p1 = p2 = p (the two AC systems of Eq. ac1 and
 * Eq. ac2), or, if aux != NULL, takes u1 and p1 from aux packed as
 * [ur1 | uth1 | uph1 | p1] in the same layouts.  Then recomputes every
 * boundary value of that level.  Setting level 0 while level 1 was never set
 * also sets level 1 to the same state (psi^{-1} := psi^0).  Page-locked
 * (pinned) host buffers are read by the device directly over the CPU-GPU
 * link; pageable ones go through one staging copy.
 * Synchronous.  Errors: YS_EINVAL (bad level / NULL field), YS_ECUDA. */
int ys_set_fields(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                  const double *uph, const double *p);
int ys_set_fields_ex(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                     const double *uph, const double *p, const double *aux);

/* Add separable forcing mode `mode` (0 <= mode < 8): f(x, t) = tau(t) F(x) with
 * tau selected by time_fn (0: 1, 1: cos t, 2: sin t, 3: cos^2 t,
 * 4: sin t cos t), F given at the unknowns in the field layouts above (T at
 * centres, f_r on r-faces, f_th on theta-faces, f_ph on phi-faces; boundary
 * entries are ignored).  The forcing enters the rates at t_n + dt/2.
 * Errors: YS_EINVAL, YS_ENOMEM, YS_ECUDA. */
int ys_set_forcing(ys_ctx *c, int mode, int time_fn, const double *f_T, const double *f_r,
                   const double *f_th, const double *f_ph);

/* Dirichlet velocity on the walls r = R1 and r = R2 (Sec. 2: the velocity is
 * prescribed on the boundary; the paper's Landau-jet runs of Sec. 5.1 use
 * the jet's own wall values), constant in time, in each patch's local basis.
 * Host arrays (FP64, copied in, caller keeps ownership), wall 0 = R1, 1 = R2:
 *   ur  [wall][patch][Nth][Nph]      u_r on the wall faces
 *   uth [wall][patch][Nth + 1][Nph]  u_theta at r = R1, R2 on theta-faces
 *   uph [wall][patch][Nth][Nph + 1]  u_phi at r = R1, R2 on phi-faces
 * u_r takes the value on the wall faces; u_theta, u_phi get the reflection
 * ghosts 2 g - x_0.  A NULL component means no-slip for that component.  The
 * boundary values of the stored levels are refreshed.
 * Errors: YS_EINVAL, YS_ENOMEM, YS_ECUDA. */
int ys_set_wall_velocity(ys_ctx *c, const double *ur, const double *uth, const double *uph);

/* Time-dependent Dirichlet wall data tau(t) W, tau one of the forcing time
 * functions (time_fn as in ys_set_forcing), for solutions with non-zero,
 * time-varying walls such as the manufactured solution of Sec. 5.1.  T:
 * [wall][patch][Nth][Nph] wall temperature at the cell-centre angles, added
 * to T_inner / T_outer (for the wall condition a T + b dT/dn of Tbc_*);
 * ur, uth, uph: wall velocity in the layouts of ys_set_wall_velocity, added
 * to the steady wall velocity.  Each state's boundary values take tau at
 * that state's time: t_n + dt for the iterate of a step, the level's own
 * time for the stored levels.  Any pointer may be NULL (that part is zero);
 * a later call replaces the data.  The boundary values of the stored levels
 * are refreshed.  A context with such data cannot join a batch (YS_EINVAL
 * from ys_batch_add).  Errors: YS_EINVAL, YS_ENOMEM, YS_ECUDA. */
int ys_set_wall_data(ys_ctx *c, int time_fn, const double *T, const double *ur, const double *uth,
                     const double *uph);

/* Set the time t_n of level 0. */
int ys_set_time(ys_ctx *c, double t);

/* Advance n_steps AC time steps, each with up to n_schwarz Schwarz /
 * splitting-error-reduction iterations (Sec. 4, Eq. er).  Per iteration:
 * exchange boundary values, defect-correct T, then u1 (r, theta, phi), p1,
 * u2 (r, theta, phi), p2, each correction through three line sweeps.
 * The work is queued on the context's stream; the call returns once the last
 * step's increment norms have been read back (with schwarz_tol > 0 it also
 * waits for the norms after every iteration).  Returns YS_EDIVERGED if one
 * of those norms is NaN or Inf, or if in any iteration of this call an
 * increment norm was not finite or, from the third iteration of a step on,
 * the largest one exceeded both 10^3 times the previous iteration's and the
 * step's first (a device-side watch after every iteration: a working defect
 * correction contracts from its second iteration on, so growth by three
 * orders of magnitude in one iteration past the first increment means it
 * diverges; growth from a second increment already at the rounding level
 * of the arithmetic stays below the first); the state then holds the
 * diverged values and the caller restarts from its own copy (ys_get_fields /
 * ys_set_fields restart exactly). */
int ys_step(ys_ctx *c, int n_steps, int n_schwarz);

/* Copy time level `level` to host buffers (u2 and p2, the second-order
 * solution); any pointer may be NULL to skip that field.  aux != NULL
 * receives [ur1 | uth1 | uph1 | p1].  Page-locked host buffers are written
 * by the device directly, pageable ones through one staging copy.
 * Synchronous.  Errors: YS_EINVAL (bad level), YS_ECUDA. */
int ys_get_fields(ys_ctx *c, int level, double *T, double *ur, double *uth, double *uph,
                  double *p, double *aux);

/* Statistics: largest l2 increment norm of the last iteration, time of
 * level 0 and steps done; any pointer may be NULL.  Synchronous. */
int ys_get_stats(ys_ctx *c, double *last_schwarz_norm, double *t, long *steps_done);

/* Per-field l2 increment norms of the last iteration (YS_NFIELDS values) and
 * the number of iterations the last step ran.  Synchronous. */
int ys_get_norms(ys_ctx *c, double *norms, int *iters_last_step);

/* Run the context's work on a caller-provided cudaStream_t (NULL = the
 * context's own stream).  The caller keeps ownership of the stream. */
int ys_set_stream(ys_ctx *c, void *stream);

/* Device-pointer variant of ys_set_fields_ex: the buffers are device memory
 * in the same layouts, read on the context's stream. */
int ys_set_fields_dev(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                      const double *uph, const double *p, const double *aux);

/* Kernel-level timing with CUDA events on the context's stream.
 * ys_profile_enable(c, 1) starts recording (clears the tallies);
 * ys_profile_read fills up to `cap` entries of names / total milliseconds /
 * launch counts (sorted as registered) and returns the number of kernel
 * classes (synchronous).  ys_launch_count returns the number of kernels the
 * context launched since creation. */
int ys_profile_enable(ys_ctx *c, int on);
int ys_profile_read(ys_ctx *c, const char **names, double *ms, long *launches, int cap);
long ys_launch_count(ys_ctx *c);
/* Diagnostic: the dense FP64 rate of the current device in TFLOP/s (2 flops
 * per FMA), measured by a kernel of independent FMA chains on every SM, timed
 * with CUDA events (synchronous; allocates 8 bytes).  The roofline
 * denominator of the FP64 form's kernels, which are bound by the FP64 pipe.
 * Errors: YS_EINVAL, YS_ENOMEM, YS_ECUDA. */
int ys_measure_fp64_rate(double *tflops);

/* Bytes of device memory held by the context. */
size_t ys_device_bytes(ys_ctx *c);
/* Host only (no GPU): the bytes of device memory ys_create_ex allocates for
 * *p, which ys_device_bytes of the new context reports until forcing modes
 * or a wall velocity are added; the serving queue admits requests by this
 * figure.  0 for parameters ys_create_ex rejects. */
size_t ys_shell_device_bytes(const ys_params *p);

/* Allocation-free preconditioner solve (the paper has no counterpart; this is
 * a library convenience).  Some callers cannot call cudaMalloc: code running
 * inside a host-side memory budget enforced by another allocator, callbacks
 * that must not trigger the driver's allocator or its implicit
 * synchronisation, and embedders that forbid device allocations after start-up.
 * This entry point allocates nothing: it applies x = P^-1 rhs, where P is the
 * product of the three 1-D line operators (I - dt/2 Ahat_d) of one unknown,
 * solved one direction after the other in this order: T along r, theta,
 * phi; u_r along theta, phi, r; u_theta along phi, r, theta; u_phi along r,
 * theta, phi.  It is meant for one shell described by
 * *prm (R1, R2, Pr as viscosity, dt, chi, overlap, Nr, Nth, Nph, and the
 * temperature wall conditions Tbc_* whose ghosts set the T factor's wall rows;
 * other fields ignored).  loc selects the unknown: 0 = T, 1 = u_r, 2 = u_theta, 3 = u_phi.
 * All pointers are caller-owned DEVICE memory in the field layouts above:
 * A_r, A_th, A_ph the advecting velocity on r-, theta- and phi-faces; rhs and
 * x in the layout of the unknown (boundary entries of rhs are ignored, those
 * of x are set to 0).  Work is queued on `stream` (a cudaStream_t, NULL = the
 * legacy default stream).
 * Scratch: one static device array of 5 * 2^18 + 14 * 264 doubles (about
 * 10.5 MB) that every GPU which loads the library holds until the process
 * exits.  Grids are limited to Nr, Nth, Nph <= 256 and at most 2^18 padded
 * elements per field (e.g. 32 x 32 x 96 per patch fits, 48 x 48 x 144 does
 * not); larger grids, bad sizes or NULL pointers return YS_EINVAL before any
 * work is queued.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, so make the first
 * call on a device before any stream capture.  A call queues only memsets and
 * kernels on `stream` (the metric tables are formed on the device) and does
 * not wait for them.  Every call shares the one array and overwrites the
 * previous call's contents (the working fields are cleared at the start of
 * each call): calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.
 * Errors: YS_EINVAL; YS_ECUDA for a failed launch of this call, and also when
 * earlier work left an error pending in the calling thread's CUDA context
 * (the pending error is cleared). */
int ys_factor_solve_static(const ys_params *prm, int loc, const double *A_r, const double *A_th,
                           const double *A_ph, const double *rhs, double *x, void *stream);

int ys_destroy(ys_ctx *c);

/* Diagnostic, host only (builds the tables without touching a device): the
 * FP64 coefficients of the 1-D line operators (I - dt/2 Ahat_d) (Sec. 3.2,
 * Sec. 4; T, u_r, u_theta, u_phi along r, theta, phi) that the
 * factorisations use for the shell *p.  The row of the operator at a point
 * whose advecting velocity component along d is a is
 * (L0 + a LA, D0, U0 - a LA) on (x_{m-1}, x_m, x_{m+1}), before the wall and
 * line-end rows are closed.  Layout: out[((3 loc + d) (Nr + 2) + i + 1)
 * (Nth + 2) + j + 1][4] = {L0, D0, U0, LA} with loc 0..3 = T, u_r, u_theta,
 * u_phi and d 0..2 = r, theta, phi; entries of points that are not unknowns
 * are zero.  *count receives the number of doubles (12 (Nr + 2) (Nth + 2) 4);
 * out = NULL only queries it.  Errors: YS_EINVAL (bad parameters, cap too
 * small, NULL count). */
int ys_line_coefficients(const ys_params *p, double *out, size_t cap, size_t *count);

/* Diagnostic, host only: the FP64 row-coefficient records of the explicit
 * residuals (Sec. 3.3) of the FP64 form for the shell *p.  Every metric factor
 * of a residual stencil depends on the row (i, j) only; a record holds, for
 * one row, the products of metric factors, spacings, dt and the physical
 * constants that multiply the stencil values, written for the two-level sums
 * S = x + x^n (so that the half-level value is S/2).  table: 0 temperature,
 * 1 u_r, 2 u_theta, 3 u_phi, 4 divergence.  Record orders:
 *   0: (S_i+1 - S_i), (S_i - S_i-1), same along theta, S_k+1 - 2 S_k + S_k-1
 *      (diffusion: RP, RM, TP, TM, PP, the minus sign of RM, TM applied by
 *      the stencil), a_r (S_i+1 - S_i-1), a_th (..), a_ph (..) with a the
 *      2-point sums of the advecting velocity (AR, AT, AP), the two
 *      deviation-form sources (zero here);
 *   4: S_r(i+1), S_r(i), S_th(j+1), S_th(j), S_ph(k+1) - S_ph(k) (R1, R0, T1,
 *      T0, P: the divergence of the half-level velocity over chi as
 *      R1 S_r(i+1) - R0 S_r(i) + T1 S_th(j+1) - T0 S_th(j) + P (..)), then the
 *      norm weight r^2 sin(theta) h / h_r of the cell;
 *   1-3: the velocity rows (orders of their kernels, not a stable interface).
 * Layout out[(i + 1) (Nth + 2) + j + 1][*record]; rows of points that are not
 * unknowns are zero.  *count receives the number of doubles; out = NULL only
 * queries.  Errors: YS_EINVAL. */
int ys_residual_coefficients(const ys_params *p, int table, double *out, size_t cap, size_t *count, int *record);

/* Diagnostic, host only: the Yin <-> Yang exchange table of one kind (Sec. 4,
 * Algorithm steps 1, 3 and 7) that the library builds for the shell *p and
 * uses on both patches.  kind: 0 temperature (theta-ghost rows and
 * phi-ghost columns, every radial cell), 1 u_r (the same points, interior
 * radial faces), 2 u_theta (edge faces j = 0, Nth and phi-ghosts), 3 u_phi
 * (edge faces k = 0, Nph and theta-ghosts), 4 the pressure ring (outermost
 * interior cells).  Each target point is one record of 12 doubles:
 * (tj, tk, j0a, k0a, wja, wka, j0b, k0b, wjb, wkb, ra, rb): the target's
 * logical (j, k); donor stencil A, the tensor bilinear stencil on the other
 * patch at the same radial index with base (j0a, k0a) and weights (wja, wka)
 * along theta and phi, of T, u_r or p (kinds 0, 1, 4) or of u_theta (2, 3);
 * stencil B, of u_phi (kinds 2, 3; zero otherwise); the target value is
 * ra A + rb B (ra = 1, rb = 0 for scalars).  *count receives the number of
 * doubles (12 per point); out = NULL only queries.  Errors: YS_EINVAL (bad
 * parameters, grid too coarse for the donor stencils, cap too small). */
int ys_exchange_table(const ys_params *p, int kind, double *out, size_t cap, size_t *count);

/* ------------------------------------------------------------------------
 * Batched ensembles.  A batch advances many independent shells (contexts
 * created with ys_create_ex and filled with ys_set_fields, uneven sizes,
 * Ra, Pr and radial grids allowed) together: every kernel class of the AC step is one launch
 * over all member shells, and a whole step is replayed from one captured CUDA
 * graph that stays valid while shells join and leave.  Members must share the
 * batch's precision, use additive Schwarz and have no forcing modes; all run
 * n_schwarz iterations per step.  A shell's fields do not depend on the other
 * members (bitwise).  While a context is in a batch only the batch steps it. */
typedef struct ys_batch ys_batch;

/* capacity: 1..4096 slots; precision YS_FP64 or YS_MIXED; n_schwarz >= 1. */
int ys_batch_create(int capacity, int precision, int n_schwarz, ys_batch **out);
/* Add a context; *slot receives its slot.  YS_EBUSY when full, YS_EINVAL on a
 * precision mismatch, multiplicative Schwarz, forcing modes or step4 (batched
 * shells run additive Schwarz without Algorithm step 4).  The caller keeps
 * ownership. */
int ys_batch_add(ys_batch *b, ys_ctx *c, int *slot);
/* Remove the shell in `slot`; its context (time, step count, levels) is
 * brought up to date and returned in *c for ys_get_fields or ys_step. */
int ys_batch_remove(ys_batch *b, int slot, ys_ctx **c);
/* Advance every member n_steps steps (asynchronous on the batch's stream). */
int ys_batch_step(ys_batch *b, int n_steps);
int ys_batch_sync(ys_batch *b);
/* l2 increment norms (YS_NFIELDS) of the member's last iteration.  Returns
 * YS_EDIVERGED (norms still written) when one is not finite, or when, in a
 * step since the member joined the batch, its largest increment norm grew
 * more than 10^3-fold from one iteration to the next after the second and
 * past the step's first increment (the same watch as ys_step). */
int ys_batch_norms(ys_batch *b, int slot, double *norms);
/* Threads per block of the line-solve launches (lines per block): 32, 64,
 * 128 (default) or 256. */
int ys_batch_set_line_threads(ys_batch *b, int threads);
/* Time trial_steps steps with each lines-per-block choice and keep the
 * fastest; the trial steps advance the members.  *chosen gets the choice. */
int ys_batch_autotune(ys_batch *b, int trial_steps, int *chosen);
/* kernel launches in one batched step (independent of the member count) */
long ys_batch_launches_per_step(ys_batch *b);
/* Kernel-class timing of batched steps: with profiling on, ys_batch_step
 * launches each step's kernels directly on the batch's stream (the same
 * kernels, arguments and order as the captured graph) with a CUDA event
 * pair around every launch; ys_batch_profile_read fills up to `cap` names /
 * total milliseconds / launch counts and returns the number of classes
 * (synchronous; a negative error code on failure).  Enabling or disabling
 * clears the tallies. */
int ys_batch_profile_enable(ys_batch *b, int on);
int ys_batch_profile_read(ys_batch *b, const char **names, double *ms, long *launches, int cap);
/* the cudaStream_t the batch runs on (for event timing by the caller) */
void *ys_batch_stream(ys_batch *b);
int ys_batch_destroy(ys_batch *b);

/* ------------------------------------------------------------------------
 * Serving with continuous batching.  Requests (one shell simulation each)
 * are admitted first come first served while a slot is free and the
 * device-memory footprint of the admitted shells stays within
 * hbm_budget_bytes; a worker thread advances all admitted shells one batched
 * step at a time, admits waiting requests and retires finished ones at every
 * step boundary.  Thread-safe.  The first request fixes the precision and
 * n_schwarz of the server; later requests must match (YS_EINVAL). */
typedef struct ys_server ys_server;

int ys_server_create(size_t hbm_budget_bytes, int max_slots, ys_server **out);
/* Queue a simulation: parameters (additive Schwarz, schwarz_tol 0, uniform
 * radial grid: r_half NULL), initial fields packed as [T | ur | uth | uph | p]
 * in the field layouts above (copied), number of steps.  *ticket identifies
 * it.  YS_EBUSY when the queue is full; YS_EINVAL if it can never fit the
 * budget or the parameters are outside these limits. */
int ys_submit(ys_server *s, const ys_params *p, const double *init_fields, int n_steps, int n_schwarz,
              uint64_t *ticket);
/* ys_submit with a deadline: a request not done deadline_s seconds after its
 * submission fails with YS_ETIMEOUT (checked at every batched step boundary,
 * while it waits in the queue and while it runs; its batch mates are not
 * affected).  deadline_s = 0: no deadline; < 0 or NaN: YS_EINVAL. */
int ys_submit_ex(ys_server *s, const ys_params *p, const double *init_fields, int n_steps, int n_schwarz,
                 double deadline_s, uint64_t *ticket);
/* Cancel a request: a queued one fails with YS_ECANCELED at once, a running
 * one at the next batched step boundary (its device state is released there;
 * its batch mates are not affected).  YS_EINVAL for an unknown ticket or one
 * that has already finished. */
int ys_cancel(ys_server *s, uint64_t ticket);
/* Most requests the queue holds while they wait for admission (1..4096,
 * default 4096); ys_submit beyond it returns YS_EBUSY. */
int ys_server_set_queue_limit(ys_server *s, int max_queued);
/* State of a request: *state = 0 queued, 1 running, 2 done, 3 failed.  Returns
 * YS_EAGAIN until it is done; when done, copies level 0 packed like the input
 * to out_fields (if not NULL) and the time from submission to completion to
 * *latency_s.  A failed request (e.g. NaN data) returns its error code; other
 * requests are not affected. */
int ys_poll(ys_server *s, uint64_t ticket, int *state, double *out_fields, double *latency_s);
/* Batched steps run, cell-updates done, requests running and queued now, and
 * the most requests that were ever running together.  Any pointer may be NULL. */
int ys_server_stats(ys_server *s, long *steps_run, double *cell_updates, int *running, int *queued,
                    int *peak_running);
int ys_server_destroy(ys_server *s);

const char *ys_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* YS_H */
