/*
 * se_mobility.h -- C ABI of the B300 Spectral Ewald far-field grand mobility.
 *
 * Computes y = M_inf . x for N spheres of radii a_i in a cubic periodic box,
 * where M_inf is the far-field grand mobility of Wang & Brady (arXiv 1506.08481)
 * including the compressible-solvent pressure-moment terms:
 *
 *   x_i = [F (3), T (3), S (5), S_tr (1)]   moments the sphere exerts on the fluid
 *   y_i = [U (3), Omega (3), E (5), E_tr (1)] translational / angular velocity,
 *                                             strain rate, expansion rate
 *
 * S and E are traceless symmetric tensors stored as coordinates on the
 * orthonormal basis (xx-yy)/sqrt2, (2zz-xx-yy)/sqrt6, (xy+yx)/sqrt2,
 * (xz+zx)/sqrt2, (yz+zy)/sqrt2.  Per particle the components are stored
 * contiguously (row-major [N][ncomp]); with ncomp < 12 only the leading
 * components are read and written (3: F->U, 6: +T->Omega, 11: +S->E, 12: +S_tr->E_tr).
 *
 * Method (paper sections and equations):
 *   Faxen laws Eqs. faxen-f/t/s/p and multipole expansion Eq. mul-expand (Sec. 2.1);
 *   Hasimoto/Beenakker split of the periodic Oseen tensor Eqs. oseen-split,
 *   oseen-ewald-rs/ws (Sec. 2.2) and of the source/pressure solutions Eq. source-split
 *   (Sec. 2.3); real-space pairs within rc from a cell list (Sec. 3.3); wave space by
 *   the Spectral Ewald method (Sec. 3.1): Gaussian spreading Eq. grid-space with the
 *   shape function Eq. shape, theta from Eq. theta-param, fast Gaussian gridding
 *   Eq. fgg-exp, 3D FFT, k-space scaling Eq. wave-result, gather by the trapezoid rule
 *   Eq. parseval-sum; particle-size terms by the hybrid approach (Sec. 3.2, default),
 *   the real-space approach (Eq. non-ortho-shape) or the wave-space approach; sheared
 *   cells (Sec. 3.2, lattice a2 = (gamma L, L, 0)); self terms Eq. uf-self.
 *   se_solve: GMRES with the block-diagonal far-field preconditioner of Sec. 4.2.
 *
 * Conventions common to all entry points:
 *   - Every function returns 0 on success or a negative SE_ERR_* code; the message
 *     of the last failure is returned by se_last_error(ctx).
 *   - Device pointers are CUDA device addresses on the context's device; the caller
 *     owns every buffer it passes; the context owns its internal scratch.
 *   - Work is enqueued on the stream given to se_create (borrowed, never destroyed)
 *     and is asynchronous unless stated otherwise.
 *   - Viscosity eta = 1 unless set with SE_OPT_ETA.
 */
#ifndef SE_MOBILITY_H
#define SE_MOBILITY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct se_ctx se_ctx;

/* error codes */
#define SE_OK                 0
#define SE_ERR_ARG           -1   /* invalid argument (null pointer, bad size, ncomp, dtype) */
#define SE_ERR_GRID          -2   /* M not of the form 2^a 3^b in [8, 512], or P outside [2, M] */
#define SE_ERR_CUTOFF        -3   /* rc <= 0 or rc >= L/2 */
#define SE_ERR_CUDA          -4   /* a CUDA runtime call failed */
#define SE_ERR_STATE         -5   /* parameters or configuration not set */
#define SE_ERR_NONFINITE     -6   /* non-finite position, radius or result */
#define SE_ERR_NOT_CONVERGED -7   /* GMRES reached maxit (x holds the last iterate) */
#define SE_ERR_NOMEM         -8   /* device allocation failed */
#define SE_ERR_TOO_LARGE     -9   /* problem larger than a fixed capacity (se_real_space_apply_noalloc) */
#define SE_ERR_OVERLAP      -10   /* two spheres overlap, |x_ij| < (a_i + a_j)(1 - 1e-12), with |x_ij| < rc */

/* dtypes of x / y */
#define SE_F32 0
#define SE_F64 1

/* options for se_set_option */
#define SE_OPT_PRECISION   1   /* compute precision of products: 0 = FP32 (default), 1 = FP64, 2 = FP64-
                                  equivalent: real-space sum, spread and gather in double-float
                                  arithmetic (pairs of FP32 numbers, ~2^-44 relative), the FFT and
                                  k-space scaling in FP64; same accuracy as 1 at a fraction of its
                                  time on B300's FP64 rate */
#define SE_OPT_SIZE_MODE   2   /* particle-size (Faxen) terms, Sec. 3.2: 0 = hybrid approach (default: target
                                  Laplacians in k-space), 1 = real-space approach (all of them in the
                                  spread/gather polynomial, Eq. non-ortho-shape), 2 = Laplacians of source and
                                  target in k-space with the torque / stresslet gradients still in the
                                  spread and gather (8 grids each way), 3 = the paper's wave-space approach
                                  (Eqs. wave-only-f-assign, wave-only-compute-1/2, parseval-sum-2): every
                                  derivative in k-space, the plain window on both sides, 20 grids each
                                  way; runs in FP32 or FP64 (SE_OPT_PRECISION 2 runs it in FP64).  A
                                  sheared cell (SE_OPT_SHEAR) needs mode 2 or 3 */
#define SE_OPT_ETA         3   /* solvent viscosity (default 1) */
#define SE_OPT_SHAPE_M     4   /* Gaussian shape parameter m of Eq. theta-param (default sqrt(pi P)) */
#define SE_OPT_RESTART     5   /* GMRES restart length, 1..1000 (default 30; the basis takes (restart + 1) N ncomp doubles) */
#define SE_OPT_PARTS       6   /* bit mask of terms: 1 real space, 2 wave space, 4 self (default 7) */
#define SE_OPT_TIMING      7   /* 1: record CUDA events around every stage of each product (default 0) */
#define SE_OPT_OVERLAP     8   /* where the real-space sum runs: 0 = on a second, high-priority stream
                                  beside the spread, 1 = beside the FFT chain, 2 = in line before the
                                  spread (the spread and gather fill every SM, so running beside them
                                  only slows them), 3 (default) = inside the gather kernel, each warp
                                  summing its particle's stored pairs before gathering, where that
                                  kernel applies (FP32, stored pair table, 11 or 12 moment components,
                                  SE_OPT_SIZE_MODE 1, unstaged gather), else as 2; results are
                                  identical */
#define SE_OPT_PC_THETA   10   /* damping theta of the spectral correction, in [0, 1]; 0 (default) = 0.9, the
                                  best single value over generated mono-, bi- and polydisperse suspensions
                                  (the best per configuration ranges from 0.8 to 0.98, which the learned
                                  preconditioner predicts; too large a value stalls the corrected cycles) */
#define SE_OPT_PC_KA      11   /* cutoff k_c a of the spectral correction, a the mean radius (default 0.9) */
#define SE_OPT_PC_CMAX    17   /* cap in [0.5, 0.99] of the largest eigenvalue of the spectral correction C
                                  (default 0.97): where the estimate of |C| (48 Lanczos steps, times 1.01)
                                  passes it, C is scaled down to it, which keeps the preconditioner positive
                                  definite */
#define SE_OPT_GATHER      9   /* gather kernel: 0 = default (currently 1), 1 = one warp per particle
                                  reading the grid through L2, 2 = one CTA per spreading bin staging
                                  the bin's support window in shared memory (slower on B300 at P = 14
                                  and 24); results agree to rounding */

#define SE_OPT_SPREAD     12   /* spreading kernel: 0 = default (FP32: 8 x 4 x 16 blocks of one warp with
                                  packed FP32 FMAs where the grid has room for them, else 8^3 tiles),
                                  1 = 8^3 tiles always, 2 = 8 x 8 x 16 tiles of two warps (FP32); results
                                  agree to rounding */

#define SE_OPT_RESIDUAL   14   /* precision of the solver's true residuals and right-hand-side products
                                  when the products run in FP32: 2 (default, double-float) or 1 (FP64) */
#define SE_OPT_SHEAR      15   /* strain gamma in [-0.5, 0.5] of the periodic cell a1 = (L, 0, 0), a2 = (gamma L,
                                  L, 0), a3 = (0, 0, L) (a cube sheared in x along y, Sec. 3.2; default 0).
                                  Needs SE_OPT_SIZE_MODE 2 or 3 (set first; SE_ERR_ARG otherwise, also for a
                                  later change of the size mode); se_set_config must follow; the spectral
                                  and learned preconditioners take the plane waves of the sheared
                                  reciprocal lattice; positions may be given in any periodic image */
#define SE_OPT_FF_TABLE   16   /* FP64-equivalent mode (SE_OPT_PRECISION 2): 1 (default) keeps a double-float
                                  copy of the FP64 real-space pair table per configuration (about 176 bytes
                                  per stored pair: 7 GB at N = 2e5, rc = 7.5, phi = 0.45), so the
                                  double-float real-space sum reads no FP64 values; 0 drops it and the sum
                                  converts the FP64 table as it reads it (same result, less memory, more time) */
#define SE_OPT_PAIR_FILL  18   /* evaluation of the FP32 real-space pair table's radial coefficients (once per
                                  configuration): 0 (default) = double-float arithmetic on the FP32 pipe
                                  (erfc through a table of Chebyshev interpolants of erfc(x) exp(x^2), exp by
                                  argument reduction and its Taylor series), with FP64 for pairs closer than
                                  0.1 or with xi r > 8.5; 1 = FP64 for every pair.  Both give the coefficients
                                  to within an FP32 rounding; changing it re-evaluates the table */
#define SE_OPT_OVERLAP_CHECK 13  /* 1 (default): se_set_config fails with SE_ERR_OVERLAP if two spheres within
                                  the real-space cutoff overlap (touching is allowed; the far-field
                                  interactions of overlapping spheres are not those of the paper, and
                                  coincident centres make them infinite); 0: no check.  The check runs
                                  with the pair-table build of the configuration's working precision */

/* product stages reported by se_stage_times */
#define SE_STAGE_PERMUTE   0   /* inputs into cell order */
#define SE_STAGE_REAL      1   /* real-space pair kernel (auxiliary stream) */
#define SE_STAGE_SPREAD    2   /* Gaussian spreading */
#define SE_STAGE_FFT_XF    3   /* forward FFT, x pass (real-to-complex) */
#define SE_STAGE_FFT_YF    4   /* forward FFT, y pass */
#define SE_STAGE_FFT_Z     5   /* forward z pass + k-space scaling + inverse z pass */
#define SE_STAGE_FFT_YI    6   /* inverse FFT, y pass */
#define SE_STAGE_FFT_XI    7   /* inverse FFT, x pass (complex-to-real) */
#define SE_STAGE_GATHER    8   /* gather + real + self, written in caller order */
#define SE_NSTAGE          9

/* preconditioners for se_solve */
#define SE_PRECOND_NONE    0
#define SE_PRECOND_BLOCK   1   /* block-diagonal self + own-image blocks (Sec. 4.2) */
#define SE_PRECOND_LEARNED 2   /* SE_PRECOND_SPECTRAL with the damping, cutoff and norm cap that the learned
                                  network predicts for the configuration (se_set_learned_weights); the
                                  plain block preconditioner without weights or in a sheared cell */
#define SE_PRECOND_SPECTRAL 3  /* block preconditioner minus a correction of the long-wavelength
                                  transverse force modes (their eigenvalues n/(eta k^2) set the
                                  iteration count), applied as a forces-only product on a coarse
                                  grid; built with three extra products.  A restart cycle that fails
                                  to halve the residual switches the rest of the solve to the block
                                  preconditioner (a damping too strong for the configuration).  Not
                                  in the paper. */

/* Create a context on CUDA device `device`; `stream` is a cudaStream_t (may be 0 for
 * the legacy default stream), borrowed for the context's lifetime.  *out receives the
 * context, or NULL on failure (SE_ERR_CUDA). */
int se_create(se_ctx **out, int device, void *stream);

/* Destroy a context and free its scratch.  Synchronises its stream.  NULL is accepted. */
int se_destroy(se_ctx *ctx);

/* Ewald/SE parameters (Sec. 3.1, Eq. theta-param; Sec. 3.3):
 *   xi  splitting parameter (> 0),  M grid points per dimension (2^a 3^b, 8..512),
 *   P   support points per dimension (2..M),  rc real-space cutoff (> 0, < L/2 at
 *   se_set_config).  Invalidates the configuration-dependent setup. */
int se_set_params(se_ctx *ctx, double xi, int M, int P, double rc);

/* Scalar options (SE_OPT_*).  Returns SE_ERR_ARG for an unknown key or a bad value. */
int se_set_option(se_ctx *ctx, int key, double value);

/* Particle configuration: N spheres, box side L; pos [N][3] and radius [N] are FP64
 * DEVICE arrays (positions anywhere, wrapped into the box).  Builds the cell list,
 * the spreading bins and (lazily) the preconditioner.  Fails with SE_ERR_ARG unless
 * 1 <= N <= 2^28 (an empty configuration included) or for null pointers, SE_ERR_CUTOFF when
 * rc >= L/2 and SE_ERR_NONFINITE for non-finite or non-positive data.  The arrays are
 * copied; the caller may free them afterwards.  Synchronises the device (work of this
 * context still in flight on any stream finishes first): the real-space pair table of the
 * previous configuration is overwritten in place while it fits (same N for its offsets; up
 * to 6% more pairs than the largest earlier table), so a sequence of configurations of one
 * N allocates and frees nothing after the first; its buffers are returned by se_destroy.
 * Equal radii are detected on the device and make the FP32 table store 13 of the 19
 * coefficients per pair. */
int se_set_config(se_ctx *ctx, int64_t N, double L, const double *pos, const double *radius);

/* y = M_inf . x.  x, y: DEVICE arrays [N][ncomp] of dtype SE_F32 or SE_F64 (both the
 * same dtype); ncomp in {3, 6, 11, 12}.  x and y must not overlap.  Asynchronous. */
int se_mobility_apply(se_ctx *ctx, int ncomp, const void *x, void *y, int dtype);

/* Same product with HOST FP64 arrays x, y [N][ncomp]: copies x to the device, applies,
 * copies y back and synchronises.  Pinned host memory gives the fastest copies. */
int se_mobility_apply_host(se_ctx *ctx, int ncomp, const double *x, double *y);

/* Solve M_inf . x = b by right-preconditioned GMRES(restart) (Sec. 4.1-4.2 with the
 * near-field resistance set to zero).  b, x: DEVICE arrays [N][ncomp] of `dtype`;
 * x holds the initial guess on entry and the solution on exit.  Krylov vectors and
 * the true residual b - M x are FP64; products run at SE_OPT_PRECISION and the final
 * residual check (one refinement restart if needed) uses an FP64 product.
 * rtol: relative residual target; maxit: maximum products; precond: SE_PRECOND_*.
 * *iters (may be NULL) receives the number of products, *relres (may be NULL) the
 * final FP64 relative residual.  Synchronises.  Returns SE_ERR_NOT_CONVERGED if
 * relres > rtol after maxit products. */
int se_solve(se_ctx *ctx, int ncomp, const void *b, void *x, int dtype, double rtol,
             int maxit, int precond, int *iters, double *relres);

/* Allocation-free real-space part.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory -- an application whose own allocator
 * reserves the device memory up front, or a latency-critical caller that cannot accept
 * the device-wide synchronisation of cudaMalloc / cudaFree.  It computes the real-space
 * pair sum of y = M_inf . x (all pairs with |x| < rc, the couplings of se_mobility_apply's
 * real-space part, FP64) for N <= SE_NOALLOC_MAX_N spheres, with the cell list and all
 * other scratch in one fixed device array of about 2 MB that every GPU loading the
 * library holds until the process exits; cells are enlarged if more than
 * SE_NOALLOC_MAX_CELLS would be needed.  It calls no allocator.
 *   device, stream : CUDA device and cudaStream_t to run on (stream may be 0)
 *   N, L           : spheres and box side;  xi, rc, eta : Ewald parameter, cutoff (< L/2),
 *                    viscosity;  pos [N][3], radius [N] : FP64 DEVICE arrays
 *   x, y           : FP64 DEVICE arrays [N][ncomp], ncomp in {3, 6, 11, 12}; y is overwritten
 * Returns SE_ERR_TOO_LARGE if N > SE_NOALLOC_MAX_N, SE_ERR_CUTOFF if rc >= L/2,
 * SE_ERR_ARG for null pointers or bad sizes, SE_ERR_NONFINITE for non-finite positions
 * or non-positive radii, SE_ERR_CUDA for a failed CUDA call of this call (a launch error
 * left pending by earlier, unrelated work is cleared on entry, not reported).  Every call
 * waits for `stream` (it reads a status flag back) and leaves the calling thread's
 * current device as it found it.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress).
 * All calls share the one array and
 * every call clears what must start at zero; calls that overlap on the GPU race on it,
 * so the caller must not run two at once. */
#define SE_NOALLOC_MAX_N     8192
#define SE_NOALLOC_MAX_CELLS 4096
int se_real_space_apply_noalloc(int device, void *stream, int64_t N, double L, double xi, double rc,
                                double eta, const double *pos, const double *radius, int ncomp,
                                const double *x, double *y);

/* Far-field Brownian displacement source: x = M^{-1/2} c for the F, T, S block of the
 * far-field grand mobility (Sec. 4.3, Eq. br-f-ff: F^B,ff and the Brownian stresslet
 * fluctuation are (2kT/dt) M^{-1/2} Psi), by the initial value problem of Eq. ivp-1 marched
 * with the explicit and implicit Euler half-steps of Eqs. ivp-forward/ivp-backward.
 *   ncomp   : 3, 6 or 11 (the symmetric positive definite F, T, S prefix)
 *   scale   : s > 0 with A = s M (the IVP is solved for A; x = sqrt(s) A^{-1/2} c); s <= 0
 *             selects 6 pi eta <a>, which puts A's translational self blocks near I
 *   nsteps  : number of steps, dtau = 1 / nsteps (the paper finds dtau = 0.1 adequate)
 *   rtol, maxit : tolerance and product limit of each of the 2 nsteps GMRES solves
 *             (shifted operators alpha I + beta M, block preconditioner of the shift;
 *             products at the context's precision with FP64 refinement)
 *   c, x    : FP64 DEVICE arrays [N][ncomp] (c is read, x is written; they may not alias)
 *   products: if not NULL, receives the number of products used
 * Returns SE_ERR_NOT_CONVERGED if a solve missed rtol (x is still written); synchronises. */
int se_brownian_ivp(se_ctx *ctx, int ncomp, double scale, int nsteps, double rtol, int maxit,
                    const double *c, double *x, int *products);

/* Rigid spheres driven by forces and torques and by an imposed strain rate E_inf
 * (Sec. 6.1): [U; Omega; E_inf] = M [F; T; S] with the stresslets S unknown; for E_inf = 0,
 * (U, Omega) = mu (F, T) with mu = M_UF - M_US M_ES^{-1} M_EF, the inverse of the FU block
 * of the far-field resistance M^{-1}.  Solved as one GMRES system for (U, Omega, S) (one
 * product per iteration, block preconditioner of that system; M [F; T; 0] in FP64).
 *   ft [N][6] (F, T; may be NULL: force- and torque-free), uw [N][6] (U, Omega), s [N][5]
 *   (S on the orthonormal basis; may be NULL): FP64 DEVICE arrays, caller order;
 *   einf: 5 HOST doubles, the imposed strain rate on the orthonormal basis (NULL: 0);
 *   iters, relres as for se_solve.
 * Returns SE_ERR_NOT_CONVERGED if rtol was missed (outputs still written); synchronises. */
int se_rigid_solve(se_ctx *ctx, const double *ft, const double *einf, double *uw, double *s, double rtol,
                   int maxit, int *iters, double *relres);

/* High-frequency shear viscosity eta_s / eta of the far-field suspension (the eta_s of
 * Eq. dst-corr): force- and torque-free rigid spheres in each of the five orthonormal
 * basis strains; eta_s / eta - 1 = sum_i S_i . e_k / (2 eta V), averaged over the five.
 * products: total products used (may be NULL).  Synchronises. */
int se_high_frequency_viscosity(se_ctx *ctx, double rtol, int maxit, double *eta_ratio, int *products);

/* Far-field short-time self-diffusivities by the matrix-free estimator of Sec. 6.1
 * (Eq. dstr-def): for random (F, T) with zero mean and unit covariance, the average of
 * (U, Omega) (F, T) over samples is diag(mu), mu as in se_rigid_solve.
 *   fr [nsamples][N][6]: the samples (FP64 DEVICE, drawn by the caller), d [N][2]: per
 *   particle the estimates of tr(mu_ii^tt)/3 and tr(mu_ii^rr)/3 (FP64 DEVICE, caller
 *   order; times kT these are the particle's translational and rotational diffusivity,
 *   to be averaged over a species by the caller); products: total products used.
 * Returns SE_ERR_NOT_CONVERGED if a solve missed rtol; synchronises. */
int se_far_field_diffusivity(se_ctx *ctx, int nsamples, const double *fr, double *d, double rtol, int maxit,
                             int *products);

/* Learned preconditioner (SE_PRECOND_LEARNED).  A small network (16 -> 64 -> 64 -> 4,
 * tanh, FP32) maps rotation- and permutation-invariant features of each sphere's radius and
 * of its neighbours inside rc (and the box size L / <a>) to per-sphere outputs whose mean
 * over the spheres sets the damping theta, the cutoff k_c <a> and the norm cap c_max of the
 * spectral correction of the Sec. 4.2 block preconditioner (clamped to [0.5, 0.985],
 * [0.4, 1.5] and [0.85, 0.985]).
 * Weights are SE_MLP_NW packed floats (layout in se_learned.cu), produced by
 * paper_1506_08481_b300/train_pc.py from the iteration counts of solves over a grid of
 * (theta, k_c <a>, c_max) on generated configurations.
 *   se_set_learned_weights: copies the HOST array w; SE_ERR_NONFINITE on NaN/Inf.
 *   se_learned_features   : DEVICE feat [N][16] in caller order for the configuration.
 *   se_mlp_forward        : DEVICE w, X [n][16] -> Y [n][4] (the outputs, unstandardised).
 *   se_mlp_grad           : gradient DEVICE grad [SE_MLP_NTRAIN] and loss [1] of the mean
 *                           squared error of the standardised outputs against Yt [n][4];
 *                           scratch >= n * 276 floats (SE_ERR_TOO_LARGE otherwise).
 *   se_mlp_adam_step      : one Adam update (beta 0.9, 0.999) of the trained parameters.
 * The network's kernels are asynchronous on `stream` except se_learned_features. */
#define SE_MLP_NW     5544
#define SE_MLP_NTRAIN 5508
int se_set_learned_weights(se_ctx *ctx, const float *w, int nw);
int se_learned_features(se_ctx *ctx, float *feat);
int se_mlp_forward(const float *w, const float *X, int n, float *Y, void *stream);
int se_mlp_grad(const float *w, const float *X, const float *Yt, int n, float *grad, float *loss,
                float *scratch, size_t scratch_floats, void *stream);
int se_mlp_adam_step(float *w, float *m, float *v, const float *grad, int step, float lr, void *stream);

/* Batches of independent boxes (uneven N, each with its own context and parameters).
 * This replaces a single batched call over ragged arrays with per-box offsets
 * (se_mobility_apply_batched(ctx, nbox, offsets, ...)): each box keeps its own context
 * (its own xi, M, P, rc and configuration), and a batch groups existing contexts.
 * se_batch_create borrows nbox configured contexts (they must outlive the batch) and
 * runs box i on the i-th (mod nstreams) of nstreams streams it creates, forked from
 * and joined back to `stream`.
 * se_batch_apply enqueues y[i] = M_inf(box i) . x[i] for every box (DEVICE arrays
 * [N_i][ncomp] of `dtype`).  use_graph selects how:
 *   0  every box's kernels are launched one by one (box i on stream i mod nstreams);
 *   1  the first call (and any call with other pointers, ncomp or dtype) runs the batch
 *      once eagerly, captures it into one CUDA graph and launches it; later calls only
 *      launch the graph;
 *   2  ONE persistent cooperative launch computes every box (FP32 boxes with their
 *      stored pair tables): per box eight phases in order (inputs, real space +
 *      spreading, five FFT passes with the k-space scaling, gather), each a list of
 *      work items; a CTA claims an item of any box whose earlier phases have finished
 *      (per-box counters, no grid-wide barrier), so the boxes' phases overlap.  The
 *      first call runs the batch eagerly and prepares the launch (captured into a graph
 *      when the runtime allows); later calls make the one launch.  A CTA that finds no
 *      ready item for longer than the wait limit (default 2 s) aborts the launch, and
 *      every CTA returns; se_batch_status reports it.
 * Asynchronous on `stream`; errors as for se_mobility_apply (SE_ERR_STATE when a box
 * does not meet mode 2's conditions), described by se_batch_last_error.
 * se_batch_status synchronises `stream` and returns SE_ERR_CUDA if a persistent launch
 * since the previous call was aborted, else SE_OK. */
typedef struct se_batch se_batch;
int se_batch_create(se_batch **out, se_ctx *const *ctx, int nbox, int nstreams, void *stream);
int se_batch_apply(se_batch *b, int ncomp, const void *const *x, void *const *y, int dtype, int use_graph);
int se_batch_destroy(se_batch *b);
int se_batch_status(se_batch *b);
const char *se_batch_last_error(const se_batch *b);

/* se_batch_set_wait_limit: the time limit (seconds, in (0, 600]) of every wait of a
 * persistent launch (mode 2) for work of an earlier phase; the next mode-2 call prepares
 * the launch again.  se_batch_inject_stall: failure-injection hook for tests of that
 * bounded wait; box >= 0 makes that box's real-space/spreading phase never count as
 * finished, so the CTAs waiting for it give up after the wait limit and the launch
 * returns with the failure that se_batch_status reports (no fault, no hang; the
 * results of that launch are not valid); box = -1 turns it off.  Both return
 * SE_ERR_ARG for a bad value. */
int se_batch_set_wait_limit(se_batch *b, double seconds);
int se_batch_inject_stall(se_batch *b, int box);

/* FP32 FMA throughput probe (no counterpart in the paper): the measured peak that the
 * ALU-bound spreading and gather kernels are compared with.  Enqueues on `stream` one
 * launch of 8 CTAs of 256 threads per SM of `device`, each thread running 8 independent
 * FMA chains of `iters` rounds; the caller times it with CUDA events on `stream`.
 *   sink : DEVICE float[1], written only in a case that never occurs (keeps the chains live)
 *   flop : receives the launch's floating-point operations (an FMA counts 2)
 *   sms  : if not NULL, receives the device's number of streaming multiprocessors
 * Returns SE_ERR_ARG for iters < 1 or null pointers, SE_ERR_CUDA for a failed launch.
 * Asynchronous; the calling thread's current device is left as it was. */
int se_fp32_fma_probe(int device, void *stream, int iters, float *sink, double *flop, int *sms);

/* Message describing the last failure on this context ("" if none).  Valid until the
 * next call on the same context.  ctx may be NULL (returns the last create failure). */
const char *se_last_error(const se_ctx *ctx);

/* Number of CUDA kernels this context has launched since creation (for accounting). */
int64_t se_kernel_launches(const se_ctx *ctx);

/* With SE_OPT_TIMING on: ms[s] (s < nstage <= SE_NSTAGE) receives the summed device
 * time of stage s over the products run since the previous call, measured with CUDA
 * events recorded on the stream that launched the stage.  Synchronises; returns the
 * number of products summed (>= 0) or a negative error code. */
int se_stage_times(se_ctx *ctx, double *ms, int nstage);

#ifdef __cplusplus
}
#endif
#endif /* SE_MOBILITY_H */
