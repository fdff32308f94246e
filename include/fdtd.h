/*
 * fdtd.h -- C ABI of the GB300 (sm_103a) FDTD + Drude adjoint library.
 *
 * The library computes, on one GPU, the hot path of time-domain topology
 * optimization of Drude-dispersive nanostructures (Hassan & Cala Lesina,
 * arXiv 2203.01462):
 *
 *   set_design   rho -> rho~ = F(rho) (Eq. 26) and the per-node material of
 *                Eq. (5a-c), evaluated inside the stencil kernels;
 *   set_damping  sigma_max of Eq. (5c) and a scale on the Drude collision
 *                rate (the artificial damping level, Sec. 2.1);
 *   forward      Yee leapfrog of Eq. (10a-c) (E, J at integer steps, H at
 *                half steps, Sec. 3.2), CPML borders, soft current source,
 *                objective W~ of Eq. (24), gap-field history for the adjoint
 *                source and the design-box field record (full history or
 *                snapshots every k steps);
 *   adjoint      the same solver in reversed time driven by eps_g E(T - tau)
 *                in the gap (Eq. 20), recomputing forward segments from
 *                snapshots when needed, with the sensitivities of
 *                Eq. (25a-c) accumulated per design node in the same pass;
 *   gradient     chain rule of Eq. (27) with the filter transpose, giving
 *                dW~/drho (ascent direction; the paper maximises W~).
 *
 * Ownership: the caller owns every device buffer.  The library allocates no
 * device memory (one mapped word of pinned host memory per context carries
 * the stability guard's flag); it carves all of its state out of the caller's workspace
 * (size from fdtd_workspace_bytes) and enqueues all work on the caller's
 * CUDA stream.  A context is used by one host thread and one stream at a
 * time.  Pointers named d_* are device pointers, h_* host pointers.
 *
 * Errors: every entry point returns an fdtd_status; nothing throws or aborts
 * across the ABI.  Calls out of order return FDTD_ESTATE.  Device-side
 * checks (density outside [0,1], a non-finite objective, the stability
 * guard) set an error word that fdtd_sync reports.
 *
 * Units: SI.  W~ follows Eq. (24) literally (eps_g dt dx^d / 2 times the sum
 * of |E|^2 over the gap nodes and steps n = 0..N; d = 2 in 2D, per unit
 * length in z; d = 3 in 3D), so it is small in absolute terms; W~ and the
 * gradient are returned in FP64 whatever the field precision.
 *
 * 2D: TM_z (Ez, Hx, Hy, Jz) on nx x ny nodes.  3D: full Yee grid on
 * nx x ny x nz nodes, Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at
 * (i, j, k+1/2); the three E components of node (i, j, k) share rho(i, j, k)
 * and the gradient sums their sensitivities.  3D takes no design filter.
 */
#ifndef FDTD_GB300_H
#define FDTD_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fdtd_status {
    FDTD_OK = 0,
    FDTD_EINVAL = 1,     /* bad argument or configuration                     */
    FDTD_ENOMEM = 2,     /* workspace smaller than fdtd_workspace_bytes       */
    FDTD_ECUDA = 3,      /* a CUDA runtime call failed                         */
    FDTD_ESTATE = 4,     /* call out of order (e.g. adjoint before forward)    */
    FDTD_EUNSTABLE = 5,  /* unstable run: a non-finite objective, or a state
                            word non-finite or above the stability-guard
                            bound (fdtd_set_stability_guard)                 */
    FDTD_ETIMEOUT = 6,   /* a bounded device wait gave up (the in-plane
                            multi-step launch: a block waited about a second
                            at a grid barrier)                               */
    FDTD_ERANGE = 7      /* a design density outside [0, 1]                    */
} fdtd_status;

/* Checkpoint storage: FDTD_SNAP_F32 keeps the field precision (lossless);
 * BF16 / F16 store 16-bit words with one scale per slab of 2048 state words
 * (lossy: the recomputed forward fields, hence the gradient, carry the
 * rounding of the restart). */
enum { FDTD_SNAP_F32 = 0, FDTD_SNAP_BF16 = 1, FDTD_SNAP_F16 = 2 };
/* Sensitivity accumulator: FDTD_ACC_F64 (one FP64 sum per design node).
 * FDTD_ACC_COMP_F32 (a compensated FP32 pair) is reserved and rejected with
 * FDTD_EINVAL: it would move the same 16 bytes per node and step. */
enum { FDTD_ACC_F64 = 0, FDTD_ACC_COMP_F32 = 1 };
enum { FDTD_SIGMA_PAPER = 0, FDTD_SIGMA_PEAK_NORMALISED = 1 };

/* Excitation g(t) = envelope(u) * sum_b sin(2 pi f0[b] u), u = t - t0.
 * FDTD_WAVE_GAUSS: envelope exp(-(u/tau)^2).
 * FDTD_WAVE_SINC_HANN (the paper's excitation, Sec. 2, Fig. 1c-d): a sinc
 * with a rectangular spectrum of width B = bandwidth, sin(pi B u)/(pi B u),
 * kept for |u| < T = lobes / B and smoothed by the Hanning window
 * (1 + cos(pi u / T)) / 2; zero outside.  t0 >= T starts it from rest. */
enum { FDTD_WAVE_GAUSS = 0, FDTD_WAVE_SINC_HANN = 1 };

/* 2D polarisation.
 * FDTD_POL_EZ: E out of plane (Ez, Hx, Hy, Jz on nx x ny nodes; the paper's
 *   2D TE case); boxes are node ranges; one design variable per node.
 * FDTD_POL_INPLANE: E in plane (the paper's 2D TM case, Sec. 3.2, in which
 *   surface plasmons exist): Ex on the edges (i+1/2, j), Ey on (i, j+1/2),
 *   Hz at cell centres, Drude Jx, Jy per edge.  Design, gap and source boxes
 *   are cell ranges [lo, hi) with hi <= n - 1 (the source box: E_x edges
 *   i < nx - 1).  The design variables are the Yee edges of the design box,
 *   as the paper assigns them: rho holds the E_x edges (i in [lo_x, hi_x),
 *   j in [lo_y, hi_y], row-major) followed by the E_y edges (i in
 *   [lo_x, hi_x], j in [lo_y, hi_y)), M_d = w (h + 1) + (w + 1) h; the gap
 *   edges are fixed (gradient 0) and W~ sums E^2 over them (Eq. 24, dx^2).
 *   The source drives E_x edges.  No design filter (filter_radius 0). */
enum { FDTD_POL_EZ = 0, FDTD_POL_INPLANE = 1 };

/* 3D plane wave by total-field / scattered-field injection (tfsf = 1; the
 * paper's 3D study illuminates at normal incidence, Sec. 3.3).  An
 * x-polarised plane wave travelling along +z enters through the faces of a
 * total-field box instead of through the source box's current: a field
 * component whose Yee position (E_x at (i+1/2, j, k), E_z at (i, j, k+1/2),
 * H_y at (i+1/2, j, k+1/2), ...) lies in the closed box
 * tf_lo <= x <= tf_hi (node units) holds the total field, every other one
 * the scattered field.  The incident field is that of a 1D column along z
 * with the grid's background layering (sub_eps below sub_hi, eps_s above),
 * the same z-CPML and PEC ends, driven by the soft E_x current of the plane
 * k = src_lo[2] with the configured waveform (the source box's x and y
 * extent is unused).  fdtd_create runs the column once on the device and
 * keeps one row of incident values per step in the workspace
 * (nsteps x (2 (tf_hi[2] - tf_lo[2] + 1) + 1) words).  Requirements
 * (FDTD_EINVAL otherwise): ndim = 3, src_comp = 0, src_lo[2] >= 1,
 * src_hi[2] = src_lo[2] + 1 <= tf_lo[2]; per axis
 * npml + 1 <= tf_lo < tf_hi <= n - npml - 2; and the box strictly around the
 * design box, tf_lo < design_lo and tf_hi >= design_hi, so that every
 * corrected component is background material.  The injection does not
 * depend on rho: the adjoint run (Eq. 20) and the sensitivities (Eq. 25)
 * are those of any other source. */

/* Problem description.  Boxes are half-open node ranges [lo, hi) per axis
 * (x, y, z); in 2D the z range must be [0, 1).  Grid: nx x ny Ez nodes in
 * 2D; nx x ny x nz Yee nodes in 3D. */
typedef struct fdtd_config {
    int ndim;                 /* 2: see pol; 3: full Yee                      */
    int nx, ny, nz;
    double dx;                /* grid step, m (dx = dy = dz, Sec. 3.2)         */
    double courant;           /* S = c0 dt / dx                                */
    int npml;                 /* CPML layers per side, PEC walls behind        */
    double pml_m;             /* CPML polynomial grading order                 */
    double pml_sigma_factor;  /* sigma_pml_max = factor (m + 1) / (eta0 dx)    */
    double pml_kappa_max;
    double pml_alpha_max;     /* S/m, linear taper                             */
    double eps_inf, omega_p, gamma_p;  /* Drude material, Eq. (1)              */
    double eps_s;             /* background relative permittivity              */
    double psi_s_ratio;       /* psi_s = ratio * omega_p^2 (paper: 0.01)       */
    double eps_g;             /* gap permittivity                              */
    int design_lo[3], design_hi[3];
    int gap_lo[3], gap_hi[3];
    int src_lo[3], src_hi[3]; /* soft current source box (Ez in 2D, src_comp   */
                              /* edges in 3D)                                 */
    int nbands;               /* 1 or 2 carriers under one envelope            */
    double f0[2];             /* carrier frequencies, Hz                       */
    double tau, t0;           /* Gaussian width (FDTD_WAVE_GAUSS) and delay, s */
    double src_amp;           /* J_src = src_amp eps0 c0 / dx g(t), A/m^2      */
    int nsteps;               /* N                                             */
    int filter_radius;        /* Gaussian filter half-width, cells; 0 = none   */
    double filter_sigma;      /* Gaussian filter standard deviation, cells     */
    int sigma_form;           /* FDTD_SIGMA_*                                  */
    double sub_eps;           /* 3D: background eps of cells with k < sub_hi   */
    int sub_hi;
    int real_bytes;           /* field precision: 4 (FP32) or 8 (FP64)         */
    int snapshot_every;       /* 0: keep the full design-box E history;        */
                              /* k > 0: checkpoint every k steps, recompute    */
    int snapshot_dtype;       /* FDTD_SNAP_*: snapshot storage precision       */
    int accum_kind;           /* FDTD_ACC_*: sensitivity accumulator           */
    int src_comp;             /* 3D: E component the source drives (0 x, 1 y, */
                              /* 2 z); the source box holds those edges      */
    int waveform;             /* FDTD_WAVE_*: envelope of the carrier(s)       */
    double bandwidth;         /* FDTD_WAVE_SINC_HANN: rectangle width B, Hz    */
    int lobes;                /* FDTD_WAVE_SINC_HANN: lobes kept per side      */
    int pol;                  /* 2D: FDTD_POL_*                                */
    int tfsf;                 /* 3D: 1 = plane wave by TFSF injection (above)  */
    int tf_lo[3], tf_hi[3];   /* total-field box, closed, node units           */
} fdtd_config;

typedef struct fdtd_ctx fdtd_ctx;

/* Run-time facts about a context. */
typedef struct fdtd_info {
    double dt;                    /* time step, s                              */
    long long n_cells;            /* grid nodes (2D) / cells (3D)              */
    long long n_design;           /* M_d, length of rho and of the gradient    */
    long long n_gap;              /* M_g                                       */
    long long launches;           /* kernels launched since create             */
    long long cell_updates;       /* cells x steps advanced since create       */
    size_t workspace_bytes;
    long long step_blocks;        /* 2D E_z: thread blocks of one step launch  */
    long long vector_blocks;      /* 2D E_z: of those, blocks whose tile and
                                     its one-node halo are clear of walls and
                                     CPML, which run the 16-byte vector path;
                                     0 and 0 in the other modes                */
} fdtd_info;

/* Bytes of device workspace a context for cfg needs (256-byte aligned
 * start expected).  Fails with FDTD_EINVAL on an invalid configuration. */
fdtd_status fdtd_workspace_bytes(const fdtd_config *cfg, size_t *bytes);

/* Create a context on the current device.  d_workspace: caller-owned device
 * memory of at least fdtd_workspace_bytes bytes, 256-byte aligned, kept
 * alive until fdtd_destroy.  stream: a cudaStream_t (NULL = legacy default
 * stream).  Builds the CPML and source tables on the host, uploads them and
 * synchronises the stream once. */
fdtd_status fdtd_create(const fdtd_config *cfg, void *d_workspace, size_t bytes,
                        void *stream, fdtd_ctx **out);

/* Set the design densities (Sec. 2.1).  d_rho: device array of n = M_d
 * values in the context's field precision (float for real_bytes 4, double
 * for 8), x fastest, then y (then z); entries inside the gap are ignored
 * (the gap is vacuum of eps_g).  Applies the filter of Eq. (26).  Checks
 * 0 <= rho <= 1 on the device and synchronises the stream: returns
 * FDTD_ERANGE if any entry is outside.  Invalidates earlier forward and
 * adjoint results. */
fdtd_status fdtd_set_design(fdtd_ctx *ctx, const void *d_rho, size_t n);

/* Artificial damping (Sec. 2.1): sigma_max of Eq. (5c) in S/m (>= 0) and a
 * factor (> 0) on the Drude collision rate.  Defaults: 0 and 1.
 * Invalidates earlier forward and adjoint results. */
fdtd_status fdtd_set_damping(fdtd_ctx *ctx, double sigma_max, double gamma_scale);

/* Terms of the sensitivity (Eq. 25a-c) that the adjoint run accumulates:
 * any non-empty OR of FDTD_TERM_PSI (Eq. 25a, through d psi_i / d rho~ =
 * psi - psi_s), FDTD_TERM_EPS (Eq. 25b, through eps_inf - eps_s) and
 * FDTD_TERM_SIGMA (Eq. 25c, through d sigma_i / d rho~).  Default
 * FDTD_TERM_ALL: the gradient of W~.  With one term selected, fdtd_gradient
 * returns F^T (Eq. 27) of that term alone, gap entries zero; the three
 * single-term gradients add up to the full one (up to rounding).  A check
 * of the adjoint term by term against a reference; the fields are not
 * affected.  FDTD_EINVAL for a mask outside 1..7.  Invalidates an earlier
 * adjoint result. */
enum { FDTD_TERM_PSI = 1, FDTD_TERM_EPS = 2, FDTD_TERM_SIGMA = 4, FDTD_TERM_ALL = 7 };
fdtd_status fdtd_set_sensitivity_terms(fdtd_ctx *ctx, int terms);

/* Stability guard of the forward solve.  Every `every` forward steps (0:
 * off; default 256) a read-only kernel checks every word of the solver
 * state (E, H, J and the CPML terms) and flags a word that is not finite or
 * whose magnitude exceeds `max_abs` (field units; 0: automatic, 1e3 x N x
 * src_amp x S x the number of bands, i.e. a thousand times the field that
 * every step's source increment could build up, which no passive
 * configuration approaches).  A flagged run is reported as FDTD_EUNSTABLE:
 * fdtd_forward returns it as soon as the host loop that enqueues the steps
 * sees the flag (through one mapped word of pinned host memory per context)
 * and stops enqueuing, after waiting for the steps already enqueued; when
 * the pass replays as a CUDA graph, fdtd_sync reports it at the end.  The
 * error word is then cleared, and the context can take a new design or new
 * settings.  The checks read the state once per `every` steps (0.2 % of the
 * forward traffic at the default) and change no result. */
fdtd_status fdtd_set_stability_guard(fdtd_ctx *ctx, int every, double max_abs);

/* Width of the Gaussian design filter (Eq. 26) of a 2D E_z context created
 * with filter_radius > 0: sigma (cells) replaces cfg->filter_sigma, the
 * window keeps the create-time radius.  Lets an optimizer continue the
 * filter (a wide filter first, a narrow one at the end) without a new
 * context.  Synchronises the stream; the design has to be set again
 * (FDTD_ESTATE until then).  FDTD_EINVAL for other contexts or sigma <= 0. */
fdtd_status fdtd_set_filter_width(fdtd_ctx *ctx, double sigma);

/* Time steps per launch.  In-plane 2D contexts (pol = FDTD_POL_INPLANE):
 * default 1 (one launch per half step).  With more than one, a run of
 * steps is one cooperative launch, one block per SM, whose half steps are
 * separated by grid-wide barriers with bounded waits (FDTD_ETIMEOUT from
 * fdtd_sync if one gives up).  Results are bit-identical either way.  On a
 * GB300 the barrier costs more than the launch boundary it replaces (about
 * 12 against 6 us per step on the paper's 491^2 geometry), hence the
 * default.  Such passes are not replayed as CUDA graphs.
 *
 * 2D E_z contexts: with steps > 1 the forward (and recompute) and the
 * full-history adjoint advance up to min(steps, 8) steps per launch (4 in
 * FP64) by temporal blocking: a block owns a square tile (16 to 32 nodes a
 * side, the smallest whose tiles fit one wave of blocks), loads it with a
 * halo of that many nodes into shared memory, advances all the steps there
 * and writes back its tile, so no block waits for another.  Small grids,
 * whose launch-per-step kernels are single partial waves, gain: the default
 * is 8 for FP32 grids of at most one 32 x 32 tile per SM (316^2: 7.1 -> 2.9
 * us per forward step) and 1 otherwise (a 640^2 grid or an FP64 one runs
 * slower blocked).  Results agree with the launch-per-step path to rounding
 * (the per-node arithmetic of its generic path).
 *
 * 3D contexts ignore the setting (see fdtd_set_wavefront). */
fdtd_status fdtd_set_steps_per_launch(fdtd_ctx *ctx, int steps);

/* 3D contexts: time steps per wavefront launch of the leapfrog (Eq. 10,
 * Sec. 3.2).  steps = 0 runs every step as two launches over the whole
 * grid, the H half step then the E half step.  steps = 1 .. 8 runs up to
 * that many steps per persistent cooperative launch (fewer when their L2
 * window would exceed half the L2): the grid is cut into z slabs of two
 * planes, and each slab's E half step runs right after the H half steps it
 * reads, and the next step's H right after the E half steps it reads, while
 * those fields are still in L2.  Blocks wait on per-slab counters of
 * finished tiles; a wait that does not end within about a second makes the
 * pass report FDTD_ETIMEOUT at fdtd_sync.  Every node's arithmetic is that
 * of the two-launch form, so the results are bit-identical.  Default 0.
 * Wavefront passes are not replayed as CUDA graphs.  Returns FDTD_EINVAL
 * for other modes or steps outside 0 .. 8, FDTD_ECUDA when the device
 * cannot run the cooperative launch. */
fdtd_status fdtd_set_wavefront(fdtd_ctx *ctx, int steps);

/* Self-test of the bounded device wait the multi-step launch uses: one
 * thread waits on a flag that nothing sets, for limit_cycles clock cycles.
 * d_words: 16 bytes of caller device memory (16-byte aligned), overwritten.
 * Returns FDTD_ETIMEOUT when the wait gave up and reported it as it should,
 * FDTD_OK if the flag was seen set, FDTD_ECUDA / FDTD_EINVAL on errors.
 * Synchronises `stream` (a cudaStream_t). */
fdtd_status fdtd_selftest_bounded_wait(void *d_words, long long limit_cycles, void *stream);

/* Forward solve of N steps.  Writes W~ (Eq. 24) to d_W (device, one double;
 * may be NULL) asynchronously.  Requires fdtd_set_design.  Returns
 * FDTD_EUNSTABLE when the stability guard stopped the pass (no W~). */
fdtd_status fdtd_forward(fdtd_ctx *ctx, double *d_W);

/* Adjoint solve (Eq. 20) with the sensitivity accumulation of Eq. (25).
 * Requires fdtd_forward since the last set_design / set_damping. */
fdtd_status fdtd_adjoint(fdtd_ctx *ctx);

/* dW~/drho (Eq. 27, with F^T) into d_grad (device, n = M_d doubles); zero
 * on gap nodes.  Requires fdtd_adjoint since the last forward. */
fdtd_status fdtd_gradient(fdtd_ctx *ctx, double *d_grad, size_t n);

/* Largest design box (M_d) that fdtd_gradient_static accepts. */
#define FDTD_STATIC_DESIGN_MAX 1048576

/* Same result as fdtd_gradient, but the two FP64 intermediates of the
 * filter-transpose passes live in a fixed array owned by the library
 * (2 x FDTD_STATIC_DESIGN_MAX doubles = 16 MiB of device memory on every GPU
 * that loads the library, kept until the process exits) instead of the
 * context's workspace; nothing is allocated.  For callers that cannot hand
 * out or grow device memory at call time.  The paper has no counterpart.
 * Only a 2D E_z context with a design filter uses the array: for it, n above
 * FDTD_STATIC_DESIGN_MAX returns FDTD_EINVAL; the other contexts need no
 * intermediates and take any n.  Call it with the device that created the
 * context current (otherwise FDTD_EINVAL).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current, so make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race on it. */
fdtd_status fdtd_gradient_static(fdtd_ctx *ctx, double *d_grad, size_t n);

/* Gap-field history E^n, n = 0..N, of the last forward run into d_out
 * (device doubles, gap nodes x fastest): 2D n = (N + 1) * M_g; 3D
 * n = (N + 1) * 3 * M_g, layout [step][component x, y, z][gap node]. */
fdtd_status fdtd_gap_history(fdtd_ctx *ctx, double *d_out, size_t n);

/* ---- optimization-loop helpers (Sec. 3.2, Eq. 28) ----
 * The paper updates the design with GCMMA; this library provides its
 * per-variable steps (below), a projected, normalised gradient-ascent step
 * as a simpler alternative, and the paper's grayness measure and final
 * thresholding. */

/* d_rho <- clip(d_rho + move * d_grad / max|d_grad|, 0, 1) on the device
 * (n = M_d; d_rho in the field precision, d_grad FP64).  A zero gradient
 * leaves rho unchanged.  Asynchronous; uses a word of the context's
 * workspace. */
fdtd_status fdtd_ascent_step(fdtd_ctx *ctx, void *d_rho, const double *d_grad, size_t n, double move);

/* Spectrum of the recorded gap field (the observation domain of Sec. 3.2,
 * whose average |E| / |E_in| is the paper's field enhancement): with the
 * e^{j w t} convention, E(w) = dt sum_{n=0..N} E^n e^{-j w n dt}, for each
 * of nf frequencies d_freqs (device, Hz) and each recorded gap value
 * (2D: M_g E_z nodes; 3D: 3 components x M_g nodes, component-major).
 * d_out (device) receives nf x ncomp x M_g complex values as (re, im)
 * double pairs, frequency-major.  Requires a forward run since the last
 * fdtd_set_design (FDTD_ESTATE otherwise); FDTD_EINVAL for null pointers,
 * nf < 1 or an empty gap.  Asynchronous. */
fdtd_status fdtd_gap_spectrum(fdtd_ctx *ctx, const double *d_freqs, int nf, double *d_out);

/* Method of moving asymptotes with the conservative inner loop of GCMMA
 * (Svanberg, Int. J. Numer. Meth. Eng. 24, 1987; SIAM J. Optim. 12, 2002),
 * the paper's design update (Sec. 3.2), for max W~ over 0 <= rho <= 1
 * written as min f, f = -scale * W~.  The host runs the loop; these two
 * calls do the per-variable work.
 *
 * d_state: caller-owned device array of 4*n doubles (x^{k-1}, x^{k-2}, L, U,
 * back to back), any content before iteration 0.  n = M_d; d_rho and
 * d_rho_new in the field precision; d_grad = dW~/drho (FP64, as from
 * fdtd_gradient); d_sums: two device doubles, overwritten.
 *
 * fdtd_mma_asymptotes, once per outer iteration k = 0, 1, ...: sets the
 * asymptotes L, U from x^k = d_rho and the two previous iterates (distance
 * 0.5 for k < 2; else 0.7x where a coordinate oscillates, 1.2x where it moves
 * monotonically, within [0.01, 10]), shifts the iterate history, and writes
 * d_sums[0] = sum |g|, d_sums[1] = the squared 2-norm of the first-order
 * optimality residual (g without the entries where a bound is active and g
 * points out of the box).
 *
 * fdtd_mma_solve, once per inner iteration: with df = -scale*g and the
 * GCMMA term raa0 > 0, writes into d_rho_new the closed-form minimiser of
 * the separable approximation p/(U-y) + q/(y-L) over
 * max(0, L+0.1(x-L), x-move) <= y <= min(1, U-0.1(U-x), x+move)
 * (0 < move <= 1); entries with g = 0 (gap nodes) keep x.  d_sums[0] =
 * f~(y) - f(x) of the approximation and d_sums[1] = sum (U-L)(y-x)^2 /
 * ((U-y)(y-L)), both for y as stored, for the caller's conservativeness test
 * f(x) + d_sums[0] >= f(y) and its raa0 update.
 *
 * Both are asynchronous on the context's stream; FDTD_EINVAL for a null
 * pointer, n != M_d, k < 0, or scale, raa0, move out of range. */
fdtd_status fdtd_mma_asymptotes(fdtd_ctx *ctx, const void *d_rho, const double *d_grad, double *d_state, size_t n,
                                int k, double *d_sums);
fdtd_status fdtd_mma_solve(fdtd_ctx *ctx, const double *d_state, const double *d_grad, size_t n, double scale,
                           double raa0, double move, void *d_rho_new, double *d_sums);

/* Design constraints of the paper's studies (Sec. 3.2, 3.4).
 *
 * fdtd_mirror_average: d_vec (device, n = M_d entries, elem_bytes 4 = float
 * or 8 = double, in the design layout of the context) becomes symmetric
 * under the mirror across the mid-plane of the design box normal to `axis`
 * (0 x, 1 y, 2 z; < ndim): each entry and its image both take their mean.
 * Applied to rho it makes a symmetric design; applied to a gradient it gives
 * the ascent direction of the symmetric design.  In the in-plane 2D mode
 * E_x edges map to E_x edges and E_y edges to E_y edges.
 *
 * fdtd_fix_design: where d_mask[k] != 0 (device bytes, n = M_d), sets
 * d_rho[k] = value (field precision; may be null) and d_grad[k] = 0 (FP64;
 * may be null): fixed material such as the silver blocks beside the gap.
 *
 * Both asynchronous; FDTD_EINVAL for bad sizes, pointers, axis or value. */
fdtd_status fdtd_mirror_average(fdtd_ctx *ctx, void *d_vec, size_t n, int elem_bytes, int axis);
fdtd_status fdtd_fix_design(fdtd_ctx *ctx, void *d_rho, double *d_grad, const unsigned char *d_mask, size_t n,
                            double value);

/* Grayness zeta = 4 rho~^T (1 - rho~) / M of the filtered design of the last
 * fdtd_set_design, gap nodes excluded (Sec. 3.2): 0 for a black-and-white
 * design, 1 for rho~ = 0.5 everywhere.  Written to d_zeta (device, one
 * double), asynchronously. */
fdtd_status fdtd_grayness(fdtd_ctx *ctx, double *d_zeta);

/* d_rho <- (d_rho >= level) ? 1 : 0 (the paper's final step, level 0.5). */
fdtd_status fdtd_threshold(fdtd_ctx *ctx, void *d_rho, size_t n, double level);

/* CUDA graphs for the time-step loops.  mode 0: every kernel is launched
 * from the host; 1: each whole forward / adjoint pass is captured into a
 * CUDA graph on its first call and replayed afterwards (the graph stays valid
 * across fdtd_set_design and fdtd_set_damping: every pointer is fixed and the
 * material coefficients live in a per-context constant-memory slot);
 * 2 (default): graphs for grids of at most 2^20 nodes, where launch latency
 * rather than bandwidth bounds a step.  Results are identical in every
 * mode.  A context holds at most one graph per pass kind. */
fdtd_status fdtd_set_graphs(fdtd_ctx *ctx, int mode);

/* L2 residency of the time-stepping state (2D E_z-out-of-plane contexts; a
 * no-op for the others).  fraction in (0, 1]: sets aside fraction x (the
 * bytes of one ping-pong pair of states) of L2 for persisting accesses
 * (cudaLimitPersistingL2CacheSize, bounded by the device maximum; a limit of
 * this process that applies to every context on the device, so the last
 * call wins) and marks the forward pair, through an access-policy window on
 * each launch of the forward run (the paired recompute + adjoint launches
 * run without one), persisting in that share and streaming elsewhere, so
 * that part of the state stays in L2 from one step to the next.  0 turns
 * the windows off, gives the set-aside back and demotes the lines marked
 * persisting; fdtd_destroy does the same for a context that has it on.
 * Results are unchanged.  FDTD_EINVAL outside [0, 1].  Default: off. */
fdtd_status fdtd_set_l2_residency(fdtd_ctx *ctx, double fraction);

/* Wait for the context's stream and report (then clear) device-side errors:
 * FDTD_ERANGE, FDTD_EUNSTABLE (a non-finite objective, or the stability
 * guard's flag), or FDTD_ECUDA for a failed kernel. */
fdtd_status fdtd_sync(fdtd_ctx *ctx);

/* One whole design evaluation from host memory: copies h_rho (M_d values in
 * the field precision) into the workspace, then set_design, forward,
 * adjoint and gradient, and copies W~ into *h_W and dW~/drho into h_grad
 * (M_d doubles).  Synchronous. */
fdtd_status fdtd_run_host(fdtd_ctx *ctx, const void *h_rho, size_t n, double *h_W, double *h_grad);

fdtd_status fdtd_get_info(const fdtd_ctx *ctx, fdtd_info *info);

const char *fdtd_status_string(fdtd_status s);

/* Release the context (host memory only; the workspace stays the caller's). */
void fdtd_destroy(fdtd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_GB300_H */
