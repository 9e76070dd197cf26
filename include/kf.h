/*
 * kf.h -- C ABI of the GB300 (sm_103a) Kalman-filter track fitter.
 *
 * Method: "A GPU-based Kalman Filter for Track Fitting" (arXiv 2105.01796).
 *   Sect. 2, Kalman filter step list: predict the state to the next measurement
 *     surface, then combine it with the measurement (gain-matrix formalism);
 *     repeat to the end of the trajectory.
 *   Sect. 2, smoother paragraph: Rauch-Tung-Striebel smoother using the
 *     Jacobians stored during the forward filter.
 *   Sect. 2, parameter list: bound parameters (loc0, loc1, phi, theta, q/p, t).
 *   Sect. 4.1: adaptive Runge-Kutta-Nystrom transport of the parameters; the
 *     covariance is transported with the transport Jacobian and the
 *     local<->global Jacobians at both surfaces.
 *   Sect. 4.2: the smoother's matrix inverse is done in double precision.
 *   Sect. 4.3: surfaces with geometry and material; a constant 3-vector field;
 *     four sets of per-track data (measurements, starting parameters, fitting
 *     configuration, fitted results with a status); boundless surfaces.
 *
 * Units: mm, GeV, tesla, ns.  |q| = 1.
 *
 * Memory: every array pointer passed to kf_fit / kf_fit_ex is a DEVICE pointer
 * on the current CUDA device, owned by the caller; kf_fit_host takes HOST
 * pointers.  The library never frees caller memory.  A kf_handle owns its
 * workspace (the per-state record the smoother reads back) and staging
 * buffers.
 *
 * Layouts (structure of arrays; T tracks, S surfaces, M states in total):
 *   offsets[T+1]         int32, states of track t are [offsets[t], offsets[t+1]);
 *                        state 0 of a track is the surface its seed lives on.
 *   seed_params[6][T]    double, bound parameters of the seed on state 0.
 *   seed_cov[21][T]      double, seed covariance, packed lower triangle in
 *                        row-major order: (0,0) (1,0) (1,1) (2,0) (2,1) ...
 *   center[3][S]         double, plane centre.
 *   rot[9][S]            double, row-major 3x3 R whose columns are the local
 *                        axes u, v and the normal n; point = c + loc0 u + loc1 v.
 *   x_over_x0[S]         double, material thickness in radiation lengths.
 *   surface_id[M]        int32 in [0, S).
 *   loc[2][M]            double, measured (loc0, loc1).
 *   cov[3][M]            double, measurement covariance (V00, V01, V11).
 *   is_hole[M]           uint8, 1 = surface crossed without a measurement.
 *   out_params[6][T]     double, smoothed parameters on state 0.
 *   out_cov[21][T]       double, smoothed covariance on state 0 (packed).
 *   out_chi2[T]          double, sum over measured states of r^T S^-1 r of
 *                        the predicted residual.
 *   out_ndf[T]           int32, 2 x number of measured states.
 *   out_status[T]        uint8, kf_track_status.
 *   out_states[6][M]     double, smoothed parameters on every state (optional).
 *
 * Errors: functions return 0 or a negative kf_error.  A per-track failure
 * does not fail the call: it sets out_status[t] and writes NaN parameters,
 * covariance and chi2 (ndf 0) for that track.  No device assert or trap is
 * ever used.  Calls on a handle are asynchronous on the given stream and a
 * handle must not be used from two host threads at once.
 */
#ifndef KF_H
#define KF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KF_ABI_VERSION 4

typedef enum {
  KF_SUCCESS = 0,
  KF_EINVAL = -1,       /* null pointer, bad size or inconsistent arguments */
  KF_ECUDA = -2,        /* a CUDA call failed; kf_last_cuda_error() has it */
  KF_ENOMEM = -3,       /* device or pinned allocation failed */
  KF_EUNSUPPORTED = -4, /* option outside what this build supports */
  KF_EDEVICE = -5,      /* a kernel's bounded wait timed out (synchronous
                           entry points; the tracks it held have status
                           KF_TRACK_TIMEOUT) */
  KF_ESIZE = -6         /* kf_fit_static: the batch does not fit its fixed
                           device block */
} kf_error;

typedef enum {
  KF_TRACK_OK = 0,
  KF_TRACK_NO_INTERSECTION = 1, /* track (nearly) parallel to a plane */
  KF_TRACK_NON_SPD = 2,         /* non-positive innovation or Cholesky pivot */
  KF_TRACK_NONFINITE = 3,       /* NaN/Inf in the result */
  KF_TRACK_BAD_INPUT = 4,       /* empty track, too many states, bad surface id */
  KF_TRACK_TIMEOUT = 5          /* not fitted: a bounded device wait of the
                                   call (the surface table's copy into shared
                                   memory) gave up */
} kf_track_status;

typedef enum {
  KF_PRECISION_FP64 = 0, /* every step in double precision */
  KF_PRECISION_MIXED = 1 /* propagation, Jacobians, covariance transport and
                            gain in float; Joseph covariance update (its
                            second-order term K W, O(eps_float |Cp|), in
                            float), chi2 and the smoother's inverse in
                            double (the two columns of the inverse the
                            smoother needs, by a 4x4 LDL^T of the non-angle
                            block and the 2x2 Schur complement of the angle
                            block); the track state between surfaces as
                            double-float pairs (about 48 bits) */
} kf_precision;

typedef struct {
  int32_t n_tracks;
  int32_t max_states;          /* upper bound on offsets[t+1]-offsets[t] */
  const int32_t* offsets;      /* [n_tracks + 1] */
  const double* seed_params;   /* [6][n_tracks] */
  const double* seed_cov;      /* [21][n_tracks] */
} kf_tracks;

typedef struct {
  int32_t n_surfaces;
  const double* center;        /* [3][n_surfaces] */
  const double* rot;           /* [9][n_surfaces] */
  const double* x_over_x0;     /* [n_surfaces] */
} kf_surfaces;

typedef struct {
  int64_t n_states;
  const int32_t* surface_id;   /* [n_states] */
  const double* loc;           /* [2][n_states] */
  const double* cov;           /* [3][n_states] */
  const uint8_t* is_hole;      /* [n_states] */
} kf_measurements;

/* Position-dependent field on a regular grid (paper Sect. 4.3 names
 * inhomogeneous fields as the general case; its studies use a constant one).
 * Grid point (i, j, l) sits at origin + (i, j, l) * spacing and holds
 * b[((l * ny + j) * nx + i) * 3 + c], c = x, y, z, in tesla.  The field at a
 * point is the trilinear interpolation of the 8 surrounding grid points;
 * points outside the grid are clamped onto its boundary.  The RKN step takes
 * the field at its stage points; its Jacobian holds those fields fixed (the
 * field-gradient term is left out). */
typedef struct {
  int32_t nx, ny, nz;          /* grid points per axis, each >= 2 */
  int32_t reserved;            /* 0 */
  double origin[3];            /* mm */
  double spacing[3];           /* mm, each > 0 */
  const double* b;             /* [nz][ny][nx][3]: device pointer (host
                                  pointer for kf_fit_host) */
} kf_field_map;

typedef struct {
  double b[3];                 /* constant field (Bx, By, Bz) in tesla */
  const kf_field_map* map;     /* NULL: the constant field b; else the map
                                  (b is then ignored).  A map needs
                                  KF_PRECISION_FP64. */
} kf_field;

/* Material of the surfaces for the energy loss (one material for all; a
 * surface's thickness is x/X0 * x0_rho in g/cm^2).  kf_default_options
 * fills silicon: the PDG's Z/A, mean excitation energy, radiation length
 * and Sternheimer density-effect parameters. */
typedef struct {
  double z_over_a;             /* mol/g */
  double i_exc;                /* mean excitation energy, GeV */
  double x0_rho;               /* radiation length, g/cm^2 */
  double sh_cbar, sh_x0, sh_x1, sh_a, sh_k, sh_delta0;
} kf_material;

typedef enum {
  KF_SMOOTHER_RTS = 0,             /* Rauch-Tung-Striebel with the stored
                                      Jacobians (Sect. 2) */
  KF_SMOOTHER_BACKWARD_FILTER = 1  /* a second Kalman filter run from the
                                      last state to the first with its own
                                      propagation, combined with the forward
                                      filter by the weighted mean (Sect. 2,
                                      Fig. 2) */
} kf_smoother;

typedef struct {
  double* params;              /* [6][n_tracks], required */
  double* cov;                 /* [21][n_tracks], required */
  double* chi2;                /* [n_tracks], required */
  int32_t* ndf;                /* [n_tracks], optional (NULL) */
  uint8_t* status;             /* [n_tracks], optional (NULL) */
  double* states;              /* [6][n_states], optional (NULL) */
} kf_outputs;

typedef struct {
  int32_t precision;           /* kf_precision */
  double mass;                 /* particle mass in GeV (default: muon) */
  double h_max;                /* longest RKN step in mm (default 50) */
  int32_t n_iter;              /* Newton corrections onto each plane (default
                                  3; 0-16).  With 0 the path length is the
                                  straight-line estimate, which the mixed
                                  path takes in FP32 (~1e-4 sigma from FP64);
                                  every end point is projected onto its plane */
  int32_t block;               /* threads per CTA, a multiple of 32 (0 = 128):
                                  up to 256, or 384 / 512 for the mixed
                                  path's min_blocks 3 / 4 variants */
  int64_t workspace_bytes;     /* cap on the handle's workspace (0 = 32 GiB);
                                  larger batches are fitted in chunks */
  int32_t schedule;            /* kf_schedule (default KF_SCHEDULE_PERSISTENT) */
  int32_t min_blocks;          /* register-cap variant: minimum resident CTAs
                                  per SM the kernel is compiled for (0 = the
                                  default variant; 3 and 4 cap registers) */
  int32_t use_graph;           /* 1: kf_fit_ex captures its launches into a
                                  CUDA graph held by the handle and replays it
                                  while every argument is unchanged (needs a
                                  non-NULL stream) */
  int32_t smoother;            /* kf_smoother (default RTS) */
  int32_t energy_loss;         /* 1: mean energy loss (Bethe, with the
                                  density effect) applied to q/p at every
                                  surface with material, with its Jacobian
                                  factor and a straggling variance on q/p
                                  (Gaussian of the Landau FWHM 4 xi) */
  double bf_scale;             /* backward filter: starting covariance is
                                  bf_scale times the last filtered one
                                  (default 1e4) */
  kf_material material;        /* for energy_loss (default silicon) */
  int32_t resident_warps;      /* persistent schedules: warps kept resident on
                                  each SM (0 = as many as fit).  With
                                  one-warp CTAs (block 32), U 32-track
                                  units and W resident warps the launch
                                  takes ceil(U / W) rounds; fewer warps
                                  that still fill the FP64 pipe can remove
                                  a part-filled last round */
  int32_t wait_limit;          /* polls of the kernels' bounded waits before
                                  they give up (0 = 2^20, about a second) */
  int32_t team_warps;          /* FP64 path: warps that share each track's
                                  work (0 or 1 = one thread per track; 2 or 4
                                  = a team: lane l of each of a CTA's warps
                                  works on track l of its 32, splitting the
                                  Jacobian columns and the matrix rows, for
                                  batches too small to fill the GPU; grid
                                  schedule, block ignored) */
  int32_t test_wait_timeout;   /* diagnostic of the timeout path (0 = off):
                                  1 announces the surface table's copy on
                                  each CTA's barrier without issuing it, so
                                  every bounded wait runs out with nothing
                                  left in flight and every track of the call
                                  gets KF_TRACK_TIMEOUT.  No fault, no hang */
} kf_options;

typedef enum {
  KF_SCHEDULE_AUTO = -1,       /* kf_fit_ex asks kf_autotune (cached per
                                  batch shape in the handle) */
  KF_SCHEDULE_GRID = 0,        /* one thread per track, one CTA per block of
                                  tracks */
  KF_SCHEDULE_PERSISTENT = 1,  /* resident CTAs; each CTA takes units of
                                  `block` tracks from a work counter until
                                  done */
  KF_SCHEDULE_SORTED = 2,      /* persistent, tracks taken longest first
                                  (counting sort by state count; for uneven
                                  tracks) */
  KF_SCHEDULE_WAVES = 3        /* grid launches: full waves of `block`-thread
                                  CTAs (every SM's resident CTAs), then one
                                  launch that spreads the remaining tracks
                                  over all SMs in smaller CTAs */
} kf_schedule;

typedef struct kf_handle kf_handle;

/* Fill *opt with the defaults: FP64, muon mass, h_max 50 mm, 3 corrections,
 * 128 threads per CTA, persistent schedule, default register variant, RTS
 * smoother, no energy loss, silicon material.
 * Method variants (smoother = KF_SMOOTHER_BACKWARD_FILTER, energy_loss = 1,
 * or a field map) run in a separate FP64 kernel: they need
 * KF_PRECISION_FP64 (KF_EUNSUPPORTED otherwise) and are not available in
 * kf_fit_static and kf_chi2_grad. */
void kf_default_options(kf_options* opt);

/* Create a handle bound to the current CUDA device.  Returns 0 or kf_error. */
int kf_create(kf_handle** handle);

/* Release the handle's workspace.  Safe on NULL. */
void kf_destroy(kf_handle* handle);

/* Fit with default options on the legacy default stream, using a library-
 * owned handle for the current device (created on first use).  Device
 * pointers.  Waits for completion before returning. */
int kf_fit(const kf_tracks* tracks, const kf_surfaces* surfaces,
           const kf_measurements* meas, const kf_field* field,
           double* out_params, double* out_cov, double* out_chi2);

/* Fit with explicit options on `stream` (a cudaStream_t, NULL = legacy
 * default stream).  Device pointers.  Asynchronous: the call returns after
 * the launches are queued.  opt may be NULL (defaults).  Each call clears the
 * handle's device error flag first; a bounded device wait that gives up
 * marks the tracks it held KF_TRACK_TIMEOUT (out_status), and so does every
 * CTA that starts after it in the same call. */
int kf_fit_ex(kf_handle* handle, const kf_tracks* tracks,
              const kf_surfaces* surfaces, const kf_measurements* meas,
              const kf_field* field, const kf_options* opt,
              const kf_outputs* out, void* stream);

/* Same as kf_fit_ex but every pointer in tracks, surfaces, meas and out is a
 * HOST pointer: the handle copies the inputs to its device buffers, fits, and
 * copies the outputs back before returning (synchronous).  Batches of at
 * least 20 000 tracks run as 2-8 chunks whose copies overlap the other
 * chunks' fits (each chunk's fit on a stream of the handle); pinned host
 * memory makes the copies asynchronous.  Results equal kf_fit_ex's.
 * Returns KF_EDEVICE when a bounded device wait of this call gave up. */
int kf_fit_host(kf_handle* handle, const kf_tracks* tracks,
                const kf_surfaces* surfaces, const kf_measurements* meas,
                const kf_field* field, const kf_options* opt,
                const kf_outputs* out, void* stream);

/* kf_fit_ex without any device allocation, for callers that cannot allocate:
 * real-time loops (a trigger farm's event loop) that must never block on the
 * CUDA allocator, and hosts that give each library a fixed memory budget up
 * front and own every other byte of device memory.  (The paper has no
 * counterpart; it is an addition of this library.)
 * Scratch space is one fixed 64 MiB block of device memory per GPU, reserved
 * for the whole life of the process once the library is loaded.  It holds
 * the packed surface table (up to 1024 surfaces) and the per-state records;
 * larger batches run as several launches on `stream`.  Returns KF_ESIZE when
 * n_surfaces > 1024 or when one track's records (max_states x 720 B in FP64,
 * max_states x 264 B in mixed precision) do not fit the block, and
 * KF_EUNSUPPORTED for schedules other than GRID and PERSISTENT and for the
 * method variants.  Device pointers, asynchronous on `stream`, same outputs
 * as kf_fit_ex.
 * The first call on a device looks up the block's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The call returns before its GPU work runs, so a bounded device wait that
 * gives up (not expected in normal operation) shows in the outputs: the
 * tracks of that launch get status KF_TRACK_TIMEOUT and NaN results.
 * Every call reuses the same block, which keeps
 * the previous call's contents: calls whose GPU work overlaps (other streams
 * or host threads) race on it and must be serialised by the caller. */
int kf_fit_static(const kf_tracks* tracks, const kf_surfaces* surfaces,
                  const kf_measurements* meas, const kf_field* field,
                  const kf_options* opt, const kf_outputs* out, void* stream);

/* Autotuner: time every launch shape (schedule x (threads per CTA, register
 * variant) pairs from 32 to 512 threads, plus CTA sizes that split this
 * batch's 32-track warp units into 1-4 nearly full waves of one CTA per SM)
 * on this batch, on `stream`, and return the fastest in *best (other fields
 * copied from *base; base may be NULL for the defaults) and its median time
 * in *best_ms (optional).  Results are cached in the handle per (precision,
 * n_tracks, max_states, n_surfaces, field along z, method variant); a cached
 * shape returns at once.  Runs the fit about 60-240 times, overwriting *out,
 * and synchronises the stream; inside a stream capture it returns the
 * defaults without timing.  The paper scans grid, block and register counts
 * by hand (Sect. 5.3.5); this automates that scan. */
int kf_autotune(kf_handle* handle, const kf_tracks* tracks,
                const kf_surfaces* surfaces, const kf_measurements* meas,
                const kf_field* field, const kf_options* base,
                const kf_outputs* out, void* stream, kf_options* best,
                double* best_ms);

/* Gradient of the summed chi2 (the adjoint of the filter; kf_grad with
 * v = W = 0).
 * L = sum_t w_t chi2_t with w_t = dl_dchi2[t] (NULL: all 1); chi2_t as
 * returned by kf_fit (predicted-residual chi2, which the smoother does not
 * change).  Computed in FP64 whatever opt->precision says.
 *   align[6][S]       alignment of every surface (NULL: all zero): shifts
 *                     (du, dv, dn) along the surface's local axes, then
 *                     rotations (alpha, beta, gamma) about them:
 *                     c' = c + R (du, dv, dn), R' = R Ru(alpha) Rv(beta) Rn(gamma).
 *   out_chi2[T]       chi2 per track at this alignment (optional).
 *   grad_seed[6][T]   dL/d seed_params (optional).
 *   grad_align[6][S]  dL/d align (optional); overwritten.
 * Method: reverse mode throughout: a reverse sweep over the states with the
 * filtered states recomputed from checkpoints every 5 states, and inside it
 * every transport recomputed with its RKN stage inputs taped and swept
 * backwards.  Launch shape: opt->team_warps as for kf_grad; one thread per
 * track with opt->block threads per CTA (a multiple of 32 up to 256; 0, and
 * opt == NULL, choose CTAs of the warp count that covers the batch in nearly
 * full waves of one CTA per SM); the other launch options do not apply.  Device pointers; asynchronous on `stream`.  Tracks that fail
 * get NaN chi2 and gradients and do not contribute to grad_align. */
int kf_chi2_grad(kf_handle* handle, const kf_tracks* tracks,
                 const kf_surfaces* surfaces, const double* align,
                 const kf_measurements* meas, const kf_field* field,
                 const kf_options* opt, const double* dl_dchi2,
                 double* out_chi2, double* grad_seed, double* grad_align,
                 void* stream);

/* Weights of the adjoint's objective (kf_grad):
 *   L = sum_t [ w_t chi2_t + sum_i v_ti x_s0,ti + sum_e W_te C_s0,te ],
 * x_s0 = out_params and C_s0 = out_cov (packed, 21) of the fit: the
 * smoothed parameters and covariance of state 0.  With torch.autograd these
 * are the incoming gradients of the three outputs. */
typedef struct {
  const double* dl_dchi2;      /* w [T]; NULL: all 1 */
  const double* dl_dparams;    /* v [6][T]; NULL: all 0 */
  const double* dl_dcov;       /* W [21][T] over the packed elements; NULL: all 0 */
} kf_grad_weights;

typedef struct {
  double* chi2;                /* [T] chi2 per track (optional) */
  double* params;              /* [6][T] x_s0 at this alignment (optional) */
  double* cov;                 /* [21][T] C_s0 at this alignment (optional) */
  double* grad_seed;           /* [6][T] dL/d seed_params (optional) */
  double* grad_align;          /* [6][S] dL/d align (optional; overwritten) */
} kf_grad_outputs;

/* The adjoint of the whole fit, filter and smoother (paper Sect. 2: the
 * filter step list and the smoother paragraph): the value and gradient of
 * L above with respect to the seed parameters and the per-surface alignment,
 * in FP64 whatever opt->precision says.  align as for kf_chi2_grad.
 * Method: reverse mode throughout, one thread per track.
 *   1. forward filter, (x_f, C_f) checkpointed every 5 states;
 *   2. RTS smoother (when params, cov or the v / W terms are asked), from
 *      the last state down, each 5-state segment's filtered states and
 *      transports recomputed from its checkpoint; smoothed checkpoints at
 *      the segment starts;
 *   3. reverse of the smoother (when v or W is given), segment by segment
 *      upwards, each segment's filtered and smoothed states recomputed from
 *      the two kinds of checkpoint; each step's contributions to the
 *      adjoints of x_f, C_f, x_p, C_p and F (79 doubles per state) are kept
 *      in the handle's scratch for
 *   4. the reverse of the filter (as kf_chi2_grad) with those contributions
 *      added at every state.
 * No filtered or smoothed state is stored beyond the checkpoints.  Scratch
 * per track: 216 B per 5 states (filter checkpoints), plus with v or W 216 B
 * per 5 states (smoothed checkpoints) and 632 B per state; a batch whose
 * scratch exceeds opt->workspace_bytes (0: 32 GiB) runs as several launches.
 * Launch shape: opt->team_warps 1 = one thread per track (CTAs as for
 * kf_chi2_grad); 2 = the pipelined form, for batches too small to fill the
 * GPU: two warps per 32 tracks, one running the forward half of the filter's
 * reverse sweep (the segments' recompute and the taped transports) one
 * transition ahead of the other, which runs the reverse half, and in the
 * smoother's passes recomputing each segment one segment ahead of the RTS
 * steps and their reverse, which the other runs (results equal
 * the one-thread form's, up to the summation order of the alignment
 * gradient); 0 (the default, and opt == NULL) = the pipelined form while
 * 2 x ceil(T / 32) warps fit in one warp per SM sub-partition (T <= 9728 on
 * 152 SMs), else one thread per track; others: KF_EUNSUPPORTED.
 * Failure behaviour as for kf_chi2_grad; a track whose smoother meets a
 * non-positive pivot gets NaN outputs and gradients.
 * Device pointers; asynchronous on `stream`. */
int kf_grad(kf_handle* handle, const kf_tracks* tracks, const kf_surfaces* surfaces, const double* align,
            const kf_measurements* meas, const kf_field* field, const kf_options* opt,
            const kf_grad_weights* weights, const kf_grad_outputs* out, void* stream);

/* Bytes of device workspace kf_fit_ex would use for this batch shape. */
int64_t kf_workspace_size(int32_t n_tracks, int32_t max_states,
                          const kf_options* opt);

/* Number of kernel launches the last kf_fit_ex / kf_fit_host on this handle
 * queued (for launch accounting). */
int32_t kf_last_launch_count(const kf_handle* handle);

/* Human-readable text of a kf_error. */
const char* kf_strerror(int code);

/* Text of the last CUDA error seen by the library on this host thread. */
const char* kf_last_cuda_error(void);

/* Diagnostic: run the device self-check of the library's numeric helpers
 * (float<->double conversions on the integer pipe, and the Newton-refined
 * double 1/sqrt and 1/x) over n_patterns inputs on the current device.
 * counts[6] (host memory) receives the mismatch counts: [0] float->double,
 * [1] double->float (round to nearest even), [2] 1/sqrt one step beyond 1e-13
 * relative, [3] 1/x one step beyond 1e-13, [4] two-step forms beyond 4 ulp,
 * [5] the full-range forms of the FP64 path (any normal double) beyond
 * 4 ulp.  All zero means the helpers behave as documented.  Synchronous. */
int kf_selftest(int64_t n_patterns, uint64_t* counts);

/* Diagnostic: device self-check of the mixed path's double-float arithmetic
 * (values carried as a pair of floats hi + lo) against FP64 arithmetic on the
 * same inputs, over n_patterns random patterns (a quarter of them with sums
 * that cancel).  counts[5] (host memory) receives the number of results off
 * by more than 2^-44 of the magnitude of their terms: [0] pair + pair,
 * [1] pair + float, [2] pair * pair, [3] the compensated dot product
 * w . r - w0 with a pair-valued r; and [4] the number of patterns whose sum
 * of the high floats alone already misses that bound (most of them: the
 * bound is out of plain float arithmetic's reach).  [0..3] all zero means
 * the arithmetic behaves as documented.  Synchronous. */
int kf_selftest_df(int64_t n_patterns, uint64_t* counts);

/* ABI version of the loaded library (KF_ABI_VERSION). */
int kf_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KF_H */
