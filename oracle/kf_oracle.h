/*
 * kf_oracle.h -- plain, slow FP64 CPU oracle of the per-track Kalman fit of
 * "A GPU-based Kalman Filter for Track Fitting" (arXiv 2105.01796).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA fitter.  Only
 * the test-suite, the package smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (paper Sect. 2, the Kalman filter step list and the RTS
 * smoother paragraph; Sect. 4.1, covariance transport with local<->global
 * Jacobians and Runge-Kutta-Nystrom propagation):
 *   for each track, states k = 0..n-1 on planar surfaces;
 *   state 0 holds the seed (prior) on its surface;
 *   predict k-1 -> k by RKN propagation in a constant field, covariance
 *   transport F C F^T and multiple-scattering noise Q_k;
 *   update with the 2D measurement (gain-matrix form, Joseph covariance);
 *   chi2_k = r^T S^-1 r of the predicted residual;
 *   then the Rauch-Tung-Striebel smoother back to state 0.
 * Method variants the paper describes (kfo_method): the smoother as a
 * backward Kalman filter combined with the forward one (Sect. 2, Fig. 2);
 * the mean energy loss with straggling noise on q/p (Sect. 1); a
 * position-dependent field given as a grid map (Sect. 4.3).
 *
 * Units: mm, GeV, tesla, ns.  Bound parameters x = (loc0, loc1, phi, theta,
 * q/p, t) (paper Sect. 2, parameter list).  Free parameters
 * f = (X, Y, Z, t, Tx, Ty, Tz, q/p).  |q| = 1.
 * Covariances: dense row-major 6x6 inside; packed lower triangle (21 values,
 * row-major: (0,0) (1,0) (1,1) (2,0) ...) at the interface.
 * Surfaces: center c[3], rotation R[9] row-major whose columns are the local
 * axes u, v and the normal n.  A point is c + loc0*u + loc1*v.
 */
#ifndef KF_ORACLE_H
#define KF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  KFO_OK = 0,
  KFO_NO_INTERSECTION = 1,
  KFO_NON_SPD = 2,
  KFO_NONFINITE = 3,
  KFO_BAD_INPUT = 4
};

/* Constants of the model (readings of the paper, listed in the design notes). */
#define KFO_KAPPA 2.99792458e-4   /* GeV / (T mm): curvature = kappa*B*q/p */
#define KFO_C_LIGHT 299.792458    /* mm / ns */

/* Field map on a regular grid (the general, position-dependent field of
 * Sect. 4.3): grid point (i, j, l) sits at origin + (i, j, l) * spacing and
 * holds b[((l * ny + j) * nx + i) * 3 + c] (tesla).  nx, ny, nz >= 2. */
typedef struct {
  int nx, ny, nz;
  double origin[3];
  double spacing[3];
  const double* b;
} kfo_field_map;

/* Material constants for the energy loss (one material for every surface;
 * a surface's thickness is x/X0 * x0_rho in g/cm^2). */
typedef struct {
  double z_over_a;   /* Z/A, mol/g */
  double i_exc;      /* mean excitation energy, GeV */
  double x0_rho;     /* radiation length, g/cm^2 */
  double sh_cbar, sh_x0, sh_x1, sh_a, sh_k, sh_delta0; /* density effect */
} kfo_material;

enum { KFO_SMOOTHER_RTS = 0, KFO_SMOOTHER_BACKWARD_FILTER = 1 };

/* Method variants (Sect. 2: smoother by a backward filter; Sect. 1: energy
 * loss in the material; Sect. 4.3: inhomogeneous field). */
typedef struct {
  int smoother;        /* KFO_SMOOTHER_* */
  double bf_scale;     /* backward filter start: bf_scale * Cf of the last state */
  int energy_loss;     /* 1: mean loss and straggling noise on q/p */
  kfo_material mat;
  const kfo_field_map* map; /* NULL: the constant field */
} kfo_method;

/* Field at r: B when map is NULL, else trilinear interpolation of the map
 * (positions outside the grid are clamped onto it). */
void kfo_field_at(const double B[3], const kfo_field_map* map,
                  const double r[3], double out[3]);

/* Density-effect correction, mean stopping power (GeV cm^2/g, unit charge),
 * Landau scale xi (GeV) for a thickness in g/cm^2. */
double kfo_density_effect(double bg, const kfo_material* m);
double kfo_bethe(double bg, double mass, const kfo_material* m);
double kfo_landau_xi(double beta, double thick, const kfo_material* m);

/* Mean energy loss through a surface (dir = +1) or its restoration
 * (dir = -1): updates *qop, returns the q/p Jacobian factor and the
 * downstream straggling variance of q/p.  KFO_NONFINITE if the particle
 * stops. */
int kfo_energy_loss(double* qop, double mass, double xx0, double cosinc,
                    const kfo_material* m, int dir, double* jac,
                    double* var_down);

/* Bound -> free on surface (c, R): f[8] and J_bf (8x6, row-major). */
void kfo_bound_to_free(const double c[3], const double R[9], const double x[6],
                       double f[8], double J[48]);

/* One RKN4 step of fixed length h in the constant field B; D (8x8) is
 * replaced by D_step * D. */
void kfo_rkn_step(double f[8], double h, const double B[3], double mass,
                  double D[64]);

/* The same step with the field of a map taken at the stage points (the
 * step Jacobian holds the stage fields fixed). */
void kfo_rkn_step_field(double f[8], double h, const double B[3],
                        const kfo_field_map* map, double mass, double D[64]);

/* Propagate free state f to the plane (c, R): ceil(|s0|/h_max) equal RKN
 * steps over the straight-line distance s0, then n_iter Newton corrections.
 * D (8x8) receives the product of the step Jacobians; *path the total length.
 * Returns a KFO_* status. */
int kfo_propagate(double f[8], const double c[3], const double R[9],
                  const double B[3], double mass, double h_max, int n_iter,
                  double D[64], double* path);

int kfo_propagate_field(double f[8], const double c[3], const double R[9],
                        const double B[3], const kfo_field_map* map,
                        double mass, double h_max, int n_iter, double D[64],
                        double* path);

/* Bound-to-bound transport of x on surface a to surface b: x_out and the
 * 6x6 Jacobian F = J_fb * P * D * J_bf.  Returns a KFO_* status. */
int kfo_transport(const double ca[3], const double Ra[9], const double x[6],
                  const double cb[3], const double Rb[9], const double B[3],
                  double mass, double h_max, int n_iter, double x_out[6],
                  double F[36], double* path);

int kfo_transport_field(const double ca[3], const double Ra[9],
                        const double x[6], const double cb[3],
                        const double Rb[9], const double B[3],
                        const kfo_field_map* map, double mass, double h_max,
                        int n_iter, double x_out[6], double F[36],
                        double* path);

/* Highland width theta0 for x/X0 = xx0 crossed at |cos(incidence)| = cosinc. */
double kfo_highland(double qop, double mass, double xx0, double cosinc);

/* Gain-matrix update with the Joseph covariance form.  V is 2x2 row-major.
 * Returns KFO_NON_SPD if det(S) <= 0. */
int kfo_update(const double xp[6], const double Cp[36], const double m[2],
               const double V[4], double xf[6], double Cf[36], double* chi2);

/* One RTS step: smoothed (xs1, Cs1) at k+1, predicted (xp1, Cp1) at k+1,
 * filtered (xf, Cf) at k and F (k -> k+1) give (xs, Cs) at k. */
int kfo_rts_step(const double xf[6], const double Cf[36], const double xp1[6],
                 const double Cp1[36], const double F1[36],
                 const double xs1[6], const double Cs1[36], double xs[6],
                 double Cs[36]);

/* Linear-Gaussian filter + smoother over n states with given transition
 * matrices F[k] (k>=1, 6x6), noise Q[k] (6x6), measurements m[k] (2),
 * V[k] (2x2) and holes.  Same update and smoother as the track fit.
 * Outputs xs[n][6], Cs[n][36], chi2[n]. */
int kfo_linear_fit(int n, const double x0[6], const double C0[36],
                   const double* F, const double* Q, const double* m,
                   const double* V, const uint8_t* hole, double* xs,
                   double* Cs, double* chi2);

/* kfo_linear_fit with the smoother chosen (KFO_SMOOTHER_*). */
int kfo_linear_fit_ex(int n, const double x0[6], const double C0[36],
                      const double* F, const double* Q, const double* m,
                      const double* V, const uint8_t* hole, int smoother,
                      double bf_scale, double* xs, double* Cs, double* chi2);

/* Full fit of one track with every intermediate: arrays of n states.
 * xp/xf/xs [n][6], Cp/Cf/Cs [n][36], F [n][36] (F[0] = identity),
 * chi2 [n].  Returns a KFO_* status. */
int kfo_fit_track(int n, const int32_t* surface_id, const double* loc,
                  const double* cov, const uint8_t* is_hole,
                  const double seed[6], const double seed_cov[36],
                  int n_surfaces, const double* center, const double* rot,
                  const double* x_over_x0, const double B[3], double mass,
                  double h_max, int n_iter, double* xp, double* Cp,
                  double* xf, double* Cf, double* xs, double* Cs, double* F,
                  double* chi2);

/* kfo_fit_track with method variants (meth NULL: the baseline method). */
int kfo_fit_track_ex(int n, const int32_t* surface_id, const double* loc,
                     const double* cov, const uint8_t* is_hole,
                     const double seed[6], const double seed_cov[36],
                     int n_surfaces, const double* center, const double* rot,
                     const double* x_over_x0, const double B[3], double mass,
                     double h_max, int n_iter, const kfo_method* meth,
                     double* xp, double* Cp, double* xf, double* Cf,
                     double* xs, double* Cs, double* F, double* chi2);

/* Batched fit:
 *   offsets[T+1]; seed_params[6][T]; seed_cov[21][T] (packed);
 *   center[S][3]; rot[S][9] (one row-major R per surface); x_over_x0[S];
 *   surface_id[M]; loc[2][M]; cov[3][M] (V00, V01, V11); is_hole[M];
 * outputs out_params[6][T], out_cov[21][T], out_chi2[T], out_ndf[T],
 * out_status[T], out_states[6][M] (nullable: smoothed parameters).
 * Tracks [t_begin, t_end) are fitted, split over n_threads POSIX threads. */
int kfo_fit_batch(int n_tracks, const int32_t* offsets,
                  const double* seed_params, const double* seed_cov,
                  int n_surfaces, const double* center, const double* rot,
                  const double* x_over_x0, int64_t n_states,
                  const int32_t* surface_id, const double* loc,
                  const double* cov, const uint8_t* is_hole, const double B[3],
                  double mass, double h_max, int n_iter, double* out_params,
                  double* out_cov, double* out_chi2, int32_t* out_ndf,
                  uint8_t* out_status, double* out_states, int t_begin,
                  int t_end, int n_threads);

/* kfo_fit_batch with method variants (meth NULL: the baseline method). */
int kfo_fit_batch_ex(int n_tracks, const int32_t* offsets,
                     const double* seed_params, const double* seed_cov,
                     int n_surfaces, const double* center, const double* rot,
                     const double* x_over_x0, int64_t n_states,
                     const int32_t* surface_id, const double* loc,
                     const double* cov, const uint8_t* is_hole,
                     const double B[3], double mass, double h_max, int n_iter,
                     const kfo_method* meth, double* out_params,
                     double* out_cov, double* out_chi2, int32_t* out_ndf,
                     uint8_t* out_status, double* out_states, int t_begin,
                     int t_end, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
