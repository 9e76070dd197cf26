/*
 * kf_oracle.c -- plain FP64 CPU oracle of the per-track Kalman fit
 * (arXiv 2105.01796).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; never by the CUDA product path.
 *
 * Everything is dense textbook algebra on 6x6 / 8x8 row-major matrices, in the
 * order the method states its steps, so it can be read against the paper:
 *   Sect. 2 (Kalman filter step list): predict to the next surface, then
 *     combine with the measurement in the gain-matrix formalism;
 *   Sect. 2 (smoother paragraph): Rauch-Tung-Striebel smoother with the
 *     Jacobians stored during the forward pass;
 *   Sect. 4.1 (parallelization strategy): Runge-Kutta-Nystrom transport of
 *     the parameters, covariance transport with the transport Jacobian and
 *     the local<->global Jacobians at both surfaces;
 *   Sect. 4.3 (data structure): constant 3-vector magnetic field, surfaces
 *     with material, boundless planes;
 *   Sect. 4.2 (precision): the smoother's inverse is done in double precision.
 * Readings where the paper is silent (frames, RKN step rule, Highland
 * multiple scattering, Joseph form, Cholesky solve) are documented in the
 * design notes of the repository.
 */
#include "kf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small dense matrix helpers                                          */
/* ------------------------------------------------------------------ */

/* C[n x p] = A[n x m] * B[m x p] (C must not alias A or B) */
static void mat_mul(const double* A, const double* B, double* C, int n, int m,
                    int p) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += A[i * m + k] * B[k * p + j];
      C[i * p + j] = s;
    }
}

static void mat_transpose(const double* A, double* AT, int n, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) AT[j * n + i] = A[i * m + j];
}

static void mat_identity(double* A, int n) {
  memset(A, 0, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i) A[i * n + i] = 1.0;
}

/* C = F * A * F^T for 6x6 */
static void sandwich6(const double* F, const double* A, double* C) {
  double FA[36], FT[36];
  mat_mul(F, A, FA, 6, 6, 6);
  mat_transpose(F, FT, 6, 6);
  mat_mul(FA, FT, C, 6, 6, 6);
}

static int all_finite(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(a[i])) return 0;
  return 1;
}

static void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* column j of R (row-major 3x3): j = 0 -> u, 1 -> v, 2 -> n */
static void rot_col(const double R[9], int j, double out[3]) {
  out[0] = R[0 * 3 + j];
  out[1] = R[1 * 3 + j];
  out[2] = R[2 * 3 + j];
}

/* ------------------------------------------------------------------ */
/* local <-> global (Sect. 4.1: "transform Jacobians between local and */
/* global track parameters at the two measurement points")            */
/* ------------------------------------------------------------------ */

/* Free vector order: 0-2 position, 3 time, 4-6 unit direction, 7 q/p.
 * Bound vector order: 0 loc0, 1 loc1, 2 phi, 3 theta, 4 q/p, 5 time. */
void kfo_bound_to_free(const double c[3], const double R[9], const double x[6],
                       double f[8], double J[48]) {
  double u[3], v[3];
  rot_col(R, 0, u);
  rot_col(R, 1, v);
  const double sp = sin(x[2]), cp = cos(x[2]);
  const double st = sin(x[3]), ct = cos(x[3]);
  for (int i = 0; i < 3; ++i) f[i] = c[i] + x[0] * u[i] + x[1] * v[i];
  f[3] = x[5];
  f[4] = cp * st;
  f[5] = sp * st;
  f[6] = ct;
  f[7] = x[4];
  if (J) {
    memset(J, 0, sizeof(double) * 48);
    for (int i = 0; i < 3; ++i) {
      J[i * 6 + 0] = u[i]; /* d pos / d loc0 */
      J[i * 6 + 1] = v[i]; /* d pos / d loc1 */
    }
    J[3 * 6 + 5] = 1.0;       /* d t / d t */
    J[4 * 6 + 2] = -sp * st;  /* d Tx / d phi */
    J[5 * 6 + 2] = cp * st;   /* d Ty / d phi */
    J[6 * 6 + 2] = 0.0;       /* d Tz / d phi */
    J[4 * 6 + 3] = cp * ct;   /* d Tx / d theta */
    J[5 * 6 + 3] = sp * ct;   /* d Ty / d theta */
    J[6 * 6 + 3] = -st;       /* d Tz / d theta */
    J[7 * 6 + 4] = 1.0;       /* d qop / d qop */
  }
}

/* Free -> bound on (c, R) for a free state lying on the plane; J_fb (6x8)
 * uses the tangent-space rows for the angles. */
static void free_to_bound(const double c[3], const double R[9],
                          const double f[8], double x[6], double J[48]) {
  double u[3], v[3], d[3];
  rot_col(R, 0, u);
  rot_col(R, 1, v);
  for (int i = 0; i < 3; ++i) d[i] = f[i] - c[i];
  x[0] = dot3(d, u);
  x[1] = dot3(d, v);
  const double phi = atan2(f[5], f[4]);
  const double theta = atan2(sqrt(f[4] * f[4] + f[5] * f[5]), f[6]);
  x[2] = phi;
  x[3] = theta;
  x[4] = f[7];
  x[5] = f[3];
  if (J) {
    const double sp = sin(phi), cp = cos(phi);
    const double st = sin(theta), ct = cos(theta);
    memset(J, 0, sizeof(double) * 48);
    for (int i = 0; i < 3; ++i) {
      J[0 * 8 + i] = u[i];
      J[1 * 8 + i] = v[i];
    }
    J[2 * 8 + 4] = -sp / st;
    J[2 * 8 + 5] = cp / st;
    J[2 * 8 + 6] = 0.0;
    J[3 * 8 + 4] = cp * ct;
    J[3 * 8 + 5] = sp * ct;
    J[3 * 8 + 6] = -st;
    J[4 * 8 + 7] = 1.0;
    J[5 * 8 + 3] = 1.0;
  }
}

/* ------------------------------------------------------------------ */
/* Runge-Kutta-Nystrom step (Sect. 4.1, Myrheim's Nystrom method)      */
/* ------------------------------------------------------------------ */

/* ------------------------------------------------------------------ */
/* magnetic field (Sect. 4.3: a constant 3-vector in the paper's      */
/* studies; position-dependent fields are named as the general case)  */
/* ------------------------------------------------------------------ */

/* Field at r: the constant B when map is NULL, else trilinear
 * interpolation of the map's grid values.  Grid point (i, j, l) sits at
 * origin + (i dx, j dy, l dz) and holds b[((l ny + j) nx + i) 3 + c].
 * Outside the grid the position is clamped onto its boundary. */
void kfo_field_at(const double B[3], const kfo_field_map* map,
                  const double r[3], double out[3]) {
  if (!map) {
    out[0] = B[0];
    out[1] = B[1];
    out[2] = B[2];
    return;
  }
  const int n[3] = {map->nx, map->ny, map->nz};
  int i0[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    double u = (r[a] - map->origin[a]) / map->spacing[a];
    if (u < 0.0) u = 0.0;
    if (u > n[a] - 1) u = n[a] - 1;
    int i = (int)floor(u);
    if (i > n[a] - 2) i = n[a] - 2;
    i0[a] = i;
    w[a] = u - i;
  }
  for (int c = 0; c < 3; ++c) out[c] = 0.0;
  for (int dl = 0; dl < 2; ++dl)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const double wt = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) *
                          (dl ? w[2] : 1.0 - w[2]);
        const int64_t idx =
            (((int64_t)(i0[2] + dl) * n[1] + (i0[1] + dj)) * n[0] + (i0[0] + di)) * 3;
        for (int c = 0; c < 3; ++c) out[c] += wt * map->b[idx + c];
      }
}

/* ------------------------------------------------------------------ */
/* Runge-Kutta-Nystrom step (Sect. 4.1, Myrheim's Nystrom method)      */
/* ------------------------------------------------------------------ */

/* Equation of motion in path length s:
 *   r'' = qop * kappa * (r' x B(r)),  t' = sqrt(1 + m^2 qop^2) / c.
 * 4-stage Nystrom step with the field taken at the stage points:
 *   k1 = a(r,            T)
 *   k2 = a(r + h/2 T + h^2/8 k1, T + h/2 k1)
 *   k3 = a(r + h/2 T + h^2/8 k1, T + h/2 k2)
 *   k4 = a(r + h T + h^2/2 k3,   T + h k3)
 *   r <- r + h T + h^2/6 (k1 + k2 + k3)
 *   T <- T + h/6 (k1 + 2 k2 + 2 k3 + k4)
 * D_step is the derivative of this map at fixed h with the stage fields
 * held at their values (exact for a constant field; the field-gradient term
 * of a map is left out), obtained by differentiating every stage (chain
 * rule) with respect to the 8 free parameters; D <- D_step * D. */
void kfo_rkn_step_field(double f[8], double h, const double B[3],
                        const kfo_field_map* map, double mass, double D[64]) {
  const double lam = f[7];
  const double r0[3] = {f[0], f[1], f[2]};
  const double T[3] = {f[4], f[5], f[6]};
  const double stage_a[4] = {0.0, 0.5, 0.5, 1.0};
  double k[4][3];
  double dk[4][3][8]; /* d k_i / d free */
  double prev_k[3] = {0, 0, 0};
  double prev_dk[3][8];
  double Bs[3];
  memset(prev_dk, 0, sizeof(prev_dk));
  for (int s = 0; s < 4; ++s) {
    const double a = stage_a[s] * h;
    /* field at the stage point (stages 2 and 3 share the midpoint) */
    if (s == 0) {
      kfo_field_at(B, map, r0, Bs);
    } else if (s == 1) {
      double rm[3];
      for (int i = 0; i < 3; ++i) rm[i] = r0[i] + 0.5 * h * T[i] + h * h / 8.0 * k[0][i];
      kfo_field_at(B, map, rm, Bs);
    } else if (s == 3) {
      double re[3];
      for (int i = 0; i < 3; ++i) re[i] = r0[i] + h * T[i] + 0.5 * h * h * k[2][i];
      kfo_field_at(B, map, re, Bs);
    }
    double Ts[3], TsxB[3];
    for (int i = 0; i < 3; ++i) Ts[i] = T[i] + a * prev_k[i];
    cross3(Ts, Bs, TsxB);
    for (int i = 0; i < 3; ++i) k[s][i] = lam * KFO_KAPPA * TsxB[i];
    /* d Ts / d free = E_T + a * d prev_k */
    double dTs[3][8];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 8; ++j)
        dTs[i][j] = (j == 4 + i ? 1.0 : 0.0) + a * prev_dk[i][j];
    /* d k = kappa * (Ts x B) d lam + lam * kappa * (d Ts x B) */
    for (int j = 0; j < 8; ++j) {
      double col[3] = {dTs[0][j], dTs[1][j], dTs[2][j]}, cxb[3];
      cross3(col, Bs, cxb);
      for (int i = 0; i < 3; ++i) {
        dk[s][i][j] = lam * KFO_KAPPA * cxb[i];
        if (j == 7) dk[s][i][j] += KFO_KAPPA * TsxB[i];
      }
    }
    for (int i = 0; i < 3; ++i) {
      prev_k[i] = k[s][i];
      for (int j = 0; j < 8; ++j) prev_dk[i][j] = dk[s][i][j];
    }
  }
  double Ds[64];
  mat_identity(Ds, 8);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 8; ++j) {
      Ds[i * 8 + j] += h * h / 6.0 * (dk[0][i][j] + dk[1][i][j] + dk[2][i][j]);
      Ds[(4 + i) * 8 + j] +=
          h / 6.0 *
          (dk[0][i][j] + 2.0 * dk[1][i][j] + 2.0 * dk[2][i][j] + dk[3][i][j]);
    }
    Ds[i * 8 + 4 + i] += h; /* d r / d T from h T */
  }
  const double g = sqrt(1.0 + mass * mass * lam * lam);
  Ds[3 * 8 + 7] += h * mass * mass * lam / (KFO_C_LIGHT * g);
  /* advance the state */
  for (int i = 0; i < 3; ++i) {
    f[i] += h * T[i] + h * h / 6.0 * (k[0][i] + k[1][i] + k[2][i]);
    f[4 + i] = T[i] + h / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
  }
  f[3] += h * g / KFO_C_LIGHT;
  if (D) {
    double tmp[64];
    mat_mul(Ds, D, tmp, 8, 8, 8);
    memcpy(D, tmp, sizeof(tmp));
  }
}

void kfo_rkn_step(double f[8], double h, const double B[3], double mass,
                  double D[64]) {
  kfo_rkn_step_field(f, h, B, NULL, mass, D);
}

/* Straight-line distance along T from r to the plane (c, n). */
static int plane_distance(const double f[8], const double c[3],
                          const double n[3], double* s) {
  const double T[3] = {f[4], f[5], f[6]};
  const double nT = dot3(n, T);
  if (!(fabs(nT) > 1e-9)) return KFO_NO_INTERSECTION;
  double d[3];
  for (int i = 0; i < 3; ++i) d[i] = c[i] - f[i];
  *s = dot3(n, d) / nT;
  return KFO_OK;
}

int kfo_propagate_field(double f[8], const double c[3], const double R[9],
                        const double B[3], const kfo_field_map* map,
                        double mass, double h_max, int n_iter, double D[64],
                        double* path) {
  double n[3];
  rot_col(R, 2, n);
  mat_identity(D, 8);
  double s0;
  int st = plane_distance(f, c, n, &s0);
  if (st) return st;
  int nsub = (int)ceil(fabs(s0) / h_max);
  if (nsub < 1) nsub = 1;
  if (nsub > 64) return KFO_NO_INTERSECTION;
  const double h = s0 / nsub;
  double total = 0.0;
  for (int i = 0; i < nsub; ++i) {
    kfo_rkn_step_field(f, h, B, map, mass, D);
    total += h;
  }
  for (int it = 0; it < n_iter; ++it) {
    double si;
    st = plane_distance(f, c, n, &si);
    if (st) return st;
    kfo_rkn_step_field(f, si, B, map, mass, D);
    total += si;
  }
  if (path) *path = total;
  return KFO_OK;
}

int kfo_propagate(double f[8], const double c[3], const double R[9],
                  const double B[3], double mass, double h_max, int n_iter,
                  double D[64], double* path) {
  return kfo_propagate_field(f, c, R, B, NULL, mass, h_max, n_iter, D, path);
}

int kfo_transport_field(const double ca[3], const double Ra[9],
                        const double x[6], const double cb[3],
                        const double Rb[9], const double B[3],
                        const kfo_field_map* map, double mass, double h_max,
                        int n_iter, double x_out[6], double F[36],
                        double* path) {
  double f[8], Jbf[48], D[64], Jfb[48];
  kfo_bound_to_free(ca, Ra, x, f, Jbf);
  int st = kfo_propagate_field(f, cb, Rb, B, map, mass, h_max, n_iter, D, path);
  if (st) return st;
  /* Path correction at the target plane.  At fixed path length the end
   * point moves by D df; the plane constraint n.(r - c) = 0 then moves the
   * path length by ds = -(n . dr)/(n . T), which moves the end state by
   * F' ds with F' = d free / ds at the end point.  Hence
   * P = I + F' (ds/dfree), ds/dfree = (-n/(n.T), 0, ..., 0). */
  double n[3];
  rot_col(Rb, 2, n);
  const double T[3] = {f[4], f[5], f[6]};
  const double nT = dot3(n, T);
  double TxB[3], Bend[3];
  kfo_field_at(B, map, f, Bend); /* field at the end point */
  cross3(T, Bend, TxB);
  double Fp[8];
  Fp[0] = T[0];
  Fp[1] = T[1];
  Fp[2] = T[2];
  Fp[3] = sqrt(1.0 + mass * mass * f[7] * f[7]) / KFO_C_LIGHT;
  for (int i = 0; i < 3; ++i) Fp[4 + i] = f[7] * KFO_KAPPA * TxB[i];
  Fp[7] = 0.0;
  double dsdf[8] = {-n[0] / nT, -n[1] / nT, -n[2] / nT, 0, 0, 0, 0, 0};
  double P[64];
  mat_identity(P, 8);
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) P[i * 8 + j] += Fp[i] * dsdf[j];
  free_to_bound(cb, Rb, f, x_out, Jfb);
  double PD[64], PDJ[48], t1[48];
  mat_mul(P, D, PD, 8, 8, 8);
  mat_mul(PD, Jbf, PDJ, 8, 8, 6);
  mat_mul(Jfb, PDJ, t1, 6, 8, 6);
  memcpy(F, t1, sizeof(double) * 36);
  return KFO_OK;
}

int kfo_transport(const double ca[3], const double Ra[9], const double x[6],
                  const double cb[3], const double Rb[9], const double B[3],
                  double mass, double h_max, int n_iter, double x_out[6],
                  double F[36], double* path) {
  return kfo_transport_field(ca, Ra, x, cb, Rb, B, NULL, mass, h_max, n_iter,
                             x_out, F, path);
}

/* ------------------------------------------------------------------ */
/* material (Sect. 4.3: surfaces carry material; multiple scattering)  */
/* ------------------------------------------------------------------ */

/* Highland/PDG width of the projected scattering angle for |q| = 1:
 *   theta0 = 13.6 MeV / (beta p) * sqrt(eps) * (1 + 0.038 ln(eps / beta^2)),
 * eps = (x/X0) / |cos(incidence)|, p = 1/|q/p|, 1/beta^2 = 1 + m^2 (q/p)^2. */
double kfo_highland(double qop, double mass, double xx0, double cosinc) {
  if (!(xx0 > 0.0)) return 0.0;
  const double p = 1.0 / fabs(qop);
  const double E = sqrt(p * p + mass * mass);
  const double beta = p / E;
  const double eps = xx0 / fabs(cosinc);
  return 0.0136 / (beta * p) * sqrt(eps) *
         (1.0 + 0.038 * log(eps / (beta * beta)));
}

/* ------------------------------------------------------------------ */
/* energy loss (Sect. 1: the fit accounts for the energy loss of the  */
/* particle in the detector material)                                 */
/* ------------------------------------------------------------------ */

#define KFO_K_BETHE 0.307075e-3     /* 4 pi N_A r_e^2 m_e c^2, GeV cm^2 / mol */
#define KFO_ME 0.51099895e-3        /* electron mass, GeV */

/* Sternheimer density-effect correction delta(beta gamma) of the PDG
 * parameterisation with X = log10(beta gamma):
 *   X >= x1:       2 ln10 X - Cbar
 *   x0 <= X < x1:  2 ln10 X - Cbar + a (x1 - X)^k
 *   X < x0:        delta0 10^(2 (X - x0)) */
double kfo_density_effect(double bg, const kfo_material* m) {
  const double X = log10(bg);
  const double two_ln10 = 2.0 * log(10.0);
  if (X >= m->sh_x1) return two_ln10 * X - m->sh_cbar;
  if (X >= m->sh_x0)
    return two_ln10 * X - m->sh_cbar + m->sh_a * pow(m->sh_x1 - X, m->sh_k);
  return m->sh_delta0 * pow(10.0, 2.0 * (X - m->sh_x0));
}

/* Mean stopping power (Bethe, unit charge) in GeV cm^2 / g:
 *   K Z/A / beta^2 [ 1/2 ln(2 me beta^2 gamma^2 Wmax / I^2) - beta^2
 *                    - delta/2 ],
 *   Wmax = 2 me beta^2 gamma^2 / (1 + 2 gamma me/M + (me/M)^2). */
double kfo_bethe(double bg, double mass, const kfo_material* m) {
  const double b2 = bg * bg / (1.0 + bg * bg);
  const double gam = sqrt(1.0 + bg * bg);
  const double r = KFO_ME / mass;
  const double wmax = 2.0 * KFO_ME * bg * bg / (1.0 + 2.0 * gam * r + r * r);
  const double arg = 2.0 * KFO_ME * bg * bg * wmax / (m->i_exc * m->i_exc);
  return KFO_K_BETHE * m->z_over_a / b2 *
         (0.5 * log(arg) - b2 - 0.5 * kfo_density_effect(bg, m));
}

/* Landau scale xi = (K/2) (Z/A) (rho x) / beta^2 in GeV for a thickness
 * rho x in g/cm^2. */
double kfo_landau_xi(double beta, double thick, const kfo_material* m) {
  return 0.5 * KFO_K_BETHE * m->z_over_a * thick / (beta * beta);
}

/* Energy loss in a surface of x/X0 = xx0 crossed at |cos(incidence)| =
 * cosinc, thickness rho x = xx0 X0rho / cosinc.  The mean loss dE is
 * evaluated at the current state's momentum.  dir = +1 (forward): the
 * particle leaves with E' = E - dE; dir = -1 (backward): the upstream energy
 * E' = E + dE is restored.  On return *qop holds the new q/p, *jac the
 * derivative d(q/p)'/d(q/p) at fixed dE, which is (p^3 E')/(p'^3 E), and
 * *var_down the straggling variance of q/p on the downstream side: the
 * energy spread is a Gaussian with the FWHM 4 xi of the Landau
 * distribution, sigma_E = 4 xi / (2 sqrt(2 ln 2)), mapped to q/p by
 * |d(q/p)/dE| = E/p^3 at the downstream energy and momentum.
 * Returns KFO_NONFINITE when the particle would stop. */
int kfo_energy_loss(double* qop, double mass, double xx0, double cosinc,
                    const kfo_material* m, int dir, double* jac,
                    double* var_down) {
  *jac = 1.0;
  *var_down = 0.0;
  if (!(xx0 > 0.0)) return KFO_OK;
  if (!(mass > 0.0)) return KFO_BAD_INPUT;
  const double thick = xx0 * m->x0_rho / fabs(cosinc);
  const double p = 1.0 / fabs(*qop);
  const double E = sqrt(p * p + mass * mass);
  const double beta = p / E;
  const double dE = kfo_bethe(p / mass, mass, m) * thick;
  const double E2 = dir > 0 ? E - dE : E + dE;
  if (!(E2 > mass)) return KFO_NONFINITE;
  const double p2 = sqrt(E2 * E2 - mass * mass);
  const double sigE = 4.0 * kfo_landau_xi(beta, thick, m) / (2.0 * sqrt(2.0 * log(2.0)));
  *jac = (p * p * p * E2) / (p2 * p2 * p2 * E);
  const double Ed = dir > 0 ? E2 : E, pd = dir > 0 ? p2 : p;
  const double dqdE = Ed / (pd * pd * pd);
  *var_down = dqdE * dqdE * sigE * sigE;
  *qop = (*qop > 0.0 ? 1.0 : -1.0) / p2;
  return KFO_OK;
}

/* ------------------------------------------------------------------ */
/* update and smoother (Sect. 2)                                       */
/* ------------------------------------------------------------------ */

int kfo_update(const double xp[6], const double Cp[36], const double m[2],
               const double V[4], double xf[6], double Cf[36], double* chi2) {
  /* H = [I2 0]: the measurement is (loc0, loc1). */
  double H[12];
  memset(H, 0, sizeof(H));
  H[0 * 6 + 0] = 1.0;
  H[1 * 6 + 1] = 1.0;
  double HT[12], CHT[12], S[4], HCHT[4];
  mat_transpose(H, HT, 2, 6);
  mat_mul(Cp, HT, CHT, 6, 6, 2);
  mat_mul(H, CHT, HCHT, 2, 6, 2);
  for (int i = 0; i < 4; ++i) S[i] = V[i] + HCHT[i];
  const double det = S[0] * S[3] - S[1] * S[2];
  if (!(det > 0.0) || !(S[0] > 0.0)) return KFO_NON_SPD;
  const double Si[4] = {S[3] / det, -S[1] / det, -S[2] / det, S[0] / det};
  double K[12];
  mat_mul(CHT, Si, K, 6, 2, 2);
  double r[2] = {m[0] - xp[0], m[1] - xp[1]};
  for (int i = 0; i < 6; ++i) xf[i] = xp[i] + K[i * 2 + 0] * r[0] + K[i * 2 + 1] * r[1];
  /* Joseph form: Cf = (I - K H) Cp (I - K H)^T + K V K^T */
  double L[36], KH[36];
  mat_mul(K, H, KH, 6, 2, 6);
  mat_identity(L, 6);
  for (int i = 0; i < 36; ++i) L[i] -= KH[i];
  double LCLT[36], KV[12], KT[12], KVKT[36];
  sandwich6(L, Cp, LCLT);
  mat_mul(K, V, KV, 6, 2, 2);
  mat_transpose(K, KT, 6, 2);
  mat_mul(KV, KT, KVKT, 6, 2, 6);
  for (int i = 0; i < 36; ++i) Cf[i] = LCLT[i] + KVKT[i];
  double Sir[2] = {Si[0] * r[0] + Si[1] * r[1], Si[2] * r[0] + Si[3] * r[1]};
  *chi2 = r[0] * Sir[0] + r[1] * Sir[1];
  return KFO_OK;
}

/* Solve A X = Bm for SPD A (6x6) and k right-hand sides (6 x k), via the
 * Cholesky factor of the Jacobi-scaled matrix Dh^-1 A Dh^-1, Dh = diag(sqrt
 * A_ii).  Returns KFO_NON_SPD on a non-positive pivot. */
static int spd_solve6(const double A[36], const double* Bm, int k, double* X) {
  double d[6], As[36], L[36];
  for (int i = 0; i < 6; ++i) {
    if (!(A[i * 6 + i] > 0.0)) return KFO_NON_SPD;
    d[i] = sqrt(A[i * 6 + i]);
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) As[i * 6 + j] = A[i * 6 + j] / (d[i] * d[j]);
  memset(L, 0, sizeof(L));
  for (int j = 0; j < 6; ++j) {
    double s = As[j * 6 + j];
    for (int q = 0; q < j; ++q) s -= L[j * 6 + q] * L[j * 6 + q];
    if (!(s > 0.0)) return KFO_NON_SPD;
    L[j * 6 + j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = As[i * 6 + j]; /* lower triangle of the scaled matrix */
      for (int q = 0; q < j; ++q) t -= L[i * 6 + q] * L[j * 6 + q];
      L[i * 6 + j] = t / L[j * 6 + j];
    }
  }
  for (int c = 0; c < k; ++c) {
    double y[6], z[6];
    /* scaled system: As (Dh X) = Dh^-1 B */
    for (int i = 0; i < 6; ++i) {
      double t = Bm[i * k + c] / d[i];
      for (int q = 0; q < i; ++q) t -= L[i * 6 + q] * y[q];
      y[i] = t / L[i * 6 + i];
    }
    for (int i = 5; i >= 0; --i) {
      double t = y[i];
      for (int q = i + 1; q < 6; ++q) t -= L[q * 6 + i] * z[q];
      z[i] = t / L[i * 6 + i];
    }
    for (int i = 0; i < 6; ++i) X[i * k + c] = z[i] / d[i];
  }
  return KFO_OK;
}

int kfo_rts_step(const double xf[6], const double Cf[36], const double xp1[6],
                 const double Cp1[36], const double F1[36],
                 const double xs1[6], const double Cs1[36], double xs[6],
                 double Cs[36]) {
  /* Smoother gain A = Cf F^T Cp1^-1, obtained from Cp1 A^T = F Cf. */
  double FC[36], AT[36], A[36];
  mat_mul(F1, Cf, FC, 6, 6, 6);
  int st = spd_solve6(Cp1, FC, 6, AT);
  if (st) return st;
  mat_transpose(AT, A, 6, 6);
  double dx[6];
  for (int i = 0; i < 6; ++i) dx[i] = xs1[i] - xp1[i];
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int j = 0; j < 6; ++j) s += A[i * 6 + j] * dx[j];
    xs[i] = xf[i] + s;
  }
  double dC[36], AdCAT[36];
  for (int i = 0; i < 36; ++i) dC[i] = Cs1[i] - Cp1[i];
  sandwich6(A, dC, AdCAT);
  for (int i = 0; i < 36; ++i) Cs[i] = Cf[i] + AdCAT[i];
  return KFO_OK;
}

/* Solve A X = Bm for a general 6x6 A (Gaussian elimination with partial
 * pivoting), k right-hand sides.  Returns KFO_NON_SPD on a zero pivot. */
static int gen_solve6(const double A[36], const double* Bm, int k, double* X) {
  double M[36];
  memcpy(M, A, sizeof(M));
  double* R = (double*)malloc(sizeof(double) * 6 * k);
  memcpy(R, Bm, sizeof(double) * 6 * k);
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (fabs(M[r * 6 + c]) > fabs(M[piv * 6 + c])) piv = r;
    if (!(fabs(M[piv * 6 + c]) > 0.0)) {
      free(R);
      return KFO_NON_SPD;
    }
    if (piv != c) {
      for (int j = 0; j < 6; ++j) {
        const double t = M[c * 6 + j];
        M[c * 6 + j] = M[piv * 6 + j];
        M[piv * 6 + j] = t;
      }
      for (int j = 0; j < k; ++j) {
        const double t = R[c * k + j];
        R[c * k + j] = R[piv * k + j];
        R[piv * k + j] = t;
      }
    }
    for (int r = c + 1; r < 6; ++r) {
      const double f = M[r * 6 + c] / M[c * 6 + c];
      for (int j = c; j < 6; ++j) M[r * 6 + j] -= f * M[c * 6 + j];
      for (int j = 0; j < k; ++j) R[r * k + j] -= f * R[c * k + j];
    }
  }
  for (int j = 0; j < k; ++j)
    for (int r = 5; r >= 0; --r) {
      double t = R[r * k + j];
      for (int q = r + 1; q < 6; ++q) t -= M[r * 6 + q] * X[q * k + j];
      X[r * k + j] = t / M[r * 6 + r];
    }
  free(R);
  return KFO_OK;
}

/* Weighted mean of two estimates of the same state (the smoothed state of
 * the two-filter smoother, Sect. 2 and Fig. 2):
 *   K = Cf (Cf + Cb)^-1,  xs = xf + K (xb - xf),  Cs = Cf - K Cf. */
static int weighted_mean(const double xf[6], const double Cf[36],
                         const double xb[6], const double Cb[36], double xs[6],
                         double Cs[36]) {
  double Sum[36], X[36], K[36], KC[36];
  for (int i = 0; i < 36; ++i) Sum[i] = Cf[i] + Cb[i];
  int st = spd_solve6(Sum, Cf, 6, X); /* X = (Cf + Cb)^-1 Cf = K^T */
  if (st) return st;
  mat_transpose(X, K, 6, 6);
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int j = 0; j < 6; ++j) s += K[i * 6 + j] * (xb[j] - xf[j]);
    xs[i] = xf[i] + s;
  }
  mat_mul(K, Cf, KC, 6, 6, 6);
  for (int i = 0; i < 36; ++i) Cs[i] = Cf[i] - KC[i];
  return KFO_OK;
}

/* Prediction callbacks: forward k-1 -> k (fills xp, Cp and the transition
 * Jacobian F) and backward k -> k-1. */
typedef int (*predict_fn)(void* ctx, int k, const double* xf_prev,
                          const double* Cf_prev, double* xp, double* Cp,
                          double* F);
typedef int (*bpredict_fn)(void* ctx, int k, const double* xb,
                           const double* Cb, double* xo, double* Co);

/* Forward filter over n states; the caller has filled xp[0], Cp[0] (the
 * prior). */
static int forward_filter(int n, predict_fn predict, void* ctx,
                          const double* m, const double* V,
                          const uint8_t* hole, double* xp, double* Cp,
                          double* xf, double* Cf, double* F, double* chi2) {
  for (int k = 0; k < n; ++k) {
    if (k > 0) {
      int st = predict(ctx, k, xf + 6 * (k - 1), Cf + 36 * (k - 1), xp + 6 * k,
                       Cp + 36 * k, F + 36 * k);
      if (st) return st;
    } else {
      mat_identity(F, 6);
    }
    chi2[k] = 0.0;
    if (hole[k]) {
      memcpy(xf + 6 * k, xp + 6 * k, sizeof(double) * 6);
      memcpy(Cf + 36 * k, Cp + 36 * k, sizeof(double) * 36);
    } else {
      int st = kfo_update(xp + 6 * k, Cp + 36 * k, m + 2 * k, V + 4 * k,
                          xf + 6 * k, Cf + 36 * k, chi2 + k);
      if (st) return st;
    }
  }
  return KFO_OK;
}

/* RTS smoother from the last filtered state back to state 0. */
static int rts_smooth(int n, const double* xp, const double* Cp,
                      const double* xf, const double* Cf, const double* F,
                      double* xs, double* Cs) {
  memcpy(xs + 6 * (n - 1), xf + 6 * (n - 1), sizeof(double) * 6);
  memcpy(Cs + 36 * (n - 1), Cf + 36 * (n - 1), sizeof(double) * 36);
  for (int k = n - 2; k >= 0; --k) {
    int st = kfo_rts_step(xf + 6 * k, Cf + 36 * k, xp + 6 * (k + 1),
                          Cp + 36 * (k + 1), F + 36 * (k + 1),
                          xs + 6 * (k + 1), Cs + 36 * (k + 1), xs + 6 * k,
                          Cs + 36 * k);
    if (st) return st;
  }
  return KFO_OK;
}

/* Backward-filter smoother (Sect. 2, Fig. 2): a second Kalman filter runs
 * from the last state to the first, with its own propagation.  It starts at
 * state n-1 from the forward-filtered parameters with the covariance
 * scale * Cf_{n-1} (a nearly uninformative start), takes the measurement of
 * each state it reaches, and its prediction onto state k is combined with
 * the forward-filtered state k by the weighted mean.  State n-1 keeps the
 * forward-filtered state (as in the RTS smoother). */
static int backward_filter_smooth(int n, bpredict_fn bpredict, void* ctx,
                                  const double* m, const double* V,
                                  const uint8_t* hole, const double* xf,
                                  const double* Cf, double scale, double* xs,
                                  double* Cs) {
  double xb[6], Cb[36];
  memcpy(xs + 6 * (n - 1), xf + 6 * (n - 1), sizeof(double) * 6);
  memcpy(Cs + 36 * (n - 1), Cf + 36 * (n - 1), sizeof(double) * 36);
  memcpy(xb, xf + 6 * (n - 1), sizeof(xb));
  for (int i = 0; i < 36; ++i) Cb[i] = scale * Cf[36 * (n - 1) + i];
  for (int k = n - 1; k >= 1; --k) {
    if (!hole[k]) {
      double xu[6], Cu[36], c2;
      int st = kfo_update(xb, Cb, m + 2 * k, V + 4 * k, xu, Cu, &c2);
      if (st) return st;
      memcpy(xb, xu, sizeof(xb));
      memcpy(Cb, Cu, sizeof(Cb));
    }
    double xo[6], Co[36];
    int st = bpredict(ctx, k, xb, Cb, xo, Co);
    if (st) return st;
    memcpy(xb, xo, sizeof(xb));
    memcpy(Cb, Co, sizeof(Cb));
    st = weighted_mean(xf + 6 * (k - 1), Cf + 36 * (k - 1), xb, Cb,
                       xs + 6 * (k - 1), Cs + 36 * (k - 1));
    if (st) return st;
  }
  return KFO_OK;
}

static int filter_smooth(int n, predict_fn predict, bpredict_fn bpredict,
                         void* ctx, const double* m, const double* V,
                         const uint8_t* hole, int smoother, double bf_scale,
                         double* xp, double* Cp, double* xf, double* Cf,
                         double* xs, double* Cs, double* F, double* chi2) {
  int st = forward_filter(n, predict, ctx, m, V, hole, xp, Cp, xf, Cf, F, chi2);
  if (st) return st;
  if (smoother == KFO_SMOOTHER_BACKWARD_FILTER)
    return backward_filter_smooth(n, bpredict, ctx, m, V, hole, xf, Cf,
                                  bf_scale, xs, Cs);
  return rts_smooth(n, xp, Cp, xf, Cf, F, xs, Cs);
}

/* linear model: xp = F xf, Cp = F Cf F^T + Q */
typedef struct {
  const double* F;
  const double* Q;
} linear_ctx;

static int predict_linear(void* vctx, int k, const double* xf_prev,
                          const double* Cf_prev, double* xp, double* Cp,
                          double* F) {
  const linear_ctx* ctx = (const linear_ctx*)vctx;
  memcpy(F, ctx->F + 36 * k, sizeof(double) * 36);
  mat_mul(F, xf_prev, xp, 6, 6, 1);
  sandwich6(F, Cf_prev, Cp);
  for (int i = 0; i < 36; ++i) Cp[i] += ctx->Q[36 * k + i];
  return KFO_OK;
}

/* backward: x_{k-1} = F_k^-1 (x_k - w_k), Cb' = F_k^-1 (Cb + Q_k) F_k^-T */
static int bpredict_linear(void* vctx, int k, const double* xb,
                           const double* Cb, double* xo, double* Co) {
  const linear_ctx* ctx = (const linear_ctx*)vctx;
  const double* Fk = ctx->F + 36 * k;
  double M[36], Y[36], YT[36];
  for (int i = 0; i < 36; ++i) M[i] = Cb[i] + ctx->Q[36 * k + i];
  int st = gen_solve6(Fk, xb, 1, xo);
  if (st) return st;
  st = gen_solve6(Fk, M, 6, Y); /* F^-1 M */
  if (st) return st;
  mat_transpose(Y, YT, 6, 6);   /* M F^-T */
  return gen_solve6(Fk, YT, 6, Co);
}

int kfo_linear_fit(int n, const double x0[6], const double C0[36],
                   const double* F, const double* Q, const double* m,
                   const double* V, const uint8_t* hole, double* xs,
                   double* Cs, double* chi2) {
  return kfo_linear_fit_ex(n, x0, C0, F, Q, m, V, hole, KFO_SMOOTHER_RTS, 0.0,
                           xs, Cs, chi2);
}

int kfo_linear_fit_ex(int n, const double x0[6], const double C0[36],
                      const double* F, const double* Q, const double* m,
                      const double* V, const uint8_t* hole, int smoother,
                      double bf_scale, double* xs, double* Cs, double* chi2) {
  double* buf = (double*)malloc(sizeof(double) * n * (6 + 36) * 3);
  double* xp = buf;
  double* xf = xp + 6 * n;
  double* Cp = xf + 6 * n;
  double* Cf = Cp + 36 * n;
  double* Fs = Cf + 36 * n;
  memcpy(xp, x0, sizeof(double) * 6);
  memcpy(Cp, C0, sizeof(double) * 36);
  linear_ctx ctx = {F, Q};
  int st = filter_smooth(n, predict_linear, bpredict_linear, &ctx, m, V, hole,
                         smoother, bf_scale, xp, Cp, xf, Cf, xs, Cs, Fs, chi2);
  free(buf);
  return st;
}

/* track model: RKN transport between the track's surfaces plus the
 * material effects of the surface reached (added before the update, so
 * state k is the state leaving surface k): multiple-scattering noise on the
 * angles and, optionally, the mean energy loss with its straggling noise on
 * q/p. */
typedef struct {
  const int32_t* surface_id;
  const double* center;
  const double* rot;
  const double* x_over_x0;
  const double* B;
  double mass, h_max;
  int n_iter;
  const kfo_method* meth; /* NULL: constant field, no energy loss */
} track_ctx;

static void unit_dir(const double x[6], double T[3]) {
  T[0] = cos(x[2]) * sin(x[3]);
  T[1] = sin(x[2]) * sin(x[3]);
  T[2] = cos(x[3]);
}

/* multiple-scattering variances of (phi, theta) for the state x crossing
 * surface sid (Highland width with the state's momentum and incidence) */
static void scattering_noise(const track_ctx* ctx, int sid, const double x[6],
                             double C[36]) {
  const double xx0 = ctx->x_over_x0[sid];
  if (!(xx0 > 0.0)) return;
  double n[3], T[3];
  rot_col(ctx->rot + 9 * sid, 2, n);
  unit_dir(x, T);
  const double th0 = kfo_highland(x[4], ctx->mass, xx0, dot3(n, T));
  const double st_ = sin(x[3]);
  C[2 * 6 + 2] += th0 * th0 / (st_ * st_);
  C[3 * 6 + 3] += th0 * th0;
}

static double incidence(const track_ctx* ctx, int sid, const double x[6]) {
  double n[3], T[3];
  rot_col(ctx->rot + 9 * sid, 2, n);
  unit_dir(x, T);
  return dot3(n, T);
}

/* scale row and column 4 (q/p) of a 6x6 matrix by g */
static void scale_qop(double C[36], double g) {
  for (int j = 0; j < 6; ++j) C[4 * 6 + j] *= g;
  for (int j = 0; j < 6; ++j) C[j * 6 + 4] *= g;
}

static int predict_track(void* vctx, int k, const double* xf_prev,
                         const double* Cf_prev, double* xp, double* Cp,
                         double* F) {
  const track_ctx* ctx = (const track_ctx*)vctx;
  const kfo_field_map* map = ctx->meth ? ctx->meth->map : NULL;
  const int sa = ctx->surface_id[k - 1], sb = ctx->surface_id[k];
  int st = kfo_transport_field(ctx->center + 3 * sa, ctx->rot + 9 * sa, xf_prev,
                               ctx->center + 3 * sb, ctx->rot + 9 * sb, ctx->B,
                               map, ctx->mass, ctx->h_max, ctx->n_iter, xp, F,
                               NULL);
  if (st) return st;
  sandwich6(F, Cf_prev, Cp);
  scattering_noise(ctx, sb, xp, Cp);
  if (ctx->meth && ctx->meth->energy_loss && ctx->x_over_x0[sb] > 0.0) {
    /* q/p' = q/p after the mean loss; F <- G F and Cp <- G Cp G^T with
     * G = diag(1, 1, 1, 1, jac, 1); then the straggling variance */
    double jac, var;
    st = kfo_energy_loss(&xp[4], ctx->mass, ctx->x_over_x0[sb],
                         incidence(ctx, sb, xp), &ctx->meth->mat, +1, &jac, &var);
    if (st) return st;
    for (int j = 0; j < 6; ++j) F[4 * 6 + j] *= jac;
    scale_qop(Cp, jac);
    Cp[4 * 6 + 4] += var;
  }
  return KFO_OK;
}

/* backward from state k (leaving surface k) to state k-1: the material of
 * surface k is undone first (its noise added, the mean loss restored), then
 * the RKN transport runs back to surface k-1 (negative path length). */
static int bpredict_track(void* vctx, int k, const double* xb,
                          const double* Cb, double* xo, double* Co) {
  const track_ctx* ctx = (const track_ctx*)vctx;
  const kfo_field_map* map = ctx->meth ? ctx->meth->map : NULL;
  const int sa = ctx->surface_id[k - 1], sb = ctx->surface_id[k];
  double x[6], C[36], F[36];
  memcpy(x, xb, sizeof(x));
  memcpy(C, Cb, sizeof(C));
  scattering_noise(ctx, sb, x, C);
  if (ctx->meth && ctx->meth->energy_loss && ctx->x_over_x0[sb] > 0.0) {
    double jac, var;
    int st = kfo_energy_loss(&x[4], ctx->mass, ctx->x_over_x0[sb],
                             incidence(ctx, sb, x), &ctx->meth->mat, -1, &jac, &var);
    if (st) return st;
    C[4 * 6 + 4] += var;
    scale_qop(C, jac);
  }
  int st = kfo_transport_field(ctx->center + 3 * sb, ctx->rot + 9 * sb, x,
                               ctx->center + 3 * sa, ctx->rot + 9 * sa, ctx->B,
                               map, ctx->mass, ctx->h_max, ctx->n_iter, xo, F,
                               NULL);
  if (st) return st;
  sandwich6(F, C, Co);
  return KFO_OK;
}

int kfo_fit_track(int n, const int32_t* surface_id, const double* loc,
                  const double* cov, const uint8_t* is_hole,
                  const double seed[6], const double seed_cov[36],
                  int n_surfaces, const double* center, const double* rot,
                  const double* x_over_x0, const double B[3], double mass,
                  double h_max, int n_iter, double* xp, double* Cp,
                  double* xf, double* Cf, double* xs, double* Cs, double* F,
                  double* chi2) {
  return kfo_fit_track_ex(n, surface_id, loc, cov, is_hole, seed, seed_cov,
                          n_surfaces, center, rot, x_over_x0, B, mass, h_max,
                          n_iter, NULL, xp, Cp, xf, Cf, xs, Cs, F, chi2);
}

int kfo_fit_track_ex(int n, const int32_t* surface_id, const double* loc,
                     const double* cov, const uint8_t* is_hole,
                     const double seed[6], const double seed_cov[36],
                     int n_surfaces, const double* center, const double* rot,
                     const double* x_over_x0, const double B[3], double mass,
                     double h_max, int n_iter, const kfo_method* meth,
                     double* xp, double* Cp, double* xf, double* Cf,
                     double* xs, double* Cs, double* F, double* chi2) {
  if (n < 1) return KFO_BAD_INPUT;
  for (int k = 0; k < n; ++k)
    if (surface_id[k] < 0 || surface_id[k] >= n_surfaces) return KFO_BAD_INPUT;
  double* V = (double*)malloc(sizeof(double) * 4 * n);
  double* m = (double*)malloc(sizeof(double) * 2 * n);
  for (int k = 0; k < n; ++k) {
    m[2 * k + 0] = loc[2 * k + 0];
    m[2 * k + 1] = loc[2 * k + 1];
    V[4 * k + 0] = cov[3 * k + 0];
    V[4 * k + 1] = cov[3 * k + 1];
    V[4 * k + 2] = cov[3 * k + 1];
    V[4 * k + 3] = cov[3 * k + 2];
  }
  memcpy(xp, seed, sizeof(double) * 6);
  memcpy(Cp, seed_cov, sizeof(double) * 36);
  track_ctx ctx = {surface_id, center, rot, x_over_x0, B, mass, h_max, n_iter, meth};
  const int smoother = meth ? meth->smoother : KFO_SMOOTHER_RTS;
  const double scale = meth ? meth->bf_scale : 0.0;
  int st = filter_smooth(n, predict_track, bpredict_track, &ctx, m, V, is_hole,
                         smoother, scale, xp, Cp, xf, Cf, xs, Cs, F, chi2);
  free(V);
  free(m);
  if (st) return st;
  if (!all_finite(xs, 6 * n) || !all_finite(Cs, 36 * n) || !all_finite(chi2, n))
    return KFO_NONFINITE;
  return KFO_OK;
}

/* ------------------------------------------------------------------ */
/* batched driver over the SoA boundary layout                         */
/* ------------------------------------------------------------------ */

typedef struct {
  int n_tracks;
  const int32_t* offsets;
  const double *seed_params, *seed_cov;
  int n_surfaces;
  const double *center, *rot, *x_over_x0;
  int64_t n_states;
  const int32_t* surface_id;
  const double *loc, *cov;
  const uint8_t* is_hole;
  const double* B;
  double mass, h_max;
  int n_iter;
  double *out_params, *out_cov, *out_chi2;
  int32_t* out_ndf;
  uint8_t* out_status;
  double* out_states;
  int t_begin, t_end;
  const kfo_method* meth;
} batch_job;

static void unpack_sym(const double* packed, int64_t stride, int64_t t,
                       double C[36]) {
  int e = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j, ++e) {
      C[i * 6 + j] = packed[e * stride + t];
      C[j * 6 + i] = packed[e * stride + t];
    }
}

static void fit_range(const batch_job* J) {
  const int64_t T = J->n_tracks;
  const int64_t M = J->n_states;
  int cap = 0;
  double* buf = NULL;
  for (int t = J->t_begin; t < J->t_end; ++t) {
    const int64_t o0 = J->offsets[t], o1 = J->offsets[t + 1];
    const int n = (int)(o1 - o0);
    int st = KFO_OK;
    int nmeas = 0;
    double chi2sum = 0.0;
    double xs0[6], Cs0[36];
    if (n < 1 || o0 < 0 || o1 > M) {
      st = KFO_BAD_INPUT;
    } else {
      if (n > cap) {
        free(buf);
        cap = n;
        buf = (double*)malloc(sizeof(double) * (size_t)cap * (6 * 3 + 36 * 4 + 1 + 2 + 3));
      }
      double* xp = buf;
      double* xf = xp + 6 * n;
      double* xs = xf + 6 * n;
      double* Cp = xs + 6 * n;
      double* Cf = Cp + 36 * n;
      double* Cs = Cf + 36 * n;
      double* F = Cs + 36 * n;
      double* chi2 = F + 36 * n;
      double* loc = chi2 + n;
      double* cov = loc + 2 * n;
      for (int k = 0; k < n; ++k) {
        loc[2 * k + 0] = J->loc[0 * M + o0 + k];
        loc[2 * k + 1] = J->loc[1 * M + o0 + k];
        cov[3 * k + 0] = J->cov[0 * M + o0 + k];
        cov[3 * k + 1] = J->cov[1 * M + o0 + k];
        cov[3 * k + 2] = J->cov[2 * M + o0 + k];
      }
      double seed[6], C0[36];
      for (int i = 0; i < 6; ++i) seed[i] = J->seed_params[i * T + t];
      unpack_sym(J->seed_cov, T, t, C0);
      st = kfo_fit_track_ex(n, J->surface_id + o0, loc, cov, J->is_hole + o0,
                            seed, C0, J->n_surfaces, J->center, J->rot,
                            J->x_over_x0, J->B, J->mass, J->h_max, J->n_iter,
                            J->meth, xp, Cp, xf, Cf, xs, Cs, F, chi2);
      if (st == KFO_OK) {
        for (int k = 0; k < n; ++k)
          if (!J->is_hole[o0 + k]) {
            ++nmeas;
            chi2sum += chi2[k];
          }
        memcpy(xs0, xs, sizeof(xs0));
        memcpy(Cs0, Cs, sizeof(Cs0));
        if (J->out_states)
          for (int k = 0; k < n; ++k)
            for (int i = 0; i < 6; ++i)
              J->out_states[i * M + o0 + k] = xs[6 * k + i];
      }
    }
    if (st != KFO_OK) {
      for (int i = 0; i < 6; ++i) xs0[i] = NAN;
      for (int i = 0; i < 36; ++i) Cs0[i] = NAN;
      chi2sum = NAN;
      nmeas = 0;
      if (J->out_states && n >= 1 && o0 >= 0 && o1 <= M)
        for (int k = 0; k < n; ++k)
          for (int i = 0; i < 6; ++i) J->out_states[i * M + o0 + k] = NAN;
    }
    for (int i = 0; i < 6; ++i) J->out_params[i * T + t] = xs0[i];
    int e = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j <= i; ++j, ++e) J->out_cov[e * T + t] = Cs0[i * 6 + j];
    J->out_chi2[t] = chi2sum;
    J->out_ndf[t] = 2 * nmeas;
    J->out_status[t] = (uint8_t)st;
  }
  free(buf);
}

static void* fit_thread(void* arg) {
  fit_range((const batch_job*)arg);
  return NULL;
}

int kfo_fit_batch(int n_tracks, const int32_t* offsets,
                  const double* seed_params, const double* seed_cov,
                  int n_surfaces, const double* center, const double* rot,
                  const double* x_over_x0, int64_t n_states,
                  const int32_t* surface_id, const double* loc,
                  const double* cov, const uint8_t* is_hole, const double B[3],
                  double mass, double h_max, int n_iter, double* out_params,
                  double* out_cov, double* out_chi2, int32_t* out_ndf,
                  uint8_t* out_status, double* out_states, int t_begin,
                  int t_end, int n_threads) {
  return kfo_fit_batch_ex(n_tracks, offsets, seed_params, seed_cov, n_surfaces,
                          center, rot, x_over_x0, n_states, surface_id, loc,
                          cov, is_hole, B, mass, h_max, n_iter, NULL,
                          out_params, out_cov, out_chi2, out_ndf, out_status,
                          out_states, t_begin, t_end, n_threads);
}

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
                     int t_end, int n_threads) {
  if (n_tracks < 0 || t_begin < 0 || t_end > n_tracks || t_begin > t_end)
    return -1;
  if (n_threads < 1) n_threads = 1;
  batch_job base = {n_tracks, offsets, seed_params, seed_cov, n_surfaces,
                    center, rot, x_over_x0, n_states, surface_id, loc, cov,
                    is_hole, B, mass, h_max, n_iter, out_params, out_cov,
                    out_chi2, out_ndf, out_status, out_states, t_begin, t_end,
                    meth};
  const int total = t_end - t_begin;
  if (n_threads == 1 || total < 2 * n_threads) {
    fit_range(&base);
    return 0;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  batch_job* jobs = (batch_job*)malloc(sizeof(batch_job) * n_threads);
  for (int i = 0; i < n_threads; ++i) {
    jobs[i] = base;
    jobs[i].t_begin = t_begin + (int)((int64_t)total * i / n_threads);
    jobs[i].t_end = t_begin + (int)((int64_t)total * (i + 1) / n_threads);
    pthread_create(&th[i], NULL, fit_thread, &jobs[i]);
  }
  for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
  free(th);
  free(jobs);
  return 0;
}
