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

/* Equation of motion in path length s for a constant field:
 *   r'' = qop * kappa * (r' x B),  t' = sqrt(1 + m^2 qop^2) / c.
 * Classic 4-stage Nystrom step:
 *   k1 = a(T), k2 = a(T + h/2 k1), k3 = a(T + h/2 k2), k4 = a(T + h k3)
 *   r <- r + h T + h^2/6 (k1 + k2 + k3)
 *   T <- T + h/6 (k1 + 2 k2 + 2 k3 + k4)
 * D_step is the exact derivative of this map at fixed h, obtained by
 * differentiating every stage (chain rule) with respect to the 8 free
 * parameters; D <- D_step * D. */
void kfo_rkn_step(double f[8], double h, const double B[3], double mass,
                  double D[64]) {
  const double lam = f[7];
  const double T[3] = {f[4], f[5], f[6]};
  const double stage_a[4] = {0.0, 0.5, 0.5, 1.0};
  double k[4][3];
  double dk[4][3][8]; /* d k_i / d free */
  double prev_k[3] = {0, 0, 0};
  double prev_dk[3][8];
  memset(prev_dk, 0, sizeof(prev_dk));
  for (int s = 0; s < 4; ++s) {
    const double a = stage_a[s] * h;
    double Ts[3], TsxB[3];
    for (int i = 0; i < 3; ++i) Ts[i] = T[i] + a * prev_k[i];
    cross3(Ts, B, TsxB);
    for (int i = 0; i < 3; ++i) k[s][i] = lam * KFO_KAPPA * TsxB[i];
    /* d Ts / d free = E_T + a * d prev_k */
    double dTs[3][8];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 8; ++j)
        dTs[i][j] = (j == 4 + i ? 1.0 : 0.0) + a * prev_dk[i][j];
    /* d k = kappa * (Ts x B) d lam + lam * kappa * (d Ts x B) */
    for (int j = 0; j < 8; ++j) {
      double col[3] = {dTs[0][j], dTs[1][j], dTs[2][j]}, cxb[3];
      cross3(col, B, cxb);
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

int kfo_propagate(double f[8], const double c[3], const double R[9],
                  const double B[3], double mass, double h_max, int n_iter,
                  double D[64], double* path) {
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
    kfo_rkn_step(f, h, B, mass, D);
    total += h;
  }
  for (int it = 0; it < n_iter; ++it) {
    double si;
    st = plane_distance(f, c, n, &si);
    if (st) return st;
    kfo_rkn_step(f, si, B, mass, D);
    total += si;
  }
  if (path) *path = total;
  return KFO_OK;
}

int kfo_transport(const double ca[3], const double Ra[9], const double x[6],
                  const double cb[3], const double Rb[9], const double B[3],
                  double mass, double h_max, int n_iter, double x_out[6],
                  double F[36], double* path) {
  double f[8], Jbf[48], D[64], Jfb[48];
  kfo_bound_to_free(ca, Ra, x, f, Jbf);
  int st = kfo_propagate(f, cb, Rb, B, mass, h_max, n_iter, D, path);
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
  double TxB[3];
  cross3(T, B, TxB);
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

/* Shared forward/backward skeleton: the caller has filled xp[0], Cp[0]
 * (the prior) and a prediction callback for k >= 1. */
typedef int (*predict_fn)(void* ctx, int k, const double* xf_prev,
                          const double* Cf_prev, double* xp, double* Cp,
                          double* F);

static int filter_smooth(int n, predict_fn predict, void* ctx,
                         const double* m, const double* V,
                         const uint8_t* hole, double* xp, double* Cp,
                         double* xf, double* Cf, double* xs, double* Cs,
                         double* F, double* chi2) {
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
  /* RTS: start from the last filtered state. */
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

int kfo_linear_fit(int n, const double x0[6], const double C0[36],
                   const double* F, const double* Q, const double* m,
                   const double* V, const uint8_t* hole, double* xs,
                   double* Cs, double* chi2) {
  double* buf = (double*)malloc(sizeof(double) * n * (6 + 36) * 3);
  double* xp = buf;
  double* xf = xp + 6 * n;
  double* Cp = xf + 6 * n;
  double* Cf = Cp + 36 * n;
  double* Fs = Cf + 36 * n;
  memcpy(xp, x0, sizeof(double) * 6);
  memcpy(Cp, C0, sizeof(double) * 36);
  linear_ctx ctx = {F, Q};
  int st = filter_smooth(n, predict_linear, &ctx, m, V, hole, xp, Cp, xf, Cf,
                         xs, Cs, Fs, chi2);
  free(buf);
  return st;
}

/* track model: RKN transport between the track's surfaces plus the
 * multiple-scattering noise of the surface reached (added before the
 * update, so state k is the direction leaving surface k). */
typedef struct {
  const int32_t* surface_id;
  const double* center;
  const double* rot;
  const double* x_over_x0;
  const double* B;
  double mass, h_max;
  int n_iter;
} track_ctx;

static int predict_track(void* vctx, int k, const double* xf_prev,
                         const double* Cf_prev, double* xp, double* Cp,
                         double* F) {
  const track_ctx* ctx = (const track_ctx*)vctx;
  const int sa = ctx->surface_id[k - 1], sb = ctx->surface_id[k];
  int st = kfo_transport(ctx->center + 3 * sa, ctx->rot + 9 * sa, xf_prev,
                         ctx->center + 3 * sb, ctx->rot + 9 * sb, ctx->B,
                         ctx->mass, ctx->h_max, ctx->n_iter, xp, F, NULL);
  if (st) return st;
  sandwich6(F, Cf_prev, Cp);
  const double xx0 = ctx->x_over_x0[sb];
  if (xx0 > 0.0) {
    double n[3], T[3];
    rot_col(ctx->rot + 9 * sb, 2, n);
    T[0] = cos(xp[2]) * sin(xp[3]);
    T[1] = sin(xp[2]) * sin(xp[3]);
    T[2] = cos(xp[3]);
    const double th0 = kfo_highland(xp[4], ctx->mass, xx0, dot3(n, T));
    const double st_ = sin(xp[3]);
    Cp[2 * 6 + 2] += th0 * th0 / (st_ * st_);
    Cp[3 * 6 + 3] += th0 * th0;
  }
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
  track_ctx ctx = {surface_id, center, rot, x_over_x0, B, mass, h_max, n_iter};
  int st = filter_smooth(n, predict_track, &ctx, m, V, is_hole, xp, Cp, xf, Cf,
                         xs, Cs, F, chi2);
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
      st = kfo_fit_track(n, J->surface_id + o0, loc, cov, J->is_hole + o0, seed,
                         C0, J->n_surfaces, J->center, J->rot, J->x_over_x0,
                         J->B, J->mass, J->h_max, J->n_iter, xp, Cp, xf, Cf,
                         xs, Cs, F, chi2);
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
  if (n_tracks < 0 || t_begin < 0 || t_end > n_tracks || t_begin > t_end)
    return -1;
  if (n_threads < 1) n_threads = 1;
  batch_job base = {n_tracks, offsets, seed_params, seed_cov, n_surfaces,
                    center, rot, x_over_x0, n_states, surface_id, loc, cov,
                    is_hole, B, mass, h_max, n_iter, out_params, out_cov,
                    out_chi2, out_ndf, out_status, out_states, t_begin, t_end};
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
