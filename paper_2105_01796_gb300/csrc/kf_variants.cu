// kf_variants.cu -- FP64 kernel of the method variants the paper describes
// besides its baseline fit (arXiv 2105.01796), one track per thread, fused
// filter + smoother like the FP64 path:
//   * smoother by a backward Kalman filter (Sect. 2, Fig. 2): a second filter
//     runs from the last state to the first with its own RKN propagation,
//     and its prediction onto each state is combined with the forward
//     filter's state by the weighted mean;
//   * energy loss in the surface material (Sect. 1): the mean (Bethe) loss
//     moves q/p at every surface with material, its Jacobian factor enters
//     the transport, and a straggling variance is added to q/p;
//   * a position-dependent field given as a grid map (Sect. 4.3): the RKN
//     stages take the trilinearly interpolated field at their own points.
// Any combination of the three runs here; the baseline method keeps its own
// tuned FP64 and mixed kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_device.cuh"
#include "kf_fp64.cuh"
#include "kf_internal.h"

namespace kfgb {
namespace {
using namespace dev;

// ---------------------------------------------------------------------------
// field
// ---------------------------------------------------------------------------

// Field at r: the constant field, or the trilinear interpolation of the map's
// 8 grid points around r (r clamped onto the grid; every index stays inside
// [0, n-1], also for a non-finite r).
__device__ __forceinline__ void field_at(const FitParams& p, const double r[3], double B[3]) {
  if (p.map_b == nullptr) {
    B[0] = p.bfield[0];
    B[1] = p.bfield[1];
    B[2] = p.bfield[2];
    return;
  }
  int idx[3];
  double w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = p.map_n[a];
    double u = (r[a] - p.map_origin[a]) * p.map_inv_spacing[a];
    u = fmin(fmax(u, 0.0), (double)(n - 1));  // NaN -> 0
    int i = (int)u;
    i = i > n - 2 ? n - 2 : i;
    idx[a] = i;
    w[a] = u - (double)i;
  }
  const size_t sx = 3, sy_ = (size_t)p.map_n[0] * 3, sz = sy_ * (size_t)p.map_n[1];
  const double* base = p.map_b + (size_t)idx[2] * sz + (size_t)idx[1] * sy_ + (size_t)idx[0] * sx;
  B[0] = B[1] = B[2] = 0.0;
#pragma unroll
  for (int dl = 0; dl < 2; ++dl)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const double wt = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) * (dl ? w[2] : 1.0 - w[2]);
        const double* q = base + dl * sz + dj * sy_ + di * sx;
#pragma unroll
        for (int c = 0; c < 3; ++c) B[c] += wt * __ldg(q + c);
      }
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------------------
// RKN step with the field at the stage points
// ---------------------------------------------------------------------------

// free-state accumulators plus the varying columns of G = D J_bf
// (columns: 0 phi, 1 theta, 2 q/p)
struct GProp {
  double r[3], T[3], t, lam;
  double gr[3][3], gT[3][3], gtl;
};

// One 4-stage Nystrom step of length h:
//   k1 = a(r, T), k2 = a(r + h/2 T + h^2/8 k1, T + h/2 k1),
//   k3 = a(same point, T + h/2 k2), k4 = a(r + h T + h^2/2 k3, T + h k3),
//   a(r, T) = (q/p) kappa T x B(r),
//   r' = r + h T + h^2/6 (k1 + k2 + k3),  T' = T + h/6 (k1 + 2 k2 + 2 k3 + k4).
// G advances by the derivative of this map with the three stage fields held
// fixed (exact for a uniform field).
__device__ __forceinline__ void rkn_step_field(const FitParams& p, GProp& s, double h, double mass) {
  const double lk = s.lam * kKappa;
  double B1[3], B2[3], B4[3];
  double TB1[3], TB2[3], TB3[3], TB4[3];  // T_s x B_s
  double T2[3], T3[3], T4[3], pt[3];
  field_at(p, s.r, B1);
  cross3(s.T, B1, TB1);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T2[i] = s.T[i] + 0.5 * h * lk * TB1[i];
    pt[i] = s.r[i] + 0.5 * h * s.T[i] + h * h / 8.0 * lk * TB1[i];
  }
  field_at(p, pt, B2);
  cross3(T2, B2, TB2);
#pragma unroll
  for (int i = 0; i < 3; ++i) T3[i] = s.T[i] + 0.5 * h * lk * TB2[i];
  cross3(T3, B2, TB3);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T4[i] = s.T[i] + h * lk * TB3[i];
    pt[i] = s.r[i] + h * s.T[i] + 0.5 * h * h * lk * TB3[i];
  }
  field_at(p, pt, B4);
  cross3(T4, B4, TB4);
  // Jacobian columns
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double g[3] = {s.gT[0][c], s.gT[1][c], s.gT[2][c]};
    double d1[3], d2[3], d3[3], d4[3], v[3], x[3];
    cross3(g, B1, x);
#pragma unroll
    for (int i = 0; i < 3; ++i) d1[i] = lk * x[i] + (c == 2 ? kKappa * TB1[i] : 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = g[i] + 0.5 * h * d1[i];
    cross3(v, B2, x);
#pragma unroll
    for (int i = 0; i < 3; ++i) d2[i] = lk * x[i] + (c == 2 ? kKappa * TB2[i] : 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = g[i] + 0.5 * h * d2[i];
    cross3(v, B2, x);
#pragma unroll
    for (int i = 0; i < 3; ++i) d3[i] = lk * x[i] + (c == 2 ? kKappa * TB3[i] : 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = g[i] + h * d3[i];
    cross3(v, B4, x);
#pragma unroll
    for (int i = 0; i < 3; ++i) d4[i] = lk * x[i] + (c == 2 ? kKappa * TB4[i] : 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      s.gr[i][c] += h * g[i] + h * h / 6.0 * (d1[i] + d2[i] + d3[i]);
      s.gT[i][c] = g[i] + h / 6.0 * (d1[i] + 2.0 * d2[i] + 2.0 * d3[i] + d4[i]);
    }
  }
  const double g2 = 1.0 + mass * mass * s.lam * s.lam;
  const double igam = rsqrt_any(g2);
  const double gam = g2 * igam;
  s.gtl += h * mass * mass * s.lam * kInvC * igam;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.r[i] += h * s.T[i] + h * h / 6.0 * lk * (TB1[i] + TB2[i] + TB3[i]);
    s.T[i] += h / 6.0 * lk * (TB1[i] + 2.0 * TB2[i] + 2.0 * TB3[i] + TB4[i]);
  }
  s.t += h * gam * kInvC;
}

__device__ __forceinline__ bool plane_distance(const GProp& s, const Surf& sb, double& out) {
  const double d = sb.n(0) * (sb.c(0) - s.r[0]) + sb.n(1) * (sb.c(1) - s.r[1]) + sb.n(2) * (sb.c(2) - s.r[2]);
  const double nT = sb.n(0) * s.T[0] + sb.n(1) * s.T[1] + sb.n(2) * s.T[2];
  if (!(fabs(nT) > 1e-9)) return false;
  out = d * rcp_any(nT);
  return true;
}

// Transport x (bound, surface a) to surface b in either direction (the path
// length comes out negative when b lies behind): prediction xp, Jacobian J,
// sin(theta) and the incidence cosine at b.
__device__ __forceinline__ int transport_field(const FitParams& p, const Surf& sa, const Surf& sb,
                                               const double x[6], double xp[6], Jac<double>& J,
                                               double& sin_theta, double& cos_inc) {
  GProp s;
  double sp, cp, st, ct;
  sincos(x[2], &sp, &cp);
  sincos(x[3], &st, &ct);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.r[i] = sa.c(i) + x[0] * sa.u(i) + x[1] * sa.v(i);
  s.T[0] = cp * st;
  s.T[1] = sp * st;
  s.T[2] = ct;
  s.t = x[5];
  s.lam = x[4];
  s.gT[0][0] = -sp * st; s.gT[1][0] = cp * st; s.gT[2][0] = 0.0;
  s.gT[0][1] = cp * ct;  s.gT[1][1] = sp * ct; s.gT[2][1] = -st;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.gT[i][2] = 0.0;
    s.gr[i][0] = s.gr[i][1] = s.gr[i][2] = 0.0;
  }
  s.gtl = 0.0;
  const double mass = p.mass;
  double s0;
  if (!plane_distance(s, sb, s0)) return ST_NO_INTERSECTION;
  const double nsub_d = ceil(fabs(s0) / p.h_max);
  if (!(nsub_d <= 64.0)) return ST_NO_INTERSECTION;
  const int nsub = nsub_d < 1.0 ? 1 : (int)nsub_d;
  const double h = s0 / nsub;
  for (int k = 0; k < nsub; ++k) rkn_step_field(p, s, h, mass);
  for (int it = 0; it < p.n_iter; ++it) {
    double si;
    if (!plane_distance(s, sb, si)) return ST_NO_INTERSECTION;
    rkn_step_field(p, s, si, mass);
  }
  // end point: bound angles and the unit direction
  const double rho2 = s.T[0] * s.T[0] + s.T[1] * s.T[1];
  const double irho = rsqrt_any(rho2);
  const double rho = rho2 * irho;
  const double phi = atan2(s.T[1], s.T[0]);
  const double theta = atan2(rho, s.T[2]);
  const double tn2 = rho2 + s.T[2] * s.T[2];
  const double itn = rsqrt_any(tn2);
  const double tn = tn2 * itn;
  const double cph = s.T[0] * irho, sph = s.T[1] * irho;
  const double sth = rho * itn, cth = s.T[2] * itn;
  const double nT = sb.n(0) * s.T[0] + sb.n(1) * s.T[1] + sb.n(2) * s.T[2];
  // path correction with F' = (T, dt/ds, (q/p) kappa T x B(end), 0)
  double Be[3], TB[3];
  field_at(p, s.r, Be);
  cross3(s.T, Be, TB);
  const double lk = s.lam * kKappa;
  const double dtds = sqrt(1.0 + mass * mass * s.lam * s.lam) * kInvC;
  const double inv_nT = rcp_any(nT);
  double Gr[3][5], GT[3][5], Gt[5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gr[i][0] = sa.u(i);
    Gr[i][1] = sa.v(i);
    Gr[i][2] = s.gr[i][0];
    Gr[i][3] = s.gr[i][1];
    Gr[i][4] = s.gr[i][2];
    GT[i][0] = 0.0;
    GT[i][1] = 0.0;
    GT[i][2] = s.gT[i][0];
    GT[i][3] = s.gT[i][1];
    GT[i][4] = s.gT[i][2];
  }
  Gt[0] = Gt[1] = Gt[2] = Gt[3] = 0.0;
  Gt[4] = s.gtl;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const double w = -(sb.n(0) * Gr[0][c] + sb.n(1) * Gr[1][c] + sb.n(2) * Gr[2][c]) * inv_nT;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i][c] += s.T[i] * w;
      GT[i][c] += lk * TB[i] * w;
    }
    Gt[c] += dtds * w;
  }
  const double inv_sth = rcp_any(sth);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    J.f[0][c] = sb.u(0) * Gr[0][c] + sb.u(1) * Gr[1][c] + sb.u(2) * Gr[2][c];
    J.f[1][c] = sb.v(0) * Gr[0][c] + sb.v(1) * Gr[1][c] + sb.v(2) * Gr[2][c];
    J.f[2][c] = (-sph * GT[0][c] + cph * GT[1][c]) * inv_sth;
    J.f[3][c] = cph * cth * GT[0][c] + sph * cth * GT[1][c] - sth * GT[2][c];
    J.ft[c] = Gt[c];
  }
  const double d0 = s.r[0] - sb.c(0), d1 = s.r[1] - sb.c(1), d2 = s.r[2] - sb.c(2);
  xp[0] = d0 * sb.u(0) + d1 * sb.u(1) + d2 * sb.u(2);
  xp[1] = d0 * sb.v(0) + d1 * sb.v(1) + d2 * sb.v(2);
  xp[2] = phi;
  xp[3] = theta;
  xp[4] = s.lam;
  xp[5] = s.t;
  sin_theta = sth;
  cos_inc = nT / tn;
  return ST_OK;
}

// C <- G F C F^T G^T with F from J (row 4 = e4, column 5 = e5) and
// G = diag(1, 1, 1, 1, g, 1); the rows of Bm = G F C go to the record when
// ws is given (the RTS smoother reads them back).
__device__ __forceinline__ void cov_transport(const Jac<double>& J, double g, double C[21], const WS* ws, int k) {
  double Cp[21];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    double brow[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double v;
      if (a == 4) {
        v = g * C[sym(4, j)];
      } else {
        v = jf(J, a, 0) * C[sym(0, j)] + jf(J, a, 1) * C[sym(1, j)] + jf(J, a, 2) * C[sym(2, j)] +
            jf(J, a, 3) * C[sym(3, j)] + jf(J, a, 4) * C[sym(4, j)];
        if (a == 5) v += C[sym(5, j)];
      }
      brow[j] = v;
      if (ws) Rec<0>::put_bm(*ws, k, a * 6 + j, v);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (c <= a) {
        double v;
        if (c == 4) {
          v = g * brow[4];
        } else {
          v = brow[0] * jf(J, c, 0) + brow[1] * jf(J, c, 1) + brow[2] * jf(J, c, 2) + brow[3] * jf(J, c, 3) +
              brow[4] * jf(J, c, 4);
          if (c == 5) v += brow[5];
        }
        Cp[sy(a, c)] = v;
      }
  }
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = Cp[e];
}

// ---------------------------------------------------------------------------
// energy loss
// ---------------------------------------------------------------------------

// Sternheimer density effect, X = log10(beta gamma):
//   X >= x1: 2 ln10 X - Cbar;  x0 <= X < x1: that + a (x1 - X)^k;
//   X < x0: delta0 10^(2 (X - x0))
__device__ __forceinline__ double density_effect(const FitParams& p, double bg) {
  const double X = log10(bg);
  const double two_ln10 = 2.0 * 2.302585092994045684;
  const double cbar = p.mat[3], x0 = p.mat[4], x1 = p.mat[5], a = p.mat[6], k = p.mat[7], d0 = p.mat[8];
  if (X >= x1) return two_ln10 * X - cbar;
  if (X >= x0) return two_ln10 * X - cbar + a * pow(x1 - X, k);
  return d0 * pow(10.0, 2.0 * (X - x0));
}

constexpr double kBetheK = 0.307075e-3;  // 4 pi N_A r_e^2 m_e c^2, GeV cm^2/mol
constexpr double kMe = 0.51099895e-3;    // electron mass, GeV

// mean stopping power, GeV cm^2/g (Bethe with the density effect)
__device__ __forceinline__ double bethe(const FitParams& p, double bg, double mass) {
  const double b2 = bg * bg / (1.0 + bg * bg);
  const double gam = sqrt(1.0 + bg * bg);
  const double r = kMe / mass;
  const double wmax = 2.0 * kMe * bg * bg / (1.0 + 2.0 * gam * r + r * r);
  const double I = p.mat[1];
  const double arg = 2.0 * kMe * bg * bg * wmax / (I * I);
  return kBetheK * p.mat[0] / b2 * (0.5 * log(arg) - b2 - 0.5 * density_effect(p, bg));
}

// The mean loss through a surface (dir = +1) or its restoration (dir = -1),
// evaluated at the current momentum; thickness x/X0 * X0rho / cos.  qop
// changes, jac = (p^3 E')/(p'^3 E), var_down = (E_d/p_d^3)^2 sigma_E^2 on the
// downstream side with sigma_E = 4 xi / (2 sqrt(2 ln 2)) (the Gaussian of the
// Landau FWHM).  ST_NONFINITE if the particle stops.
__device__ __forceinline__ int energy_loss(const FitParams& p, double& qop, double xx0, double cos_inc, int dir,
                                           double& jac, double& var_down) {
  jac = 1.0;
  var_down = 0.0;
  const double mass = p.mass;
  const double thick = xx0 * p.mat[2] / fabs(cos_inc);
  const double pm = 1.0 / fabs(qop);
  const double E = sqrt(pm * pm + mass * mass);
  const double beta = pm / E;
  const double dE = bethe(p, pm / mass, mass) * thick;
  const double E2 = dir > 0 ? E - dE : E + dE;
  if (!(E2 > mass)) return ST_NONFINITE;
  const double p2 = sqrt(E2 * E2 - mass * mass);
  const double xi = 0.5 * kBetheK * p.mat[0] * thick / (beta * beta);
  const double sigE = 4.0 * xi / (2.0 * sqrt(2.0 * 0.693147180559945309));
  jac = (pm * pm * pm * E2) / (p2 * p2 * p2 * E);
  const double Ed = dir > 0 ? E2 : E, pd = dir > 0 ? p2 : pm;
  const double dqdE = Ed / (pd * pd * pd);
  var_down = dqdE * dqdE * sigE * sigE;
  qop = (qop > 0.0 ? 1.0 : -1.0) / p2;
  return ST_OK;
}

// multiple-scattering variances of (phi, theta) for a state with |q/p| = la
// crossing a surface of x/X0 = xx0 at incidence cos_inc
__device__ __forceinline__ void add_scattering(const FitParams& p, double la, double xx0, double cos_inc,
                                               double sin_th, double C[21]) {
  const double th0 = highland<double>(la, p.mass * p.mass, xx0, cos_inc);
  const double q = th0 * th0;
  C[sy(2, 2)] += q / (sin_th * sin_th);
  C[sy(3, 3)] += q;
}

// X = S^-1 B for SPD S (packed) and a symmetric right-hand side B (packed),
// through the Cholesky factor of the Jacobi-scaled D^-1/2 S D^-1/2; K = X^T.
__device__ __forceinline__ int spd_solve_sym(const double S[21], const double B[21], double X[6][6]) {
  double L[21];
  double id[6];  // 1 / sqrt(S_ii), the Jacobi scaling
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (!(S[sy(i, i)] > 0.0)) return ST_NON_SPD;
    id[i] = rsqrt_any(S[sy(i, i)]);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j <= i) L[sy(i, j)] = S[sy(i, j)] * (id[i] * id[j]);
  double idg[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double dj = L[sy(j, j)];
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (q < j) dj -= L[sy(j, q)] * L[sy(j, q)];
    if (!(dj > 0.0)) return ST_NON_SPD;
    idg[j] = rsqrt_any(dj);
    L[sy(j, j)] = dj * idg[j];
#pragma unroll
    for (int r = 0; r < 6; ++r)
      if (r > j) {
        double v = L[sy(r, j)];
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (q < j) v -= L[sy(r, q)] * L[sy(j, q)];
        L[sy(r, j)] = v * idg[j];
      }
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double y[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double v = B[sym(r, c)] * id[r];
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (q < r) v -= L[sy(r, q)] * y[q];
      y[r] = v * idg[r];
    }
    double z[6];
#pragma unroll
    for (int r = 5; r >= 0; --r) {
      double v = y[r];
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (q > r) v -= L[sy(q, r)] * z[q];
      z[r] = v * idg[r];
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) X[r][c] = z[r] * id[r];
  }
  return ST_OK;
}

// ---------------------------------------------------------------------------
// the fused fit
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fit_one_variants(const FitParams& p, const double* s_surf, int i) {
  const int t = track_of(p, i);
  const size_t TT = (size_t)p.n_tracks_total;
  const WS ws{p.ws64, p.ws32, (size_t)p.n_tracks, kRec64Fp64, 0, i};
  const int64_t o0 = p.offsets[t], o1 = p.offsets[t + 1];
  const int n = (int)(o1 - o0);
  int status = ST_OK;
  if (!(o1 > o0) || o0 < 0 || o1 > p.n_states || n > p.max_states) status = ST_BAD_INPUT;
  if (status == ST_OK)
    for (int k = 0; k < n; ++k) {
      const int sid = p.surface_id[o0 + k];
      if (sid < 0 || sid >= p.n_surfaces) status = ST_BAD_INPUT;
    }
  double xs[6], Cs[21];
  double chi2sum = 0.0;
  int nmeas = 0;
  if (status == ST_OK) {
    // ------------------------------------------------ forward filter
    double x[6], C[21];
#pragma unroll
    for (int e = 0; e < 6; ++e) x[e] = p.seed_params[e * TT + t];
#pragma unroll
    for (int e = 0; e < 21; ++e) C[e] = p.seed_cov[e * TT + t];
    int sid_prev = p.surface_id[o0];
    for (int k = 0; k < n && status == ST_OK; ++k) {
      const int sid = p.surface_id[o0 + k];
      double xp[6];
      if (k == 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) xp[e] = x[e];
      } else {
        const Surf sa{s_surf + sid_prev * kSurfStride}, sb{s_surf + sid * kSurfStride};
        Jac<double> J;
        double sin_th, cos_inc;
        status = transport_field(p, sa, sb, x, xp, J, sin_th, cos_inc);
        if (status != ST_OK) break;
        // material of surface k (before the update): scattering with the
        // arriving momentum, then the mean loss and its straggling
        const double xx0 = sb.xx0();
        const double la = fabs(xp[4]);
        double g = 1.0, var_q = 0.0;
        if (p.energy_loss && xx0 > 0.0) {
          status = energy_loss(p, xp[4], xx0, cos_inc, +1, g, var_q);
          if (status != ST_OK) break;
        }
        cov_transport(J, g, C, &ws, k);
        if (xx0 > 0.0) add_scattering(p, la, xx0, cos_inc, sin_th, C);
        C[sy(4, 4)] += var_q;
      }
      // record the prediction (C now holds Cp)
#pragma unroll
      for (int e = 0; e < 6; ++e) ws.d(k, Rec<0>::XP + e) = xp[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) ws.d(k, Rec<0>::CP + e) = C[e];
      if (!p.is_hole[o0 + k]) {
        const double m[2] = {p.loc[o0 + k], p.loc[p.n_states + o0 + k]};
        const double V[3] = {p.cov[o0 + k], p.cov[p.n_states + o0 + k], p.cov[2 * p.n_states + o0 + k]};
        double c2 = 0.0, Cu[21];
        status = kalman_update<double>(xp, C, m, V, x, Cu, c2);
        if (status != ST_OK) break;
#pragma unroll
        for (int e = 0; e < 21; ++e) C[e] = Cu[e];
        chi2sum += c2;
        ++nmeas;
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) x[e] = xp[e];
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) ws.d(k, Rec<0>::XF + e) = x[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) Rec<0>::put_cf(ws, k, e, C[e]);
      sid_prev = sid;
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) xs[e] = x[e];
#pragma unroll
    for (int e = 0; e < 21; ++e) Cs[e] = C[e];

    if (status == ST_OK && p.smoother == 0) {
      // ------------------------------------------------ RTS smoother
      status = rts_smooth_fp64(ws, n, xs, Cs, p.out_states, p.n_states, o0);
    } else if (status == ST_OK) {
      // ------------------------------------------------ backward filter
      // starts at the last state from the forward-filtered parameters with
      // bf_scale times their covariance; the last state keeps the forward
      // filtered state
      if (p.out_states)
#pragma unroll
        for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + n - 1] = x[e];
      double xb[6], Cb[21];
#pragma unroll
      for (int e = 0; e < 6; ++e) xb[e] = x[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) Cb[e] = p.bf_scale * C[e];
      for (int k = n - 1; k >= 1 && status == ST_OK; --k) {
        if (!p.is_hole[o0 + k]) {
          const double m[2] = {p.loc[o0 + k], p.loc[p.n_states + o0 + k]};
          const double V[3] = {p.cov[o0 + k], p.cov[p.n_states + o0 + k], p.cov[2 * p.n_states + o0 + k]};
          double c2, xu[6], Cu[21];
          status = kalman_update<double>(xb, Cb, m, V, xu, Cu, c2);
          if (status != ST_OK) break;
#pragma unroll
          for (int e = 0; e < 6; ++e) xb[e] = xu[e];
#pragma unroll
          for (int e = 0; e < 21; ++e) Cb[e] = Cu[e];
        }
        // material of surface k at the backward state: its scattering noise,
        // then the mean loss restored (straggling on the downstream side)
        const Surf sk{s_surf + p.surface_id[o0 + k] * kSurfStride};
        const Surf sj{s_surf + p.surface_id[o0 + k - 1] * kSurfStride};
        const double xx0 = sk.xx0();
        if (xx0 > 0.0) {
          double sp, cp, st, ct;
          sincos(xb[2], &sp, &cp);
          sincos(xb[3], &st, &ct);
          const double cos_inc = sk.n(0) * cp * st + sk.n(1) * sp * st + sk.n(2) * ct;
          add_scattering(p, fabs(xb[4]), xx0, cos_inc, st, Cb);
          if (p.energy_loss) {
            double g, var_q;
            status = energy_loss(p, xb[4], xx0, cos_inc, -1, g, var_q);
            if (status != ST_OK) break;
            Cb[sy(4, 4)] += var_q;
#pragma unroll
            for (int j = 0; j < 6; ++j) Cb[sym(4, j)] *= g;
            Cb[sy(4, 4)] *= g;
          }
        }
        // back-propagation to surface k-1
        Jac<double> J;
        double xo[6], sin_th, cos_inc;
        status = transport_field(p, sk, sj, xb, xo, J, sin_th, cos_inc);
        if (status != ST_OK) break;
        cov_transport(J, 1.0, Cb, nullptr, 0);
#pragma unroll
        for (int e = 0; e < 6; ++e) xb[e] = xo[e];
        // weighted mean with the forward-filtered state k-1:
        //   K = Cf (Cf + Cb)^-1, xs = xf + K (xb - xf), Cs = Cf - K Cf
        double Cf[21], Ssum[21], xf[6];
#pragma unroll
        for (int e = 0; e < 21; ++e) {
          Cf[e] = Rec<0>::get_cf(ws, k - 1, e);
          Ssum[e] = Cf[e] + Cb[e];
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) xf[e] = ws.d(k - 1, Rec<0>::XF + e);
        double X[6][6];  // (Cf + Cb)^-1 Cf = K^T
        status = spd_solve_sym(Ssum, Cf, X);
        if (status != ST_OK) break;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q < 6; ++q) acc += X[q][r] * (xb[q] - xf[q]);
          xs[r] = xf[r] + acc;
        }
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
          for (int c = 0; c < 6; ++c)
            if (c <= r) {
              double acc = 0.0;
#pragma unroll
              for (int q = 0; q < 6; ++q) acc += X[q][r] * Cf[sym(q, c)];
              Cs[sy(r, c)] = Cf[sy(r, c)] - acc;
            }
        if (p.out_states)
#pragma unroll
          for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + k - 1] = xs[e];
      }
    }
    if (status == ST_OK) {
      bool fin = isfinite(chi2sum);
#pragma unroll
      for (int e = 0; e < 6; ++e) fin = fin && isfinite(xs[e]);
#pragma unroll
      for (int e = 0; e < 21; ++e) fin = fin && isfinite(Cs[e]);
      if (!fin) status = ST_NONFINITE;
    }
  }
  if (status != ST_OK) {
    const double nan = qnan();
#pragma unroll
    for (int e = 0; e < 6; ++e) xs[e] = nan;
#pragma unroll
    for (int e = 0; e < 21; ++e) Cs[e] = nan;
    chi2sum = nan;
    nmeas = 0;
    if (p.out_states && n >= 1 && o0 >= 0 && o1 <= p.n_states && n <= p.max_states)
      for (int k = 0; k < n; ++k)
        for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + k] = nan;
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) p.out_params[e * TT + t] = xs[e];
#pragma unroll
  for (int e = 0; e < 21; ++e) p.out_cov[e * TT + t] = Cs[e];
  p.out_chi2[t] = chi2sum;
  if (p.out_ndf) p.out_ndf[t] = 2 * nmeas;
  if (p.out_status) p.out_status[t] = (uint8_t)status;
}

struct VariantBody {
  static constexpr int kStride = kSurfStride;
  static __device__ __forceinline__ void run(const FitParams& p, const double* s_surf, int i) {
    fit_one_variants(p, s_surf, i);
  }
};

}  // namespace

cudaError_t launch_fit_variants(const FitParams& p, int block, cudaStream_t stream, int* launched) {
  if (launched) *launched = 0;
  if (p.n_tracks <= 0) return cudaSuccess;
  return dev::launch_body<VariantBody, 1>(p, block ? block : 128, stream, launched);
}

}  // namespace kfgb
