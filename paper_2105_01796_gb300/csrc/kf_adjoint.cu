// kf_adjoint.cu -- gradients of the summed chi2 of the Kalman fit with
// respect to per-surface alignment parameters and the seed parameters.
//
// Objective: L = sum_t w_t sum_k chi2_{t,k}, chi2_k = r_k^T S_k^-1 r_k of the
// predicted residual (paper Sect. 2 filter step list; the chi2 quality
// metric of the smoother paragraph).  chi2 depends only on the forward
// filter, so the smoother contributes nothing to this gradient.
//
// Method (reverse mode over the states, forward mode inside one transport):
//   forward:  FP64 filter; (x_f, C_f) checkpointed every kSeg states.
//   backward: for each segment, last first, recompute its filtered states
//     from the checkpoint; then for k = last .. 1 of the segment
//       1. recompute the transport k-1 -> k (x_p, F, Q) and C_p = F C_f F^T + Q
//       2. reverse through chi2_k and the gain-matrix update (exact algebra):
//          adjoints of (x_f,k, C_f,k) -> adjoints of (x_p,k, C_p,k)
//       3. reverse through C_p = F C_f F^T + Q: Lambda_Cf = F^T Lambda_Cp F,
//          lambda_F = 2 Lambda_Cp F C_f, lambda_Q = Lambda_Cp
//       4. the transport's sensitivities to the 18 inputs it depends on
//          (x_f,k-1; the alignment of surfaces k-1 and k) by dual numbers
//          carrying two tangent directions per pass (9 passes), contracted at
//          once with (lambda_xp, lambda_F, lambda_Q): this includes the
//          derivative of F itself.
//     state 0: reverse through its update; x_p,0 is the seed.
// Alignment of a surface (shifts along its local axes, then rotations about
// them):  c' = c + R (du, dv, dn),  R' = R Ru(alpha) Rv(beta) Rn(gamma).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_device.cuh"
#include "kf_internal.h"

namespace kfgb {
namespace {
using namespace dev;

constexpr int kSeg = 8;  // states per checkpoint segment (about sqrt(n) for n ~ 30-60)

// ---------------------------------------------------------------------------
// dual numbers: value + N directional derivatives (forward-mode AD)
// ---------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  __device__ Dual() {}
  __device__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};

template <int N> __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> __device__ __forceinline__ Dual<N> operator+(double b, const Dual<N>& a) { return a + b; }
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> __device__ __forceinline__ Dual<N> operator-(double b, const Dual<N>& a) { return (-a) + b; }
template <int N> __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N> __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> __device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> __device__ __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> __device__ __forceinline__ Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }

template <int N> __device__ __forceinline__ Dual<N> chain(const Dual<N>& a, double f, double df) {
  Dual<N> r; r.v = f;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> sqrt(const Dual<N>& a) {
  const double s = ::sqrt(a.v);
  return chain(a, s, 0.5 / s);
}
template <int N> __device__ __forceinline__ Dual<N> sin(const Dual<N>& a) { return chain(a, ::sin(a.v), ::cos(a.v)); }
template <int N> __device__ __forceinline__ Dual<N> cos(const Dual<N>& a) { return chain(a, ::cos(a.v), -::sin(a.v)); }
template <int N> __device__ __forceinline__ Dual<N> log(const Dual<N>& a) { return chain(a, ::log(a.v), 1.0 / a.v); }
template <int N> __device__ __forceinline__ Dual<N> fabs(const Dual<N>& a) { return a.v < 0.0 ? -a : a; }
template <int N> __device__ __forceinline__ Dual<N> atan2(const Dual<N>& y, const Dual<N>& x) {
  Dual<N> r; r.v = ::atan2(y.v, x.v);
  const double id = 1.0 / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) * id;
  return r;
}
// the double overloads stay visible next to the Dual templates
using ::atan2;
using ::cos;
using ::fabs;
using ::log;
using ::sin;
using ::sqrt;

__device__ __forceinline__ double val(double x) { return x; }
template <int N> __device__ __forceinline__ double val(const Dual<N>& x) { return x.v; }

// ---------------------------------------------------------------------------
// geometry with alignment
// ---------------------------------------------------------------------------
template <class S>
struct Plane {
  S c[3];
  S R[9];  // row-major, columns u, v, n
  __device__ const S& u(int i) const { return R[3 * i + 0]; }
  __device__ const S& v(int i) const { return R[3 * i + 1]; }
  __device__ const S& n(int i) const { return R[3 * i + 2]; }
};

// c' = c + R (du, dv, dn); R' = R Ru(alpha) Rv(beta) Rn(gamma)
template <class S>
__device__ __forceinline__ Plane<S> aligned_plane(const Surf& s, const S a[6]) {
  Plane<S> p;
#pragma unroll
  for (int i = 0; i < 3; ++i) p.c[i] = s.c(i) + s.R(i, 0) * a[0] + s.R(i, 1) * a[1] + s.R(i, 2) * a[2];
  const S ca = cos(a[3]), sa = sin(a[3]), cb = cos(a[4]), sb = sin(a[4]), cg = cos(a[5]), sg = sin(a[5]);
  // M = Ru Rv Rn
  S M[9];
  // Ru = [[1,0,0],[0,ca,-sa],[0,sa,ca]], Rv = [[cb,0,sb],[0,1,0],[-sb,0,cb]], Rn = [[cg,-sg,0],[sg,cg,0],[0,0,1]]
  // Rv Rn:
  const S vn[9] = {cb * cg, -(cb * sg), sb, sg, cg, S(0.0), -(sb * cg), sb * sg, cb};
  // Ru (Rv Rn):
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    M[0 * 3 + j] = vn[0 * 3 + j];
    M[1 * 3 + j] = ca * vn[1 * 3 + j] - sa * vn[2 * 3 + j];
    M[2 * 3 + j] = sa * vn[1 * 3 + j] + ca * vn[2 * 3 + j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) p.R[3 * i + j] = s.R(i, 0) * M[0 * 3 + j] + s.R(i, 1) * M[1 * 3 + j] + s.R(i, 2) * M[2 * 3 + j];
  return p;
}

// ---------------------------------------------------------------------------
// the transport, generic in the scalar type (double or Dual<N>); same
// arithmetic as the FP64 fit kernel
// ---------------------------------------------------------------------------
template <class S>
struct PropS {
  S r[3], T[3], t, lam;
  S gr[3][3], gT[3][3], gtl;
};

template <class S>
__device__ __forceinline__ void crossB(const S v[3], const double B[3], const S& lk, S out[3]) {
  out[0] = (v[1] * B[2] - v[2] * B[1]) * lk;
  out[1] = (v[2] * B[0] - v[0] * B[2]) * lk;
  out[2] = (v[0] * B[1] - v[1] * B[0]) * lk;
}

template <class S>
__device__ __forceinline__ void rkn_step_s(PropS<S>& s, const S& h, const double B[3], double mass) {
  const S h2 = h * h * 0.5, h3 = h * h * h * (1.0 / 6.0), h4 = h * h * h * h * (1.0 / 24.0);
  const S lk = s.lam * kKappa;
  const S one(1.0);
  S a1[3], a2[3], a3[3], a4[3];
  crossB(s.T, B, lk, a1);
  crossB(a1, B, lk, a2);
  crossB(a2, B, lk, a3);
  crossB(a3, B, lk, a4);
  S u0[3], u1[3], u2[3], u3[3];
  crossB(s.T, B, S(kKappa), u0);
  crossB(u0, B, lk, u1);
  crossB(u1, B, lk, u2);
  crossB(u2, B, lk, u3);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const S g[3] = {s.gT[0][c], s.gT[1][c], s.gT[2][c]};
    S b1[3], b2[3], b3[3], b4[3];
    crossB(g, B, lk, b1);
    crossB(b1, B, lk, b2);
    crossB(b2, B, lk, b3);
    crossB(b3, B, lk, b4);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S dr = h * g[i] + h2 * b1[i] + h3 * b2[i] + h4 * b3[i];
      S nt = g[i] + h * b1[i] + h2 * b2[i] + h3 * b3[i] + h4 * b4[i];
      if (c == 2) {
        dr += h2 * u0[i] + h * h * h * (1.0 / 3.0) * u1[i] + h * h * h * h * 0.125 * u2[i];
        nt += h * u0[i] + h * h * u1[i] + h * h * h * 0.5 * u2[i] + h * h * h * h * (1.0 / 6.0) * u3[i];
      }
      s.gr[i][c] += dr;
      s.gT[i][c] = nt;
    }
  }
  const S gam = sqrt(one + s.lam * s.lam * (mass * mass));
  s.gtl += h * (s.lam * (mass * mass * kInvC)) / gam;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.r[i] = s.r[i] + h * s.T[i] + (h2 * a1[i] + h3 * a2[i] + h4 * a3[i]);
    s.T[i] = s.T[i] + (h * a1[i] + h2 * a2[i] + h3 * a3[i] + h4 * a4[i]);
  }
  s.t = s.t + h * gam * kInvC;
}

template <class S>
struct JacS {
  S f[4][5];  // rows loc0, loc1, phi, theta over columns loc0..q/p
  S ft[5];    // time row
};

// transport x on plane a to plane b; also the Highland variances of b
template <class S>
__device__ int transport_s(const Plane<S>& pa, const Plane<S>& pb, const S x[6], const double B[3], double mass,
                           double h_max, int n_iter, double xx0, S xp[6], JacS<S>& J, S& qphi, S& qth) {
  PropS<S> s;
  const S sp = sin(x[2]), cp = cos(x[2]), st = sin(x[3]), ct = cos(x[3]);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.r[i] = pa.c[i] + x[0] * pa.u(i) + x[1] * pa.v(i);
  s.T[0] = cp * st;
  s.T[1] = sp * st;
  s.T[2] = ct;
  s.t = x[5];
  s.lam = x[4];
  s.gT[0][0] = -(sp * st); s.gT[1][0] = cp * st; s.gT[2][0] = S(0.0);
  s.gT[0][1] = cp * ct;    s.gT[1][1] = sp * ct; s.gT[2][1] = -st;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.gT[i][2] = S(0.0);
    s.gr[i][0] = S(0.0);
    s.gr[i][1] = S(0.0);
    s.gr[i][2] = S(0.0);
  }
  s.gtl = S(0.0);
  auto dist = [&](S& out) -> bool {
    const S d = pb.n(0) * (pb.c[0] - s.r[0]) + pb.n(1) * (pb.c[1] - s.r[1]) + pb.n(2) * (pb.c[2] - s.r[2]);
    const S nT = pb.n(0) * s.T[0] + pb.n(1) * s.T[1] + pb.n(2) * s.T[2];
    if (!(::fabs(val(nT)) > 1e-9)) return false;
    out = d / nT;
    return true;
  };
  S s0;
  if (!dist(s0)) return ST_NO_INTERSECTION;
  const double nsub_d = ::ceil(::fabs(val(s0)) / h_max);
  if (!(nsub_d <= 64.0)) return ST_NO_INTERSECTION;
  const int nsub = nsub_d < 1.0 ? 1 : (int)nsub_d;
  const S h = s0 / (double)nsub;
  for (int k = 0; k < nsub; ++k) rkn_step_s(s, h, B, mass);
  for (int it = 0; it < n_iter; ++it) {
    S si;
    if (!dist(si)) return ST_NO_INTERSECTION;
    rkn_step_s(s, si, B, mass);
  }
  const S rho2 = s.T[0] * s.T[0] + s.T[1] * s.T[1];
  const S phi = atan2(s.T[1], s.T[0]);
  const S rho = sqrt(rho2);
  const S theta = atan2(rho, s.T[2]);
  const S tn = sqrt(rho2 + s.T[2] * s.T[2]);
  const S cph = s.T[0] / rho, sph = s.T[1] / rho, sth = rho / tn, cth = s.T[2] / tn;
  const S nT = pb.n(0) * s.T[0] + pb.n(1) * s.T[1] + pb.n(2) * s.T[2];
  // path correction
  const S lk = s.lam * kKappa;
  S AT[3];
  crossB(s.T, B, lk, AT);
  const S dtds = sqrt(S(1.0) + s.lam * s.lam * (mass * mass)) * kInvC;
  S Gr[3][5], GT[3][5], Gt[5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gr[i][0] = pa.u(i);
    Gr[i][1] = pa.v(i);
    Gr[i][2] = s.gr[i][0];
    Gr[i][3] = s.gr[i][1];
    Gr[i][4] = s.gr[i][2];
    GT[i][0] = S(0.0);
    GT[i][1] = S(0.0);
    GT[i][2] = s.gT[i][0];
    GT[i][3] = s.gT[i][1];
    GT[i][4] = s.gT[i][2];
  }
  Gt[0] = S(0.0); Gt[1] = S(0.0); Gt[2] = S(0.0); Gt[3] = S(0.0);
  Gt[4] = s.gtl;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const S w = -(pb.n(0) * Gr[0][c] + pb.n(1) * Gr[1][c] + pb.n(2) * Gr[2][c]) / nT;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i][c] += s.T[i] * w;
      GT[i][c] += AT[i] * w;
    }
    Gt[c] += dtds * w;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    J.f[0][c] = pb.u(0) * Gr[0][c] + pb.u(1) * Gr[1][c] + pb.u(2) * Gr[2][c];
    J.f[1][c] = pb.v(0) * Gr[0][c] + pb.v(1) * Gr[1][c] + pb.v(2) * Gr[2][c];
    J.f[2][c] = (cph * GT[1][c] - sph * GT[0][c]) / sth;
    J.f[3][c] = cph * cth * GT[0][c] + sph * cth * GT[1][c] - sth * GT[2][c];
    J.ft[c] = Gt[c];
  }
  const S d0 = s.r[0] - pb.c[0], d1 = s.r[1] - pb.c[1], d2 = s.r[2] - pb.c[2];
  xp[0] = d0 * pb.u(0) + d1 * pb.u(1) + d2 * pb.u(2);
  xp[1] = d0 * pb.v(0) + d1 * pb.v(1) + d2 * pb.v(2);
  xp[2] = phi;
  xp[3] = theta;
  xp[4] = s.lam;
  xp[5] = s.t;
  // multiple scattering at b (Highland, unit direction of the prediction)
  if (xx0 > 0.0) {
    const S l = fabs(s.lam);
    const S g2 = S(1.0) + l * l * (mass * mass);
    const S eps = xx0 / fabs(nT / tn);
    const S th0 = 0.0136 * l * sqrt(g2) * sqrt(eps) * (1.0 + 0.038 * log(eps * g2));
    qth = th0 * th0;
    qphi = qth / (sth * sth);
  } else {
    qth = S(0.0);
    qphi = S(0.0);
  }
  return ST_OK;
}

// F as a dense 6x6 (row 4 = e4, column 5 = e5)
__device__ __forceinline__ void dense_F(const JacS<double>& J, double F[6][6]) {
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double v = 0.0;
      if (r < 4 && c < 5) v = J.f[r][c];
      if (r == 5 && c < 5) v = J.ft[c];
      if (r == c && (r == 4 || r == 5)) v = 1.0;
      F[r][c] = v;
    }
}

// gain-matrix update (FP64, Joseph form as in the fit kernels)
__device__ __forceinline__ int update_fwd(const double xp[6], const double Cp[21], const double m[2],
                                          const double V[3], double xf[6], double Cf[21], double& chi2) {
  const double S00 = V[0] + Cp[sy(0, 0)], S01 = V[1] + Cp[sy(1, 0)], S11 = V[2] + Cp[sy(1, 1)];
  const double det = S00 * S11 - S01 * S01;
  if (!(det > 0.0) || !(S00 > 0.0)) return ST_NON_SPD;
  const double idet = 1.0 / det;
  const double r0 = m[0] - xp[0], r1 = m[1] - xp[1];
  chi2 = (S11 * r0 * r0 - 2.0 * S01 * r0 * r1 + S00 * r1 * r1) * idet;
  const double i00 = S11 * idet, i01 = -S01 * idet, i11 = S00 * idet;
  double K[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double c0 = Cp[sym(i, 0)], c1 = Cp[sym(i, 1)];
    K[i][0] = c0 * i00 + c1 * i01;
    K[i][1] = c0 * i01 + c1 * i11;
    xf[i] = xp[i] + K[i][0] * r0 + K[i][1] * r1;
  }
  double W[2][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    W[0][j] = S00 * K[j][0] + S01 * K[j][1] - Cp[sym(0, j)];
    W[1][j] = S01 * K[j][0] + S11 * K[j][1] - Cp[sym(1, j)];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j <= i)
        Cf[sy(i, j)] = Cp[sy(i, j)] + K[i][0] * W[0][j] + K[i][1] * W[1][j] - Cp[sym(0, i)] * K[j][0] -
                       Cp[sym(1, i)] * K[j][1];
  return ST_OK;
}

// Reverse through one measured update (exact arithmetic of the update):
//   P = Cp H^T, S = V + H Cp H^T, Si = S^-1, K = P Si, r = m - H xp,
//   xf = xp + K r, Cf = Cp - P Si P^T, chi2 = r^T Si r (weight w).
// In: lf, Lf (adjoints of xf, Cf; Lf symmetric, full-matrix convention).
// Out: lp, Lp (adjoints of xp, Cp), Lp symmetric.
__device__ void update_adj(const double xp[6], const double Cp[21], const double m[2], const double V[3], double w,
                           const double lf[6], const double Lf[6][6], double lp[6], double Lp[6][6]) {
  const double S00 = V[0] + Cp[sy(0, 0)], S01 = V[1] + Cp[sy(1, 0)], S11 = V[2] + Cp[sy(1, 1)];
  const double idet = 1.0 / (S00 * S11 - S01 * S01);
  const double Si[2][2] = {{S11 * idet, -S01 * idet}, {-S01 * idet, S00 * idet}};
  const double r[2] = {m[0] - xp[0], m[1] - xp[1]};
  double P[6][2], K[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    P[i][0] = Cp[sym(i, 0)];
    P[i][1] = Cp[sym(i, 1)];
    K[i][0] = P[i][0] * Si[0][0] + P[i][1] * Si[1][0];
    K[i][1] = P[i][0] * Si[0][1] + P[i][1] * Si[1][1];
  }
  // lambda_r = K^T lf + 2 w Si r
  double lr[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    double v = 2.0 * w * (Si[a][0] * r[0] + Si[a][1] * r[1]);
#pragma unroll
    for (int i = 0; i < 6; ++i) v += K[i][a] * lf[i];
    lr[a] = v;
  }
  // lambda_K = lf r^T; lambda_P = lambda_K Si - 2 Lf P Si
  double lP[6][2];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double LfP[2] = {0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      LfP[0] += Lf[i][j] * P[j][0];
      LfP[1] += Lf[i][j] * P[j][1];
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const double lK0 = lf[i] * r[0], lK1 = lf[i] * r[1];
      lP[i][b] = lK0 * Si[0][b] + lK1 * Si[1][b] - 2.0 * (LfP[0] * Si[0][b] + LfP[1] * Si[1][b]);
    }
  }
  // Lambda_Si = w r r^T + P^T lambda_K - P^T Lf P  (then symmetrised)
  double LSi[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      double v = w * r[a] * r[b];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        v += P[i][a] * lf[i] * r[b];
        double LfPb = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) LfPb += Lf[i][j] * P[j][b];
        v -= P[i][a] * LfPb;
      }
      LSi[a][b] = v;
    }
  const double s01 = 0.5 * (LSi[0][1] + LSi[1][0]);
  LSi[0][1] = s01;
  LSi[1][0] = s01;
  // Lambda_S = -Si LSi Si
  double T2[2][2], LS[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) T2[a][b] = LSi[a][0] * Si[0][b] + LSi[a][1] * Si[1][b];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) LS[a][b] = -(Si[a][0] * T2[0][b] + Si[a][1] * T2[1][b]);
  // assemble Lp = Lf + lambda_P H (columns 0,1) + Lambda_S (block 0:2), symmetrised
  double L[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double v = Lf[i][j];
      if (j < 2) v += lP[i][j];
      if (i < 2 && j < 2) v += LS[i][j];
      L[i][j] = v;
    }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) Lp[i][j] = 0.5 * (L[i][j] + L[j][i]);
  // lp = lf - H^T lambda_r
#pragma unroll
  for (int i = 0; i < 6; ++i) lp[i] = lf[i] - (i < 2 ? lr[i] : 0.0);
}

struct GradParams {
  FitParams f;          // geometry, inputs, options (outputs unused)
  const double* align;  // [6][S] or null (zero alignment)
  const double* dl_dchi2;  // [T] or null (all ones)
  double* chi2;         // [T] or null
  double* grad_seed;    // [6][T] or null
  double* grad_align;   // [6][S] or null (accumulated with atomicAdd; zeroed by the host)
  double* ckpt;         // [n_ckpt][27][T]
  int32_t n_ckpt;
};

template <class S>
__device__ __forceinline__ void load_align(const GradParams& g, int sid, S a[6]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) a[e] = S(g.align ? g.align[(size_t)e * g.f.n_surfaces + sid] : 0.0);
}

// values of the transport k-1 -> k with the aligned planes
__device__ __forceinline__ int transport_values(const GradParams& g, const double* s_surf, int sa, int sb,
                                                const double x[6], double xp[6], JacS<double>& J, double& qp,
                                                double& qt) {
  double aa[6], ab[6];
  load_align(g, sa, aa);
  load_align(g, sb, ab);
  const Plane<double> pa = aligned_plane<double>(Surf{s_surf + sa * kSurfStride}, aa);
  const Plane<double> pb = aligned_plane<double>(Surf{s_surf + sb * kSurfStride}, ab);
  const double B[3] = {g.f.bfield[0], g.f.bfield[1], g.f.bfield[2]};
  return transport_s<double>(pa, pb, x, B, g.f.mass, g.f.h_max, g.f.n_iter,
                             Surf{s_surf + sb * kSurfStride}.xx0(), xp, J, qp, qt);
}

__device__ __forceinline__ void cov_transport(const double F[6][6], const double Cf[21], double qp, double qt,
                                              double Cp[21]) {
  double FC[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += F[i][q] * Cf[sym(q, j)];
      FC[i][j] = v;
    }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j <= i) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += FC[i][q] * F[j][q];
        Cp[sy(i, j)] = v;
      }
  Cp[sy(2, 2)] += qp;
  Cp[sy(3, 3)] += qt;
}

// add v to grad_align[e][sid] (all 32 lanes of the warp call this together;
// inactive lanes pass act = false).  When every active lane is on the same
// surface the warp adds its sum once; otherwise each active lane adds.
__device__ __forceinline__ void add_align_grad(double* grad, int n_surf, int sid, int e, double v, bool act) {
  const unsigned full = 0xffffffffu;
  const unsigned any = __ballot_sync(full, act);
  if (any == 0u) return;
  const int lead = __ffs(any) - 1;
  const int sid0 = __shfl_sync(full, sid, lead);
  if (__all_sync(full, !act || sid == sid0)) {
    double sum = act ? v : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(full, sum, o);
    if ((int)(threadIdx.x & 31) == lead) atomicAdd(&grad[(size_t)e * n_surf + sid0], sum);
  } else if (act) {
    atomicAdd(&grad[(size_t)e * n_surf + sid], v);
  }
}

__global__ void __launch_bounds__(128) kf_grad_kernel(const GradParams g) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* s_surf = reinterpret_cast<double*>(smem_raw);
  __shared__ __align__(8) uint64_t s_mbar;
  const FitParams& p = g.f;
  const bool staged = stage_surfaces(s_surf, p.surf, (uint32_t)(p.n_surfaces * kSurfStride * 8), &s_mbar,
                                     p.error_flag);
  if (!staged) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in_range = t < p.n_tracks;
  const int tt = in_range ? t : 0;
  const size_t TT = (size_t)p.n_tracks;
  const int64_t o0 = p.offsets[tt], o1 = p.offsets[tt + 1];
  const int n = (int)(o1 - o0);
  int status = in_range ? ST_OK : ST_BAD_INPUT;
  if (!(o1 > o0) || o0 < 0 || o1 > p.n_states || n > p.max_states) status = ST_BAD_INPUT;
  if (status == ST_OK)
    for (int k = 0; k < n; ++k) {
      const int sid = p.surface_id[o0 + k];
      if (sid < 0 || sid >= p.n_surfaces) status = ST_BAD_INPUT;
    }
  const double w = (g.dl_dchi2 && in_range) ? g.dl_dchi2[tt] : 1.0;
  auto ck = [&](int j, int e) -> double& { return g.ckpt[((size_t)j * 27 + e) * TT + tt]; };
  auto meas = [&](int k, double m[2], double V[3]) {
    m[0] = p.loc[o0 + k];
    m[1] = p.loc[p.n_states + o0 + k];
    V[0] = p.cov[o0 + k];
    V[1] = p.cov[p.n_states + o0 + k];
    V[2] = p.cov[2 * p.n_states + o0 + k];
  };

  // ---------------------------------------------------------- forward
  double chi2sum = 0.0;
  double x[6], C[21];
  if (status == ST_OK) {
#pragma unroll
    for (int e = 0; e < 6; ++e) x[e] = p.seed_params[e * TT + tt];
#pragma unroll
    for (int e = 0; e < 21; ++e) C[e] = p.seed_cov[e * TT + tt];
    for (int k = 0; k < n && status == ST_OK; ++k) {
      double xp[6], Cp[21];
      if (k == 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) xp[e] = x[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp[e] = C[e];
      } else {
        JacS<double> J;
        double qp, qt, F[6][6];
        status = transport_values(g, s_surf, p.surface_id[o0 + k - 1], p.surface_id[o0 + k], x, xp, J, qp, qt);
        if (status != ST_OK) break;
        dense_F(J, F);
        cov_transport(F, C, qp, qt, Cp);
      }
      if (!p.is_hole[o0 + k]) {
        double m[2], V[3], c2 = 0.0;
        meas(k, m, V);
        status = update_fwd(xp, Cp, m, V, x, C, c2);
        chi2sum += c2;
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) x[e] = xp[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) C[e] = Cp[e];
      }
      if (k % kSeg == 0 && k / kSeg < g.n_ckpt) {
#pragma unroll
        for (int e = 0; e < 6; ++e) ck(k / kSeg, e) = x[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) ck(k / kSeg, 6 + e) = C[e];
      }
    }
  }
  if (in_range && g.chi2) g.chi2[tt] = status == ST_OK ? chi2sum : qnan();
  const bool want = (g.grad_seed || g.grad_align);

  // ---------------------------------------------------------- backward
  double lf[6] = {0, 0, 0, 0, 0, 0};
  double Lf[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) Lf[i][j] = 0.0;
  const int n_seg = (status == ST_OK && want) ? (n - 1 + kSeg - 1) / kSeg : 0;
  // the loop runs in lock-step over the warp's maximum segment count so that
  // the alignment-gradient reduction sees whole warps
  int n_seg_warp = n_seg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_seg_warp = max(n_seg_warp, __shfl_xor_sync(0xffffffffu, n_seg_warp, o));
  for (int sg = n_seg_warp - 1; sg >= 0; --sg) {
    const bool seg_active = sg < n_seg;
    const int s0 = sg * kSeg;
    const int s1 = seg_active ? min(s0 + kSeg, n - 1) : s0;  // last state of the segment
    // recompute the filtered states s0 .. s1-1 of the segment
    double bx[kSeg][6], bC[kSeg][21];
    if (seg_active) {
#pragma unroll
      for (int e = 0; e < 6; ++e) bx[0][e] = ck(sg, e);
#pragma unroll
      for (int e = 0; e < 21; ++e) bC[0][e] = ck(sg, 6 + e);
#pragma unroll
      for (int i = 1; i < kSeg; ++i) {
        if (s0 + i < s1) {
          const int k = s0 + i;
          double xp[6], Cp[21], F[6][6], qp, qt;
          JacS<double> J;
          transport_values(g, s_surf, p.surface_id[o0 + k - 1], p.surface_id[o0 + k], bx[i - 1], xp, J, qp, qt);
          dense_F(J, F);
          cov_transport(F, bC[i - 1], qp, qt, Cp);
          if (!p.is_hole[o0 + k]) {
            double m[2], V[3], c2;
            meas(k, m, V);
            update_fwd(xp, Cp, m, V, bx[i], bC[i], c2);
          } else {
#pragma unroll
            for (int e = 0; e < 6; ++e) bx[i][e] = xp[e];
#pragma unroll
            for (int e = 0; e < 21; ++e) bC[i][e] = Cp[e];
          }
        }
      }
    }
    // reverse over the transitions k = s1 .. s0+1
#pragma unroll 1
    for (int k = s0 + kSeg; k > s0; --k) {
      const bool act = seg_active && k <= s1;
      const int i = act ? k - 1 - s0 : 0;
      const int sa = act ? p.surface_id[o0 + k - 1] : 0, sbi = act ? p.surface_id[o0 + k] : 0;
      double lp[6], Lp[6][6];
      double xprev[6], Cprev[21];
#pragma unroll
      for (int e = 0; e < 6; ++e) xprev[e] = act ? bx[i][e] : 0.0;
#pragma unroll
      for (int e = 0; e < 21; ++e) Cprev[e] = act ? bC[i][e] : 0.0;
      double F[6][6];
      if (act) {
        double xp[6], Cp[21], qp, qt;
        JacS<double> J;
        transport_values(g, s_surf, sa, sbi, xprev, xp, J, qp, qt);
        dense_F(J, F);
        cov_transport(F, Cprev, qp, qt, Cp);
        if (!p.is_hole[o0 + k]) {
          double m[2], V[3];
          meas(k, m, V);
          update_adj(xp, Cp, m, V, w, lf, Lf, lp, Lp);
        } else {
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            lp[a] = lf[a];
#pragma unroll
            for (int b = 0; b < 6; ++b) Lp[a][b] = Lf[a][b];
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          lp[a] = 0.0;
#pragma unroll
          for (int b = 0; b < 6; ++b) {
            Lp[a][b] = 0.0;
            F[a][b] = (a == b) ? 1.0 : 0.0;
          }
        }
      }
      // lambda_F = 2 Lp F Cf (only rows 0-3, 5 and columns 0-4 of F vary)
      double lF[6][6];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        double LF[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          double v = 0.0;
#pragma unroll
          for (int q = 0; q < 6; ++q) v += Lp[a][q] * F[q][c];
          LF[c] = v;
        }
#pragma unroll
        for (int b = 0; b < 6; ++b) {
          double v = 0.0;
#pragma unroll
          for (int c = 0; c < 6; ++c) v += LF[c] * Cprev[sym(c, b)];
          lF[a][b] = 2.0 * v;
        }
      }
      // sensitivities of the transport to its 18 inputs, two per pass
      double lx[6];
#pragma unroll 1
      for (int pass = 0; pass < 9; ++pass) {
        double gdir[2] = {0.0, 0.0};
        if (act) {
          Dual<2> xd[6], aa[6], ab[6];
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            xd[e] = Dual<2>(xprev[e]);
            const double va = g.align ? g.align[(size_t)e * p.n_surfaces + sa] : 0.0;
            const double vb = g.align ? g.align[(size_t)e * p.n_surfaces + sbi] : 0.0;
            aa[e] = Dual<2>(va);
            ab[e] = Dual<2>(vb);
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int dir = 2 * pass + q;
            if (dir < 6) xd[dir].d[q] = 1.0;
            else if (dir < 12) aa[dir - 6].d[q] = 1.0;
            else ab[dir - 12].d[q] = 1.0;
          }
          const Plane<Dual<2>> pa = aligned_plane<Dual<2>>(Surf{s_surf + sa * kSurfStride}, aa);
          const Plane<Dual<2>> pb = aligned_plane<Dual<2>>(Surf{s_surf + sbi * kSurfStride}, ab);
          const double B[3] = {p.bfield[0], p.bfield[1], p.bfield[2]};
          Dual<2> xpd[6], qpd, qtd;
          JacS<Dual<2>> Jd;
          transport_s<Dual<2>>(pa, pb, xd, B, p.mass, p.h_max, p.n_iter, Surf{s_surf + sbi * kSurfStride}.xx0(),
                               xpd, Jd, qpd, qtd);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            double v = Lp[2][2] * qpd.d[q] + Lp[3][3] * qtd.d[q];
#pragma unroll
            for (int e = 0; e < 6; ++e) v += lp[e] * xpd[e].d[q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 5; ++c) v += lF[r][c] * Jd.f[r][c].d[q];
#pragma unroll
            for (int c = 0; c < 5; ++c) v += lF[5][c] * Jd.ft[c].d[q];
            gdir[q] = v;
          }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int dir = 2 * pass + q;
          if (dir < 6) {
            lx[dir] = gdir[q];
          } else if (g.grad_align) {
            const int sid = dir < 12 ? sa : sbi;
            add_align_grad(g.grad_align, p.n_surfaces, sid, (dir - 6) % 6, gdir[q], act);
          }
        }
      }
      if (act) {
        // Lambda_Cf = F^T Lp F
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          lf[a] = lx[a];
          double LFa[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < 6; ++q) v += Lp[c][q] * F[q][a];
            LFa[c] = v;
          }
#pragma unroll
          for (int b = 0; b < 6; ++b) {
            double v = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) v += F[c][b] * LFa[c];
            Lf[a][b] = v;  // (F^T Lp F)[b][a], symmetric
          }
        }
      }
    }
  }
  // state 0: reverse through its update; x_p,0 is the seed
  if (in_range && g.grad_seed) {
    double gs[6];
    if (status == ST_OK && want) {
      if (!p.is_hole[o0]) {
        double m[2], V[3], lp[6], Lp[6][6], Cp0[21], xp0[6];
        meas(0, m, V);
#pragma unroll
        for (int e = 0; e < 6; ++e) xp0[e] = p.seed_params[e * TT + tt];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp0[e] = p.seed_cov[e * TT + tt];
        update_adj(xp0, Cp0, m, V, w, lf, Lf, lp, Lp);
#pragma unroll
        for (int e = 0; e < 6; ++e) gs[e] = lp[e];
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) gs[e] = lf[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < 6; ++e) gs[e] = qnan();
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) g.grad_seed[e * TT + tt] = gs[e];
  }
}

}  // namespace

cudaError_t launch_grad(const FitParams& f, const double* align, const double* dl_dchi2, double* chi2,
                        double* grad_seed, double* grad_align, double* ckpt, int n_ckpt, cudaStream_t stream) {
  GradParams g;
  g.f = f;
  g.align = align;
  g.dl_dchi2 = dl_dchi2;
  g.chi2 = chi2;
  g.grad_seed = grad_seed;
  g.grad_align = grad_align;
  g.ckpt = ckpt;
  g.n_ckpt = n_ckpt;
  const size_t smem = (size_t)f.n_surfaces * kSurfStride * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kf_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int block = 64;
  const int grid = (f.n_tracks + block - 1) / block;
  kf_grad_kernel<<<grid, block, smem, stream>>>(g);
  return cudaGetLastError();
}

int grad_segment_length() { return kSeg; }

}  // namespace kfgb
