// kf_adjoint.cu -- gradients of the summed chi2 of the Kalman fit with
// respect to per-surface alignment parameters and the seed parameters.
//
// Objective: L = sum_t w_t sum_k chi2_{t,k}, chi2_k = r_k^T S_k^-1 r_k of the
// predicted residual (paper Sect. 2 filter step list; the chi2 quality
// metric of the smoother paragraph).  chi2 depends only on the forward
// filter, so the smoother contributes nothing to this gradient.
//
// Method (reverse mode throughout):
//   forward:  FP64 filter; (x_f, C_f) checkpointed every kSeg states.
//   backward: for each segment, last first, recompute its filtered states
//     from the checkpoint; then for k = last .. 1 of the segment
//       1. recompute the transport k-1 -> k (x_p, F, Q) and C_p = F C_f F^T + Q
//       2. reverse through chi2_k and the gain-matrix update (exact algebra):
//          adjoints of (x_f,k, C_f,k) -> adjoints of (x_p,k, C_p,k)
//       3. reverse through C_p = F C_f F^T + Q: Lambda_Cf = F^T Lambda_Cp F,
//          lambda_F = 2 Lambda_Cp F C_f, lambda_Q = Lambda_Cp
//       4. one reverse sweep through the transport (its RKN steps recorded
//          on a small tape) gives the adjoints of its 18 inputs (x_f,k-1; the
//          alignment of surfaces k-1 and k) for the contraction with
//          (lambda_xp, lambda_F, lambda_Q): this includes the derivative of
//          F itself, since the sweep runs through the code that forms F.
//     state 0: reverse through its update; x_p,0 is the seed.
// Alignment of a surface (shifts along its local axes, then rotations about
// them):  c' = c + R (du, dv, dn),  R' = R Ru(alpha) Rv(beta) Rn(gamma).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_device.cuh"
#include "kf_fp64.cuh"
#include "kf_internal.h"

namespace kfgb {
namespace {
using namespace dev;

constexpr int kSeg = 5;  // states per checkpoint segment (about sqrt(n) for n ~ 20-40)


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

// c' = c + R (du, dv, dn); R' = R Ru(alpha) Rv(beta) Rn(gamma); cs holds the
// cosines and sines of the three angles (cos alpha, sin alpha, cos beta, ...)
__device__ __forceinline__ Plane<double> aligned_plane(const Surf& s, const double a[6], const double cs[6]) {
  using S = double;
  Plane<S> p;
#pragma unroll
  for (int i = 0; i < 3; ++i) p.c[i] = s.c(i) + s.R(i, 0) * a[0] + s.R(i, 1) * a[1] + s.R(i, 2) * a[2];
  const S ca = cs[0], sa = cs[1], cb = cs[2], sb = cs[3], cg = cs[4], sg = cs[5];
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

// the cosines and sines of every surface's alignment angles, once per call:
// out[2 m][s] = cos(angle m), out[2 m + 1][s] = sin(angle m), m = 0, 1, 2
__global__ void align_trig_kernel(int n_surfaces, const double* __restrict__ align, double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_surfaces) return;
  for (int m = 0; m < 3; ++m) {
    double sn, cn;
    sincos(align[(size_t)(3 + m) * n_surfaces + s], &sn, &cn);
    out[(size_t)(2 * m) * n_surfaces + s] = cn;
    out[(size_t)(2 * m + 1) * n_surfaces + s] = sn;
  }
}

// ---------------------------------------------------------------------------
// the transport (generic in the scalar type; used with double); same
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
  const S g2 = one + s.lam * s.lam * (mass * mass);
  const S igam = rsqrt_any(g2);
  const S gam = g2 * igam;
  s.gtl += h * (s.lam * (mass * mass * kInvC)) * igam;
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

// ---------------------------------------------------------------------------
// reverse mode through one transport
//
// The gradient of a scalar of the transport's outputs,
//   phi = lxp . xp + sum lJ . F + lq_phi q_phi + lq_theta q_theta,
// with respect to the transport's inputs (x and the two aligned planes) is
// taken by one reverse sweep over the arithmetic of transport_tape
// (RKN steps with their Jacobian columns, plane intersections, end frame,
// path correction, free -> bound, Highland noise).  The second derivatives
// that the F term brings in are exact: the reverse sweep runs through the
// code that forms F.
// ---------------------------------------------------------------------------
constexpr int kTape = 16;  // RKN steps recorded per transport (more are recomputed)

struct StepIn {  // state entering one RKN step
  double r[3], T[3], gT[3][3], h;
};

struct Tape {
  StepIn st[kTape];
  int n_steps, nsub;
  double s0;
};

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// A(v) = lk (v x B)
__device__ __forceinline__ void Aop(const double v[3], const double B[3], double lk, double o[3]) {
  o[0] = (v[1] * B[2] - v[2] * B[1]) * lk;
  o[1] = (v[2] * B[0] - v[0] * B[2]) * lk;
  o[2] = (v[0] * B[1] - v[1] * B[0]) * lk;
}

// reverse of o = A(v): vbar += lk (B x obar), lkbar += (v x B) . obar
__device__ __forceinline__ void Aop_rev(const double v[3], const double B[3], double lk, const double ob[3],
                                        double vb[3], double& lkb) {
  double bx[3], vx[3];
  cross3(B, ob, bx);
  cross3(v, B, vx);
#pragma unroll
  for (int i = 0; i < 3; ++i) vb[i] += lk * bx[i];
  lkb += vx[0] * ob[0] + vx[1] * ob[1] + vx[2] * ob[2];
}

// Reverse of one RKN step.  In: the step's input state (T, gT, lam, h) and
// the adjoints of its outputs (Tb = adjoint of T', gTb = of gT'; the
// additive parts r, t, gr, gtl pass their adjoints rb, tb, grb, gtlb through
// unchanged).  Out: Tb, gTb replaced by the adjoints of the inputs; lamb and
// hb accumulated.
__device__ void rkn_rev(const StepIn& in, double lam, const double B[3], double mass, const double rb[3],
                        double tb, const double grb[3][3], double gtlb, double Tb[3], double gTb[3][3],
                        double& lamb, double& hb) {
  const double h = in.h;
  const double h2 = h * h * 0.5, h3 = h * h * h * (1.0 / 6.0), h4 = h * h * h * h * (1.0 / 24.0);
  const double lk = lam * kKappa;
  const double* T = in.T;
  double a1[3], a2[3], a3[3], a4[3], u0[3], u1[3], u2[3], u3[3];
  Aop(T, B, lk, a1);
  Aop(a1, B, lk, a2);
  Aop(a2, B, lk, a3);
  Aop(a3, B, lk, a4);
  Aop(T, B, kKappa, u0);
  Aop(u0, B, lk, u1);
  Aop(u1, B, lk, u2);
  Aop(u2, B, lk, u3);
  double lkb = 0.0;
  double Tin_b[3], a1b[3], a2b[3], a3b[3], a4b[3], u0b[3] = {0, 0, 0}, u1b[3] = {0, 0, 0}, u2b[3] = {0, 0, 0},
                                                   u3b[3] = {0, 0, 0};
  // t' = t + h gam / c;  gtl' = gtl + h lam m^2 / (c gam)
  const double m2 = mass * mass;
  const double g2 = 1.0 + lam * lam * m2;
  const double igam = rsqrt_any(g2), gam = g2 * igam;
  double gamb = tb * h * kInvC - gtlb * h * lam * m2 * kInvC * igam * igam;
  hb += tb * gam * kInvC + gtlb * lam * m2 * kInvC * igam;
  lamb += gtlb * h * m2 * kInvC * igam;
  lamb += gamb * lam * m2 * igam;
  // r' = r + h T + h2 a1 + h3 a2 + h4 a3;  T' = T + h a1 + h2 a2 + h3 a3 + h4 a4
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Tin_b[i] = Tb[i] + h * rb[i];
    a1b[i] = h2 * rb[i] + h * Tb[i];
    a2b[i] = h3 * rb[i] + h2 * Tb[i];
    a3b[i] = h4 * rb[i] + h3 * Tb[i];
    a4b[i] = h4 * Tb[i];
    hb += rb[i] * (T[i] + h * a1[i] + 0.5 * h * h * a2[i] + h * h * h * (1.0 / 6.0) * a3[i]);
    hb += Tb[i] * (a1[i] + h * a2[i] + 0.5 * h * h * a3[i] + h * h * h * (1.0 / 6.0) * a4[i]);
  }
  // Jacobian columns
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double v[3] = {in.gT[0][c], in.gT[1][c], in.gT[2][c]};
    double b1[3], b2[3], b3[3], b4[3];
    Aop(v, B, lk, b1);
    Aop(b1, B, lk, b2);
    Aop(b2, B, lk, b3);
    Aop(b3, B, lk, b4);
    double vb[3], b1b[3], b2b[3], b3b[3], b4b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double rho = grb[i][c], nu = gTb[i][c];
      vb[i] = h * rho + nu;
      b1b[i] = h2 * rho + h * nu;
      b2b[i] = h3 * rho + h2 * nu;
      b3b[i] = h4 * rho + h3 * nu;
      b4b[i] = h4 * nu;
      hb += rho * (v[i] + h * b1[i] + 0.5 * h * h * b2[i] + h * h * h * (1.0 / 6.0) * b3[i]);
      hb += nu * (b1[i] + h * b2[i] + 0.5 * h * h * b3[i] + h * h * h * (1.0 / 6.0) * b4[i]);
      if (c == 2) {
        u0b[i] += h2 * rho + h * nu;
        u1b[i] += h * h * h * (1.0 / 3.0) * rho + h * h * nu;
        u2b[i] += h * h * h * h * 0.125 * rho + h * h * h * 0.5 * nu;
        u3b[i] += h * h * h * h * (1.0 / 6.0) * nu;
        hb += rho * (h * u0[i] + h * h * u1[i] + 0.5 * h * h * h * u2[i]);
        hb += nu * (u0[i] + 2.0 * h * u1[i] + 1.5 * h * h * u2[i] + (2.0 / 3.0) * h * h * h * u3[i]);
      }
    }
    Aop_rev(b3, B, lk, b4b, b3b, lkb);
    Aop_rev(b2, B, lk, b3b, b2b, lkb);
    Aop_rev(b1, B, lk, b2b, b1b, lkb);
    Aop_rev(v, B, lk, b1b, vb, lkb);
#pragma unroll
    for (int i = 0; i < 3; ++i) gTb[i][c] = vb[i];
  }
  Aop_rev(u2, B, lk, u3b, u2b, lkb);
  Aop_rev(u1, B, lk, u2b, u1b, lkb);
  Aop_rev(u0, B, lk, u1b, u0b, lkb);
  {
    double dummy = 0.0;
    Aop_rev(T, B, kKappa, u0b, Tin_b, dummy);  // u0 = kappa (T x B)
  }
  Aop_rev(a3, B, lk, a4b, a3b, lkb);
  Aop_rev(a2, B, lk, a3b, a2b, lkb);
  Aop_rev(a1, B, lk, a2b, a1b, lkb);
  Aop_rev(T, B, lk, a1b, Tin_b, lkb);
  lamb += kKappa * lkb;
#pragma unroll
  for (int i = 0; i < 3; ++i) Tb[i] = Tin_b[i];
}

__device__ __forceinline__ void save_step(const PropS<double>& s, double h, StepIn& o) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.r[i] = s.r[i];
    o.T[i] = s.T[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) o.gT[i][c] = s.gT[i][c];
  }
  o.h = h;
}

// The transport x on plane a -> plane b (the same arithmetic as the FP64
// fit kernel) with the Highland variances of b; with TAPE, the state
// entering each RKN step is recorded (the first kTape) for the reverse sweep.
template <bool TAPE>
__device__ int transport_tape(const Plane<double>& pa, const Plane<double>& pb, const double x[6],
                              const double B[3], double mass, double h_max, int n_iter, double xx0, double xp[6],
                              JacS<double>& J, double& qphi, double& qth, Tape* tp, PropS<double>& s_end) {
  PropS<double> s;
  const double sp = sin(x[2]), cp = cos(x[2]), st = sin(x[3]), ct = cos(x[3]);
#pragma unroll
  for (int i = 0; i < 3; ++i) s.r[i] = pa.c[i] + x[0] * pa.u(i) + x[1] * pa.v(i);
  s.T[0] = cp * st;
  s.T[1] = sp * st;
  s.T[2] = ct;
  s.t = x[5];
  s.lam = x[4];
  s.gT[0][0] = -(sp * st); s.gT[1][0] = cp * st; s.gT[2][0] = 0.0;
  s.gT[0][1] = cp * ct;    s.gT[1][1] = sp * ct; s.gT[2][1] = -st;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.gT[i][2] = 0.0;
    s.gr[i][0] = s.gr[i][1] = s.gr[i][2] = 0.0;
  }
  s.gtl = 0.0;
  auto dist = [&](double& out) -> bool {
    const double d = pb.n(0) * (pb.c[0] - s.r[0]) + pb.n(1) * (pb.c[1] - s.r[1]) + pb.n(2) * (pb.c[2] - s.r[2]);
    const double nT = pb.n(0) * s.T[0] + pb.n(1) * s.T[1] + pb.n(2) * s.T[2];
    if (!(::fabs(nT) > 1e-9)) return false;
    out = d * rcp_any(nT);
    return true;
  };
  double s0;
  if (!dist(s0)) return ST_NO_INTERSECTION;
  const double nsub_d = ::ceil(::fabs(s0) / h_max);
  if (!(nsub_d <= 64.0)) return ST_NO_INTERSECTION;
  const int nsub = nsub_d < 1.0 ? 1 : (int)nsub_d;
  const double h = s0 / (double)nsub;
  if (TAPE) {
    tp->nsub = nsub;
    tp->s0 = s0;
  }
  int ns = 0;
  for (int k = 0; k < nsub; ++k, ++ns) {
    if (TAPE && ns < kTape) save_step(s, h, tp->st[ns]);
    rkn_step_s<double>(s, h, B, mass);
  }
  for (int it = 0; it < n_iter; ++it, ++ns) {
    double si;
    if (!dist(si)) return ST_NO_INTERSECTION;
    if (TAPE && ns < kTape) save_step(s, si, tp->st[ns]);
    rkn_step_s<double>(s, si, B, mass);
  }
  if (TAPE) {
    tp->n_steps = ns;
    s_end = s;
  }
  // the end frame and the outputs
  const double rho2 = s.T[0] * s.T[0] + s.T[1] * s.T[1];
  const double irho = rsqrt_any(rho2);
  const double rho = rho2 * irho;
  const double phi = atan2(s.T[1], s.T[0]);
  const double theta = atan2(rho, s.T[2]);
  const double tn2 = rho2 + s.T[2] * s.T[2];
  const double itn = rsqrt_any(tn2);
  const double tn = tn2 * itn;
  const double cph = s.T[0] * irho, sph = s.T[1] * irho, sth = rho * itn, cth = s.T[2] * itn;
  const double nT = pb.n(0) * s.T[0] + pb.n(1) * s.T[1] + pb.n(2) * s.T[2];
  const double inv_nT = rcp_any(nT), inv_sth = rcp_any(sth);
  const double lk = s.lam * kKappa;
  double AT[3];
  crossB(s.T, B, lk, AT);
  const double dtds = sqrt(1.0 + s.lam * s.lam * (mass * mass)) * kInvC;
  double Gr[3][5], GT[3][5], Gt[5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gr[i][0] = pa.u(i);
    Gr[i][1] = pa.v(i);
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
    const double w = -(pb.n(0) * Gr[0][c] + pb.n(1) * Gr[1][c] + pb.n(2) * Gr[2][c]) * inv_nT;
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
    J.f[2][c] = (cph * GT[1][c] - sph * GT[0][c]) * inv_sth;
    J.f[3][c] = cph * cth * GT[0][c] + sph * cth * GT[1][c] - sth * GT[2][c];
    J.ft[c] = Gt[c];
  }
  const double d0 = s.r[0] - pb.c[0], d1 = s.r[1] - pb.c[1], d2 = s.r[2] - pb.c[2];
  xp[0] = d0 * pb.u(0) + d1 * pb.u(1) + d2 * pb.u(2);
  xp[1] = d0 * pb.v(0) + d1 * pb.v(1) + d2 * pb.v(2);
  xp[2] = phi;
  xp[3] = theta;
  xp[4] = s.lam;
  xp[5] = s.t;
  if (xx0 > 0.0) {
    const double l = ::fabs(s.lam);
    const double g2 = 1.0 + l * l * (mass * mass);
    const double eps = xx0 * ::fabs(tn * inv_nT);
    const double ge = g2 * eps;
    const double th0 = 0.0136 * l * (ge * rsqrt_any(ge)) * (1.0 + 0.038 * log(ge));
    qth = th0 * th0;
    qphi = qth * (inv_sth * inv_sth);
  } else {
    qth = 0.0;
    qphi = 0.0;
  }
  return ST_OK;
}

// Adjoints of the transport's inputs for the output adjoints (lxp, lJ, lJt,
// lqp, lqt), from the tape and end state of transport_tape on the same
// inputs.  Outputs: lx[6] and the adjoints of the planes' centres and
// rotations (row-major 3x3 whose columns are u, v, n).
__device__ void transport_rev(const Plane<double>& pa, const Plane<double>& pb, const double x[6], const double B[3],
                              double mass, double xx0, const Tape& tp, const PropS<double>& s,
                              const double lxp[6], const double lJ[4][5], const double lJt[5], double lqp,
                              double lqt, double lx[6], double lca[3], double lRa[9], double lcb[3],
                              double lRb[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) lca[i] = lcb[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) lRa[i] = lRb[i] = 0.0;
  // adjoints of the end state
  double rb[3] = {0, 0, 0}, Tb[3] = {0, 0, 0}, tb = lxp[5], lamb = lxp[4], grb[3][3], gTb[3][3], gtlb = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) grb[i][c] = gTb[i][c] = 0.0;
  double nbb[3] = {0, 0, 0}, ubb[3] = {0, 0, 0}, vbb[3] = {0, 0, 0};  // plane b axes
  double uab[3] = {0, 0, 0}, vab[3] = {0, 0, 0};                       // plane a axes
  const double m2 = mass * mass;
  // ---- end frame values (recomputed)
  const double rho2 = s.T[0] * s.T[0] + s.T[1] * s.T[1];
  const double irho = rsqrt_any(rho2), rho = rho2 * irho, irho2 = irho * irho;
  const double tn2 = rho2 + s.T[2] * s.T[2];
  const double itn = rsqrt_any(tn2), tn = tn2 * itn, itn2 = itn * itn;
  const double cph = s.T[0] * irho, sph = s.T[1] * irho, sth = rho * itn, cth = s.T[2] * itn;
  const double nT = pb.n(0) * s.T[0] + pb.n(1) * s.T[1] + pb.n(2) * s.T[2];
  const double inv_nT = rcp_any(nT), inv_sth = rcp_any(sth);
  const double lk = s.lam * kKappa;
  double AT[3];
  crossB(s.T, B, lk, AT);
  const double g2_e = 1.0 + s.lam * s.lam * m2;
  const double igam_e = rsqrt_any(g2_e);
  const double dtds = g2_e * igam_e * kInvC;
  double Gr0[3][5], GT0[3][5], w[5], Gr[3][5], GT[3][5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gr0[i][0] = pa.u(i);
    Gr0[i][1] = pa.v(i);
    Gr0[i][2] = s.gr[i][0];
    Gr0[i][3] = s.gr[i][1];
    Gr0[i][4] = s.gr[i][2];
    GT0[i][0] = 0.0;
    GT0[i][1] = 0.0;
    GT0[i][2] = s.gT[i][0];
    GT0[i][3] = s.gT[i][1];
    GT0[i][4] = s.gT[i][2];
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    w[c] = -(pb.n(0) * Gr0[0][c] + pb.n(1) * Gr0[1][c] + pb.n(2) * Gr0[2][c]) * inv_nT;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i][c] = Gr0[i][c] + s.T[i] * w[c];
      GT[i][c] = GT0[i][c] + AT[i] * w[c];
    }
  }
  double nTb = 0.0, cphb = 0.0, sphb = 0.0, cthb = 0.0, sthb = 0.0, phib = lxp[2], thetab = lxp[3], tnb = 0.0;
  // ---- Highland noise
  if (xx0 > 0.0) {
    const double l = ::fabs(s.lam);
    const double g2 = 1.0 + l * l * m2;
    const double icinc = tn * inv_nT;  // 1 / cos(incidence)
    const double eps = xx0 * ::fabs(icinc);
    const double ge = g2 * eps;
    const double Lg = 1.0 + 0.038 * log(ge);
    const double iLg = rcp_any(Lg), ig2 = rcp_any(g2), ieps = rcp_any(eps);
    const double th0 = 0.0136 * l * (ge * rsqrt_any(ge)) * Lg;
    const double is2 = inv_sth * inv_sth;
    const double qthb = lqt + lqp * is2;
    sthb += lqp * (-2.0 * th0 * th0 * is2 * inv_sth);
    const double th0b = 2.0 * th0 * qthb;
    const double dl = th0 * (rcp_any(l) + l * m2 * ig2 + 0.038 * (2.0 * l * m2 * ig2) * iLg);
    const double deps = th0 * ieps * (0.5 + 0.038 * iLg);
    lamb += th0b * dl * (s.lam >= 0.0 ? 1.0 : -1.0);
    const double cb = th0b * deps * (-eps * icinc);
    nTb += cb * itn;
    tnb -= cb * nT * itn2;
  }
  // ---- outputs xp
  {
    const double d[3] = {s.r[0] - pb.c[0], s.r[1] - pb.c[1], s.r[2] - pb.c[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double db = lxp[0] * pb.u(i) + lxp[1] * pb.v(i);
      ubb[i] += lxp[0] * d[i];
      vbb[i] += lxp[1] * d[i];
      rb[i] += db;
      lcb[i] -= db;
    }
  }
  // ---- J = projections of the corrected G columns
  double Grb[3][5], GTb[3][5], Gtb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const double l0 = lJ[0][c], l1 = lJ[1][c], l2 = lJ[2][c], l3 = lJ[3][c];
    const double q = l2 * inv_sth;
    const double f2 = (cph * GT[1][c] - sph * GT[0][c]) * inv_sth;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Grb[i][c] = l0 * pb.u(i) + l1 * pb.v(i);
      ubb[i] += l0 * Gr[i][c];
      vbb[i] += l1 * Gr[i][c];
    }
    GTb[0][c] = -q * sph + l3 * cph * cth;
    GTb[1][c] = q * cph + l3 * sph * cth;
    GTb[2][c] = -l3 * sth;
    cphb += q * GT[1][c] + l3 * cth * GT[0][c];
    sphb += -q * GT[0][c] + l3 * cth * GT[1][c];
    sthb += -l2 * f2 * inv_sth - l3 * GT[2][c];
    cthb += l3 * (cph * GT[0][c] + sph * GT[1][c]);
    Gtb[c] = lJt[c];
  }
  // ---- path correction: G = G0 + (T, AT, dtds) w, w = -(n.Gr0)/nT
  double ATb[3] = {0, 0, 0}, dtdsb = 0.0;
  double Gr0b[3][5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const double wb = Grb[0][c] * s.T[0] + Grb[1][c] * s.T[1] + Grb[2][c] * s.T[2] + GTb[0][c] * AT[0] +
                      GTb[1][c] * AT[1] + GTb[2][c] * AT[2] + Gtb[c] * dtds;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Tb[i] += w[c] * Grb[i][c];
      ATb[i] += w[c] * GTb[i][c];
      Gr0b[i][c] = Grb[i][c] - wb * pb.n(i) * inv_nT;
      nbb[i] += -wb * Gr0[i][c] * inv_nT;
    }
    dtdsb += w[c] * Gtb[c];
    nTb += -wb * w[c] * inv_nT;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    uab[i] += Gr0b[i][0];
    vab[i] += Gr0b[i][1];
    grb[i][0] = Gr0b[i][2];
    grb[i][1] = Gr0b[i][3];
    grb[i][2] = Gr0b[i][4];
    gTb[i][0] = GTb[i][2];
    gTb[i][1] = GTb[i][3];
    gTb[i][2] = GTb[i][4];
  }
  gtlb = Gtb[4];
  // AT = lk (T x B); dtds = sqrt(1 + lam^2 m^2) / c
  {
    double lkb = 0.0;
    Aop_rev(s.T, B, lk, ATb, Tb, lkb);
    lamb += kKappa * lkb;
    lamb += dtdsb * s.lam * m2 * kInvC * igam_e;
  }
  // nT = n . T
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    nbb[i] += nTb * s.T[i];
    Tb[i] += nTb * pb.n(i);
  }
  // end angles and direction cosines
  {
    double rhob = 0.0, rho2b = 0.0;
    Tb[0] += cphb * irho;
    rhob -= cphb * s.T[0] * irho2;
    Tb[1] += sphb * irho;
    rhob -= sphb * s.T[1] * irho2;
    rhob += sthb * itn;
    tnb -= sthb * rho * itn2;
    Tb[2] += cthb * itn;
    tnb -= cthb * s.T[2] * itn2;
    // theta = atan2(rho, T2)
    rhob += thetab * s.T[2] * itn2;
    Tb[2] -= thetab * rho * itn2;
    // tn = sqrt(rho2 + T2^2)
    rho2b += tnb * 0.5 * itn;
    Tb[2] += tnb * s.T[2] * itn;
    rho2b += rhob * 0.5 * irho;
    // phi = atan2(T1, T0)
    Tb[1] += phib * s.T[0] * irho2;
    Tb[0] -= phib * s.T[1] * irho2;
    Tb[0] += 2.0 * s.T[0] * rho2b;
    Tb[1] += 2.0 * s.T[1] * rho2b;
  }
  // ---- reverse over the RKN steps, last first
  const int nsteps = tp.n_steps;
  double hb_main = 0.0;  // adjoint of the main steps' common length h = s0 / nsub
  for (int j = nsteps - 1; j >= 0; --j) {
    StepIn in;
    if (j < kTape) {
      in = tp.st[j];
    } else {
      // beyond the tape: recompute the forward from the last recorded step
      PropS<double> q;
      const StepIn& base = tp.st[kTape - 1];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        q.r[i] = base.r[i];
        q.T[i] = base.T[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          q.gT[i][c] = base.gT[i][c];
          q.gr[i][c] = 0.0;
        }
      }
      q.t = 0.0;
      q.gtl = 0.0;
      q.lam = x[4];
      double hj = base.h;
      for (int k = kTape - 1; k < j; ++k) {
        rkn_step_s<double>(q, hj, B, mass);
        if (k + 1 < tp.nsub) {
          hj = tp.s0 / (double)tp.nsub;
        } else {
          hj = (pb.n(0) * (pb.c[0] - q.r[0]) + pb.n(1) * (pb.c[1] - q.r[1]) + pb.n(2) * (pb.c[2] - q.r[2])) /
               (pb.n(0) * q.T[0] + pb.n(1) * q.T[1] + pb.n(2) * q.T[2]);
        }
      }
      save_step(q, hj, in);
    }
    double hb = 0.0;
    rkn_rev(in, x[4], B, mass, rb, tb, grb, gtlb, Tb, gTb, lamb, hb);
    if (j >= tp.nsub) {
      // correction step: si = (n.(c - r))/(n.T) of the state entering it
      const double nTi = pb.n(0) * in.T[0] + pb.n(1) * in.T[1] + pb.n(2) * in.T[2];
      const double inTi = rcp_any(nTi);
      const double db = hb * inTi, nTib = -hb * in.h * inTi;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        nbb[i] += db * (pb.c[i] - in.r[i]) + nTib * in.T[i];
        lcb[i] += db * pb.n(i);
        rb[i] -= db * pb.n(i);
        Tb[i] += nTib * pb.n(i);
      }
    } else {
      hb_main += hb;
    }
  }
  // ---- the main steps' length: h = s0 / nsub, s0 = (n.(c - r0))/(n.T0) of
  // the start state (whose adjoints rb, Tb now are)
  {
    const StepIn& st0 = tp.st[0];
    const double s0b = hb_main / (double)tp.nsub;
    const double nT0 = pb.n(0) * st0.T[0] + pb.n(1) * st0.T[1] + pb.n(2) * st0.T[2];
    const double inT0 = rcp_any(nT0);
    const double db = s0b * inT0, nT0b = -s0b * tp.s0 * inT0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      nbb[i] += db * (pb.c[i] - st0.r[i]) + nT0b * st0.T[i];
      lcb[i] += db * pb.n(i);
      rb[i] -= db * pb.n(i);
      Tb[i] += nT0b * pb.n(i);
    }
  }
  // ---- the start: r = ca + x0 ua + x1 va; T and the G columns from the
  // angles; t = x5; q/p = x4
  {
    const double sp = sin(x[2]), cp = cos(x[2]), st = sin(x[3]), ct = cos(x[3]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lca[i] += rb[i];
      uab[i] += x[0] * rb[i];
      vab[i] += x[1] * rb[i];
    }
    lx[0] = rb[0] * pa.u(0) + rb[1] * pa.u(1) + rb[2] * pa.u(2);
    lx[1] = rb[0] * pa.v(0) + rb[1] * pa.v(1) + rb[2] * pa.v(2);
    // dT/dphi = (-sp st, cp st, 0), dT/dtheta = (cp ct, sp ct, -st);
    // gT[:,0] = dT/dphi, gT[:,1] = dT/dtheta
    lx[2] = Tb[0] * (-sp * st) + Tb[1] * (cp * st) + gTb[0][0] * (-cp * st) + gTb[1][0] * (-sp * st) +
            gTb[0][1] * (-sp * ct) + gTb[1][1] * (cp * ct);
    lx[3] = Tb[0] * (cp * ct) + Tb[1] * (sp * ct) - Tb[2] * st + gTb[0][0] * (-sp * ct) + gTb[1][0] * (cp * ct) +
            gTb[0][1] * (-cp * st) + gTb[1][1] * (-sp * st) + gTb[2][1] * (-ct);
    lx[4] = lamb;
    lx[5] = tb;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lRa[3 * i + 0] += uab[i];
    lRa[3 * i + 1] += vab[i];
    lRb[3 * i + 0] += ubb[i];
    lRb[3 * i + 1] += vbb[i];
    lRb[3 * i + 2] += nbb[i];
  }
}

// Reverse of aligned_plane: adjoints of the plane's centre lc and rotation lR
// (row-major) -> adjoints of its 6 alignment parameters (accumulated in ga).
//   c' = c + R (du, dv, dn):        d(du, dv, dn) = R^T lc
//   R' = R M, M = Ru(al) Rv(be) Rn(ga):  lM = R^T lR, d(angle) = <lM, dM/d(angle)>
__device__ __forceinline__ void aligned_plane_rev(const Surf& s, const double cs[6], const double lc[3],
                                                  const double lR[9], double ga[6]) {
#pragma unroll
  for (int e = 0; e < 3; ++e) ga[e] += s.R(0, e) * lc[0] + s.R(1, e) * lc[1] + s.R(2, e) * lc[2];
  double lM[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) lM[i][j] = s.R(0, i) * lR[0 * 3 + j] + s.R(1, i) * lR[1 * 3 + j] + s.R(2, i) * lR[2 * 3 + j];
  const double ca = cs[0], sa = cs[1], cb = cs[2], sb = cs[3], cg = cs[4], sg = cs[5];
  const double Ru[3][3] = {{1, 0, 0}, {0, ca, -sa}, {0, sa, ca}};
  const double Rv[3][3] = {{cb, 0, sb}, {0, 1, 0}, {-sb, 0, cb}};
  const double Rn[3][3] = {{cg, -sg, 0}, {sg, cg, 0}, {0, 0, 1}};
  const double dRu[3][3] = {{0, 0, 0}, {0, -sa, -ca}, {0, ca, -sa}};
  const double dRv[3][3] = {{-sb, 0, cb}, {0, 0, 0}, {-cb, 0, -sb}};
  const double dRn[3][3] = {{-sg, -cg, 0}, {cg, -sg, 0}, {0, 0, 0}};
  auto mul3 = [](const double X[3][3], const double Y[3][3], double Z[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Z[i][j] = X[i][0] * Y[0][j] + X[i][1] * Y[1][j] + X[i][2] * Y[2][j];
  };
  double VN[3][3], dVN[3][3], VdN[3][3], D[3][3];
  mul3(Rv, Rn, VN);
  mul3(dRv, Rn, dVN);
  mul3(Rv, dRn, VdN);
  double acc[3] = {0.0, 0.0, 0.0};
  mul3(dRu, VN, D);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[0] += lM[i][j] * D[i][j];
  mul3(Ru, dVN, D);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[1] += lM[i][j] * D[i][j];
  mul3(Ru, VdN, D);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[2] += lM[i][j] * D[i][j];
  ga[3] += acc[0];
  ga[4] += acc[1];
  ga[5] += acc[2];
}

struct GradParams {
  FitParams f;          // geometry, inputs, options (outputs unused); a
                        // launch covers tracks [track0, track0 + n_tracks)
                        // of n_tracks_total
  const double* align;  // [6][S] or null (zero alignment)
  const double* align_cs;  // [6][S] cosines and sines of the alignment angles (with align)
  const double* dl_dchi2;    // [T] or null (all ones)
  const double* dl_dparams;  // [6][T] or null: weights of the smoothed state-0 parameters
  const double* dl_dcov;     // [21][T] or null: weights of its packed covariance
  double* chi2;         // [T] or null
  double* out_params;   // [6][T] or null: smoothed parameters of state 0
  double* out_cov;      // [21][T] or null: smoothed covariance of state 0
  double* grad_seed;    // [6][T] or null
  double* grad_align;   // [6][S] or null (accumulated with atomicAdd; zeroed by the host)
  double* ckpt;         // [n_ckpt][27][n_tracks]: filtered checkpoints
  double* sck;          // [n_ckpt + 1][27][n_tracks]: smoothed checkpoints
  double* sadj;         // [max_states][kSmRec][n_tracks]: the smoother's adjoint contributions
  double* pipe;         // [kPipeScratch][n_tracks]: hand-off slots of the pipelined form (or null)
  int32_t n_ckpt;
};

// the alignment of surface sid and the cosines and sines of its angles
__device__ __forceinline__ void load_align(const GradParams& g, int sid, double a[6], double cs[6]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) a[e] = g.align ? g.align[(size_t)e * g.f.n_surfaces + sid] : 0.0;
#pragma unroll
  for (int e = 0; e < 6; ++e) cs[e] = g.align ? g.align_cs[(size_t)e * g.f.n_surfaces + sid] : ((e & 1) ? 0.0 : 1.0);
}

// values of the transport k-1 -> k with the aligned planes
__device__ __forceinline__ int transport_values(const GradParams& g, const double* s_surf, int sa, int sb,
                                                const double x[6], double xp[6], JacS<double>& J, double& qp,
                                                double& qt) {
  double aa[6], ab[6], ca[6], cb[6];
  load_align(g, sa, aa, ca);
  load_align(g, sb, ab, cb);
  const Plane<double> pa = aligned_plane(Surf{s_surf + sa * kSurfStride}, aa, ca);
  const Plane<double> pb = aligned_plane(Surf{s_surf + sb * kSurfStride}, ab, cb);
  const double B[3] = {g.f.bfield[0], g.f.bfield[1], g.f.bfield[2]};
  PropS<double> s_end;
  return transport_tape<false>(pa, pb, x, B, g.f.mass, g.f.h_max, g.f.n_iter, Surf{s_surf + sb * kSurfStride}.xx0(),
                               xp, J, qp, qt, nullptr, s_end);
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

// ---------------------------------------------------------------------------
// the RTS smoother step and its reverse (paper Sect. 2, smoother paragraph)
// ---------------------------------------------------------------------------

// Cholesky factor L (packed lower) of an SPD 6x6 C and the reciprocals of its
// diagonal; false on a non-positive pivot.
__device__ __forceinline__ bool chol6(const double C[21], double L[21], double idg[6]) {
  bool ok = true;
#pragma unroll
  for (int e = 0; e < 21; ++e) L[e] = C[e];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double dj = L[sy(j, j)];
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (q < j) dj -= L[sy(j, q)] * L[sy(j, q)];
    if (!(dj > 0.0)) ok = false;
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
  return ok;
}

// G = C^-1 (packed) from the Cholesky factor: Y = L^-1 (lower), G = Y^T Y.
__device__ __forceinline__ void chol6_inverse(const double L[21], const double idg[6], double G[21]) {
  double Y[21];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    Y[sy(j, j)] = idg[j];
#pragma unroll
    for (int r = 0; r < 6; ++r)
      if (r > j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (q >= j && q < r) v += L[sy(r, q)] * Y[sy(q, j)];
        Y[sy(r, j)] = -v * idg[r];
      }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j <= i) {
        double v = 0.0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
          if (r >= i) v += Y[sy(r, i)] * Y[sy(r, j)];
        G[sy(i, j)] = v;
      }
}

// What the reverse of one smoother step needs from its forward: M = G F with
// G = Cp_{k+1}^-1, and dx = xs_{k+1} - xp_{k+1}, dC = Cs_{k+1} - Cp_{k+1}.
struct RtsKeep {
  double M[36], G[21], dx[6], dC[21];
};

// One RTS step from the smoothed state k+1 (xs, Cs) to state k:
//   A = Cf_k F^T Cp_{k+1}^-1 = Cf_k M^T,  M = Cp_{k+1}^-1 F,
//   xs_k = xf_k + A (xs_{k+1} - xp_{k+1}),  Cs_k = Cf_k + A (Cs_{k+1} - Cp_{k+1}) A^T.
// F is the transport k -> k+1, xp, Cp its prediction.
__device__ __noinline__ int rts_step_fwd(const double xf[6], const double Cf[21], const double xp[6], const double Cp[21],
                            const JacS<double>& J, double xs[6], double Cs[21], RtsKeep* keep) {
  double L[21], idg[6], G[21];
  if (!chol6(Cp, L, idg)) return ST_NON_SPD;
  chol6_inverse(L, idg, G);
  double F[6][6];
  dense_F(J, F);
  double M[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += G[sym(i, q)] * F[q][j];
      M[i][j] = v;
    }
  double A[6][6];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += Cf[sym(r, q)] * M[c][q];
      A[r][c] = v;
    }
  double dx[6], dC[21];
#pragma unroll
  for (int e = 0; e < 6; ++e) dx[e] = xs[e] - xp[e];
#pragma unroll
  for (int e = 0; e < 21; ++e) dC[e] = Cs[e] - Cp[e];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double v = xf[r];
#pragma unroll
    for (int c = 0; c < 6; ++c) v += A[r][c] * dx[c];
    xs[r] = v;
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double z[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += A[r][q] * dC[sym(q, c)];
      z[c] = v;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (c <= r) {
        double v = Cf[sy(r, c)];
#pragma unroll
        for (int q = 0; q < 6; ++q) v += z[q] * A[c][q];
        Cs[sy(r, c)] = v;
      }
  }
  if (keep) {
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) keep->M[i * 6 + j] = M[i][j];
#pragma unroll
    for (int e = 0; e < 21; ++e) {
      keep->G[e] = G[e];
      keep->dC[e] = dC[e];
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) keep->dx[e] = dx[e];
  }
  return ST_OK;
}

// Contributions of one smoother step to the adjoints of the filter's
// quantities (symmetric matrices in the full-matrix convention, stored
// packed): [0..5] x_f,k, [6..26] C_f,k, [27..32] x_p,k+1, [33..53] C_p,k+1,
// [54..73] F_{k+1} rows 0-3 x columns 0-4, [74..78] its time row.
constexpr int kSmXF = 0, kSmCF = 6, kSmXP = 27, kSmCP = 33, kSmF = 54, kSmRec = 79;

// Reverse of rts_step_fwd.  In: lxs, Ls, the adjoints of xs_k, Cs_k (Ls
// symmetric).  Out: lxs, Ls become the adjoints of xs_{k+1}, Cs_{k+1}; c[]
// receives the step's contributions (layout above).  With LA the adjoint of
// the gain A:
//   LA = lxs dx^T + 2 Ls A dC;  l_dx = A^T lxs;  L_dC = A^T Ls A
//   x_f: lxs;  C_f: Ls + sym(LA M);  F: G LA^T Cf;
//   x_p: -l_dx;  C_p: -L_dC - sym(A^T LA G);  next: lxs = l_dx, Ls = L_dC.
__device__ __noinline__ void rts_step_rev(const double Cf[21], const RtsKeep& r, double lxs[6], double Ls[6][6],
                             double c[kSmRec]) {
  double A[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += Cf[sym(i, q)] * r.M[j * 6 + q];
      A[i][j] = v;
    }
  // LsA = Ls A, then LA = lxs dx^T + 2 (Ls A) dC
  double LA[6][6];
  {
    double LsA[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += Ls[i][q] * A[q][j];
        LsA[i][j] = v;
      }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += LsA[i][q] * r.dC[sym(q, j)];
        LA[i][j] = lxs[i] * r.dx[j] + 2.0 * v;
      }
    // L_dC = A^T (Ls A)
    double LdC[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += A[q][i] * LsA[q][j];
        LdC[i][j] = v;
      }
    // x_f and C_f (direct terms), before Ls is replaced
#pragma unroll
    for (int e = 0; e < 6; ++e) c[kSmXF + e] = lxs[e];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (j <= i) c[kSmCF + sy(i, j)] = Ls[i][j];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) Ls[i][j] = 0.5 * (LdC[i][j] + LdC[j][i]);
  }
  // l_dx = A^T lxs
  double ldx[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) v += A[q][j] * lxs[q];
    ldx[j] = v;
  }
  // C_f += sym(LA M)
  {
    double T[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += LA[i][q] * r.M[q * 6 + j];
        T[i][j] = v;
      }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (j <= i) c[kSmCF + sy(i, j)] += 0.5 * (T[i][j] + T[j][i]);
  }
  // F: G LA^T Cf (rows 0-3 and 5, columns 0-4)
  {
    double LtC[6][6];  // LA^T Cf
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += LA[q][i] * Cf[sym(q, j)];
        LtC[i][j] = v;
      }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i == 4) continue;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += r.G[sym(i, q)] * LtC[q][j];
        c[i == 5 ? kSmF + 20 + j : kSmF + i * 5 + j] = v;
      }
    }
  }
  // x_p and C_p: -l_dx, -L_dC - sym(A^T LA G)
  {
    double ATL[6][6];  // A^T LA
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += A[q][i] * LA[q][j];
        ATL[i][j] = v;
      }
    double T[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += ATL[i][q] * r.G[sym(q, j)];
        T[i][j] = v;
      }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (j <= i) c[kSmCP + sy(i, j)] = -Ls[i][j] - 0.5 * (T[i][j] + T[j][i]);
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    c[kSmXP + e] = -ldx[e];
    lxs[e] = ldx[e];
  }
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

// Per-thread view of one track's inputs and of its slices of the scratch
// arrays (inputs and outputs are [.][n_tracks_total] at track tg, scratch is
// [.][n_tracks] of the launch at track tl).
struct TrackIO {
  const GradParams* g;
  int64_t o0;
  int tg, tl;
  size_t TG, TL;
  __device__ double& ck(int j, int e) const { return g->ckpt[((size_t)j * 27 + e) * TL + tl]; }
  __device__ double& sck(int j, int e) const { return g->sck[((size_t)j * 27 + e) * TL + tl]; }
  __device__ double& sadj(int k, int e) const { return g->sadj[((size_t)k * kSmRec + e) * TL + tl]; }
  __device__ void meas(int k, double m[2], double V[3]) const {
    const FitParams& p = g->f;
    m[0] = p.loc[o0 + k];
    m[1] = p.loc[p.n_states + o0 + k];
    V[0] = p.cov[o0 + k];
    V[1] = p.cov[p.n_states + o0 + k];
    V[2] = p.cov[2 * p.n_states + o0 + k];
  }
  __device__ int sid(int k) const { return g->f.surface_id[o0 + k]; }
  __device__ bool hole(int k) const { return g->f.is_hole[o0 + k] != 0; }
};

// Recompute segment [s0, s0 + L] of a track from its filtered checkpoint j:
// the filtered states s0 .. s0+L-1 (fx, fC) and the transports i: s0+i ->
// s0+i+1 (their predictions px, pC and Jacobians pJ), i = 0 .. L-1.  The
// arithmetic is the forward pass's, so it succeeds where that did.
__device__ __noinline__ void recompute_segment(const TrackIO& io, const double* s_surf, int j, int s0, int L,
                                  double fx[kSeg][6], double fC[kSeg][21], double px[kSeg][6],
                                  double pC[kSeg][21], JacS<double> pJ[kSeg]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) fx[0][e] = io.ck(j, e);
#pragma unroll
  for (int e = 0; e < 21; ++e) fC[0][e] = io.ck(j, 6 + e);
#pragma unroll 1
  for (int i = 0; i < L; ++i) {
    const int k = s0 + i + 1;
    double qp, qt, F[6][6];
    transport_values(*io.g, s_surf, io.sid(k - 1), io.sid(k), fx[i], px[i], pJ[i], qp, qt);
    dense_F(pJ[i], F);
    cov_transport(F, fC[i], qp, qt, pC[i]);
    if (i + 1 < L) {
      if (!io.hole(k)) {
        double m[2], V[3], c2;
        io.meas(k, m, V);
        update_fwd(px[i], pC[i], m, V, fx[i + 1], fC[i + 1], c2);
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) fx[i + 1][e] = px[i][e];
#pragma unroll
        for (int e = 0; e < 21; ++e) fC[i + 1][e] = pC[i][e];
      }
    }
  }
}

// adds the smoother's contributions to the adjoints of x_f,k and C_f,k
__device__ __forceinline__ void add_sm_filtered(const TrackIO& io, int k, double lf[6], double Lf[6][6]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) lf[e] += io.sadj(k, kSmXF + e);
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const double v = io.sadj(k, kSmCF + sy(i, j));
      Lf[i][j] += v;
      if (j < i) Lf[j][i] += v;
    }
}

// The filtered states s0 .. s1-1 of a segment, from its checkpoint j.
__device__ __forceinline__ void recompute_filtered(const TrackIO& io, const double* s_surf, int j, int s0, int s1,
                                                   double bx[kSeg][6], double bC[kSeg][21]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) bx[0][e] = io.ck(j, e);
#pragma unroll
  for (int e = 0; e < 21; ++e) bC[0][e] = io.ck(j, 6 + e);
#pragma unroll
  for (int i = 1; i < kSeg; ++i) {
    if (s0 + i < s1) {
      const int k = s0 + i;
      double xp[6], Cp[21], F[6][6], qp, qt;
      JacS<double> J;
      transport_values(*io.g, s_surf, io.sid(k - 1), io.sid(k), bx[i - 1], xp, J, qp, qt);
      dense_F(J, F);
      cov_transport(F, bC[i - 1], qp, qt, Cp);
      if (!io.hole(k)) {
        double m[2], V[3], c2;
        io.meas(k, m, V);
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

// One filtered state: transition k-1 -> k from (xi, Ci) and the update at k.
__device__ __forceinline__ void step_filtered(const TrackIO& io, const double* s_surf, int k, const double xi[6],
                                              const double Ci[21], double xo[6], double Co[21]) {
  double xp[6], Cp[21], F[6][6], qp, qt;
  JacS<double> J;
  transport_values(*io.g, s_surf, io.sid(k - 1), io.sid(k), xi, xp, J, qp, qt);
  dense_F(J, F);
  cov_transport(F, Ci, qp, qt, Cp);
  if (!io.hole(k)) {
    double m[2], V[3], c2;
    io.meas(k, m, V);
    update_fwd(xp, Cp, m, V, xo, Co, c2);
  } else {
#pragma unroll
    for (int e = 0; e < 6; ++e) xo[e] = xp[e];
#pragma unroll
    for (int e = 0; e < 21; ++e) Co[e] = Cp[e];
  }
}

// What the reverse of transition k-1 -> k needs from its forward: the
// filtered state it starts from, the prediction, the Jacobian, and the
// transport's tape and end state.
struct TransitionFwd {
  double xprev[6], Cprev[21], xp[6], Cp[21];
  JacS<double> J;
  Tape tp;
  PropS<double> s_end;
};

__device__ __forceinline__ void aligned_planes(const GradParams& g, const double* s_surf, int sa, int sb,
                                               double ca[6], double cb[6], Plane<double>& pa, Plane<double>& pb) {
  double aa[6], ab[6];
  load_align(g, sa, aa, ca);
  load_align(g, sb, ab, cb);
  pa = aligned_plane(Surf{s_surf + sa * kSurfStride}, aa, ca);
  pb = aligned_plane(Surf{s_surf + sb * kSurfStride}, ab, cb);
}

// the forward of transition k: the taped transport from (xprev, Cprev)
__device__ __forceinline__ void transition_forward(const GradParams& g, const TrackIO& io, const double* s_surf, int k,
                                                   const double xprev[6], const double Cprev[21], TransitionFwd& tf) {
  const FitParams& p = g.f;
  const int sa = io.sid(k - 1), sb = io.sid(k);
  double ca[6], cb[6];
  Plane<double> pa, pb;
  aligned_planes(g, s_surf, sa, sb, ca, cb, pa, pb);
  const double B[3] = {p.bfield[0], p.bfield[1], p.bfield[2]};
  const double xxb = Surf{s_surf + sb * kSurfStride}.xx0();
#pragma unroll
  for (int e = 0; e < 6; ++e) tf.xprev[e] = xprev[e];
#pragma unroll
  for (int e = 0; e < 21; ++e) tf.Cprev[e] = Cprev[e];
  double qp, qt, F[6][6];
  transport_tape<true>(pa, pb, xprev, B, p.mass, p.h_max, p.n_iter, xxb, tf.xp, tf.J, qp, qt, &tf.tp, tf.s_end);
  dense_F(tf.J, F);
  cov_transport(F, Cprev, qp, qt, tf.Cp);
}

// The reverse of transition k: lf, Lf (adjoints of x_f,k, C_f,k) become
// those of x_f,k-1, C_f,k-1; galign receives the adjoints of the alignment
// of surfaces k-1 (0..5) and k (6..11).
__device__ __forceinline__ void transition_reverse(const GradParams& g, const TrackIO& io, const double* s_surf, int k,
                                                   double w, bool use_sm, const TransitionFwd& tf, double lf[6],
                                                   double Lf[6][6], double galign[12]) {
  const FitParams& p = g.f;
  const int sa = io.sid(k - 1), sbi = io.sid(k);
  double ca[6], cb[6];
  Plane<double> pa, pb;
  aligned_planes(g, s_surf, sa, sbi, ca, cb, pa, pb);
  const double B[3] = {p.bfield[0], p.bfield[1], p.bfield[2]};
  const double xxb = Surf{s_surf + sbi * kSurfStride}.xx0();
  double F[6][6];
  dense_F(tf.J, F);
  double lp[6], Lp[6][6];
  if (use_sm) add_sm_filtered(io, k, lf, Lf);
  if (!io.hole(k)) {
    double m[2], V[3];
    io.meas(k, m, V);
    update_adj(tf.xp, tf.Cp, m, V, w, lf, Lf, lp, Lp);
  } else {
#pragma unroll
    for (int a2 = 0; a2 < 6; ++a2) {
      lp[a2] = lf[a2];
#pragma unroll
      for (int b2 = 0; b2 < 6; ++b2) Lp[a2][b2] = Lf[a2][b2];
    }
  }
  if (use_sm) {
    // the smoother's direct use of x_p,k and C_p,k
#pragma unroll
    for (int e = 0; e < 6; ++e) lp[e] += io.sadj(k, kSmXP + e);
#pragma unroll
    for (int a2 = 0; a2 < 6; ++a2)
#pragma unroll
      for (int b2 = 0; b2 <= a2; ++b2) {
        const double v = io.sadj(k, kSmCP + sy(a2, b2));
        Lp[a2][b2] += v;
        if (b2 < a2) Lp[b2][a2] += v;
      }
  }
  // lambda_F = 2 Lp F Cf (only rows 0-3, 5 and columns 0-4 of F vary)
  double lF[6][6];
#pragma unroll
  for (int a2 = 0; a2 < 6; ++a2) {
    double LF[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += Lp[a2][q] * F[q][c];
      LF[c] = v;
    }
#pragma unroll
    for (int b2 = 0; b2 < 6; ++b2) {
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < 6; ++c) v += LF[c] * tf.Cprev[sym(c, b2)];
      lF[a2][b2] = 2.0 * v;
    }
  }
  // reverse sweep through the transport: adjoints of x_f,k-1 and of both
  // planes' alignment, contracted with (lambda_xp, lambda_F, Lambda_Q)
  double lx[6];
  {
    double lJ[4][5], lJt[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
#pragma unroll
      for (int r = 0; r < 4; ++r) lJ[r][c] = lF[r][c] + (use_sm ? io.sadj(k, kSmF + r * 5 + c) : 0.0);
      lJt[c] = lF[5][c] + (use_sm ? io.sadj(k, kSmF + 20 + c) : 0.0);
    }
    double lca[3], lRa[9], lcb[3], lRb[9];
    transport_rev(pa, pb, tf.xprev, B, p.mass, xxb, tf.tp, tf.s_end, lp, lJ, lJt, Lp[2][2], Lp[3][3], lx, lca, lRa,
                  lcb, lRb);
    aligned_plane_rev(Surf{s_surf + sa * kSurfStride}, ca, lca, lRa, galign);
    aligned_plane_rev(Surf{s_surf + sbi * kSurfStride}, cb, lcb, lRb, galign + 6);
  }
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

// Hand-off slot of the pipelined reverse, [field][n_tracks] doubles:
// xprev 6 | Cprev 21 | xp 6 | Cp 21 | J 25 | n_steps, nsub, s0 | end state 27
// | the recorded steps (16 doubles each, as many as were recorded).
constexpr int kSlotFixed = 6 + 21 + 6 + 21 + 25 + 3 + 27;
constexpr int kSlot = kSlotFixed + 16 * kTape;

// Hand-off slot of one recomputed segment in the pipelined smoother passes:
// for each of its kSeg transitions the filtered state and covariance, the
// prediction and its covariance, and the transport Jacobian
// ([fx 6 | fC 21 | px 6 | pC 21 | J 25] doubles per transition and track).
constexpr int kSegRec = 6 + 21 + 6 + 21 + 25;
constexpr int kSegSlot = kSeg * kSegRec;
// the pipelined form's hand-off scratch per track: two transition slots
// (pass B) or two segment slots and the last filtered state (passes S, R)
constexpr int kPipeScratch = 2 * kSlot > 2 * kSegSlot + 27 ? 2 * kSlot : 2 * kSegSlot + 27;

__device__ __forceinline__ void seg_write(double* slot, size_t TL, int tl, int L, const double fx[kSeg][6],
                                          const double fC[kSeg][21], const double px[kSeg][6],
                                          const double pC[kSeg][21], const JacS<double> pJ[kSeg]) {
#pragma unroll 1
  for (int i = 0; i < L; ++i) {
    double* q = slot + (size_t)i * kSegRec * TL + tl;
#pragma unroll
    for (int e = 0; e < 6; ++e) q[(size_t)e * TL] = fx[i][e];
#pragma unroll
    for (int e = 0; e < 21; ++e) q[(size_t)(6 + e) * TL] = fC[i][e];
#pragma unroll
    for (int e = 0; e < 6; ++e) q[(size_t)(27 + e) * TL] = px[i][e];
#pragma unroll
    for (int e = 0; e < 21; ++e) q[(size_t)(33 + e) * TL] = pC[i][e];
#pragma unroll
    for (int e = 0; e < 20; ++e) q[(size_t)(54 + e) * TL] = pJ[i].f[e / 5][e % 5];
#pragma unroll
    for (int e = 0; e < 5; ++e) q[(size_t)(74 + e) * TL] = pJ[i].ft[e];
  }
}

__device__ __forceinline__ void seg_read(const double* slot, size_t TL, int tl, int L, double fx[kSeg][6],
                                         double fC[kSeg][21], double px[kSeg][6], double pC[kSeg][21],
                                         JacS<double> pJ[kSeg]) {
#pragma unroll 1
  for (int i = 0; i < L; ++i) {
    const double* q = slot + (size_t)i * kSegRec * TL + tl;
#pragma unroll
    for (int e = 0; e < 6; ++e) fx[i][e] = q[(size_t)e * TL];
#pragma unroll
    for (int e = 0; e < 21; ++e) fC[i][e] = q[(size_t)(6 + e) * TL];
#pragma unroll
    for (int e = 0; e < 6; ++e) px[i][e] = q[(size_t)(27 + e) * TL];
#pragma unroll
    for (int e = 0; e < 21; ++e) pC[i][e] = q[(size_t)(33 + e) * TL];
#pragma unroll
    for (int e = 0; e < 20; ++e) pJ[i].f[e / 5][e % 5] = q[(size_t)(54 + e) * TL];
#pragma unroll
    for (int e = 0; e < 5; ++e) pJ[i].ft[e] = q[(size_t)(74 + e) * TL];
  }
}

__device__ __forceinline__ void slot_write(double* slot, size_t TL, int tl, const TransitionFwd& tf) {
  int o = 0;
  auto put = [&](double v) { slot[(size_t)(o++) * TL + tl] = v; };
#pragma unroll
  for (int e = 0; e < 6; ++e) put(tf.xprev[e]);
#pragma unroll
  for (int e = 0; e < 21; ++e) put(tf.Cprev[e]);
#pragma unroll
  for (int e = 0; e < 6; ++e) put(tf.xp[e]);
#pragma unroll
  for (int e = 0; e < 21; ++e) put(tf.Cp[e]);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) put(tf.J.f[r][c]);
#pragma unroll
  for (int c = 0; c < 5; ++c) put(tf.J.ft[c]);
  put((double)tf.tp.n_steps);
  put((double)tf.tp.nsub);
  put(tf.tp.s0);
  const PropS<double>& e = tf.s_end;
#pragma unroll
  for (int i = 0; i < 3; ++i) put(e.r[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) put(e.T[i]);
  put(e.t);
  put(e.lam);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) put(e.gr[i][c]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) put(e.gT[i][c]);
  put(e.gtl);
  const int ns = min(tf.tp.n_steps, kTape);
  for (int j = 0; j < ns; ++j) {
    double* q = slot + (size_t)(kSlotFixed + 16 * j) * TL + tl;
    const StepIn& st = tf.tp.st[j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      q[(size_t)i * TL] = st.r[i];
      q[(size_t)(3 + i) * TL] = st.T[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) q[(size_t)(6 + 3 * i + c) * TL] = st.gT[i][c];
    }
    q[(size_t)15 * TL] = st.h;
  }
}

__device__ __forceinline__ void slot_read(const double* slot, size_t TL, int tl, TransitionFwd& tf) {
  int o = 0;
  auto get = [&]() { return slot[(size_t)(o++) * TL + tl]; };
#pragma unroll
  for (int e = 0; e < 6; ++e) tf.xprev[e] = get();
#pragma unroll
  for (int e = 0; e < 21; ++e) tf.Cprev[e] = get();
#pragma unroll
  for (int e = 0; e < 6; ++e) tf.xp[e] = get();
#pragma unroll
  for (int e = 0; e < 21; ++e) tf.Cp[e] = get();
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) tf.J.f[r][c] = get();
#pragma unroll
  for (int c = 0; c < 5; ++c) tf.J.ft[c] = get();
  tf.tp.n_steps = (int)get();
  tf.tp.nsub = (int)get();
  tf.tp.s0 = get();
  PropS<double>& e = tf.s_end;
#pragma unroll
  for (int i = 0; i < 3; ++i) e.r[i] = get();
#pragma unroll
  for (int i = 0; i < 3; ++i) e.T[i] = get();
  e.t = get();
  e.lam = get();
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) e.gr[i][c] = get();
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) e.gT[i][c] = get();
  e.gtl = get();
  const int ns = min(tf.tp.n_steps, kTape);
  for (int j = 0; j < ns; ++j) {
    const double* q = slot + (size_t)(kSlotFixed + 16 * j) * TL + tl;
    StepIn& st = tf.tp.st[j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      st.r[i] = q[(size_t)i * TL];
      st.T[i] = q[(size_t)(3 + i) * TL];
#pragma unroll
      for (int c = 0; c < 3; ++c) st.gT[i][c] = q[(size_t)(6 + 3 * i + c) * TL];
    }
    st.h = q[(size_t)15 * TL];
  }
}

// Register-cap variants as for the fit kernels: MINB 1 may use 255
// registers (up to 8 warps per SM), 3 caps at 168 (12 warps) and 4 at 128
// (16 warps; the tape then spills to local memory).
//
// Passes (one thread per track):
//   F  forward filter, filtered checkpoints every kSeg states, chi2;
//   S  (smoothed outputs or their adjoints asked) the RTS smoother from the
//      last state down, segment by segment, each segment's filtered states
//      and transports recomputed from its checkpoint; smoothed checkpoints
//      at the segment starts; the smoothed state 0 is the output;
//   R  (adjoints of the smoothed outputs asked) the reverse of the smoother,
//      segment by segment upwards: the segment's states recomputed from both
//      kinds of checkpoint, then each step reversed; the contributions to
//      the adjoints of the filter's quantities go to sadj;
//   B  the reverse of the filter, segment by segment downwards (states
//      recomputed from the checkpoints, transports re-run with a tape), with
//      sadj added in at every state.
// PIPE: a CTA of two warps per 32 tracks (lane l of both on track l).  The
// second warp runs pass F; in S and R it recomputes each segment one segment
// ahead of the first warp, which runs the RTS steps and their reverse on
// what the second left in a segment slot (two slots, one barrier per
// segment); in B it runs the forward half of every transition (the
// segment's recompute, the taped transport) one transition ahead, and the
// first warp the reverse half (the reverse of the update and of the
// transport) on what the second left in a slot (two slots, one barrier per
// transition).  For batches too small to fill the GPU: a warp
// instruction costs an SM sub-partition's FP64 pipe the same at any number
// of active lanes, so the split has to go across warps.
template <int MINB, bool PIPE>
__global__ void __launch_bounds__(PIPE ? 64 : max_threads_of(MINB), 1) kf_grad_kernel(const GradParams g) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* s_surf = reinterpret_cast<double*>(smem_raw);
  __shared__ __align__(8) uint64_t s_mbar;
  const FitParams& p = g.f;
  const bool staged = stage_surfaces(s_surf, p.surf, (uint32_t)(p.n_surfaces * kSurfStride * 8), &s_mbar,
                                     p.error_flag, p.wait_limit, p.skip_stage_copy != 0);
  const int t = PIPE ? blockIdx.x * 32 + (int)(threadIdx.x & 31) : blockIdx.x * blockDim.x + threadIdx.x;
  const bool in_range = t < p.n_tracks;
  // the warp that runs pass F (both warps without PIPE)
  const bool run_fwd = !PIPE || threadIdx.x >= 32;
  TrackIO io;
  io.g = &g;
  io.tl = in_range ? t : 0;
  io.tg = p.track0 + io.tl;
  io.TG = (size_t)p.n_tracks_total;
  io.TL = (size_t)p.n_tracks;
  const int tg = io.tg;
  const size_t TG = io.TG;
  if (!staged) {
    // a bounded wait of this call gave up: this CTA's tracks get NaN chi2,
    // smoothed outputs and seed gradients and add nothing to the alignment
    // gradient (the whole CTA returns here, so no warp-wide reduction below
    // is entered)
    if (in_range) {
      if (g.chi2) g.chi2[tg] = qnan();
      if (g.grad_seed)
        for (int e = 0; e < 6; ++e) g.grad_seed[(size_t)e * TG + tg] = qnan();
      if (g.out_params)
        for (int e = 0; e < 6; ++e) g.out_params[(size_t)e * TG + tg] = qnan();
      if (g.out_cov)
        for (int e = 0; e < 21; ++e) g.out_cov[(size_t)e * TG + tg] = qnan();
    }
    return;
  }
  const int64_t o0 = p.offsets[tg], o1 = p.offsets[tg + 1];
  io.o0 = o0;
  const int n = (int)(o1 - o0);
  int status = in_range ? ST_OK : ST_BAD_INPUT;
  if (!(o1 > o0) || o0 < 0 || o1 > p.n_states || n > p.max_states) status = ST_BAD_INPUT;
  if (status == ST_OK)
    for (int k = 0; k < n; ++k) {
      const int sid = p.surface_id[o0 + k];
      if (sid < 0 || sid >= p.n_surfaces) status = ST_BAD_INPUT;
    }
  const double w = (g.dl_dchi2 && in_range) ? g.dl_dchi2[tg] : 1.0;
  const bool want = (g.grad_seed || g.grad_align);
  const bool sm_adj = want && (g.dl_dparams || g.dl_dcov);
  const bool sm_fwd = sm_adj || g.out_params || g.out_cov;

  // ---------------------------------------------------------- F: forward
  double chi2sum = 0.0;
  double x[6], C[21];
  if (status == ST_OK && run_fwd) {
#pragma unroll
    for (int e = 0; e < 6; ++e) x[e] = p.seed_params[e * TG + tg];
#pragma unroll
    for (int e = 0; e < 21; ++e) C[e] = p.seed_cov[e * TG + tg];
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
        status = transport_values(g, s_surf, io.sid(k - 1), io.sid(k), x, xp, J, qp, qt);
        if (status != ST_OK) break;
        dense_F(J, F);
        cov_transport(F, C, qp, qt, Cp);
      }
      if (!io.hole(k)) {
        double m[2], V[3], c2 = 0.0;
        io.meas(k, m, V);
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
        for (int e = 0; e < 6; ++e) io.ck(k / kSeg, e) = x[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) io.ck(k / kSeg, 6 + e) = C[e];
      }
    }
  }
  // segments: sg covers the transitions s0+1 .. s1, s0 = sg kSeg,
  // s1 = min(s0 + kSeg, n - 1); its filtered checkpoint is state s0
  const int n_seg_trk = status == ST_OK ? (n - 1 + kSeg - 1) / kSeg : 0;

  if constexpr (!PIPE) {
    // ---------------------------------------------------------- S: smoother
    if (sm_fwd && status == ST_OK && run_fwd) {
      double xs[6], Cs[21];  // x_s,n-1 = x_f,n-1
  #pragma unroll
      for (int e = 0; e < 6; ++e) xs[e] = x[e];
  #pragma unroll
      for (int e = 0; e < 21; ++e) Cs[e] = C[e];
      if (sm_adj) {
  #pragma unroll
        for (int e = 0; e < 6; ++e) io.sck(n_seg_trk, e) = xs[e];
  #pragma unroll
        for (int e = 0; e < 21; ++e) io.sck(n_seg_trk, 6 + e) = Cs[e];
      }
  #pragma unroll 1
      for (int sg = n_seg_trk - 1; sg >= 0 && status == ST_OK; --sg) {
        const int s0 = sg * kSeg, L = min(s0 + kSeg, n - 1) - s0;
        double fx[kSeg][6], fC[kSeg][21], px[kSeg][6], pC[kSeg][21];
        JacS<double> pJ[kSeg];
        recompute_segment(io, s_surf, sg, s0, L, fx, fC, px, pC, pJ);
  #pragma unroll 1
        for (int i = L - 1; i >= 0 && status == ST_OK; --i)
          status = rts_step_fwd(fx[i], fC[i], px[i], pC[i], pJ[i], xs, Cs, nullptr);
        if (sm_adj && sg > 0) {
  #pragma unroll
          for (int e = 0; e < 6; ++e) io.sck(sg, e) = xs[e];
  #pragma unroll
          for (int e = 0; e < 21; ++e) io.sck(sg, 6 + e) = Cs[e];
        }
      }
      if (in_range && g.out_params)
  #pragma unroll
        for (int e = 0; e < 6; ++e) g.out_params[e * TG + tg] = status == ST_OK ? xs[e] : qnan();
      if (in_range && g.out_cov)
  #pragma unroll
        for (int e = 0; e < 21; ++e) g.out_cov[e * TG + tg] = status == ST_OK ? Cs[e] : qnan();
    } else if (in_range && run_fwd) {
      if (g.out_params)
        for (int e = 0; e < 6; ++e) g.out_params[e * TG + tg] = qnan();
      if (g.out_cov)
        for (int e = 0; e < 21; ++e) g.out_cov[e * TG + tg] = qnan();
    }
    if (in_range && g.chi2 && run_fwd) g.chi2[tg] = status == ST_OK ? chi2sum : qnan();

    // ---------------------------------------------------------- R: smoother reverse
    if (sm_adj && status == ST_OK && run_fwd) {
      double lxs[6], Ls[6][6];
  #pragma unroll
      for (int e = 0; e < 6; ++e) lxs[e] = g.dl_dparams ? g.dl_dparams[e * TG + tg] : 0.0;
      // the weight W_e of a packed covariance element e = (i, j), i > j, stands
      // for both C_ij and C_ji in the full-matrix convention: W_e / 2 each
  #pragma unroll
      for (int i = 0; i < 6; ++i)
  #pragma unroll
        for (int j = 0; j <= i; ++j) {
          const double v = g.dl_dcov ? g.dl_dcov[sy(i, j) * TG + tg] : 0.0;
          Ls[i][j] = Ls[j][i] = (i == j) ? v : 0.5 * v;
        }
  #pragma unroll 1
      for (int sg = 0; sg < n_seg_trk; ++sg) {
        const int s0 = sg * kSeg, L = min(s0 + kSeg, n - 1) - s0;
        double fx[kSeg][6], fC[kSeg][21], px[kSeg][6], pC[kSeg][21];
        JacS<double> pJ[kSeg];
        recompute_segment(io, s_surf, sg, s0, L, fx, fC, px, pC, pJ);
        double xs[6], Cs[21];
  #pragma unroll
        for (int e = 0; e < 6; ++e) xs[e] = io.sck(sg + 1, e);
  #pragma unroll
        for (int e = 0; e < 21; ++e) Cs[e] = io.sck(sg + 1, 6 + e);
        RtsKeep keep[kSeg];
  #pragma unroll 1
        for (int i = L - 1; i >= 0; --i) rts_step_fwd(fx[i], fC[i], px[i], pC[i], pJ[i], xs, Cs, &keep[i]);
  #pragma unroll 1
        for (int i = 0; i < L; ++i) {
          double c[kSmRec];
          rts_step_rev(fC[i], keep[i], lxs, Ls, c);
          const int k = s0 + i;
  #pragma unroll
          for (int e = 0; e < kSmXP; ++e) io.sadj(k, e) = c[e];
  #pragma unroll
          for (int e = kSmXP; e < kSmRec; ++e) io.sadj(k + 1, e) = c[e];
        }
      }
      // the last state: x_s,n-1 = x_f,n-1, C_s,n-1 = C_f,n-1
  #pragma unroll
      for (int e = 0; e < 6; ++e) io.sadj(n - 1, kSmXF + e) = lxs[e];
  #pragma unroll
      for (int i = 0; i < 6; ++i)
  #pragma unroll
        for (int j = 0; j <= i; ++j) io.sadj(n - 1, kSmCF + sy(i, j)) = Ls[i][j];
    }
  } else {
    // Pipelined smoother passes: the forward warp recomputes the filter's
    // segments (transports and updates from the checkpoints) one segment
    // ahead; the other warp runs the RTS steps on what it left in one of two
    // segment slots (one barrier per segment, both warps the same count).
    const bool fwd_warp = threadIdx.x >= 32;
    const int lane = threadIdx.x & 31;
    __shared__ int s_status[32];
    // the filter's status, from the forward warp to the other
    if (fwd_warp) s_status[lane] = status;
    __syncthreads();
    status = s_status[lane];
    __syncthreads();
    const int nseg_f = status == ST_OK ? n_seg_trk : 0;  // the same in both warps
    auto warp_max = [](int v) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
      return v;
    };
    const size_t seg_stride = (size_t)kSegSlot * io.TL;
    double* const hand = g.pipe + 2 * seg_stride;  // the last filtered state
    // ---------------------------------------------------------- S: smoother
    double xs[6], Cs[21];
    if (sm_fwd) {
      if (fwd_warp && status == ST_OK) {
#pragma unroll
        for (int e = 0; e < 6; ++e) hand[(size_t)e * io.TL + io.tl] = x[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) hand[(size_t)(6 + e) * io.TL + io.tl] = C[e];
      }
      __syncthreads();
      if (!fwd_warp && status == ST_OK) {
#pragma unroll
        for (int e = 0; e < 6; ++e) xs[e] = hand[(size_t)e * io.TL + io.tl];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cs[e] = hand[(size_t)(6 + e) * io.TL + io.tl];
        if (sm_adj) {
#pragma unroll
          for (int e = 0; e < 6; ++e) io.sck(nseg_f, e) = xs[e];
#pragma unroll
          for (int e = 0; e < 21; ++e) io.sck(nseg_f, 6 + e) = Cs[e];
        }
      }
      const int n_items = warp_max(nseg_f);
      for (int j = 0; j <= n_items; ++j) {
        if (fwd_warp && j < n_items) {
          const int sg = n_items - 1 - j;
          if (sg < nseg_f) {
            const int s0 = sg * kSeg, L = min(s0 + kSeg, n - 1) - s0;
            double fx[kSeg][6], fC[kSeg][21], px[kSeg][6], pC[kSeg][21];
            JacS<double> pJ[kSeg];
            recompute_segment(io, s_surf, sg, s0, L, fx, fC, px, pC, pJ);
            seg_write(g.pipe + (size_t)(j & 1) * seg_stride, io.TL, io.tl, L, fx, fC, px, pC, pJ);
          }
        }
        if (!fwd_warp && j >= 1) {
          const int sg = n_items - j;
          if (sg < nseg_f && status == ST_OK) {
            const int s0 = sg * kSeg, L = min(s0 + kSeg, n - 1) - s0;
            double fx[kSeg][6], fC[kSeg][21], px[kSeg][6], pC[kSeg][21];
            JacS<double> pJ[kSeg];
            seg_read(g.pipe + (size_t)((j - 1) & 1) * seg_stride, io.TL, io.tl, L, fx, fC, px, pC, pJ);
#pragma unroll 1
            for (int i = L - 1; i >= 0 && status == ST_OK; --i)
              status = rts_step_fwd(fx[i], fC[i], px[i], pC[i], pJ[i], xs, Cs, nullptr);
            if (sm_adj && sg > 0) {
#pragma unroll
              for (int e = 0; e < 6; ++e) io.sck(sg, e) = xs[e];
#pragma unroll
              for (int e = 0; e < 21; ++e) io.sck(sg, 6 + e) = Cs[e];
            }
          }
        }
        __syncthreads();
      }
      if (!fwd_warp && in_range) {
        if (g.out_params)
#pragma unroll
          for (int e = 0; e < 6; ++e) g.out_params[e * TG + tg] = status == ST_OK ? xs[e] : qnan();
        if (g.out_cov)
#pragma unroll
          for (int e = 0; e < 21; ++e) g.out_cov[e * TG + tg] = status == ST_OK ? Cs[e] : qnan();
      }
    }
    // ---------------------------------------------------------- R: smoother reverse
    if (sm_adj) {
      double lxs[6], Ls[6][6];
      if (!fwd_warp) {
#pragma unroll
        for (int e = 0; e < 6; ++e) lxs[e] = g.dl_dparams ? g.dl_dparams[e * TG + tg] : 0.0;
        // W_e of a packed off-diagonal element stands for C_ij and C_ji: W_e / 2 each
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int j = 0; j <= i; ++j) {
            const double v = g.dl_dcov ? g.dl_dcov[sy(i, j) * TG + tg] : 0.0;
            Ls[i][j] = Ls[j][i] = (i == j) ? v : 0.5 * v;
          }
      }
      const int n_items = warp_max(nseg_f);
      for (int j = 0; j <= n_items; ++j) {
        if (fwd_warp && j < n_items) {
          const int sg = j;
          if (sg < nseg_f) {
            const int s0 = sg * kSeg, L = min(s0 + kSeg, n - 1) - s0;
            double fx[kSeg][6], fC[kSeg][21], px[kSeg][6], pC[kSeg][21];
            JacS<double> pJ[kSeg];
            recompute_segment(io, s_surf, sg, s0, L, fx, fC, px, pC, pJ);
            seg_write(g.pipe + (size_t)(j & 1) * seg_stride, io.TL, io.tl, L, fx, fC, px, pC, pJ);
          }
        }
        if (!fwd_warp && j >= 1) {
          const int sg = j - 1;
          if (sg < nseg_f && status == ST_OK) {
            const int s0 = sg * kSeg, L = min(s0 + kSeg, n - 1) - s0;
            double fx[kSeg][6], fC[kSeg][21], px[kSeg][6], pC[kSeg][21];
            JacS<double> pJ[kSeg];
            seg_read(g.pipe + (size_t)((j - 1) & 1) * seg_stride, io.TL, io.tl, L, fx, fC, px, pC, pJ);
            double xr[6], Cr[21];
#pragma unroll
            for (int e = 0; e < 6; ++e) xr[e] = io.sck(sg + 1, e);
#pragma unroll
            for (int e = 0; e < 21; ++e) Cr[e] = io.sck(sg + 1, 6 + e);
            RtsKeep keep[kSeg];
#pragma unroll 1
            for (int i = L - 1; i >= 0; --i) rts_step_fwd(fx[i], fC[i], px[i], pC[i], pJ[i], xr, Cr, &keep[i]);
#pragma unroll 1
            for (int i = 0; i < L; ++i) {
              double c[kSmRec];
              rts_step_rev(fC[i], keep[i], lxs, Ls, c);
              const int k = s0 + i;
#pragma unroll
              for (int e = 0; e < kSmXP; ++e) io.sadj(k, e) = c[e];
#pragma unroll
              for (int e = kSmXP; e < kSmRec; ++e) io.sadj(k + 1, e) = c[e];
            }
          }
        }
        __syncthreads();
      }
      if (!fwd_warp && status == ST_OK) {
        // the last state: x_s,n-1 = x_f,n-1, C_s,n-1 = C_f,n-1
#pragma unroll
        for (int e = 0; e < 6; ++e) io.sadj(n - 1, kSmXF + e) = lxs[e];
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int j = 0; j <= i; ++j) io.sadj(n - 1, kSmCF + sy(i, j)) = Ls[i][j];
      }
    }
    // the smoother's status (an RTS step may fail), back to the forward warp
    __syncthreads();
    if (!fwd_warp) s_status[lane] = status;
    __syncthreads();
    status = s_status[lane];
    if (in_range && g.chi2 && fwd_warp) g.chi2[tg] = status == ST_OK ? chi2sum : qnan();
  }

  // ---------------------------------------------------------- B: filter reverse
  double lf[6] = {0, 0, 0, 0, 0, 0};
  double Lf[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) Lf[i][j] = 0.0;
  const int n_seg = (status == ST_OK && want) ? n_seg_trk : 0;
  const bool use_sm = sm_adj && status == ST_OK;
  // the loop runs in lock-step over the warp's maximum segment count so that
  // the alignment-gradient reduction sees whole warps (with PIPE both warps
  // hold the same 32 tracks and find the same count)
  int n_seg_warp = n_seg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_seg_warp = max(n_seg_warp, __shfl_xor_sync(0xffffffffu, n_seg_warp, o));
  auto add_galign = [&](int k, bool act, const double galign[12]) {
    if (!g.grad_align) return;
    const int sa = act ? io.sid(k - 1) : 0, sbi = act ? io.sid(k) : 0;
#pragma unroll 1
    for (int e = 0; e < 12; ++e) add_align_grad(g.grad_align, p.n_surfaces, e < 6 ? sa : sbi, e % 6, galign[e], act);
  };
  if (!PIPE) {
    for (int sg = n_seg_warp - 1; sg >= 0; --sg) {
      const bool seg_active = sg < n_seg;
      const int s0 = sg * kSeg;
      const int s1 = seg_active ? min(s0 + kSeg, n - 1) : s0;  // last state of the segment
      // the filtered states s0 .. s1-1 of the segment
      double bx[kSeg][6], bC[kSeg][21];
      if (seg_active) recompute_filtered(io, s_surf, sg, s0, s1, bx, bC);
      // reverse over the transitions k = s1 .. s0+1
#pragma unroll 1
      for (int k = s0 + kSeg; k > s0; --k) {
        const bool act = seg_active && k <= s1;
        double galign[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) galign[e] = 0.0;
        if (act) {
          TransitionFwd tf;
          transition_forward(g, io, s_surf, k, bx[k - 1 - s0], bC[k - 1 - s0], tf);
          transition_reverse(g, io, s_surf, k, w, use_sm, tf, lf, Lf, galign);
        }
        add_galign(k, act, galign);
      }
    }
  } else {
    // item j is transition k of segment sg, in the order above; the forward
    // warp produces item j into slot j % 2 while the reverse warp consumes
    // item j - 1 from the other slot; one barrier per item (both warps run
    // the same n_items + 1 iterations).  The forward warp recomputes the
    // filtered states of the next segment (below) one per item while it
    // produces the current segment's items, so no item carries a whole
    // segment's recompute (only the first segment is recomputed at once).
    const bool fwd_warp = threadIdx.x >= 32;
    const int n_items = n_seg_warp * kSeg;
    const size_t slot_stride = (size_t)kSlot * io.TL;
    double bx[2][kSeg][6], bC[2][kSeg][21];  // by segment parity
    for (int j = 0; j <= n_items; ++j) {
      if (fwd_warp && j < n_items) {
        const int sg = n_seg_warp - 1 - j / kSeg, q = j % kSeg;
        const int s0 = sg * kSeg, k = s0 + kSeg - q;
        const bool seg_active = sg < n_seg;
        const int s1 = seg_active ? min(s0 + kSeg, n - 1) : s0;
        const int cur = sg & 1, nxt = cur ^ 1;
        if (j == 0 && seg_active) recompute_filtered(io, s_surf, sg, s0, s1, bx[cur], bC[cur]);
        if (sg > 0 && sg - 1 < n_seg && q + 1 < kSeg) {
          // state q + 1 of segment sg - 1 (its checkpoint first)
          const int s0n = (sg - 1) * kSeg, s1n = min(s0n + kSeg, n - 1);
          if (q == 0) {
#pragma unroll
            for (int e = 0; e < 6; ++e) bx[nxt][0][e] = io.ck(sg - 1, e);
#pragma unroll
            for (int e = 0; e < 21; ++e) bC[nxt][0][e] = io.ck(sg - 1, 6 + e);
          }
          if (s0n + q + 1 < s1n)
            step_filtered(io, s_surf, s0n + q + 1, bx[nxt][q], bC[nxt][q], bx[nxt][q + 1], bC[nxt][q + 1]);
        }
        if (seg_active && k <= s1) {
          TransitionFwd tf;
          transition_forward(g, io, s_surf, k, bx[cur][k - 1 - s0], bC[cur][k - 1 - s0], tf);
          slot_write(g.pipe + (size_t)(j & 1) * slot_stride, io.TL, io.tl, tf);
        }
      }
      if (!fwd_warp && j >= 1) {
        const int jj = j - 1;
        const int sg = n_seg_warp - 1 - jj / kSeg;
        const int s0 = sg * kSeg, k = s0 + kSeg - jj % kSeg;
        const bool seg_active = sg < n_seg;
        const int s1 = seg_active ? min(s0 + kSeg, n - 1) : s0;
        const bool act = seg_active && k <= s1;
        double galign[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) galign[e] = 0.0;
        if (act) {
          TransitionFwd tf;
          slot_read(g.pipe + (size_t)(jj & 1) * slot_stride, io.TL, io.tl, tf);
          transition_reverse(g, io, s_surf, k, w, use_sm, tf, lf, Lf, galign);
        }
        add_galign(k, act, galign);
      }
      __syncthreads();
    }
  }
  if (PIPE && run_fwd) return;  // the reverse warp finishes the track
  // state 0: reverse through its update; x_p,0 is the seed
  if (in_range && g.grad_seed) {
    double gs[6];
    if (status == ST_OK && want) {
      if (use_sm) add_sm_filtered(io, 0, lf, Lf);
      if (!io.hole(0)) {
        double m[2], V[3], lp[6], Lp[6][6], Cp0[21], xp0[6];
        io.meas(0, m, V);
#pragma unroll
        for (int e = 0; e < 6; ++e) xp0[e] = p.seed_params[e * TG + tg];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp0[e] = p.seed_cov[e * TG + tg];
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
    for (int e = 0; e < 6; ++e) g.grad_seed[e * TG + tg] = gs[e];
  }
}

}  // namespace

template <int MINB, bool PIPE>
cudaError_t launch_grad_v(const GradParams& g, int block, cudaStream_t stream) {
  const FitParams& f = g.f;
  const size_t smem = (size_t)f.n_surfaces * kSurfStride * sizeof(double);
  auto kern = kf_grad_kernel<MINB, PIPE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (PIPE) {
    kern<<<(f.n_tracks + 31) / 32, 64, smem, stream>>>(g);
    return cudaGetLastError();
  }
  if (block <= 0) {
    // CTAs of w warps, one per SM per wave, w the smallest count (within the
    // warps this variant's registers allow per SM) that covers the batch's
    // 32-track warp units in r full waves: the last wave is nearly full
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long wmax = max_threads_of(MINB) / 32;
    const long long units = ((long long)f.n_tracks + 31) / 32;
    long long w = wmax;
    for (long long r = 1; r <= 1024; ++r) {
      w = (units + r * nsm - 1) / (r * nsm);
      if (w <= wmax) break;
    }
    block = 32 * (int)(w < 1 ? 1 : (w > wmax ? wmax : w));
  }
  const int grid = (f.n_tracks + block - 1) / block;
  kern<<<grid, block, smem, stream>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_align_trig(int n_surfaces, const double* align, double* out, cudaStream_t stream) {
  align_trig_kernel<<<(n_surfaces + 127) / 128, 128, 0, stream>>>(n_surfaces, align, out);
  return cudaGetLastError();
}

size_t grad_scratch_doubles(int max_states, bool smoother, bool smoother_adjoint, bool pipelined) {
  const size_t n_ckpt = ((size_t)max_states + kSeg - 1) / kSeg;
  size_t d = 27 * n_ckpt;
  if (smoother_adjoint) d += 27 * (n_ckpt + 1) + (size_t)kSmRec * (size_t)max_states;
  if (pipelined) d += (size_t)kPipeScratch;
  (void)smoother;  // the smoother alone keeps no per-track scratch
  return d;
}

cudaError_t launch_grad(const FitParams& f, const GradArgs& a, double* scratch, int block, int min_blocks,
                        bool pipelined, cudaStream_t stream) {
  GradParams g;
  g.f = f;
  g.align = a.align;
  g.align_cs = a.align_cs;
  g.dl_dchi2 = a.dl_dchi2;
  g.dl_dparams = a.dl_dparams;
  g.dl_dcov = a.dl_dcov;
  g.chi2 = a.chi2;
  g.out_params = a.params;
  g.out_cov = a.cov;
  g.grad_seed = a.grad_seed;
  g.grad_align = a.grad_align;
  const size_t T = (size_t)f.n_tracks;
  g.n_ckpt = (f.max_states + kSeg - 1) / kSeg;
  g.ckpt = scratch;
  // the smoother's checkpoints and contributions follow when its adjoint is
  // asked; the hand-off slots come last
  const bool sm_adj = (a.grad_seed || a.grad_align) && (a.dl_dparams || a.dl_dcov);
  g.sck = scratch + 27 * (size_t)g.n_ckpt * T;
  g.sadj = g.sck + 27 * (size_t)(g.n_ckpt + 1) * T;
  g.pipe = nullptr;
  if (pipelined) g.pipe = sm_adj ? g.sadj + (size_t)kSmRec * (size_t)f.max_states * T : g.sck;
  if (pipelined) return launch_grad_v<1, true>(g, 64, stream);
  switch (min_blocks) {
    case 4: return launch_grad_v<4, false>(g, block, stream);
    case 3: return launch_grad_v<3, false>(g, block, stream);
    default: return launch_grad_v<1, false>(g, block, stream);
  }
}

}  // namespace kfgb
