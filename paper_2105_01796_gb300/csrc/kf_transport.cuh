// kf_transport.cuh -- the FP64 path's RKN propagation with the columns of
// its transport Jacobian (paper Sect. 4.1), shared by the one-thread-per-track
// kernel (kf_kernels.cu) and the track-team kernel (kf_team.cu).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "kf_device.cuh"
#include "kf_fp64.cuh"

namespace kfgb {
namespace dev {

// ---------------------------------------------------------------------------
// propagation state: free parameters (double accumulators) plus the columns
// of G = D * J_bf that vary along the path.  Columns: 0 phi, 1 theta, 2 q/p.
// ---------------------------------------------------------------------------
template <typename R>
struct Prop {
  double r[3], T[3], t;
  double lam;
  R gr[3][3];  // position rows, column c
  R gT[3][3];  // direction rows, column c
  R gtl;       // time row, q/p column
};

// One 4-stage Nystrom step of length h in the constant field.  With
// A v = (q/p) kappa (v x B) the four stages give
//   T' = (I + hA + h^2A^2/2 + h^3A^3/6 + h^4A^4/24) T = Stt T
//   r' = r + (hI + h^2A/2 + h^3A^2/6 + h^4A^3/24) T  = r + Srt T
// (the classic RKN4 combination k1+2k2+2k3+k4 and k1+k2+k3 of the stage
// accelerations).  G advances by the exact derivative of this step:
//   position rows += Srt * direction rows (+ dSrt/dlam T on the q/p column)
//   direction rows = Stt * direction rows (+ dStt/dlam T on the q/p column)
//   time row (q/p column) += h m^2 lam / (c sqrt(1 + m^2 lam^2)).
// CMASK selects the Jacobian columns that are advanced (bit c: column c);
// the others are left as they are (a team of warps splits them).
template <typename R, bool BZ, int CMASK = 7>
__device__ __forceinline__ void rkn_step(Prop<R>& s, double h, const double B[3], double mass) {
  const R hr = (R)h;
  const R h2 = hr * hr * R(0.5);
  const R h3 = hr * hr * hr * R(1.0 / 6.0);
  const R h4 = hr * hr * hr * hr * R(1.0 / 24.0);
  const R lk = (R)(s.lam * kKappa);
  const R bs[3] = {lk * (R)B[0], lk * (R)B[1], lk * (R)B[2]};
  const R kB[3] = {(R)(kKappa * B[0]), (R)(kKappa * B[1]), (R)(kKappa * B[2])};
  // value
  const R Tr[3] = {(R)s.T[0], (R)s.T[1], (R)s.T[2]};
  R a1[3], a2[3], a3[3], a4[3];
  applyA<R, BZ>(bs, Tr, a1);
  applyA<R, BZ>(bs, a1, a2);
  applyA<R, BZ>(bs, a2, a3);
  applyA<R, BZ>(bs, a3, a4);
  // q/p derivative seed: u = kappa (T x B)
  R u0[3], u1[3], u2[3], u3[3];
  applyA<R, BZ>(kB, Tr, u0);
  applyA<R, BZ>(bs, u0, u1);
  applyA<R, BZ>(bs, u1, u2);
  applyA<R, BZ>(bs, u2, u3);
  // Jacobian columns
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (!(CMASK & (1 << c))) continue;
    R g[3] = {s.gT[0][c], s.gT[1][c], s.gT[2][c]};
    R b1[3], b2[3], b3[3], b4[3];
    applyA<R, BZ>(bs, g, b1);
    applyA<R, BZ>(bs, b1, b2);
    applyA<R, BZ>(bs, b2, b3);
    applyA<R, BZ>(bs, b3, b4);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R dr = hr * g[i] + h2 * b1[i] + h3 * b2[i] + h4 * b3[i];
      R nt = g[i] + hr * b1[i] + h2 * b2[i] + h3 * b3[i] + h4 * b4[i];
      if (c == 2) {
        dr += h2 * u0[i] + hr * hr * hr * R(1.0 / 3.0) * u1[i] + hr * hr * hr * hr * R(0.125) * u2[i];
        nt += hr * u0[i] + hr * hr * u1[i] + hr * hr * hr * R(0.5) * u2[i] +
              hr * hr * hr * hr * R(1.0 / 6.0) * u3[i];
      }
      s.gr[i][c] += dr;
      s.gT[i][c] = nt;
    }
  }
  // sqrt(1 + m^2 lam^2) and its reciprocal from one Newton-refined 1/sqrt
  const double g2 = 1.0 + mass * mass * s.lam * s.lam;
  const double igam = rsqrt_any(g2);
  const R gam = (R)(g2 * igam);
  if (CMASK & 4) s.gtl += hr * (R)(mass * mass * s.lam * kInvC * igam);
  // advance the double accumulators with float (mixed) increments
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R dr = h2 * a1[i] + h3 * a2[i] + h4 * a3[i];
    const R dT = hr * a1[i] + h2 * a2[i] + h3 * a3[i] + h4 * a4[i];
    s.r[i] = fma(h, s.T[i], s.r[i]) + (double)dr;
    s.T[i] += (double)dT;
  }
  s.t += (double)(hr * gam * (R)kInvC);
}

// signed straight-line distance along T from r to the plane (c, n)
template <typename R>
__device__ __forceinline__ bool plane_step(const Prop<R>& s, const Surf& sb, double& out) {
  const double d = sb.n(0) * (sb.c(0) - s.r[0]) + sb.n(1) * (sb.c(1) - s.r[1]) + sb.n(2) * (sb.c(2) - s.r[2]);
  const double nT = sb.n(0) * s.T[0] + sb.n(1) * s.T[1] + sb.n(2) * s.T[2];
  if (!(fabs(nT) > 1e-9)) return false;
  out = d * rcp_any(nT);
  return true;
}

}  // namespace dev
}  // namespace kfgb
