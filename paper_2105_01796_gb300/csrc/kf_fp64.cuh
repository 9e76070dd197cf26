// kf_fp64.cuh -- double-precision building blocks shared by the FP64 fit
// kernel and the method-variant kernel: the transport Jacobian layout, the
// per-state workspace record, the gain-matrix update with the Joseph form and
// the Rauch-Tung-Striebel smoother over the stored records (paper Sect. 2).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_device.cuh"
#include "kf_internal.h"

namespace kfgb {
namespace dev {

// 1/sqrt(x) (x > 0) and 1/x (x != 0) for the whole double range: the
// argument is scaled by a power of two into [1, 4) (resp. [1, 2)) on the
// integer pipe, the two-step Newton form runs there, and the result is
// scaled back.  Arguments with extreme exponents (zero, subnormal, Inf, NaN)
// take CUDA's double operations, so NaN and Inf propagate as usual.
__device__ __forceinline__ double rsqrt_any(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e < -1000 || e > 1000) return 1.0 / sqrt(x);
  const int k = e >> 1;
  const double r = rsqrt_nr<2>(__hiloint2double(hi - (k << 21), __double2loint(x)));
  return __hiloint2double(__double2hiint(r) - (k << 20), __double2loint(r));
}

__device__ __forceinline__ double rcp_any(double x) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e < -1000 || e > 1000) return 1.0 / x;
  const double r = rcp_nr<2>(__hiloint2double(hi - (e << 20), __double2loint(x)));
  return __hiloint2double(__double2hiint(r) - (e << 20), __double2loint(r));
}

// ---------------------------------------------------------------------------
// transport Jacobian F of one transition: rows 0..3 and 5 over columns 0..4
// are stored; row 4 (q/p) is e4 times the energy-loss factor, column 5 is e5.
// ---------------------------------------------------------------------------
template <typename R>
struct Jac {
  R f[4][5];   // rows loc0, loc1, phi, theta over columns 0..4
  R ft[5];     // time row over columns 0..4 (column 5 of that row is 1)
};

// element (r, c) of F for r in {0..3, 5}, c in 0..4 (a value select, so the
// struct stays in registers when r and c are compile-time constants)
template <typename R>
__device__ __forceinline__ R jf(const Jac<R>& J, int r, int c) { return r == 5 ? J.ft[c] : J.f[r][c]; }

// ---------------------------------------------------------------------------
// workspace access: record element e of state k for chunk track i
// ---------------------------------------------------------------------------
struct WS {
  double* w64;
  float* w32;
  size_t nt;
  int rec64, rec32;
  int i;
  __device__ double& d(int k, int e) const { return w64[((size_t)k * rec64 + e) * nt + i]; }
  __device__ float& f(int k, int e) const { return w32[((size_t)k * rec32 + e) * nt + i]; }
};

// Storage of the record fields whose precision depends on the path.
template <int PREC> struct Rec;
template <> struct Rec<0> {
  static constexpr int XP = 0, XF = 6, CP = 12, CF = 33, BM = 54;
  __device__ static void put_cf(const WS& w, int k, int e, double v) { w.d(k, CF + e) = v; }
  __device__ static double get_cf(const WS& w, int k, int e) { return w.d(k, CF + e); }
  __device__ static void put_bm(const WS& w, int k, int e, double v) { w.d(k, BM + e) = v; }
  __device__ static double get_bm(const WS& w, int k, int e) { return w.d(k, BM + e); }
};

// ---------------------------------------------------------------------------
// gain-matrix update with the Joseph covariance form (double precision for
// the covariance and chi2; the gain in R).  Cp, Cf packed lower triangles.
//   S = V + H Cp H^T, K = Cp H^T S^-1, xf = xp + K r
//   Cf = (I-KH) Cp (I-KH)^T + K V K^T
//      = Cp + K W - (H Cp)^T K^T,  W = S K^T - H Cp   (expanded, exact for any K)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int kalman_update(const double xp[6], const double Cp[21], const double m[2],
                                             const double V[3], double xf[6], double Cf[21],
                                             double& chi2) {
  const double S00 = V[0] + Cp[sy(0, 0)], S01 = V[1] + Cp[sy(1, 0)], S11 = V[2] + Cp[sy(1, 1)];
  const double det = S00 * S11 - S01 * S01;
  if (!(det > 0.0) || !(S00 > 0.0)) return ST_NON_SPD;
  const double idet = rcp_any(det);
  const double r0 = m[0] - xp[0], r1 = m[1] - xp[1];
  chi2 = (S11 * r0 * r0 - 2.0 * S01 * r0 * r1 + S00 * r1 * r1) * idet;
  // gain in R
  const R i00 = (R)(S11 * idet), i01 = (R)(-S01 * idet), i11 = (R)(S00 * idet);
  double K[6][2];
  const R rr0 = (R)r0, rr1 = (R)r1;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const R c0 = (R)Cp[sym(i, 0)], c1 = (R)Cp[sym(i, 1)];
    const R k0 = c0 * i00 + c1 * i01;
    const R k1 = c0 * i01 + c1 * i11;
    K[i][0] = (double)k0;
    K[i][1] = (double)k1;
    xf[i] = xp[i] + (double)(k0 * rr0 + k1 * rr1);
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
    for (int j = 0; j < 6; ++j) if (j <= i) {
      double v = Cp[sy(i, j)];
      v = fma(K[i][0], W[0][j], v);
      v = fma(K[i][1], W[1][j], v);
      v = fma(-Cp[sym(0, i)], K[j][0], v);
      v = fma(-Cp[sym(1, i)], K[j][1], v);
      Cf[sy(i, j)] = v;
    }
  return ST_OK;
}


// ---------------------------------------------------------------------------
// RTS smoother over the stored records (Sect. 2): for k = n-2 .. 0
//   A = Cf_k F^T Cp_{k+1}^-1 (from the Cholesky factor of Cp_{k+1} and the
//       stored Bm = F Cf_k),
//   xs_k = xf_k + A (xs_{k+1} - xp_{k+1}),  Cs_k = Cf_k + A (Cs_{k+1} - Cp_{k+1}) A^T.
// xs, Cs enter as the last filtered state and leave as the smoothed state 0;
// the smoothed parameters of every state go to out_states when it is set.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rts_smooth_fp64(const WS& ws, int n, double xs[6], double Cs[21],
                                               double* out_states, int64_t n_states, int64_t o0) {
  int status = ST_OK;
  if (out_states)
#pragma unroll
    for (int e = 0; e < 6; ++e) out_states[e * n_states + o0 + n - 1] = xs[e];
  for (int k = n - 2; k >= 0 && status == ST_OK; --k) {
    // dC = Cs_{k+1} - Cp_{k+1}; L = chol(Cp_{k+1})
    double L[21], dC[21];
#pragma unroll
    for (int e = 0; e < 21; ++e) {
      L[e] = ws.d(k + 1, Rec<0>::CP + e);
      dC[e] = Cs[e] - L[e];
    }
    double idg[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double dj = L[sy(j, j)];
#pragma unroll
      for (int q = 0; q < 6; ++q) if (q < j) dj -= L[sy(j, q)] * L[sy(j, q)];
      if (!(dj > 0.0)) status = ST_NON_SPD;
      idg[j] = rsqrt_any(dj);  // Newton-refined, double rounding level
      const double ljj = dj * idg[j];
      L[sy(j, j)] = ljj;
#pragma unroll
      for (int r = 0; r < 6; ++r) if (r > j) {
        double v = L[sy(r, j)];
#pragma unroll
        for (int q = 0; q < 6; ++q) if (q < j) v -= L[sy(r, q)] * L[sy(j, q)];
        L[sy(r, j)] = v * idg[j];
      }
    }
    if (status != ST_OK) break;
    // X = Cp^-1 Bm (column by column); the smoother gain is A = X^T
    double X[6][6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double y[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        double v = Rec<0>::get_bm(ws, k + 1, r * 6 + c);
#pragma unroll
        for (int q = 0; q < 6; ++q) if (q < r) v -= L[sy(r, q)] * y[q];
        y[r] = v * idg[r];
      }
#pragma unroll
      for (int r = 5; r >= 0; --r) {
        double v = y[r];
#pragma unroll
        for (int q = 0; q < 6; ++q) if (q > r) v -= L[sy(q, r)] * X[q][c];
        X[r][c] = v * idg[r];
      }
    }
    // xs_k = xf_k + A (xs_{k+1} - xp_{k+1})
    double d[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) d[e] = xs[e] - ws.d(k + 1, Rec<0>::XP + e);
    double Ar[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) Ar[r][c] = X[c][r];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 6; ++c) acc += Ar[r][c] * d[c];
      xs[r] = ws.d(k, Rec<0>::XF + r) + acc;
    }
    // Cs_k = Cf_k + A dC A^T
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double z[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc += Ar[r][q] * dC[sym(q, c)];
        z[c] = acc;
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) if (c <= r) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc += z[q] * Ar[c][q];
        Cs[sy(r, c)] = Rec<0>::get_cf(ws, k, sy(r, c)) + acc;
      }
    }
    if (out_states)
#pragma unroll
      for (int e = 0; e < 6; ++e) out_states[e * n_states + o0 + k] = xs[e];
  }
  return status;
}

}  // namespace dev
}  // namespace kfgb
