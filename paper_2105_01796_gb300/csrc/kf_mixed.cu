// kf_mixed.cu -- the mixed-precision fit kernel (sm_103a).
//
// Same method as the FP64 kernel (paper Sect. 2 filter step list and RTS
// smoother; Sect. 4.1 RKN transport with local<->global Jacobians; Sect. 4.2
// double-precision inverter), arranged for a part whose FP64 pipe is a
// small fraction of its FP32 pipe:
//   * FP32: RKN stages, the step Jacobians, path correction, the 6x6
//     transport F C F^T, the Highland noise, the gain K, the smoother gain
//     algebra and the smoothed covariance.
//   * FP64: the Joseph covariance update, chi2, the LDL^T factorisation
//     of the predicted covariance and its solves (the smoother's inverse).
//   * Double-float pairs of FP32 values (about 48 bits): the track's point,
//     direction, angles, q/p and time between surfaces, which only receive
//     FP32 increments and meet the plane geometry (split the same way in
//     this kernel's own surface table) in dot products; no FP64 instruction
//     is spent on them.
//   * float<->double conversions run on the integer pipe (dev::f2d/d2f);
//     FP64 1/sqrt and 1/x come from float seeds refined by a Newton step.
//   * The direction is carried as (phi, theta) with their cosines and
//     sines; propagation and updates change them by small rotations, so no
//     trigonometry of the carried angles runs after the seed.
//
// Smoother in noise-rank form.  With Cp' = F Cf F^T + Q (Q non-zero only in
// the (phi, theta) block) the RTS gain A = Cf F^T Cp'^-1 equals
//   A = F^-1 (I - Q Cp'^-1),
// and the smoothed covariance Cs = Cf + A (Cs' - Cp') A^T equals
//   Cs = F^-1 (Q - Q Cp'^-1 Q) F^-T + A Cs' A^T,
// a sum of two positive semi-definite terms (no cancellation against Cf).
// Only the (phi, theta) columns of Cp'^-1 are needed: one FP64 LDL^T
// factorisation of a 4x4 block and two FP64 triangular-solve pairs per state.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_device.cuh"
#include "kf_internal.h"

namespace kfgb {
namespace {
using namespace dev;

// per-state record: x_p in FP64 (written for state 0, and for every state
// when the smoothed states are output); in FP32 the transport Jacobian, the
// scattering variances, the filter increment and the predicted covariance
// (its values are FP32 products, so the float copy is exact; the smoother
// promotes them for its FP64 inverse)
constexpr int XP = 0;                                           // ws64 fields
constexpr int FJ = 0, QPHI = 25, QTH = 26, DXF = 27, CPF = 33;  // ws32 fields

// ---- double-float ("df") values: an unevaluated sum hi + lo of two floats
// with |lo| <= ulp(hi) / 2, about 48 significant bits.  Error-free
// transformations: Knuth's TwoSum, Dekker's Fast2Sum and the exact product
// from one FMA; sums and products of df values as in Dekker (1971), dot
// products as Dot2 of Ogita, Rump and Oishi (2005).  The _rn intrinsics keep
// the compiler from contracting or reassociating these steps.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// exact for |a| >= |b| or a = 0
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// x + f (the final TwoSum keeps the pair normalised under cancellation)
__device__ __forceinline__ DF df_add_f(DF x, float f) {
  const DF s = two_sum(x.hi, f);
  return two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
// x + y, with the low parts summed exactly as well
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  const DF t = two_sum(x.lo, y.lo);
  const DF u = two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
// x * y (the lo * lo term is below the pair's resolution)
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const DF p = two_prod(x.hi, y.hi);
  return fast_two_sum(p.hi, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo)));
}
// float value (hi + lo rounded)
__device__ __forceinline__ float df_f(DF x) { return __fadd_rn(x.hi, x.lo); }
// conversions: to FP64 exactly, from FP64 as the nearest float and the
// nearest float to the rest
__device__ __forceinline__ double df_to_d(DF x) { return f2d(x.hi) + f2d(x.lo); }
__device__ __forceinline__ DF df_from_d(double v) {
  const float h = d2f(v);
  return {h, d2f(v - f2d(h))};
}
// w . r - w0 for a vector w given as hi / lo float arrays and a df offset
// w0: Dot2 (the products split exactly by FMA, the running sum by TwoSum,
// every error term gathered in one float), as accurate as a dot product in
// twice the float precision; the wl * r.lo terms are below that
__device__ __forceinline__ DF df_dot(const float* wh, const float* wl, DF w0, const DF r[3]) {
  float s = -w0.hi, c = -w0.lo;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const DF p = two_prod(wh[i], r[i].hi);
    const DF q = two_sum(s, p.hi);
    s = q.hi;
    c = __fadd_rn(c, __fadd_rn(q.lo, p.lo));
    c = __fmaf_rn(wh[i], r[i].lo, c);
    c = __fmaf_rn(wl[i], r[i].hi, c);
  }
  return two_sum(s, c);
}

// this kernel's surface record (32 floats, layout in kf_internal.h)
struct SurfM {
  const float* f;  // shared memory
  __device__ const float* nh() const { return f; }
  __device__ const float* uh() const { return f + 3; }
  __device__ const float* vh() const { return f + 6; }
  __device__ const float* nl() const { return f + 10; }
  __device__ const float* ul() const { return f + 13; }
  __device__ const float* vl() const { return f + 16; }
  __device__ float nf(int i) const { return f[i]; }
  __device__ float uf(int i) const { return f[3 + i]; }
  __device__ float vf(int i) const { return f[6 + i]; }
  __device__ float xx0f() const { return f[9]; }
  __device__ DF nc() const { return {f[19], f[22]}; }
  __device__ DF uc() const { return {f[20], f[23]}; }
  __device__ DF vc() const { return {f[21], f[24]}; }
  __device__ DF c(int i) const { return {f[25 + i], f[28 + i]}; }
  __device__ DF u(int i) const { return {f[3 + i], f[13 + i]}; }
  __device__ DF v(int i) const { return {f[6 + i], f[16 + i]}; }
};
__device__ __forceinline__ SurfM surf_m(const double* s_surf, int sid) {
  return SurfM{reinterpret_cast<const float*>(s_surf + (size_t)sid * kSurfStrideM)};
}

struct WSM {
  double* w64;
  float* w32;
  size_t nt;
  int i;
  __device__ double& d(int k, int e) const { return w64[((size_t)k * kRec64Mixed + e) * nt + i]; }
  __device__ float& f(int k, int e) const { return w32[((size_t)k * kRec32Mixed + e) * nt + i]; }
};

// direction: the angles and the unit direction vector, all df
struct Dir {
  DF phi, theta;
  DF T[3];  // (cos phi sin theta, sin phi sin theta, cos theta), unit up to rounding
};

// float cosines and sines of the direction's angles, from T
__device__ __forceinline__ void dir_cs(const DF T[3], float& cp, float& sp, float& ct, float& st) {
  const float t0 = T[0].hi, t1 = T[1].hi, t2 = T[2].hi;
  const float rho = sqrtf(t0 * t0 + t1 * t1);
  const float irho = 1.0f / rho, itn = rsqrtf(rho * rho + t2 * t2);
  cp = t0 * irho;
  sp = t1 * irho;
  st = rho * itn;
  ct = t2 * itn;
}

// FP32 Jacobian columns along the path (G = D J_bf): phi, theta, q/p
struct Cols {
  float gr[3][3], gT[3][3], gtl;
};

struct JacF {
  float f[4][5];  // rows loc0, loc1, phi, theta over columns loc0..q/p
  float ft[5];    // time row over columns loc0..q/p
};

// element (r, c) of F for r in {0..3, 5}, c in 0..4 (a value select, so the
// struct stays in registers when r and c are compile-time constants)
__device__ __forceinline__ float jf(const JacF& J, int r, int c) { return r == 5 ? J.ft[c] : J.f[r][c]; }

// G advance for one RKN4 step of length h (FP32): direction rows <- Stt g,
// position rows += Srt g, plus the q/p column's dStt/dlam T, dSrt/dlam T.
template <bool BZ>
__device__ __forceinline__ void cols_step(Cols& g, float h, const float bs[3], const float kB[3],
                                          const float T[3], float dtl) {
  const float h2 = h * h * 0.5f, h3 = h * h * h * (1.0f / 6.0f), h4 = h * h * h * h * (1.0f / 24.0f);
  float u0[3], u1[3], u2[3], u3[3];
  applyA<float, BZ>(kB, T, u0);
  applyA<float, BZ>(bs, u0, u1);
  applyA<float, BZ>(bs, u1, u2);
  applyA<float, BZ>(bs, u2, u3);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float v[3] = {g.gT[0][c], g.gT[1][c], g.gT[2][c]};
    float b1[3], b2[3], b3[3], b4[3];
    applyA<float, BZ>(bs, v, b1);
    applyA<float, BZ>(bs, b1, b2);
    applyA<float, BZ>(bs, b2, b3);
    applyA<float, BZ>(bs, b3, b4);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float dr = h * v[i] + h2 * b1[i] + h3 * b2[i] + h4 * b3[i];
      float nt = v[i] + h * b1[i] + h2 * b2[i] + h3 * b3[i] + h4 * b4[i];
      if (c == 2) {
        dr += h2 * u0[i] + h * h * h * (1.0f / 3.0f) * u1[i] + h * h * h * h * 0.125f * u2[i];
        nt += h * u0[i] + h * h * u1[i] + h * h * h * 0.5f * u2[i] + h * h * h * h * (1.0f / 6.0f) * u3[i];
      }
      g.gr[i][c] += dr;
      g.gT[i][c] = nt;
    }
  }
  g.gtl += h * dtl;
}

// value increments of one RKN4 step: dr_curv = (Srt - hI) T, dT = (Stt - I) T
template <bool BZ>
__device__ __forceinline__ void value_step(float h, const float bs[3], const float T[3], float dr[3],
                                           float dT[3]) {
  const float h2 = h * h * 0.5f, h3 = h * h * h * (1.0f / 6.0f), h4 = h * h * h * h * (1.0f / 24.0f);
  float a1[3], a2[3], a3[3], a4[3];
  applyA<float, BZ>(bs, T, a1);
  applyA<float, BZ>(bs, a1, a2);
  applyA<float, BZ>(bs, a2, a3);
  applyA<float, BZ>(bs, a3, a4);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dr[i] = h2 * a1[i] + h3 * a2[i] + h4 * a3[i];
    dT[i] = h * a1[i] + h2 * a2[i] + h3 * a3[i] + h4 * a4[i];
  }
}

// float cosines and sines of the direction's angles, carried with it
struct CS {
  float cp, sp, ct, st;
};

// sin(a) and cos(a) - 1 for a small float angle: series for |a| <= 0.1
// (truncation below 3e-12 relative), sincosf otherwise
__device__ __forceinline__ void sin_cosm1(float a, float& s, float& cm1) {
  if (fabsf(a) <= 0.1f) {
    const float a2 = a * a;
    s = a * (1.0f - a2 * (1.0f / 6.0f) * (1.0f - a2 * (1.0f / 20.0f) * (1.0f - a2 * (1.0f / 42.0f))));
    cm1 = -0.5f * a2 * (1.0f - a2 * (1.0f / 12.0f) * (1.0f - a2 * (1.0f / 30.0f) * (1.0f - a2 * (1.0f / 56.0f))));
  } else {
    float sh, ch;
    sincosf(0.5f * a, &sh, &ch);
    s = 2.0f * sh * ch;
    cm1 = -2.0f * sh * sh;
  }
}

// atan2(y, x) for a small angle (x > 0, |y| <= 0.1 x): series of atan(y/x)
// (truncation below 1e-10 relative); atan2f otherwise
__device__ __forceinline__ float small_atan2(float y, float x) {
  if (x > 0.0f && fabsf(y) <= 0.1f * x) {
    const float q = y / x, q2 = q * q;
    return q * (1.0f - q2 * (1.0f / 3.0f - q2 * (1.0f / 5.0f - q2 * (1.0f / 7.0f - q2 * (1.0f / 9.0f)))));
  }
  return atan2f(y, x);
}

// The filter's increments of the state that the next transport applies
// (zero after a hole): in-plane move of the point, change of the unit
// direction, and the increments of phi, theta and t.
struct Pend {
  float r[3], T[3], phi, theta, t;
};

// change of the unit direction when (phi, theta) turn by small increments
// (a, b): every term is proportional to the increments, so FP32 carries it
// with full relative precision.  cs enters as the cosines / sines of the
// old angles and leaves as those of the new ones.
__device__ __forceinline__ void turn_inc(CS& cs, float a, float b, float out[3]) {
  float sa, ca1, sb, cb1;  // sin, cos - 1
  sin_cosm1(a, sa, ca1);
  sin_cosm1(b, sb, cb1);
  const float cp = cs.cp, sp = cs.sp, ct = cs.ct, st = cs.st;
  const float dcp = cp * ca1 - sp * sa, dsp = sp * ca1 + cp * sa;
  const float dct = ct * cb1 - st * sb, dst = st * cb1 + ct * sb;
  out[0] = cp * dst + dcp * st + dcp * dst;
  out[1] = sp * dst + dsp * st + dsp * dst;
  out[2] = dct;
  cs.cp = cp + dcp;
  cs.sp = sp + dsp;
  cs.ct = ct + dct;
  cs.st = st + dst;
}


// Transport the filtered state on surface a to surface b.  The filtered
// state is the predicted one (point r0, direction d, time x[5]) plus the
// filter's pending FP32 increments pd; x[4] is the filtered q/p.
template <bool BZ>
__device__ __forceinline__ int transport_mixed(const SurfM& sa, const SurfM& sb, const DF r0[3], const DF x[6],
                               const Dir& d, const Pend& pd, CS& cs, const float Bf[3], float m2, float h_max,
                               int n_iter, DF xp[6], DF rp[3], Dir& dp, JacF& J, float& sin_th,
                               float& cos_inc) {
  // The point and the direction stay df (predicted values of surface a);
  // everything that moves them here (the pending filter increments, the RKN
  // curvature terms, the direction change accT, the plane corrections) is
  // summed in FP32 and added once at the end.
  DF r[3] = {r0[0], r0[1], r0[2]};
  const DF* Td = d.T;
  const float T0f[3] = {Td[0].hi + (Td[0].lo + pd.T[0]), Td[1].hi + (Td[1].lo + pd.T[1]),
                        Td[2].hi + (Td[2].lo + pd.T[2])};
  const float lam = df_f(x[4]);
  const float lk = lam * (float)kKappa;
  const float bs[3] = {lk * Bf[0], lk * Bf[1], lk * Bf[2]};
  const float kB[3] = {(float)kKappa * Bf[0], (float)kKappa * Bf[1], (float)kKappa * Bf[2]};
  const float gam = sqrtf(1.0f + m2 * lam * lam);
  const float dtds = gam * (float)kInvC;
  const float dtl = m2 * lam * (float)kInvC / gam;  // d(dt/ds)/dlam
  Cols g;
  {
    const float cpf = cs.cp, spf = cs.sp, ctf = cs.ct, stf = cs.st;
    g.gT[0][0] = -spf * stf; g.gT[1][0] = cpf * stf; g.gT[2][0] = 0.0f;
    g.gT[0][1] = cpf * ctf;  g.gT[1][1] = spf * ctf; g.gT[2][1] = -stf;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g.gT[i][2] = 0.0f;
      g.gr[i][0] = g.gr[i][1] = g.gr[i][2] = 0.0f;
    }
    g.gtl = 0.0f;
  }
  const float nb[3] = {sb.nf(0), sb.nf(1), sb.nf(2)};
  float accT[3] = {0.0f, 0.0f, 0.0f};  // T_end - T_start
  float accR[3] = {0.0f, 0.0f, 0.0f};  // r_end - r_start - s0 T_start
  float tinc = 0.0f;                    // t_end - t_start
  // main steps over the straight-line distance s0: the position moves by
  // s0 T_start (df) plus the FP32 offsets of the curvature and of the
  // direction change
  DF s0d, dist;
  {
    dist = df_neg(df_dot(sb.nh(), sb.nl(), sb.nc(), r));  // n.c - n.r
    const float nT = nb[0] * T0f[0] + nb[1] * T0f[1] + nb[2] * T0f[2];
    if (!(fabsf(nT) > 1e-9f)) return ST_NO_INTERSECTION;
    const float s0 = (df_f(dist) - (nb[0] * pd.r[0] + nb[1] * pd.r[1] + nb[2] * pd.r[2])) / nT;
    const float nsub_f = ceilf(fabsf(s0) / h_max);
    if (!(nsub_f <= 64.0f)) return ST_NO_INTERSECTION;
    const int nsub = nsub_f < 1.0f ? 1 : (int)nsub_f;
    const float h = s0 / (float)nsub;
    s0d = two_prod(h, (float)nsub);  // exact: nsub is a small integer
    for (int k = 0; k < nsub; ++k) {
      const float Tf[3] = {T0f[0] + accT[0], T0f[1] + accT[1], T0f[2] + accT[2]};
      cols_step<BZ>(g, h, bs, kB, Tf, dtl);
      float dr[3], dT[3];
      value_step<BZ>(h, bs, Tf, dr, dT);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        accR[i] += h * accT[i] + dr[i];
        accT[i] += dT[i];
      }
      tinc += h * dtds;
    }
  }
  // Newton corrections onto the plane, as float offsets from the main end.
  // The main end is r_main = r0 + s0 Td + off with the FP32 offset
  // off = pd.r + s0 pd.T + accR; the remaining distance is
  // n.(c - r_main) = dist - s0 (n.Td) - n.off.
  const float s0f = s0d.hi;
  float off[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) off[i] = pd.r[i] + s0f * pd.T[i] + accR[i];
  {
    const DF nTd = df_dot(sb.nh(), sb.nl(), DF{0.0f, 0.0f}, Td);
    const float dmf = df_f(df_add(dist, df_neg(df_mul(s0d, nTd)))) - (nb[0] * off[0] + nb[1] * off[1] + nb[2] * off[2]);
    const float Tm[3] = {T0f[0] + accT[0], T0f[1] + accT[1], T0f[2] + accT[2]};
    float orr[3] = {0.0f, 0.0f, 0.0f}, oT[3] = {0.0f, 0.0f, 0.0f}, ot = 0.0f;
    for (int it = 0; it < n_iter; ++it) {
      const float Tc[3] = {Tm[0] + oT[0], Tm[1] + oT[1], Tm[2] + oT[2]};
      const float dist = dmf - (nb[0] * orr[0] + nb[1] * orr[1] + nb[2] * orr[2]);
      const float nT = nb[0] * Tc[0] + nb[1] * Tc[1] + nb[2] * Tc[2];
      if (!(fabsf(nT) > 1e-9f)) return ST_NO_INTERSECTION;
      const float si = dist / nT;
      if (it == 0) {
        cols_step<BZ>(g, si, bs, kB, Tc, dtl);
      } else {
        // later corrections are tiny (|si| ~ |s1|^2 curvature): the columns
        // take their first-order terms in si only (position += si dir, and
        // the q/p column's direction += si d(A T)/dlam); the rest is
        // O(si k B) relative, far below FP32 resolution
        float u0[3];
        applyA<float, BZ>(kB, Tc, u0);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int i = 0; i < 3; ++i) g.gr[i][c] += si * g.gT[i][c];
#pragma unroll
        for (int i = 0; i < 3; ++i) g.gT[i][2] += si * u0[i];
        g.gtl += si * dtl;
      }
      float dr[3], dT[3];
      value_step<BZ>(si, bs, Tc, dr, dT);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        orr[i] += si * Tc[i] + dr[i];
        oT[i] += dT[i];
      }
      ot += si * dtds;
    }
    // the bound state lives on the plane: the end point is projected onto it
    // along n by the distance the corrections leave (a few 1e-4 mm after one
    // correction, nothing after two; the whole curvature miss with none)
    const float drem = dmf - (nb[0] * orr[0] + nb[1] * orr[1] + nb[2] * orr[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      r[i] = df_add_f(df_add(r[i], df_mul(s0d, Td[i])), off[i] + orr[i] + drem * nb[i]);
      accT[i] += oT[i];
    }
    tinc += ot;
  }
  const DF t = df_add_f(x[5], pd.t + tinc);
  // end angles: the rotation from the start to the end direction, computed in
  // FP32 from the start direction c and its change a = accT (no cancellation
  // of large terms):
  //   tan dphi = (c0 a1 - c1 a0) / (rho^2 + c0 a0 + c1 a1),
  //   tan dtheta = (c2 drho - rho a2) / (c2 (c2 + a2) + rho (rho + drho)),
  // with rho = |(c0, c1)| and drho the change of rho; the df angles and
  // their cosines / sines then turn by these increments.
  {
    const float c0 = T0f[0], c1 = T0f[1], c2 = T0f[2];
    const float a0 = accT[0], a1 = accT[1], a2 = accT[2];
    const float rho_sq = c0 * c0 + c1 * c1;
    const float dphi = small_atan2(c0 * a1 - c1 * a0, rho_sq + c0 * a0 + c1 * a1);
    const float drho_sq = 2.0f * (c0 * a0 + c1 * a1) + a0 * a0 + a1 * a1;
    const float rho = sqrtf(rho_sq), rho_end = sqrtf(rho_sq + drho_sq);
    const float drho = drho_sq / (rho + rho_end);
    const float dth = small_atan2(c2 * drho - rho * a2, c2 * (c2 + a2) + rho * (rho + drho));
    DF phi = df_add_f(d.phi, pd.phi + dphi);
    // keep phi in (-pi, pi]: pi as the df pair (nearest float, rest)
    constexpr float kPiHi = 3.14159274101257324f, kPiLo = -8.742278000372475e-08f;
    if (phi.hi > kPiHi || (phi.hi == kPiHi && phi.lo > kPiLo))
      phi = df_add(phi, DF{-2.0f * kPiHi, -2.0f * kPiLo});
    else if (phi.hi < -kPiHi || (phi.hi == -kPiHi && phi.lo <= -kPiLo))
      phi = df_add(phi, DF{2.0f * kPiHi, 2.0f * kPiLo});
    dp.phi = phi;
    dp.theta = df_add_f(d.theta, pd.theta + dth);
#pragma unroll
    for (int i = 0; i < 3; ++i) dp.T[i] = df_add_f(Td[i], pd.T[i] + accT[i]);
  }
  rp[0] = r[0];
  rp[1] = r[1];
  rp[2] = r[2];
  xp[0] = df_dot(sb.uh(), sb.ul(), sb.uc(), r);
  xp[1] = df_dot(sb.vh(), sb.vl(), sb.vc(), r);
  xp[2] = dp.phi;
  xp[3] = dp.theta;
  xp[4] = x[4];
  xp[5] = t;

  // path correction and free -> bound Jacobian (FP32)
  float cph, sph, cth, sth;
  dir_cs(dp.T, cph, sph, cth, sth);
  cs = CS{cph, sph, cth, sth};
  const float Tu[3] = {cph * sth, sph * sth, cth};
  const float nT = nb[0] * Tu[0] + nb[1] * Tu[1] + nb[2] * Tu[2];
  float AT[3];
  applyA<float, BZ>(bs, Tu, AT);
  const float inv_nT = 1.0f / nT;
  float Gr[3][5], GT[3][5], Gt[5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gr[i][0] = sa.uf(i);
    Gr[i][1] = sa.vf(i);
    Gr[i][2] = g.gr[i][0];
    Gr[i][3] = g.gr[i][1];
    Gr[i][4] = g.gr[i][2];
    GT[i][0] = 0.0f;
    GT[i][1] = 0.0f;
    GT[i][2] = g.gT[i][0];
    GT[i][3] = g.gT[i][1];
    GT[i][4] = g.gT[i][2];
  }
  Gt[0] = Gt[1] = Gt[2] = Gt[3] = 0.0f;
  Gt[4] = g.gtl;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const float w = -(nb[0] * Gr[0][c] + nb[1] * Gr[1][c] + nb[2] * Gr[2][c]) * inv_nT;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i][c] += Tu[i] * w;
      GT[i][c] += AT[i] * w;
    }
    Gt[c] += dtds * w;
  }
  const float ub[3] = {sb.uf(0), sb.uf(1), sb.uf(2)};
  const float vb[3] = {sb.vf(0), sb.vf(1), sb.vf(2)};
  const float inv_sth = 1.0f / sth;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    J.f[0][c] = ub[0] * Gr[0][c] + ub[1] * Gr[1][c] + ub[2] * Gr[2][c];
    J.f[1][c] = vb[0] * Gr[0][c] + vb[1] * Gr[1][c] + vb[2] * Gr[2][c];
    J.f[2][c] = (-sph * GT[0][c] + cph * GT[1][c]) * inv_sth;
    J.f[3][c] = cph * cth * GT[0][c] + sph * cth * GT[1][c] - sth * GT[2][c];
    J.ft[c] = Gt[c];
  }
  sin_th = sth;
  cos_inc = nT;
  return ST_OK;
}

// 6x6 inverse of the transport Jacobian F in FP32, using its structure
// (q/p row = e4, time column = e5):  with F11 the loc/angle 4x4 block,
//   F^-1 = [[F11^-1, -F11^-1 f12, 0], [0, 1, 0], [-ft F11^-1, ft F11^-1 f12 - ft4, 1]].
// F11^-1 by 2x2 blocks (the loc-loc and angle-angle blocks are near identity):
//   F11 = [[P, Qb], [Rb, S]], Z = (S - Rb P^-1 Qb)^-1,
//   F11^-1 = [[P^-1 + P^-1 Qb Z Rb P^-1, -P^-1 Qb Z], [-Z Rb P^-1, Z]].
__device__ __forceinline__ void inv2(const float a[2][2], float o[2][2]) {
  const float id = 1.0f / (a[0][0] * a[1][1] - a[0][1] * a[1][0]);
  o[0][0] = a[1][1] * id;
  o[0][1] = -a[0][1] * id;
  o[1][0] = -a[1][0] * id;
  o[1][1] = a[0][0] * id;
}

__device__ __forceinline__ void mul2(const float a[2][2], const float b[2][2], float o[2][2]) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) o[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j];
}

__device__ __forceinline__ void invert_F(const float F[25], float Fi[6][6]) {
  float P[2][2], Qb[2][2], Rb[2][2], S[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      P[i][j] = F[i * 5 + j];
      Qb[i][j] = F[i * 5 + 2 + j];
      Rb[i][j] = F[(2 + i) * 5 + j];
      S[i][j] = F[(2 + i) * 5 + 2 + j];
    }
  float Pi[2][2], PiQ[2][2], RPi[2][2], Sc[2][2], Z[2][2], t1[2][2], t2[2][2];
  inv2(P, Pi);
  mul2(Pi, Qb, PiQ);
  mul2(Rb, Pi, RPi);
  mul2(Rb, PiQ, t1);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) Sc[i][j] = S[i][j] - t1[i][j];
  inv2(Sc, Z);
  float M[4][4];
  mul2(PiQ, Z, t1);  // P^-1 Qb Z
  mul2(t1, RPi, t2);  // P^-1 Qb Z Rb P^-1
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      M[i][j] = Pi[i][j] + t2[i][j];
      M[i][2 + j] = -t1[i][j];
      M[2 + i][2 + j] = Z[i][j];
    }
  mul2(Z, RPi, t2);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) M[2 + i][j] = -t2[i][j];
  // assemble
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float mf = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      Fi[i][j] = M[i][j];
      mf += M[i][j] * F[j * 5 + 4];
    }
    Fi[i][4] = -mf;
    Fi[i][5] = 0.0f;
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) Fi[4][j] = (j == 4) ? 1.0f : 0.0f;
  float tf = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float v = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) v += F[20 + q] * M[q][j];
    Fi[5][j] = -v;
    tf += v * F[j * 5 + 4];
  }
  Fi[5][4] = tf - F[24];
  Fi[5][5] = 1.0f;
}

// Columns phi and theta of Cp^-1 in FP64, by block elimination with the
// angle block last: a = (loc0, loc1, q/p, t), b = (phi, theta).
//   X = Caa^-1 Cab (4x4 LDL^T, two solves), Sig = Cbb - Cab^T X (the 2x2
//   Schur complement), then (Cp^-1)[b][b] = Sig^-1, (Cp^-1)[a][b] = -X Sig^-1.
// Cp is SPD iff the four pivots of Caa and Sig are positive.  Returns false
// otherwise.  w[0] = Cp^-1 e_phi, w[1] = Cp^-1 e_theta (6 each).
__device__ __forceinline__ bool angle_columns_of_inverse(const double Cp[21], double w[2][6]) {
  constexpr int ia[4] = {0, 1, 4, 5};
  // LDL^T of the 4x4 block (no square roots): U = L D below the diagonal
  double L[4][4], U[4][4], iD[4];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    double dj = Cp[sym(ia[j], ia[j])];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < j) dj = fma(-U[j][q], L[j][q], dj);
    if (!dpos(dj)) {
      ok = false;
      dj = 1.0;
    }
    iD[j] = rcp_nr<1>(dj);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r > j) {
        double u = Cp[sym(ia[r], ia[j])];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < j) u = fma(-U[r][q], L[j][q], u);
        U[r][j] = u;
        L[r][j] = u * iD[j];
      }
    }
  }
  // X = Caa^-1 Cab: unit-lower forward solve, scaling by D^-1, unit-upper
  // backward solve
  double X[4][2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    double y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double v = Cp[sym(ia[r], 2 + m)];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < r) v = fma(-L[r][q], y[q], v);
      y[r] = v;
    }
#pragma unroll
    for (int r = 3; r >= 0; --r) {
      double v = y[r] * iD[r];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q > r) v = fma(-L[q][r], X[q][m], v);
      X[r][m] = v;
    }
  }
  double s00 = Cp[sy(2, 2)], s01 = Cp[sy(3, 2)], s11 = Cp[sy(3, 3)];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    s00 = fma(-Cp[sym(ia[r], 2)], X[r][0], s00);
    s01 = fma(-Cp[sym(ia[r], 2)], X[r][1], s01);
    s11 = fma(-Cp[sym(ia[r], 3)], X[r][1], s11);
  }
  const double det = fma(s00, s11, -s01 * s01);
  if (!dpos(det) || !dpos(s00)) {
    ok = false;
  }
  const double idet = rcp_nr<1>(det);
  const double i00 = s11 * idet, i01 = -s01 * idet, i11 = s00 * idet;
  w[0][2] = i00;
  w[0][3] = i01;
  w[1][2] = i01;
  w[1][3] = i11;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    w[0][ia[r]] = -fma(X[r][0], i00, X[r][1] * i01);
    w[1][ia[r]] = -fma(X[r][0], i01, X[r][1] * i11);
  }
  return ok;
}

template <bool BZ>
__device__ __forceinline__ void fit_one_mixed(const FitParams& p, const double* s_surf, int i) {
  const int t = track_of(p, i);
  const size_t TT = (size_t)p.n_tracks_total;
  const WSM ws{p.ws64, p.ws32, (size_t)p.n_tracks, i};
  const int64_t o0 = p.offsets[t], o1 = p.offsets[t + 1];
  const int n = (int)(o1 - o0);
  int status = ST_OK;
  if (!(o1 > o0) || o0 < 0 || o1 > p.n_states || n > p.max_states) status = ST_BAD_INPUT;
  if (status == ST_OK)
    for (int k = 0; k < n; ++k) {
      const int sid = p.surface_id[o0 + k];
      if (sid < 0 || sid >= p.n_surfaces) status = ST_BAD_INPUT;
    }
  const float m2 = (float)(p.mass * p.mass);
  const float h_max = (float)p.h_max;
  // the field as floats, once per track (copied to registers: taking the
  // address of a kernel parameter would move the parameter block to local
  // memory)
  const float Bf[3] = {(float)p.bfield[0], (float)p.bfield[1], (float)p.bfield[2]};

  double xs[6];
  double Cs_out[21];
  double chi2sum = 0.0;
  int nmeas = 0;
  if (status == ST_OK) {
    // ------------------------------------------------ forward filter
    // Between states the df state is the prediction of the last surface
    // (point r, direction d, time x[5]) plus the filter's FP32 increments
    // in pd, which the next transport applies; the filtered q/p is x[4].
    // The filtered covariance is kept in FP32 between states: it only feeds
    // the FP32 transport F Cf F^T (the Joseph update produces it in FP64).
    DF x[6], r[3];
    Pend pd = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, 0.0f, 0.0f, 0.0f};
    CS cs;  // float cosines / sines of the filtered direction
    float Cf[21];
    float dx[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // x_f - x_p of the last state
    Dir d;
    {
      double xs0[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        xs0[e] = p.seed_params[e * TT + t];
        x[e] = df_from_d(xs0[e]);
      }
      d.phi = x[2];
      d.theta = x[3];
      double sp, cp, st, ct;
      sincos(xs0[2], &sp, &cp);  // the only FP64 trigonometry of the track
      sincos(xs0[3], &st, &ct);
      d.T[0] = df_from_d(cp * st);
      d.T[1] = df_from_d(sp * st);
      d.T[2] = df_from_d(ct);
      cs = CS{d2f(cp), d2f(sp), d2f(ct), d2f(st)};
    }
    int sid_prev = p.surface_id[o0];
    {
      const SurfM s0 = surf_m(s_surf, sid_prev);
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = df_add(s0.c(c), df_add(df_mul(x[0], s0.u(c)), df_mul(x[1], s0.v(c))));
    }
    for (int k = 0; k < n && status == ST_OK; ++k) {
      const int sid = p.surface_id[o0 + k];
      DF xp[6], rp[3];
      double Cp[21];
      float Cpf[21];
      Dir dp;
      if (k == 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) xp[e] = x[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) {
          Cp[e] = p.seed_cov[e * TT + t];
          Cpf[e] = d2f(Cp[e]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) rp[c] = r[c];
        dp = d;
      } else {
        const SurfM sa = surf_m(s_surf, sid_prev), sb = surf_m(s_surf, sid);
        JacF J;
        float sin_th, cos_inc;
        status = transport_mixed<BZ>(sa, sb, r, x, d, pd, cs, Bf, m2, h_max, p.n_iter, xp, rp, dp, J, sin_th,
                                     cos_inc);
        if (status != ST_OK) break;
        const float* Cr = Cf;
        // Cp = F Cf F^T, rows of Bm = F Cf formed on the fly
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          float brow[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            float v;
            if (a == 4) {
              v = Cr[sym(4, j)];
            } else {
              v = jf(J, a, 0) * Cr[sym(0, j)] + jf(J, a, 1) * Cr[sym(1, j)] + jf(J, a, 2) * Cr[sym(2, j)] +
                  jf(J, a, 3) * Cr[sym(3, j)] + jf(J, a, 4) * Cr[sym(4, j)];
              if (a == 5) v += Cr[sym(5, j)];
            }
            brow[j] = v;
          }
#pragma unroll
          for (int c = 0; c < 6; ++c)
            if (c <= a) {
              float v;
              if (c == 4) {
                v = brow[4];
              } else {
                v = brow[0] * jf(J, c, 0) + brow[1] * jf(J, c, 1) + brow[2] * jf(J, c, 2) +
                    brow[3] * jf(J, c, 3) + brow[4] * jf(J, c, 4);
                if (c == 5) v += brow[5];
              }
              Cpf[sy(a, c)] = v;
            }
        }
        // multiple scattering of surface k, added before the update
        float qphi = 0.0f, qth = 0.0f;
        const float xx0 = sb.xx0f();
        if (xx0 > 0.0f) {
          const float th0 = highland<float>(fabsf(x[4].hi), m2, xx0, cos_inc);
          qth = th0 * th0;
          qphi = qth / (sin_th * sin_th);
          Cpf[sy(2, 2)] += qphi;
          Cpf[sy(3, 3)] += qth;
        }
#pragma unroll
        for (int e = 0; e < 20; ++e) ws.f(k, FJ + e) = J.f[e / 5][e % 5];
#pragma unroll
        for (int e = 0; e < 5; ++e) ws.f(k, FJ + 20 + e) = J.ft[e];
        ws.f(k, QPHI) = qphi;
        ws.f(k, QTH) = qth;
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp[e] = f2d(Cpf[e]);
      }
      if (k == 0 || p.out_states) {
#pragma unroll
        for (int e = 0; e < 6; ++e) ws.d(k, XP + e) = df_to_d(xp[e]);
      }
      if (k > 0) {
#pragma unroll
        for (int e = 0; e < 21; ++e) ws.f(k, CPF + e) = Cpf[e];
      }
      const SurfM sk = surf_m(s_surf, sid);
      if (!p.is_hole[o0 + k]) {
        // gain-matrix update: gain in FP32, Joseph covariance (but its K W term)
        // and chi2 in FP64
        const double m0 = p.loc[o0 + k], m1 = p.loc[p.n_states + o0 + k];
        const double V0 = p.cov[o0 + k], V1 = p.cov[p.n_states + o0 + k], V2 = p.cov[2 * p.n_states + o0 + k];
        const double S00 = V0 + Cp[sy(0, 0)], S01 = V1 + Cp[sy(1, 0)], S11 = V2 + Cp[sy(1, 1)];
        const double det = fma(S00, S11, -S01 * S01);
        if (!dpos(det) || !dpos(S00)) {
          status = ST_NON_SPD;
          break;
        }
        const double idet = rcp_nr<1>(det);
        const double r0 = (m0 - f2d(xp[0].hi)) - f2d(xp[0].lo), r1 = (m1 - f2d(xp[1].hi)) - f2d(xp[1].lo);
        const double u = fma(S11, r0, -S01 * r1), v = fma(S00, r1, -S01 * r0);
        chi2sum += fma(r0, u, r1 * v) * idet;
        ++nmeas;
        const float idf = d2f(idet);
        const float i00 = d2f(S11) * idf, i01 = -d2f(S01) * idf, i11 = d2f(S00) * idf;
        const float r0f = d2f(r0), r1f = d2f(r1);
        double K[6][2];
        float Kf[6][2];
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          const float c0 = Cpf[sym(e, 0)], c1 = Cpf[sym(e, 1)];
          const float k0 = c0 * i00 + c1 * i01, k1 = c0 * i01 + c1 * i11;
          Kf[e][0] = k0;
          Kf[e][1] = k1;
          K[e][0] = f2d(k0);
          K[e][1] = f2d(k1);
          dx[e] = k0 * r0f + k1 * r1f;
        }
        // Joseph form, expanded: Cf = Cp - (H Cp)^T K^T + K W with
        // W = S K^T - H Cp.  For the exact gain W = 0; here W is the residual
        // of the gain equation left by the FP32 gain, O(eps32 |H Cp|), so
        // the term K W is O(eps32 |Cp|).  FP64 takes the cancelling part
        // (Cp - (H Cp)^T K^T, and W itself); K W is summed in FP32 onto the
        // rounded result, which carries it to O(eps32^2 |Cp|).
        float Wf[2][6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          Wf[0][j] = d2f(fma(S00, K[j][0], fma(S01, K[j][1], -Cp[sym(0, j)])));
          Wf[1][j] = d2f(fma(S01, K[j][0], fma(S11, K[j][1], -Cp[sym(1, j)])));
        }
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b < 6; ++b)
            if (b <= a) {
              double v = Cp[sy(a, b)];
              v = fma(-Cp[sym(0, a)], K[b][0], v);
              v = fma(-Cp[sym(1, a)], K[b][1], v);
              Cf[sy(a, b)] = d2f(v) + (Kf[a][0] * Wf[0][b] + Kf[a][1] * Wf[1][b]);
            }
        // the filtered state: the prediction plus the increments, which stay
        // pending in FP32 (the point moves in the plane by (dx0, dx1)); only
        // q/p is updated here
#pragma unroll
        for (int c = 0; c < 3; ++c) pd.r[c] = dx[0] * sk.uf(c) + dx[1] * sk.vf(c);
        turn_inc(cs, dx[2], dx[3], pd.T);
        pd.phi = dx[2];
        pd.theta = dx[3];
        pd.t = dx[5];
        x[4] = df_add_f(xp[4], dx[4]);
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) dx[e] = 0.0f;
#pragma unroll
        for (int e = 0; e < 21; ++e) Cf[e] = Cpf[e];
        pd = Pend{{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, 0.0f, 0.0f, 0.0f};
        x[4] = xp[4];
      }
      // the df state moves to the prediction of surface k
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = rp[c];
      d = dp;
      x[5] = xp[5];
#pragma unroll
      for (int e = 0; e < 6; ++e) ws.f(k, DXF + e) = dx[e];
      sid_prev = sid;
    }

    // ------------------------------------------------ RTS smoother
    // The recursion runs on FP32 offsets: with dxf_k = x_f,k - x_p,k (the
    // filter increment) and off_k = x_s,k - x_f,k,
    //   x_s,k+1 - x_p,k+1 = dxf_{k+1} + off_{k+1},  off_k = A_k (that),
    // and x_s,k = x_p,k + dxf_k + off_k is formed in FP64 only for output.
    if (status == ST_OK) {
      float Cs[21];
      float off[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int e = 0; e < 21; ++e) Cs[e] = Cf[e];
      if (p.out_states)
#pragma unroll
        for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + n - 1] = ws.d(n - 1, XP + e) + f2d(dx[e]);
      for (int k = n - 2; k >= 0 && status == ST_OK; --k) {
        // FP64: the (phi, theta) columns of Cp_{k+1}^-1
        double Cp1[21];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp1[e] = f2d(ws.f(k + 1, CPF + e));
        double w[2][6];
        if (!angle_columns_of_inverse(Cp1, w)) {
          status = ST_NON_SPD;
          break;
        }
        // noise-rank pieces: Q Cp^-1 rows (phi, theta) and N = Q - Q Cp^-1 Q
        const float qp = ws.f(k + 1, QPHI), qt = ws.f(k + 1, QTH);
        const double qpd = f2d(qp), qtd = f2d(qt);
        float qw[2][6];
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          qw[0][e] = qp * d2f(w[0][e]);
          qw[1][e] = qt * d2f(w[1][e]);
        }
        const float Npp = d2f(qpd * fma(-qpd, w[0][2], 1.0));
        const float Ntt = d2f(qtd * fma(-qtd, w[1][3], 1.0));
        const float Npt = d2f(-qpd * qtd * w[1][2]);
        // F^-1 and the gain A = F^-1 - F^-1[:,phi] qw_phi^T - F^-1[:,theta] qw_theta^T
        float Fr[25];
#pragma unroll
        for (int e = 0; e < 25; ++e) Fr[e] = ws.f(k + 1, FJ + e);
        float Fi[6][6];
        invert_F(Fr, Fi);
        float A[6][6];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int c = 0; c < 6; ++c) A[a][c] = Fi[a][c] - Fi[a][2] * qw[0][c] - Fi[a][3] * qw[1][c];
        // off_k = A (dxf_{k+1} + off_{k+1})
        float dd[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) dd[e] = ws.f(k + 1, DXF + e) + off[e];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          float acc = 0.0f;
#pragma unroll
          for (int c = 0; c < 6; ++c) acc += A[a][c] * dd[c];
          off[a] = acc;
        }
        // Cs_k = F^-1 N F^-T (N on the (phi, theta) block) + A Cs_{k+1} A^T
        float Cn[21];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          float z[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            float acc = 0.0f;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc += A[a][q] * Cs[sym(q, c)];
            z[c] = acc;
          }
          const float a2 = Fi[a][2] * Npp + Fi[a][3] * Npt, a3 = Fi[a][2] * Npt + Fi[a][3] * Ntt;
#pragma unroll
          for (int c = 0; c < 6; ++c)
            if (c <= a) {
              float acc = a2 * Fi[c][2] + a3 * Fi[c][3];
#pragma unroll
              for (int q = 0; q < 6; ++q) acc += z[q] * A[c][q];
              Cn[sy(a, c)] = acc;
            }
        }
#pragma unroll
        for (int e = 0; e < 21; ++e) Cs[e] = Cn[e];
        if (p.out_states || k == 0) {
          float tot[6];
#pragma unroll
          for (int e = 0; e < 6; ++e) tot[e] = ws.f(k, DXF + e) + off[e];
#pragma unroll
          for (int e = 0; e < 6; ++e) xs[e] = ws.d(k, XP + e) + f2d(tot[e]);
          if (p.out_states)
#pragma unroll
            for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + k] = xs[e];
        }
      }
      if (n == 1) {
        // the filtered state 0: the seed plus the filter increment
#pragma unroll
        for (int e = 0; e < 6; ++e) xs[e] = p.seed_params[e * TT + t] + f2d(dx[e]);
#pragma unroll
        for (int e = 0; e < 21; ++e) Cs_out[e] = f2d(Cf[e]);
      } else {
#pragma unroll
        for (int e = 0; e < 21; ++e) Cs_out[e] = f2d(Cs[e]);
      }
    }
    if (status == ST_OK) {
      bool fin = isfinite(chi2sum);
#pragma unroll
      for (int e = 0; e < 6; ++e) fin = fin && isfinite(xs[e]);
#pragma unroll
      for (int e = 0; e < 21; ++e) fin = fin && isfinite(Cs_out[e]);
      if (!fin) status = ST_NONFINITE;
    }
  }
  if (status != ST_OK) {
    const double nan = qnan();
#pragma unroll
    for (int e = 0; e < 6; ++e) xs[e] = nan;
#pragma unroll
    for (int e = 0; e < 21; ++e) Cs_out[e] = nan;
    chi2sum = nan;
    nmeas = 0;
    if (p.out_states && n >= 1 && o0 >= 0 && o1 <= p.n_states && n <= p.max_states)
      for (int k = 0; k < n; ++k)
        for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + k] = nan;
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) p.out_params[e * TT + t] = xs[e];
#pragma unroll
  for (int e = 0; e < 21; ++e) p.out_cov[e * TT + t] = Cs_out[e];
  p.out_chi2[t] = chi2sum;
  if (p.out_ndf) p.out_ndf[t] = 2 * nmeas;
  if (p.out_status) p.out_status[t] = (uint8_t)status;
}

template <bool BZ>
struct MixedBody {
  static constexpr int kStride = kSurfStrideM;
  static __device__ __forceinline__ void run(const FitParams& p, const double* s_surf, int i) {
    fit_one_mixed<BZ>(p, s_surf, i);
  }
};

template <bool BZ>
cudaError_t launch_m(const FitParams& p, int block, int min_blocks, cudaStream_t stream, int* launched) {
  switch (min_blocks) {
    case 4: return launch_body<MixedBody<BZ>, 4>(p, block, stream, launched);
    case 3: return launch_body<MixedBody<BZ>, 3>(p, block, stream, launched);
    default: return launch_body<MixedBody<BZ>, 1>(p, block, stream, launched);
  }
}

}  // namespace

cudaError_t launch_fit_mixed(const FitParams& p, int block, int min_blocks, cudaStream_t stream, int* launched) {
  const bool bz = p.bfield[0] == 0.0 && p.bfield[1] == 0.0;
  // this kernel's table follows the FP64 table in the packed buffer
  FitParams q = p;
  q.surf = p.surf + (size_t)p.n_surfaces * kSurfStride;
  return bz ? launch_m<true>(q, block, min_blocks, stream, launched)
            : launch_m<false>(q, block, min_blocks, stream, launched);
}

}  // namespace kfgb

// ---------------------------------------------------------------------------
// self-check of the numeric helpers against the hardware conversions and
// CUDA's double-precision sqrt / division (no fit involved)
// ---------------------------------------------------------------------------
namespace kfgb {
namespace {
using namespace dev;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// counters: [0] f2d mismatches, [1] d2f mismatches, [2] rsqrt_nr<1> beyond
// 1e-13 relative, [3] rcp_nr<1> beyond 1e-13, [4] rsqrt_nr<2>/rcp_nr<2> beyond
// 4 ulp (2^-50 relative)
__global__ void selftest_kernel(long long n, unsigned long long* counters) {
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long c[5] = {0, 0, 0, 0, 0};
  for (long long i = i0; i < n; i += stride) {
    const uint64_t z = mix64((uint64_t)i);
    // f2d over random float bit patterns (subnormals excluded by design)
    const float f = __uint_as_float((uint32_t)z);
    const uint32_t fe = ((uint32_t)z >> 23) & 0xffu;
    if (fe != 0u) {
      const double a = f2d(f), b = (double)f;
      if (__double_as_longlong(a) != __double_as_longlong(b) && !(a != a && b != b)) ++c[0];
    }
    // d2f over doubles in and around the float range
    const double x = __longlong_as_double((long long)((z & 0x800fffffffffffffULL) |
                                                      ((uint64_t)(896 - 8 + (int)((z >> 52) % 272)) << 52)));
    const float g1 = d2f(x);
    const float g2 = __double2float_rn(x);
    const bool sub = fabs(x) < 1.1754943508222875e-38;  // float subnormal range flushes to 0
    if (!sub && __float_as_uint(g1) != __float_as_uint(g2)) ++c[1];
    // Newton helpers on positive values across 1e-30 .. 1e30
    const double y = exp2((double)((int)(z % 180) - 90)) * (1.0 + (double)((z >> 20) & 0xfffff) / 1048576.0);
    const double rs_ref = 1.0 / sqrt(y), rc_ref = 1.0 / y;
    if (fabs(rsqrt_nr<1>(y) - rs_ref) > 1e-13 * rs_ref) ++c[2];
    if (fabs(rcp_nr<1>(y) - rc_ref) > 1e-13 * rc_ref) ++c[3];
    if (fabs(rsqrt_nr<2>(y) - rs_ref) > 8.9e-16 * rs_ref || fabs(rcp_nr<2>(y) - rc_ref) > 8.9e-16 * rc_ref) ++c[4];
  }
  for (int k = 0; k < 5; ++k)
    if (c[k]) atomicAdd(&counters[k], c[k]);
}
}  // namespace

// the double-float helpers against FP64 arithmetic on the same (df-exact)
// inputs; counters: [0] df_add, [1] df_add_f, [2] df_mul, [3] df_dot off by
// more than 2^-44 of the magnitude of their terms; [4] the patterns whose
// sum of the float parts alone (hi + hi) already misses that bound, which
// shows the bound is out of plain FP32's reach.  Every fourth pattern makes
// the sum cancel (b close to -a).
__global__ void df_selftest_kernel(long long n, unsigned long long* counters) {
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long c[5] = {0, 0, 0, 0, 0};
  // a double of magnitude 2^-10 .. 2^14 with a random sign and mantissa
  auto rnd = [](uint64_t z) {
    const double m = 1.0 + (double)((z >> 12) & 0xfffffffffULL) * 0x1p-36;
    return ((z & 1) ? -m : m) * exp2((double)((int)((z >> 1) % 25) - 10));
  };
  const double tol = 0x1p-44;
  for (long long i = i0; i < n; i += stride) {
    const uint64_t z = mix64((uint64_t)i);
    const double a = rnd(z), b0 = rnd(mix64(z)), f0 = rnd(mix64(z + 1));
    const double b = (i & 3) == 0 ? -a * (1.0 + rnd(mix64(z + 2)) * 0x1p-30) : b0;
    const DF A = df_from_d(a), B = df_from_d(b);
    const double ad = df_to_d(A), bd = df_to_d(B);
    const double sd = df_to_d(df_add(A, B));
    if (!(fabs(sd - (ad + bd)) <= tol * (fabs(ad) + fabs(bd)))) ++c[0];
    if (!(fabs((double)(A.hi + B.hi) - (ad + bd)) <= tol * (fabs(ad) + fabs(bd)))) ++c[4];
    const float f = __double2float_rn((i & 3) == 1 ? -ad : f0);
    const double s2 = df_to_d(df_add_f(A, f));
    if (!(fabs(s2 - (ad + (double)f)) <= tol * (fabs(ad) + fabs((double)f)))) ++c[1];
    const double pd = df_to_d(df_mul(A, B));
    if (!(fabs(pd - ad * bd) <= tol * fabs(ad * bd))) ++c[2];
    float wh[3], wl[3];
    DF r[3];
    double ref = 0.0, mag = 0.0;
    for (int k = 0; k < 3; ++k) {
      const DF w = df_from_d(rnd(mix64(z + 3 + k)));
      wh[k] = w.hi;
      wl[k] = w.lo;
      r[k] = df_from_d(rnd(mix64(z + 7 + k)));
      const double t = df_to_d(w) * df_to_d(r[k]);
      ref += t;
      mag += fabs(t);
    }
    const DF w0 = df_from_d((i & 3) == 2 ? ref : rnd(mix64(z + 11)));
    ref -= df_to_d(w0);
    mag += fabs(df_to_d(w0));
    const double dd = df_to_d(df_dot(wh, wl, w0, r));
    if (!(fabs(dd - ref) <= tol * mag)) ++c[3];
  }
  for (int k = 0; k < 5; ++k)
    if (c[k]) atomicAdd(&counters[k], c[k]);
}

cudaError_t launch_selftest_df(long long n, unsigned long long* counters, cudaStream_t stream) {
  df_selftest_kernel<<<152 * 4, 256, 0, stream>>>(n, counters);
  return cudaGetLastError();
}

cudaError_t launch_selftest(long long n, unsigned long long* counters, cudaStream_t stream) {
  selftest_kernel<<<152 * 4, 256, 0, stream>>>(n, counters);
  return cudaGetLastError();
}
}  // namespace kfgb
