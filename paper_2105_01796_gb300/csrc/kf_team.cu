// kf_team.cu -- the FP64 fit with each track's work shared by a team of W
// warps (W = 2 or 4), for batches too small to fill the GPU (paper Sect. 4.1:
// parallelism inside one track's fit, for small batches).
//
// On this part an FP64 warp instruction holds its SM sub-partition's FP64
// pipe for the same time whatever the number of active lanes (measured: 79.6
// cycles per DFMA warp instruction with 32, 16, 8, 4, 2 or 1 active lanes),
// and one warp of the one-thread-per-track kernel keeps that pipe busy on its
// own: a batch of fewer tracks than sub-partitions x 32 runs at one warp's
// FP64 instruction count per state (about 2400).  Splitting a track over the
// lanes of one warp cannot shorten that; splitting it over W warps, each on
// its own sub-partition, can.
//
// Lane l of each of a CTA's W warps works on track l of the CTA's 32.  The
// warps all propagate the state (point, direction, time) and take the same
// discrete decisions; they split
//   * the Jacobian columns of the RKN steps, the path correction and the
//     free -> bound projection (by column of F),
//   * Bm = F Cf and Cp = Bm F^T, the Joseph update, the smoother's triangular
//     solves (by column of Cp^-1 Bm, i.e. by row of the gain A) and
//     Cs = Cf + A (Cs' - Cp') A^T (by row),
// and exchange F, Cp, Cf, A and Cs through shared memory.  The 32 tracks of a
// CTA step through the states in lockstep (a track with fewer states, or one
// that failed, idles at its barriers).  The arithmetic of every element is
// that of the one-thread-per-track FP64 kernel (kf_kernels.cu), so the
// results are the same up to the order of a few sums.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_device.cuh"
#include "kf_fp64.cuh"
#include "kf_internal.h"
#include "kf_transport.cuh"

namespace kfgb {
namespace {
using namespace dev;

constexpr int kTeamTracks = 32;
// shared exchange buffers per CTA, [field][32 tracks] doubles
// F 25 | Cp 21 | Cf (also Cs) 21 | A 36 | sin/cos of the next transport's
// start angles 4 | the end angles (phi, theta) and the scattering variance 3
constexpr int kShF = 0, kShCp = 25, kShCf = 46, kShA = 67, kShTrig = 103, kShAng = 107, kShFields = 110;

// The transcendental functions of the state (the sine and cosine of the
// start angles, atan2 of the end direction, the Highland width) are computed
// by one warp, the one with the least split work, and read by the others
// after the barriers that follow them anyway.
template <int W>
__host__ __device__ constexpr int trig_owner() { return W - 1; }

// owner warp of matrix row r (rows hold 1..6 lower-triangle elements; the
// split balances them: W = 2: 11 / 10, W = 4: 6 / 6 / 6 / 3)
template <int W>
__host__ __device__ constexpr int row_owner(int r) {
  return W == 2 ? ((r == 5 || r == 3 || r == 0) ? 0 : 1)
                : (r == 5 ? 0 : (r == 4 || r == 0) ? 1 : (r == 3 || r == 1) ? 2 : 3);
}
// owner warp of column j of F (0 loc0, 1 loc1, 2 phi, 3 theta, 4 q/p); the
// phi, theta and q/p columns are the ones the RKN steps carry
template <int W>
__host__ __device__ constexpr int col_owner(int j) {
  return W == 2 ? ((j == 2 || j == 3) ? 0 : 1) : (j == 2 ? 0 : j == 3 ? 1 : j == 4 ? 2 : 3);
}
template <int W>
__host__ __device__ constexpr int col_mask(int w) {
  return (col_owner<W>(0) == w ? 1 : 0) | (col_owner<W>(1) == w ? 2 : 0) | (col_owner<W>(2) == w ? 4 : 0) |
         (col_owner<W>(3) == w ? 8 : 0) | (col_owner<W>(4) == w ? 16 : 0);
}

// The transport of kf_kernels.cu for the F columns in FMASK: the state is
// propagated in full, the Jacobian columns of FMASK only; those columns of F
// go to shared memory (sF[(r * 5 + c) * 32 + lane], time row at r = 4).
// sc = (sin phi, cos phi, sin theta, cos theta) of x; the end angles phi,
// theta go to sAng when ANG (their owner warp), else xp[2], xp[3] are left
// for the caller to read from sAng after the barrier.
template <bool BZ, int FMASK, bool ANG>
__device__ __forceinline__ int transport_cols(const Surf& sa, const Surf& sb, const double x[6], const double sc[4],
                                              const double B[3], double mass, double h_max, int n_iter,
                                              double xp[6], double* sF, double* sAng, int lane, double& sin_theta,
                                              double& cos_inc) {
  using R = double;
  constexpr int CMASK = (FMASK >> 2) & 7;
  Prop<R> s;
  const double sp = sc[0], cp = sc[1], st = sc[2], ct = sc[3];
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
  double s0;
  if (!plane_step(s, sb, s0)) return ST_NO_INTERSECTION;
  const double nsub_d = ceil(fabs(s0) / h_max);
  if (!(nsub_d <= 64.0)) return ST_NO_INTERSECTION;
  const int nsub = nsub_d < 1.0 ? 1 : (int)nsub_d;
  const double h = s0 / nsub;
  for (int k = 0; k < nsub; ++k) rkn_step<R, BZ, CMASK>(s, h, B, mass);
  for (int it = 0; it < n_iter; ++it) {
    double si;
    if (!plane_step(s, sb, si)) return ST_NO_INTERSECTION;
    rkn_step<R, BZ, CMASK>(s, si, B, mass);
  }
  const double rho2 = s.T[0] * s.T[0] + s.T[1] * s.T[1];
  const double irho = rsqrt_any(rho2);
  const double rho = rho2 * irho;
  if (ANG) {
    sAng[0 * kTeamTracks + lane] = atan2(s.T[1], s.T[0]);
    sAng[1 * kTeamTracks + lane] = atan2(rho, s.T[2]);
  }
  const double itn = rsqrt_any(rho2 + s.T[2] * s.T[2]);
  const double tn = (rho2 + s.T[2] * s.T[2]) * itn;
  const double cph = s.T[0] * irho, sph = s.T[1] * irho;
  const double sth = rho * itn, cth = s.T[2] * itn;
  const double nT = sb.n(0) * s.T[0] + sb.n(1) * s.T[1] + sb.n(2) * s.T[2];
  const double lk = s.lam * kKappa;
  const double bs[3] = {lk * B[0], lk * B[1], lk * B[2]};
  double AT[3];
  applyA<R, BZ>(bs, s.T, AT);
  const double dtds = sqrt(1.0 + mass * mass * s.lam * s.lam) * kInvC;
  const double inv_nT = rcp_any(nT);
  const double inv_sth = rcp_any(sth);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (!(FMASK & (1 << c))) continue;
    double Gr[3], GT[3], Gt;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i] = c == 0 ? sa.u(i) : c == 1 ? sa.v(i) : s.gr[i][c - 2];
      GT[i] = c < 2 ? 0.0 : s.gT[i][c - 2];
    }
    Gt = c == 4 ? s.gtl : 0.0;
    const double wc = -(sb.n(0) * Gr[0] + sb.n(1) * Gr[1] + sb.n(2) * Gr[2]) * inv_nT;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i] += s.T[i] * wc;
      GT[i] += AT[i] * wc;
    }
    Gt += dtds * wc;
    sF[(0 * 5 + c) * kTeamTracks + lane] = sb.u(0) * Gr[0] + sb.u(1) * Gr[1] + sb.u(2) * Gr[2];
    sF[(1 * 5 + c) * kTeamTracks + lane] = sb.v(0) * Gr[0] + sb.v(1) * Gr[1] + sb.v(2) * Gr[2];
    sF[(2 * 5 + c) * kTeamTracks + lane] = (-sph * GT[0] + cph * GT[1]) * inv_sth;
    sF[(3 * 5 + c) * kTeamTracks + lane] = cph * cth * GT[0] + sph * cth * GT[1] - sth * GT[2];
    sF[(4 * 5 + c) * kTeamTracks + lane] = Gt;
  }
  const double d0 = s.r[0] - sb.c(0), d1 = s.r[1] - sb.c(1), d2 = s.r[2] - sb.c(2);
  xp[0] = d0 * sb.u(0) + d1 * sb.u(1) + d2 * sb.u(2);
  xp[1] = d0 * sb.v(0) + d1 * sb.v(1) + d2 * sb.v(2);
  xp[4] = s.lam;
  xp[5] = s.t;
  sin_theta = sth;
  cos_inc = nT / tn;
  return ST_OK;
}

template <bool BZ, int W, int w>
__device__ __forceinline__ int transport_warp(const Surf& sa, const Surf& sb, const double x[6], const double sc[4],
                                              const double B[3], double mass, double h_max, int n_iter,
                                              double xp[6], double* sF, double* sAng, int lane, double& sin_theta,
                                              double& cos_inc) {
  return transport_cols<BZ, col_mask<W>(w), w == trig_owner<W>()>(sa, sb, x, sc, B, mass, h_max, n_iter, xp, sF,
                                                                   sAng, lane, sin_theta, cos_inc);
}

// F element (r, c), r in {0..3, 5}, c in 0..4, from shared memory
__device__ __forceinline__ double shf(const double* sF, int r, int c, int lane) {
  return sF[((r == 5 ? 4 : r) * 5 + c) * kTeamTracks + lane];
}

// One CTA: the 32 tracks of slots [base, base + 32), W warps.
template <bool BZ, int W>
__device__ void fit_team(const FitParams& p, const double* s_surf, double* sh, int base) {
  using RC = Rec<0>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = base + lane;
  const bool valid = i < p.n_tracks;
  const int t = valid ? track_of(p, i) : 0;
  const size_t TT = (size_t)p.n_tracks_total;
  const WS ws{p.ws64, p.ws32, (size_t)p.n_tracks, kRec64Fp64, 0, valid ? i : 0};
  double* sF = sh + kShF * kTeamTracks;
  double* sCp = sh + kShCp * kTeamTracks;
  double* sCf = sh + kShCf * kTeamTracks;
  double* sA = sh + kShA * kTeamTracks;
  double* sTrig = sh + kShTrig * kTeamTracks;
  double* sAng = sh + kShAng * kTeamTracks;
  int64_t o0 = 0, o1 = 0;
  int n = 0;
  int status = valid ? ST_OK : ST_BAD_INPUT;
  if (valid) {
    o0 = p.offsets[t];
    o1 = p.offsets[t + 1];
    n = (int)(o1 - o0);
    if (!(o1 > o0) || o0 < 0 || o1 > p.n_states || n > p.max_states) status = ST_BAD_INPUT;
    if (status == ST_OK)
      for (int k = 0; k < n; ++k) {
        const int sid = p.surface_id[o0 + k];
        if (sid < 0 || sid >= p.n_surfaces) status = ST_BAD_INPUT;
      }
  }
  // the CTA's longest track sets the lockstep count (the same in every warp)
  int nmax = status == ST_OK ? n : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
  const double Bf[3] = {p.bfield[0], p.bfield[1], p.bfield[2]};

  double x[6], C[21];
  double chi2sum = 0.0;
  int nmeas = 0;
  if (status == ST_OK) {
#pragma unroll
    for (int e = 0; e < 6; ++e) x[e] = p.seed_params[e * TT + t];
#pragma unroll
    for (int e = 0; e < 21; ++e) C[e] = p.seed_cov[e * TT + t];
  }
  // ------------------------------------------------ forward filter
  for (int k = 0; k < nmax; ++k) {
    bool act = status == ST_OK && k < n;
    double xp[6], Cp[21];
    if (k == 0) {
#pragma unroll
      for (int e = 0; e < 6; ++e) xp[e] = x[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) Cp[e] = C[e];
    } else {
      double sin_th = 1.0, cos_inc = 1.0;
      if (act) {
        const Surf sa{s_surf + p.surface_id[o0 + k - 1] * kSurfStride}, sb{s_surf + p.surface_id[o0 + k] * kSurfStride};
        int st = ST_OK;
        double sc[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) sc[e] = sTrig[e * kTeamTracks + lane];
#define KF_TEAM_TRANSPORT(WW) \
  transport_warp<BZ, W, WW>(sa, sb, x, sc, Bf, p.mass, p.h_max, p.n_iter, xp, sF, sAng, lane, sin_th, cos_inc)
        switch (w) {
          case 0: st = KF_TEAM_TRANSPORT(0); break;
          case 1: st = KF_TEAM_TRANSPORT(1); break;
          case 2: st = KF_TEAM_TRANSPORT((W > 2 ? 2 : 1)); break;
          default: st = KF_TEAM_TRANSPORT((W > 3 ? 3 : 1)); break;
        }
#undef KF_TEAM_TRANSPORT
        status = st;
        act = st == ST_OK;
        // multiple scattering of surface k: theta0^2 (added before the update)
        if (act && w == trig_owner<W>()) {
          const double xx0 = sb.xx0();
          double q = 0.0;
          if (xx0 > 0.0) {
            const double th0 = highland<double>(fabs(x[4]), p.mass * p.mass, xx0, cos_inc);
            q = th0 * th0;
          }
          sAng[2 * kTeamTracks + lane] = q;
        }
      }
      __syncthreads();  // F, the end angles and theta0^2 complete
      double q_ms = 0.0;
      if (act) {
        xp[2] = sAng[0 * kTeamTracks + lane];
        xp[3] = sAng[1 * kTeamTracks + lane];
        q_ms = sAng[2 * kTeamTracks + lane];
      }
      if (act) {
        // Bm = F Cf_{k-1} and Cp = Bm F^T for the rows this warp owns
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          if (row_owner<W>(r) != w) continue;
          double brow[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            double v;
            if (r == 4) {
              v = C[sym(4, j)];
            } else {
              v = shf(sF, r, 0, lane) * C[sym(0, j)] + shf(sF, r, 1, lane) * C[sym(1, j)] +
                  shf(sF, r, 2, lane) * C[sym(2, j)] + shf(sF, r, 3, lane) * C[sym(3, j)] +
                  shf(sF, r, 4, lane) * C[sym(4, j)];
              if (r == 5) v += C[sym(5, j)];
            }
            brow[j] = v;
            RC::put_bm(ws, k, r * 6 + j, v);
          }
#pragma unroll
          for (int c = 0; c <= r; ++c) {
            double v;
            if (c == 4) {
              v = brow[4];
            } else {
              v = brow[0] * shf(sF, c, 0, lane) + brow[1] * shf(sF, c, 1, lane) + brow[2] * shf(sF, c, 2, lane) +
                  brow[3] * shf(sF, c, 3, lane) + brow[4] * shf(sF, c, 4, lane);
              if (c == 5) v += brow[5];
            }
            sCp[sy(r, c) * kTeamTracks + lane] = v;
          }
        }
      }
      __syncthreads();  // Cp complete
      if (act) {
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp[e] = sCp[e * kTeamTracks + lane];
        if (q_ms > 0.0) {
          Cp[sy(2, 2)] += q_ms / (sin_th * sin_th);
          Cp[sy(3, 3)] += q_ms;
        }
      }
    }
    // record the prediction (owners write their rows)
    if (act) {
      if (w == 0)
#pragma unroll
        for (int e = 0; e < 6; ++e) ws.d(k, RC::XP + e) = xp[e];
#pragma unroll
      for (int r = 0; r < 6; ++r)
        if (row_owner<W>(r) == w)
#pragma unroll
          for (int c = 0; c <= r; ++c) ws.d(k, RC::CP + sy(r, c)) = Cp[sy(r, c)];
    }
    // update: gain and x_f in every warp, the Joseph rows split
    const bool meas = act && !p.is_hole[o0 + k];
    if (meas) {
      const double m[2] = {p.loc[o0 + k], p.loc[p.n_states + o0 + k]};
      const double V[3] = {p.cov[o0 + k], p.cov[p.n_states + o0 + k], p.cov[2 * p.n_states + o0 + k]};
      const double S00 = V[0] + Cp[sy(0, 0)], S01 = V[1] + Cp[sy(1, 0)], S11 = V[2] + Cp[sy(1, 1)];
      const double det = S00 * S11 - S01 * S01;
      if (!(det > 0.0) || !(S00 > 0.0)) {
        status = ST_NON_SPD;
      } else {
        const double idet = rcp_any(det);
        const double r0 = m[0] - xp[0], r1 = m[1] - xp[1];
        chi2sum += (S11 * r0 * r0 - 2.0 * S01 * r0 * r1 + S00 * r1 * r1) * idet;
        ++nmeas;
        const double i00 = S11 * idet, i01 = -S01 * idet, i11 = S00 * idet;
        double K[6][2];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const double c0 = Cp[sym(a, 0)], c1 = Cp[sym(a, 1)];
          K[a][0] = c0 * i00 + c1 * i01;
          K[a][1] = c0 * i01 + c1 * i11;
          x[a] = xp[a] + (K[a][0] * r0 + K[a][1] * r1);
        }
        double Wm[2][6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          Wm[0][j] = S00 * K[j][0] + S01 * K[j][1] - Cp[sym(0, j)];
          Wm[1][j] = S01 * K[j][0] + S11 * K[j][1] - Cp[sym(1, j)];
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          if (row_owner<W>(r) != w) continue;
#pragma unroll
          for (int c = 0; c <= r; ++c) {
            double v = Cp[sy(r, c)];
            v = fma(K[r][0], Wm[0][c], v);
            v = fma(K[r][1], Wm[1][c], v);
            v = fma(-Cp[sym(0, r)], K[c][0], v);
            v = fma(-Cp[sym(1, r)], K[c][1], v);
            sCf[sy(r, c) * kTeamTracks + lane] = v;
            RC::put_cf(ws, k, sy(r, c), v);
          }
        }
      }
    } else if (act) {
#pragma unroll
      for (int e = 0; e < 6; ++e) x[e] = xp[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) C[e] = Cp[e];
#pragma unroll
      for (int r = 0; r < 6; ++r)
        if (row_owner<W>(r) == w)
#pragma unroll
          for (int c = 0; c <= r; ++c) RC::put_cf(ws, k, sy(r, c), Cp[sy(r, c)]);
    }
    // the start angles' sines and cosines for the next transport
    if (act && status == ST_OK && w == trig_owner<W>() && k + 1 < n) {
      double sp, cp, st, ct;
      sincos(x[2], &sp, &cp);
      sincos(x[3], &st, &ct);
      sTrig[0 * kTeamTracks + lane] = sp;
      sTrig[1 * kTeamTracks + lane] = cp;
      sTrig[2 * kTeamTracks + lane] = st;
      sTrig[3 * kTeamTracks + lane] = ct;
    }
    __syncthreads();  // Cf and the start angles complete
    if (meas && status == ST_OK)
#pragma unroll
      for (int e = 0; e < 21; ++e) C[e] = sCf[e * kTeamTracks + lane];
    if (act && status == ST_OK && w == 0)
#pragma unroll
      for (int e = 0; e < 6; ++e) ws.d(k, RC::XF + e) = x[e];
  }

  // ------------------------------------------------ RTS smoother
  double xs[6], Cs[21];
  if (status == ST_OK) {
#pragma unroll
    for (int e = 0; e < 6; ++e) xs[e] = x[e];
#pragma unroll
    for (int e = 0; e < 21; ++e) Cs[e] = C[e];
    if (p.out_states && w == 0)
#pragma unroll
      for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + n - 1] = xs[e];
  }
  for (int k = nmax - 2; k >= 0; --k) {
    bool act = status == ST_OK && k + 1 < n;
    double L[21], idg[6], dC[21];
    if (act) {
#pragma unroll
      for (int e = 0; e < 21; ++e) {
        L[e] = ws.d(k + 1, RC::CP + e);
        dC[e] = Cs[e] - L[e];
      }
      // Cholesky of Cp_{k+1} (every warp)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double dj = L[sy(j, j)];
#pragma unroll
        for (int q = 0; q < j; ++q) dj -= L[sy(j, q)] * L[sy(j, q)];
        if (!(dj > 0.0)) status = ST_NON_SPD;
        idg[j] = rsqrt_any(dj);
        L[sy(j, j)] = dj * idg[j];
#pragma unroll
        for (int r = j + 1; r < 6; ++r) {
          double v = L[sy(r, j)];
#pragma unroll
          for (int q = 0; q < j; ++q) v -= L[sy(r, q)] * L[sy(j, q)];
          L[sy(r, j)] = v * idg[j];
        }
      }
      act = status == ST_OK;
      // the columns of X = Cp^-1 Bm this warp owns (column c of X = row c of A)
      if (act)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          if (row_owner<W>(c) != w) continue;
          double y[6], X[6];
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            double v = RC::get_bm(ws, k + 1, r * 6 + c);
#pragma unroll
            for (int q = 0; q < r; ++q) v -= L[sy(r, q)] * y[q];
            y[r] = v * idg[r];
          }
#pragma unroll
          for (int r = 5; r >= 0; --r) {
            double v = y[r];
#pragma unroll
            for (int q = r + 1; q < 6; ++q) v -= L[sy(q, r)] * X[q];
            X[r] = v * idg[r];
          }
#pragma unroll
          for (int r = 0; r < 6; ++r) sA[(c * 6 + r) * kTeamTracks + lane] = X[r];
        }
    }
    __syncthreads();  // A complete
    if (act) {
      double Ar[6][6];
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) Ar[r][c] = sA[(r * 6 + c) * kTeamTracks + lane];
      double d[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) d[e] = xs[e] - ws.d(k + 1, RC::XP + e);
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc += Ar[r][c] * d[c];
        xs[r] = ws.d(k, RC::XF + r) + acc;
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        if (row_owner<W>(r) != w) continue;
        double z[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q < 6; ++q) acc += Ar[r][q] * dC[sym(q, c)];
          z[c] = acc;
        }
#pragma unroll
        for (int c = 0; c <= r; ++c) {
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q < 6; ++q) acc += z[q] * Ar[c][q];
          sCf[sy(r, c) * kTeamTracks + lane] = RC::get_cf(ws, k, sy(r, c)) + acc;
        }
      }
    }
    __syncthreads();  // Cs complete
    if (act) {
#pragma unroll
      for (int e = 0; e < 21; ++e) Cs[e] = sCf[e * kTeamTracks + lane];
      if (p.out_states && w == 0)
#pragma unroll
        for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + o0 + k] = xs[e];
    }
  }
  if (!valid || w != 0) return;
  if (status == ST_OK) {
    bool fin = isfinite(chi2sum);
#pragma unroll
    for (int e = 0; e < 6; ++e) fin = fin && isfinite(xs[e]);
#pragma unroll
    for (int e = 0; e < 21; ++e) fin = fin && isfinite(Cs[e]);
    if (!fin) status = ST_NONFINITE;
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

// One CTA of W warps per 32 tracks; dynamic shared memory: the surface table,
// then the exchange buffers.
template <bool BZ, int W>
__global__ void __launch_bounds__(32 * W, 1) team_kernel(const FitParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* s_surf = reinterpret_cast<double*>(smem_raw);
  double* sh = s_surf + (size_t)p.n_surfaces * kSurfStride;
  __shared__ __align__(8) uint64_t s_mbar;
  const bool ok = stage_surfaces(s_surf, p.surf, (uint32_t)(p.n_surfaces * kSurfStride * 8), &s_mbar,
                                 p.error_flag, p.wait_limit, p.skip_stage_copy != 0);
  const int base = blockIdx.x * kTeamTracks;
  if (!ok) {
    const int i = base + (int)threadIdx.x;
    if (threadIdx.x < kTeamTracks && i < p.n_tracks) write_failed_track(p, i, ST_TIMEOUT);
    return;
  }
  fit_team<BZ, W>(p, s_surf, sh, base);
}

template <bool BZ, int W>
cudaError_t launch_team_v(const FitParams& p, cudaStream_t stream) {
  const size_t smem = (size_t)p.n_surfaces * kSurfStride * sizeof(double) +
                      (size_t)kShFields * kTeamTracks * sizeof(double);
  auto kern = team_kernel<BZ, W>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = (p.n_tracks + kTeamTracks - 1) / kTeamTracks;
  kern<<<grid, 32 * W, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fit_team(const FitParams& p, int team_warps, cudaStream_t stream, int* launched) {
  if (launched) *launched = 0;
  if (p.n_tracks <= 0) return cudaSuccess;
  const bool bz = p.bfield[0] == 0.0 && p.bfield[1] == 0.0;
  if (launched) *launched = 1;
  if (team_warps == 4) return bz ? launch_team_v<true, 4>(p, stream) : launch_team_v<false, 4>(p, stream);
  return bz ? launch_team_v<true, 2>(p, stream) : launch_team_v<false, 2>(p, stream);
}

}  // namespace kfgb
