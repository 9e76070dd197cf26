// kf_kernels.cu -- the FP64 fit kernel (sm_103a) of the Kalman-filter track
// fit (arXiv 2105.01796): forward filter (Runge-Kutta-Nystrom propagation in
// a constant field, Jacobian transport, multiple-scattering noise, gain-matrix
// update with the Joseph covariance form, chi2) and the Rauch-Tung-Striebel
// smoother, fused into one launch with one track per thread, every step in
// double precision; plus the small helper kernels (surface packing, the
// length sort of the sorted schedule, a self-check).  The mixed-precision
// kernel is in kf_mixed.cu, the method variants in kf_variants.cu.
// Paper references: Sect. 2 (filter step list, RTS smoother with the stored
// Jacobians), Sect. 4.1 (RKN transport; local<->global Jacobians at both
// surfaces), Sect. 4.2 (double-precision inverter), Sect. 4.3 (surfaces in
// global memory accessed once; constant field).
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


// ---------------------------------------------------------------------------
// transport x (bound, on surface a) to surface b.  Returns the bound
// prediction xp, the 6x6 Jacobian F (row 4 = e4 and column 5 = e5 implied),
// and the unit-direction quantities the noise needs.
// ---------------------------------------------------------------------------
template <typename R, bool BZ>
__device__ __forceinline__ int transport(const Surf& sa, const Surf& sb, const double x[6], const double B[3],
                         double mass, double h_max, int n_iter, double xp[6], Jac<R>& J,
                         R& sin_theta, R& cos_inc) {
  Prop<R> s;
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
  // G columns phi, theta: direction rows = dT/dphi, dT/dtheta; q/p column 0
  s.gT[0][0] = (R)(-sp * st); s.gT[1][0] = (R)(cp * st); s.gT[2][0] = R(0);
  s.gT[0][1] = (R)(cp * ct);  s.gT[1][1] = (R)(sp * ct); s.gT[2][1] = (R)(-st);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.gT[i][2] = R(0);
    s.gr[i][0] = s.gr[i][1] = s.gr[i][2] = R(0);
  }
  s.gtl = R(0);

  double s0;
  if (!plane_step(s, sb, s0)) return ST_NO_INTERSECTION;
  const double nsub_d = ceil(fabs(s0) / h_max);
  if (!(nsub_d <= 64.0)) return ST_NO_INTERSECTION;
  const int nsub = nsub_d < 1.0 ? 1 : (int)nsub_d;
  const double h = s0 / nsub;
  for (int k = 0; k < nsub; ++k) rkn_step<R, BZ>(s, h, B, mass);
  for (int it = 0; it < n_iter; ++it) {
    double si;
    if (!plane_step(s, sb, si)) return ST_NO_INTERSECTION;
    rkn_step<R, BZ>(s, si, B, mass);
  }

  // end point: unit direction and bound angles
  // square roots and quotients of the end frame from Newton-refined
  // reciprocal square roots (two steps: double rounding level)
  const double rho2 = s.T[0] * s.T[0] + s.T[1] * s.T[1];
  const double irho_d = rsqrt_any(rho2);
  const double rho_d = rho2 * irho_d;
  const double phi = atan2(s.T[1], s.T[0]);
  const double theta = atan2(rho_d, s.T[2]);
  const R Tr[3] = {(R)s.T[0], (R)s.T[1], (R)s.T[2]};
  const double itn_d = rsqrt_any(rho2 + s.T[2] * s.T[2]);
  const R rho = (R)rho_d;
  const R tn = (R)((rho2 + s.T[2] * s.T[2]) * itn_d);
  const R cph = Tr[0] * (R)irho_d, sph = Tr[1] * (R)irho_d;
  const R sth = rho * (R)itn_d, cth = Tr[2] * (R)itn_d;
  const R nb[3] = {(R)sb.n(0), (R)sb.n(1), (R)sb.n(2)};
  const R nT = nb[0] * Tr[0] + nb[1] * Tr[1] + nb[2] * Tr[2];

  // path correction: dfree += F' w, w = -(n . position rows) / (n . T),
  // F' = (T, dt/ds, A T, 0) at the end point.
  const R lk = (R)(s.lam * kKappa);
  const R bs[3] = {lk * (R)B[0], lk * (R)B[1], lk * (R)B[2]};
  R AT[3];
  applyA<R, BZ>(bs, Tr, AT);
  const R dtds = (R)(sqrt(1.0 + mass * mass * s.lam * s.lam) * kInvC);
  const R inv_nT = (R)rcp_any((double)nT);
  // columns 0..4: loc0, loc1, phi, theta, q/p; full G columns after correction
  R Gr[3][5], GT[3][5], Gt[5];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gr[i][0] = (R)sa.u(i);
    Gr[i][1] = (R)sa.v(i);
    Gr[i][2] = s.gr[i][0];
    Gr[i][3] = s.gr[i][1];
    Gr[i][4] = s.gr[i][2];
    GT[i][0] = R(0);
    GT[i][1] = R(0);
    GT[i][2] = s.gT[i][0];
    GT[i][3] = s.gT[i][1];
    GT[i][4] = s.gT[i][2];
  }
  Gt[0] = Gt[1] = Gt[2] = Gt[3] = R(0);
  Gt[4] = s.gtl;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const R w = -(nb[0] * Gr[0][c] + nb[1] * Gr[1][c] + nb[2] * Gr[2][c]) * inv_nT;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gr[i][c] += Tr[i] * w;
      GT[i][c] += AT[i] * w;
    }
    Gt[c] += dtds * w;
  }
  // free -> bound at b
  const R ub[3] = {(R)sb.u(0), (R)sb.u(1), (R)sb.u(2)};
  const R vb[3] = {(R)sb.v(0), (R)sb.v(1), (R)sb.v(2)};
  const R inv_sth = (R)rcp_any((double)sth);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    J.f[0][c] = ub[0] * Gr[0][c] + ub[1] * Gr[1][c] + ub[2] * Gr[2][c];
    J.f[1][c] = vb[0] * Gr[0][c] + vb[1] * Gr[1][c] + vb[2] * Gr[2][c];
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


// ---------------------------------------------------------------------------
// the fused fit kernel
// ---------------------------------------------------------------------------
template <bool BZ>
__device__ __forceinline__ void fit_one_fp64(const FitParams& p, const double* s_surf, int i) {
  using R = double;
  using RC = Rec<0>;
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
      double xp[6], Cp[21];
      if (k == 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) xp[e] = x[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp[e] = C[e];
      } else {
        const Surf sa{s_surf + sid_prev * kSurfStride}, sb{s_surf + sid * kSurfStride};
        Jac<R> J;
        R sin_th, cos_inc;
        // field copied to registers: taking the address of a kernel parameter
        // would move the parameter block to local memory
        const double Bf[3] = {p.bfield[0], p.bfield[1], p.bfield[2]};
        status = transport<R, BZ>(sa, sb, x, Bf, p.mass, p.h_max, p.n_iter, xp, J, sin_th, cos_inc);
        if (status != ST_OK) break;
        // Bm = F Cf_{k-1}; Cp = Bm F^T + Q.  F rows 0..3 and 5 over columns
        // 0..4 are J; row 4 = e4; column 5 = e5.
        R Cr[21];
#pragma unroll
        for (int e = 0; e < 21; ++e) Cr[e] = (R)C[e];
        R Cpr[21];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          R brow[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            R v;
            if (r == 4) {
              v = Cr[sym(4, j)];
            } else {
              v = jf(J, r, 0) * Cr[sym(0, j)] + jf(J, r, 1) * Cr[sym(1, j)] + jf(J, r, 2) * Cr[sym(2, j)] +
                  jf(J, r, 3) * Cr[sym(3, j)] + jf(J, r, 4) * Cr[sym(4, j)];
              if (r == 5) v += Cr[sym(5, j)];
            }
            brow[j] = v;
            RC::put_bm(ws, k, r * 6 + j, brow[j]);
          }
#pragma unroll
          for (int c = 0; c < 6; ++c) if (c <= r) {
            R v;
            if (c == 4) {
              v = brow[4];
            } else {
              v = brow[0] * jf(J, c, 0) + brow[1] * jf(J, c, 1) + brow[2] * jf(J, c, 2) + brow[3] * jf(J, c, 3) +
                  brow[4] * jf(J, c, 4);
              if (c == 5) v += brow[5];
            }
            Cpr[sy(r, c)] = v;
          }
        }
        // multiple scattering of surface k (added before the update)
        const R xx0 = (R)sb.xx0();
        if (xx0 > R(0)) {
          const R th0 = highland<R>((R)fabs(x[4]), (R)(p.mass * p.mass), xx0, cos_inc);
          const R q = th0 * th0;
          Cpr[sy(2, 2)] += q / (sin_th * sin_th);
          Cpr[sy(3, 3)] += q;
        }
#pragma unroll
        for (int e = 0; e < 21; ++e) Cp[e] = (double)Cpr[e];
      }
      // record the prediction
#pragma unroll
      for (int e = 0; e < 6; ++e) ws.d(k, RC::XP + e) = xp[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) ws.d(k, RC::CP + e) = Cp[e];
      // update
      if (!p.is_hole[o0 + k]) {
        const double m[2] = {p.loc[o0 + k], p.loc[p.n_states + o0 + k]};
        const double V[3] = {p.cov[o0 + k], p.cov[p.n_states + o0 + k], p.cov[2 * p.n_states + o0 + k]};
        double c2 = 0.0;
        status = kalman_update<R>(xp, Cp, m, V, x, C, c2);
        if (status != ST_OK) break;
        chi2sum += c2;
        ++nmeas;
      } else {
#pragma unroll
        for (int e = 0; e < 6; ++e) x[e] = xp[e];
#pragma unroll
        for (int e = 0; e < 21; ++e) C[e] = Cp[e];
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) ws.d(k, RC::XF + e) = x[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) RC::put_cf(ws, k, e, (R)C[e]);
      sid_prev = sid;
    }

    // ------------------------------------------------ RTS smoother
    if (status == ST_OK) {
#pragma unroll
      for (int e = 0; e < 6; ++e) xs[e] = x[e];
#pragma unroll
      for (int e = 0; e < 21; ++e) Cs[e] = C[e];
      status = rts_smooth_fp64(ws, n, xs, Cs, p.out_states, p.n_states, o0);
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

// self-check of the full-range Newton helpers against CUDA's double 1/sqrt
// and 1/x over positive and negative values across 1e-300 .. 1e300;
// counter: cases beyond 4 ulp
__global__ void selftest_any_kernel(long long n, unsigned long long* counter) {
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long c = 0;
  for (long long i = i0; i < n; i += stride) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;
    z ^= z >> 29;
    const double y = exp2((double)((int)(z % 1990) - 995)) * (1.0 + (double)((z >> 20) & 0xfffff) / 1048576.0);
    const double rs_ref = 1.0 / sqrt(y), rc_ref = 1.0 / y;
    if (fabs(rsqrt_any(y) - rs_ref) > 8.9e-16 * rs_ref) ++c;
    if (fabs(rcp_any(y) - rc_ref) > 8.9e-16 * rc_ref) ++c;
    if (fabs(rcp_any(-y) + rc_ref) > 8.9e-16 * rc_ref) ++c;
  }
  if (c) atomicAdd(counter, c);
}

__global__ void pack_surfaces_kernel(int n, const double* __restrict__ center, const double* __restrict__ rot,
                                     const double* __restrict__ xx0, double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double* o = out + (size_t)s * kSurfStride;
  for (int i = 0; i < 3; ++i) o[i] = center[(size_t)i * n + s];
  for (int i = 0; i < 9; ++i) o[3 + i] = rot[(size_t)i * n + s];
  o[12] = xx0[s];
  // n.c, u.c, v.c (column j of R is o[3 + 3 i + j], i = 0..2)
  for (int j = 0; j < 3; ++j) o[13 + (j + 1) % 3] = o[3 + j] * o[0] + o[6 + j] * o[1] + o[9 + j] * o[2];
  // float copies of n, u, v and x/X0
  float* f = reinterpret_cast<float*>(o + 16);
  for (int i = 0; i < 3; ++i) {
    f[i] = (float)o[3 + 3 * i + 2];
    f[3 + i] = (float)o[3 + 3 * i + 0];
    f[6 + i] = (float)o[3 + 3 * i + 1];
  }
  f[9] = (float)o[12];
  for (int i = 10; i < 16; ++i) f[i] = 0.0f;
  // the mixed kernel's table: each FP64 value v as hi = (float)v and
  // lo = (float)(v - hi)
  float* m = reinterpret_cast<float*>(out + (size_t)n * kSurfStride + (size_t)s * kSurfStrideM);
  auto split = [](double v, float* hi, float* lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
  };
  for (int i = 0; i < 3; ++i) {
    split(o[3 + 3 * i + 2], &m[i], &m[10 + i]);      // n
    split(o[3 + 3 * i + 0], &m[3 + i], &m[13 + i]);  // u
    split(o[3 + 3 * i + 1], &m[6 + i], &m[16 + i]);  // v
    split(o[13 + i], &m[19 + i], &m[22 + i]);        // n.c, u.c, v.c
    split(o[i], &m[25 + i], &m[28 + i]);             // c
  }
  m[9] = (float)o[12];
  m[31] = 0.0f;
}

template <bool BZ>
struct Fp64Body {
  static constexpr int kStride = kSurfStride;
  static __device__ __forceinline__ void run(const FitParams& p, const double* s_surf, int i) {
    fit_one_fp64<BZ>(p, s_surf, i);
  }
};

template <bool BZ>
cudaError_t launch_fp64(const FitParams& p, int block, int min_blocks, cudaStream_t stream, int* launched) {
  (void)min_blocks;  // a register cap below 255 spills this kernel heavily
  return launch_body<Fp64Body<BZ>, 1>(p, block, stream, launched);
}

// counting sort of tracks by state count (longest first)
__global__ void length_hist_kernel(int n, int max_states, const int32_t* __restrict__ offsets,
                                   int32_t* __restrict__ hist) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int len = offsets[t + 1] - offsets[t];
  len = len < 0 ? 0 : (len > max_states ? max_states + 1 : len);
  atomicAdd(&hist[max_states + 1 - len], 1);  // bin 0 = longest
}

__global__ void length_scan_kernel(int nbins, int32_t* hist) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < nbins; ++b) {
      const int c = hist[b];
      hist[b] = acc;
      acc += c;
    }
  }
}

__global__ void length_scatter_kernel(int n, int max_states, const int32_t* __restrict__ offsets,
                                      int32_t* __restrict__ hist, int32_t* __restrict__ order) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int len = offsets[t + 1] - offsets[t];
  len = len < 0 ? 0 : (len > max_states ? max_states + 1 : len);
  const int slot = atomicAdd(&hist[max_states + 1 - len], 1);
  order[slot] = t;
}

}  // namespace

cudaError_t launch_selftest_any(long long n, unsigned long long* counter, cudaStream_t stream) {
  selftest_any_kernel<<<152 * 4, 256, 0, stream>>>(n, counter);
  return cudaGetLastError();
}

cudaError_t launch_pack_surfaces(int n_surfaces, const double* center, const double* rot,
                                 const double* x_over_x0, double* packed, cudaStream_t stream) {
  const int block = 128;
  pack_surfaces_kernel<<<(n_surfaces + block - 1) / block, block, 0, stream>>>(n_surfaces, center, rot,
                                                                              x_over_x0, packed);
  return cudaGetLastError();
}

cudaError_t launch_fit_mixed(const FitParams& p, int block, int min_blocks, cudaStream_t stream, int* launched);

cudaError_t launch_fit(const FitParams& p, int precision, int block, int min_blocks, cudaStream_t stream,
                       int* launched) {
  if (launched) *launched = 0;
  if (p.n_tracks <= 0) return cudaSuccess;
  if (block <= 0) block = 128;
  const bool bz = p.bfield[0] == 0.0 && p.bfield[1] == 0.0;
  if (precision == 0 && p.team_warps > 1) return launch_fit_team(p, p.team_warps, stream, launched);
  if (precision == 0) return bz ? launch_fp64<true>(p, block, min_blocks, stream, launched)
                                : launch_fp64<false>(p, block, min_blocks, stream, launched);
  return launch_fit_mixed(p, block, min_blocks, stream, launched);
}

cudaError_t launch_length_order(int n_tracks, int max_states, const int32_t* offsets, int32_t* hist,
                                int32_t* order, cudaStream_t stream) {
  if (n_tracks <= 0) return cudaSuccess;
  const int nbins = max_states + 2;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * nbins, stream);
  if (e != cudaSuccess) return e;
  const int block = 256, grid = (n_tracks + block - 1) / block;
  length_hist_kernel<<<grid, block, 0, stream>>>(n_tracks, max_states, offsets, hist);
  length_scan_kernel<<<1, 32, 0, stream>>>(nbins, hist);
  length_scatter_kernel<<<grid, block, 0, stream>>>(n_tracks, max_states, offsets, hist, order);
  return cudaGetLastError();
}

}  // namespace kfgb
