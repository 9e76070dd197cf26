// kf_device.cuh -- device helpers shared by the FP64 and mixed fit kernels.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_internal.h"

namespace kfgb {
namespace dev {

constexpr double kKappa = 2.99792458e-4;   // GeV / (T mm): curvature = kappa B q/p
constexpr double kInvC = 1.0 / 299.792458;  // ns / mm

enum : int { ST_OK = 0, ST_NO_INTERSECTION = 1, ST_NON_SPD = 2, ST_NONFINITE = 3, ST_BAD_INPUT = 4, ST_TIMEOUT = 5 };

constexpr int kDefaultWaitLimit = 1 << 20;  // polls of a bounded wait

// packed lower-triangle index
__host__ __device__ constexpr int sy(int i, int j) { return i * (i + 1) / 2 + j; }
__host__ __device__ constexpr int sym(int i, int j) { return i >= j ? sy(i, j) : sy(j, i); }

// ---------------------------------------------------------------------------
// surface table staging: one bulk (TMA) copy global -> shared per CTA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// True when a bounded wait of this call gave up somewhere (the flag is reset
// at the start of every call).
__device__ __forceinline__ bool call_failed(const int32_t* error_flag) {
  return *reinterpret_cast<const volatile int32_t*>(error_flag) != 0;
}

// Every thread of the CTA calls this.  Returns false (in every thread) if
// the bounded wait on the copy's mbarrier gave up after wait_limit polls
// (<= 0: the default) in any thread -- the error flag is then set -- or if
// the flag was already set by another CTA of the call.  skip_copy (a
// diagnostic of the timeout path) announces the copy's bytes on the barrier
// but issues no copy, so the wait runs out with nothing in flight.
__device__ __forceinline__ bool stage_surfaces(double* s_surf, const double* g_surf, uint32_t nbytes,
                                               uint64_t* mbar, int32_t* error_flag, int wait_limit = 0,
                                               bool skip_copy = false) {
  const uint32_t bar = smem_addr(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(nbytes) : "memory");
    if (!skip_copy)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(s_surf)),
          "l"(g_surf), "r"(nbytes), "r"(bar)
          : "memory");
  }
  const int limit = wait_limit > 0 ? wait_limit : kDefaultWaitLimit;
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(0u)
        : "memory");
  }
  // one verdict for the whole CTA (its threads poll independently and could
  // disagree near the limit; the callers' barriers need every thread)
  const bool mine = __syncthreads_and(done) != 0;
  if (!mine && threadIdx.x == 0) atomicExch(error_flag, 1);
  // a CTA that starts after another CTA's wait of this call gave up fits
  // nothing either: a copy that a timed-out CTA left in flight could land in
  // shared memory that this CTA has been given
  return __syncthreads_and(mine && !call_failed(error_flag)) != 0;
}

struct Surf {
  const double* d;  // points into shared memory
  __device__ double c(int i) const { return d[i]; }
  __device__ double R(int i, int j) const { return d[3 + 3 * i + j]; }
  __device__ double u(int i) const { return R(i, 0); }
  __device__ double v(int i) const { return R(i, 1); }
  __device__ double n(int i) const { return R(i, 2); }
  __device__ double xx0() const { return d[12]; }
  __device__ double nc() const { return d[13]; }  // n . c
  __device__ double uc() const { return d[14]; }  // u . c
  __device__ double vc() const { return d[15]; }  // v . c
  __device__ const float* f() const { return reinterpret_cast<const float*>(d + 16); }
  __device__ float nf(int i) const { return f()[i]; }
  __device__ float uf(int i) const { return f()[3 + i]; }
  __device__ float vf(int i) const { return f()[6 + i]; }
  __device__ float xx0f() const { return f()[9]; }
};

// out = v x bs, with bs = (q/p) kappa B: the operator A of dT/ds = A T
template <typename R, bool BZ>
__device__ __forceinline__ void applyA(const R bs[3], const R v[3], R out[3]) {
  if (BZ) {
    out[0] = v[1] * bs[2];
    out[1] = -v[0] * bs[2];
    out[2] = R(0);
  } else {
    out[0] = v[1] * bs[2] - v[2] * bs[1];
    out[1] = v[2] * bs[0] - v[0] * bs[2];
    out[2] = v[0] * bs[1] - v[1] * bs[0];
  }
}

// Highland width for |q| = 1:
//   theta0 = 13.6 MeV/(beta p) sqrt(eps) (1 + 0.038 ln(eps/beta^2)),
//   eps = (x/X0)/|cos incidence|, 1/(beta p) = |q/p| sqrt(1 + m^2 (q/p)^2).
template <typename R>
__device__ __forceinline__ R highland(R lam_abs, R m2, R xx0, R cos_inc) {
  const R g2 = R(1) + m2 * lam_abs * lam_abs;  // 1/beta^2
  const R eps = xx0 / fabs(cos_inc);
  return R(0.0136) * lam_abs * sqrt(g2) * sqrt(eps) * (R(1) + R(0.038) * log(eps * g2));
}

// ---------------------------------------------------------------------------
// float <-> double conversions on the integer pipe.  On this part the
// hardware F2F conversions issue on the (narrow) FP64 pipe; these use plain
// 32-bit integer operations instead.
//   f2d: exact for normal floats and zero; float subnormals become 0;
//        Inf/NaN preserved.
//   d2f: round to nearest even; |x| < 2^-126 becomes 0 (no float subnormals);
//        overflow gives Inf; NaN preserved.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f2d(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t a = b & 0x7fffffffu;
  // normal numbers: the high word is the float's exponent and mantissa moved
  // down by 3 bits with the exponent rebiased by 1023 - 127 = 896
  uint32_t hi = (a >> 3) + 0x38000000u;
  uint32_t lo = b << 29;
  // Inf and NaN: all-ones exponent (a NaN keeps a mantissa bit, in either word)
  if (a >= 0x7f800000u) hi = (a >> 3) | 0x7ff00000u;
  // zero, and the float subnormals, become zero
  if (a < 0x00800000u) hi = lo = 0u;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

__device__ __forceinline__ float d2f(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t ah = hi & 0x7fffffffu;
  // the float's exponent and 23 mantissa bits: the high word and the top 3
  // bits of the low word, shifted up by 3, with the exponent rebiased by
  // -896 (added modulo 2^32 as 2^32 - 896 * 2^23; the field it lands in is
  // right whenever the result is a normal float)
  uint32_t r = __funnelshift_l(lo, ah, 3) + 0x40000000u;
  // round to nearest even on the 29 dropped bits (a carry into the exponent
  // is the correct result, up to Inf)
  const uint32_t rem = lo & 0x1fffffffu;
  r += (rem + (r & 1u)) > 0x10000000u ? 1u : 0u;
  if (ah < 0x38100000u) r = 0u;            // |x| < 2^-126
  if (ah >= 0x47f00000u) r = 0x7f800000u;  // |x| >= 2^128, Inf
  if (ah > 0x7ff00000u || (ah == 0x7ff00000u && lo != 0u)) r = 0x7fc00000u;  // NaN
  return __uint_as_float(r | (hi & 0x80000000u));
}

// Double-precision 1/sqrt(x) and 1/x for positive normal x within the float
// range: a float seed refined by Newton-Raphson steps in double,
//   rsqrt: y <- y + y (1 - x y^2) / 2,   rcp: y <- y + y (1 - x y).
// One step leaves a relative error below 1e-13 (the seed is accurate to a few
// float ulps and each step squares the error); two steps reach double
// rounding level.
// y / 2 for a positive normal double, by decrementing the exponent field on
// the integer pipe
__device__ __forceinline__ double half_pos(double y) {
  return __hiloint2double(__double2hiint(y) - 0x00100000, __double2loint(y));
}

template <int STEPS>
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = f2d(rsqrtf(d2f(x)));
#pragma unroll
  for (int i = 0; i < STEPS; ++i) {
    const double e = fma(-x * y, y, 1.0);
    y = fma(half_pos(y), e, y);
  }
  return y;
}

// x > 0 (false for NaN), decided on the integer pipe: positive doubles order
// like their bit patterns, and NaNs lie above +Inf
__device__ __forceinline__ bool dpos(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}

template <int STEPS>
__device__ __forceinline__ double rcp_nr(double x) {
  double y = f2d(__frcp_rn(d2f(x)));
#pragma unroll
  for (int i = 0; i < STEPS; ++i) {
    const double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
  }
  return y;
}

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000ULL); }

// track fitted by slot i of a launch
__device__ __forceinline__ int track_of(const FitParams& p, int i) {
  return p.order ? p.order[p.track0 + i] : p.track0 + i;
}

// Outputs of a track the launch could not fit: NaN parameters, covariance,
// chi2 and smoothed states, ndf 0, the given status.
__device__ __forceinline__ void write_failed_track(const FitParams& p, int i, int status) {
  const int t = track_of(p, i);
  const size_t TT = (size_t)p.n_tracks_total;
  const double nan = qnan();
#pragma unroll
  for (int e = 0; e < 6; ++e) p.out_params[e * TT + t] = nan;
#pragma unroll
  for (int e = 0; e < 21; ++e) p.out_cov[e * TT + t] = nan;
  p.out_chi2[t] = nan;
  if (p.out_ndf) p.out_ndf[t] = 0;
  if (p.out_status) p.out_status[t] = (uint8_t)status;
  if (p.out_states) {
    const int64_t o0 = p.offsets[t], o1 = p.offsets[t + 1];
    if (o0 >= 0 && o1 > o0 && o1 <= p.n_states && o1 - o0 <= p.max_states)
      for (int64_t k = o0; k < o1; ++k)
        for (int e = 0; e < 6; ++e) p.out_states[e * p.n_states + k] = nan;
  }
}

// The fit kernel: stage the surface table once per CTA, then either one
// track per thread over the grid (work_counter == nullptr) or a persistent
// loop in which every CTA takes blockDim-track units from a global counter
// until the batch is exhausted (balances uneven tracks).
// Body::run(p, s_surf, i) fits slot i.  A CTA whose staging wait gave up, or
// that starts after another CTA's did, writes its tracks as failed
// (status ST_TIMEOUT) instead of fitting them.
template <class Body, int MINB>
__global__ void __launch_bounds__(max_threads_of(MINB), 1) fit_kernel(const FitParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* s_surf = reinterpret_cast<double*>(smem_raw);
  __shared__ __align__(8) uint64_t s_mbar;
  const bool ok = stage_surfaces(s_surf, p.surf, (uint32_t)(p.n_surfaces * Body::kStride * 8), &s_mbar,
                                 p.error_flag, p.wait_limit, p.skip_stage_copy != 0);
  // One call site for both schedules. A grid CTA fits its own blockDim
  // tracks once; a persistent CTA keeps taking blockDim-track units. The
  // whole CTA takes a unit together, so its warps start every unit in step
  // and run the same stretch of the (large) kernel body at the same time,
  // which keeps the instruction fetches shared; the loop condition is
  // uniform over the CTA, so every thread reaches both barriers.
  __shared__ int s_unit;
  const bool persistent = p.work_counter != nullptr;
  int base = blockIdx.x * blockDim.x;
  for (;;) {
    if (persistent) {
      if (threadIdx.x == 0) s_unit = atomicAdd(p.work_counter, 1);
      __syncthreads();
      base = s_unit * blockDim.x;
      __syncthreads();  // all have read s_unit before it is overwritten
    }
    if (base >= p.n_tracks) break;
    const int i = base + threadIdx.x;
    if (i < p.n_tracks) {
      if (ok)
        Body::run(p, s_surf, i);
      else
        write_failed_track(p, i, ST_TIMEOUT);
    }
    if (!persistent) break;
  }
}

// Launch the fit of p.n_tracks tracks: the persistent grid (resident CTAs on
// every SM) when p.work_counter is set; else one thread per track, either
// as one grid or, with p.waves, as full waves of `block`-thread CTAs plus
// one launch that spreads the rest over all SMs.  *launched (optional) gets
// the number of launches queued.
template <class Body, int MINB>
cudaError_t launch_body(const FitParams& p, int block, cudaStream_t stream, int* launched = nullptr) {
  const size_t smem = (size_t)p.n_surfaces * Body::kStride * sizeof(double);
  auto kern = fit_kernel<Body, MINB>;
  if (launched) *launched = 1;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int grid = (p.n_tracks + block - 1) / block;
  if (p.work_counter || p.waves) {
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (p.work_counter) {
      long long resident = (long long)nsm * occ;
      if (p.resident_warps > 0) {
        const long long want = ((long long)nsm * p.resident_warps * 32 + block - 1) / block;
        if (want < resident) resident = want;
      }
      if (grid > resident) grid = (int)resident;
    } else {
      // full waves of `block`-thread CTAs (every SM's resident CTAs), then
      // the remainder spread over all SMs in one wave of smaller CTAs, so
      // that the last wave leaves no SM idle
      const long long per_wave = (long long)nsm * occ * block;
      const long long full = ((long long)p.n_tracks / per_wave) * per_wave;
      const long long rest = (long long)p.n_tracks - full;
      if (full > 0 && rest > 0) {
        const long long rest_warps = (rest + 31) / 32;
        long long b2 = 32 * ((rest_warps + (long long)nsm * occ - 1) / ((long long)nsm * occ));
        if (b2 > block) b2 = block;
        FitParams a = p;
        a.n_tracks = (int32_t)full;
        kern<<<(int)(full / block), block, smem, stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        FitParams b = p;
        b.track0 = p.track0 + (int32_t)full;
        b.n_tracks = (int32_t)rest;
        kern<<<(int)((rest + b2 - 1) / b2), (int)b2, smem, stream>>>(b);
        if (launched) *launched = 2;
        return cudaGetLastError();
      }
    }
  }
  kern<<<grid, block, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace kfgb
