// Internal interface between the C ABI (kf_api.cu) and the kernels
// (kf_kernels.cu).  Not part of the public header.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kfgb {

// Packed surface record staged into shared memory: 24 doubles (192 B, a
// whole number of 16-byte units for the bulk copy):
//   doubles [0..2] centre c, [3..11] R row-major (columns u, v, n), [12] x/X0,
//           [13] n.c, [14] u.c, [15] v.c
//   floats at double offset 16: [0..2] n, [3..5] u, [6..8] v, [9] x/X0
//           (float copies)
// The mixed kernel stages a table of its own, 32 floats (128 B) per surface,
// packed after the FP64 table in the same buffer ([n_surfaces][kSurfStride]
// doubles, then [n_surfaces][kSurfStrideM] doubles): every FP64 quantity as
// a double-float pair hi + lo (hi = the nearest float, lo = the nearest
// float to the rest), so it converts nothing per step:
//   [0..2] n hi, [3..5] u hi, [6..8] v hi, [9] x/X0,
//   [10..12] n lo, [13..15] u lo, [16..18] v lo,
//   [19..21] (n.c, u.c, v.c) hi, [22..24] (n.c, u.c, v.c) lo,
//   [25..27] c hi, [28..30] c lo, [31] 0
constexpr int kSurfStride = 24;
constexpr int kSurfStrideM = 16;
constexpr int kSurfPacked = kSurfStride + kSurfStrideM;  // doubles per surface in the packed buffer
constexpr int kMaxSurfaces = 1024;  // 192 KiB of shared memory (FP64 table)

// Per-state record the forward pass writes and the RTS pass reads back.
// FP64 path, all in ws64:  xp 6 | xf 6 | Cp 21 | Cf 21 | Bm 36   (90 doubles)
//   Bm = F_k * Cf_{k-1}: the right-hand side of the smoother-gain solve.
// Mixed path, ws64:        xp 6                                   (6 doubles)
//             ws32:        F 25 | q_phi | q_theta | dxf 6 | Cp 21 (54 floats)
//   xp is written for state 0 always and for the others only when smoothed
//   states are output.
//   F_k: rows loc0, loc1, phi, theta over columns 0..4 (20), then the time
//   row over columns 0..4 (5); q = the multiple-scattering variances added to
//   Var(phi) and Var(theta) at state k; dxf = x_f - x_p (the filter's
//   increment, zero on a hole); Cp = the predicted covariance of state k
//   (FP32 products, so exact as floats; states k >= 1).
// Register-cap variants of the fit kernels ("min_blocks"): variant 1 (the
// default) may use 255 registers, 3 caps at 168 and 4 at 128, i.e. the
// registers of 1, 3 or 4 CTAs of 128 threads per SM. Each variant accepts
// CTAs of up to the threads those registers allow.
constexpr int max_threads_of(int min_blocks) { return min_blocks == 4 ? 512 : min_blocks == 3 ? 384 : 256; }
// largest CTA a launch may ask for: only the mixed kernel has the capped
// variants; the FP64 and method-variant kernels are variant 1
inline int max_block(bool mixed, int min_blocks) { return max_threads_of(mixed ? min_blocks : 1); }

constexpr int kRec64Fp64 = 90;
constexpr int kRec64Mixed = 6;
constexpr int kRec32Mixed = 54;

struct FitParams {
  int32_t n_tracks;        // tracks in this launch (chunk)
  int32_t track0;          // global index of the chunk's first track
  int32_t n_tracks_total;  // row stride of [k][n_tracks_total] inputs/outputs
  int32_t max_states;      // states per track the workspace holds
  const int32_t* offsets;
  const double* seed_params;
  const double* seed_cov;
  int32_t n_surfaces;
  const double* surf;      // packed [n_surfaces][kSurfStride]
  int64_t n_states;
  const int32_t* surface_id;
  const double* loc;
  const double* cov;
  const uint8_t* is_hole;
  double bfield[3];
  double mass;
  double h_max;
  int32_t n_iter;
  double* out_params;
  double* out_cov;
  double* out_chi2;
  int32_t* out_ndf;
  uint8_t* out_status;
  double* out_states;
  double* ws64;            // [max_states][rec64][n_tracks]
  float* ws32;             // [max_states][rec32][n_tracks] (mixed only)
  int32_t* error_flag;     // set to 1 when a bounded device wait gives up
  int32_t wait_limit;      // polls of a bounded wait (0 = the default)
  int32_t skip_stage_copy; // diagnostic: announce but skip the surface-table
                           // copy, so that every staging wait runs out
  int32_t* work_counter;   // non-null: persistent launch, warps take 32-track
                           // units from this counter (zeroed before launch)
  const int32_t* order;    // non-null: slot s fits track order[s]
  int32_t resident_warps;  // persistent launch: warps per SM (0 = occupancy)
  int32_t waves;           // grid launch split into full waves + one spread wave (host side)
  int32_t team_warps;      // FP64 path: > 1 shares each track over that many warps (host side)
  // method variants (the FP64 variant kernel)
  int32_t smoother;        // 0 RTS, 1 backward filter + weighted mean
  int32_t energy_loss;     // 1: mean loss and straggling on q/p
  double bf_scale;         // backward filter start: bf_scale * Cf_{n-1}
  double mat[9];           // z_over_a, i_exc, x0_rho, Sternheimer cbar, x0,
                           // x1, a, k, delta0
  int32_t map_n[3];        // field-map grid points per axis
  double map_origin[3];
  double map_inv_spacing[3];
  const double* map_b;     // null: the constant field bfield
};

// Record a failed CUDA call for kf_last_cuda_error() and map it to a
// kf_error code (KF_ENOMEM for allocation failures, else KF_ECUDA).
int cuda_fail(cudaError_t e, const char* what);

// True when the options or the field ask for a method variant.
inline bool wants_variants(int smoother, int energy_loss, const void* map) {
  return smoother != 0 || energy_loss != 0 || map != nullptr;
}

// Pack the SoA surface table into [S][kSurfStride] doubles followed by the
// mixed kernel's [S][kSurfStrideM] (packed must hold S * kSurfPacked doubles).
cudaError_t launch_pack_surfaces(int n_surfaces, const double* center,
                                 const double* rot, const double* x_over_x0,
                                 double* packed, cudaStream_t stream);

// Check the integer-pipe conversions and the Newton 1/sqrt, 1/x helpers on n
// patterns; counters[0..4] receive the mismatch counts.
cudaError_t launch_selftest(long long n, unsigned long long* counters, cudaStream_t stream);
// Check the mixed kernel's double-float arithmetic against FP64 on n
// patterns; counters[0..3] receive the counts beyond 2^-44, counters[4] the
// patterns a plain float sum already misses.
cudaError_t launch_selftest_df(long long n, unsigned long long* counters, cudaStream_t stream);
// The full-range 1/sqrt and 1/x helpers of the FP64 path; counter[0] gets
// the cases beyond 4 ulp.
cudaError_t launch_selftest_any(long long n, unsigned long long* counter, cudaStream_t stream);

// One fused filter + smoother launch over p.n_tracks tracks.  min_blocks
// selects the register-cap variant (__launch_bounds__ minimum CTAs per SM;
// 0 = the default variant).
// *launched (optional) gets the number of kernel launches queued.
cudaError_t launch_fit(const FitParams& p, int precision, int block, int min_blocks,
                       cudaStream_t stream, int* launched = nullptr);

// The FP64 fit with each track's work shared by a team of 2 or 4 warps
// (kf_team.cu): one CTA per 32 tracks, grid schedule.
cudaError_t launch_fit_team(const FitParams& p, int team_warps, cudaStream_t stream, int* launched = nullptr);

// The FP64 kernel of the method variants (kf_variants.cu): backward-filter
// smoother, energy loss, field map; same records as the FP64 path.
cudaError_t launch_fit_variants(const FitParams& p, int block, cudaStream_t stream, int* launched = nullptr);

// Inputs and outputs of the adjoint (kf_adjoint.cu): the objective
// L = sum_t [w_t chi2_t + v_t . x_s0,t + W_t . C_s0,t] (x_s0, C_s0 the
// smoothed parameters and packed covariance of state 0) and its gradient
// with respect to the seeds and the per-surface alignment.
struct GradArgs {
  const double* align;       // [6][S] or null (zero)
  const double* align_cs;    // [6][S] cosines and sines of its angles (launch_align_trig)
  const double* dl_dchi2;    // w [T] or null (ones)
  const double* dl_dparams;  // v [6][T] or null (zero)
  const double* dl_dcov;     // W [21][T] or null (zero)
  double* chi2;              // [T] or null
  double* params;            // [6][T] or null: x_s0
  double* cov;               // [21][T] or null: C_s0
  double* grad_seed;         // [6][T] or null
  double* grad_align;        // [6][S] or null: accumulated (the caller zeroes it)
};

// The cosines and sines of every surface's three alignment angles, out[6][S]
// (cos alpha, sin alpha, cos beta, sin beta, cos gamma, sin gamma).
cudaError_t launch_align_trig(int n_surfaces, const double* align, double* out, cudaStream_t stream);

// Scratch doubles per track of one adjoint launch: the filtered checkpoints,
// with the smoother's adjoint the smoothed checkpoints and its per-state
// contributions, and in the pipelined form two hand-off slots.
size_t grad_scratch_doubles(int max_states, bool smoother, bool smoother_adjoint, bool pipelined);

// One launch over tracks [f.track0, f.track0 + f.n_tracks) of
// f.n_tracks_total; scratch holds grad_scratch_doubles(...) x f.n_tracks.
// pipelined: two warps per 32 tracks (the forward and the reverse half of
// the filter's reverse sweep on separate warps), block ignored.
cudaError_t launch_grad(const FitParams& f, const GradArgs& a, double* scratch, int block, int min_blocks,
                        bool pipelined, cudaStream_t stream);

// Counting sort of the tracks by state count, longest first:
// order[0..n_tracks) receives track indices.  hist needs max_states + 2 ints.
cudaError_t launch_length_order(int n_tracks, int max_states, const int32_t* offsets,
                                int32_t* hist, int32_t* order, cudaStream_t stream);

}  // namespace kfgb
