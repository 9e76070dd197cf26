// kf_static.cu -- kf_fit_static: the fit without any device allocation.
//
// Some callers cannot allocate device memory: real-time trigger loops that
// must never block on the CUDA allocator, and hosts that hand the library a
// fixed memory budget up front and own every other byte of device memory.  For them this entry point uses one fixed
// block of device memory that lives in this file for the whole life of the
// process: every GPU that loads the library keeps kStaticBytes reserved until
// the process exits.  The caller still owns and passes all inputs and
// outputs.
//
// What the static block holds: the packed surface table, the error flag word
// the kernels raise if a bounded wait gives up, and the per-state records the
// smoother reads back.  Batches whose
// records do not fit are fitted in several launches on the caller's stream,
// one after another, reusing the same block.
//
// Set-up: the first call on a device looks up the device address of the
// block with cudaGetSymbolAddress (host code cannot use the array's name as a
// device pointer) and caches it.  Make that first call on each device before
// capturing a stream.
//
// Sharing: all calls share the one block and it keeps whatever the last call
// left in it.  Calls whose GPU work overlaps in time (other streams, other
// host threads) race on it; serialise them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/kf.h"
#include "kf_internal.h"

using namespace kfgb;

namespace {

constexpr size_t kStaticBytes = size_t(64) << 20;  // 64 MiB per device
constexpr size_t kSurfBytes = size_t(kMaxSurfaces) * kSurfPacked * sizeof(double);
constexpr size_t kFlagBytes = 256;
constexpr size_t kRecordBytes = kStaticBytes - kSurfBytes - kFlagBytes;

static __device__ __align__(256) unsigned char g_static_block[kStaticBytes];

std::mutex g_mu;
void* g_block_ptr[64] = {nullptr};

// device address of the static block on the current device (set up once)
cudaError_t static_block(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_block_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_block);
    if (e != cudaSuccess) return e;
    g_block_ptr[dev] = p;
  }
  *out = g_block_ptr[dev];
  return cudaSuccess;
}

size_t rec_bytes(int precision) {
  return precision == KF_PRECISION_FP64 ? kRec64Fp64 * sizeof(double)
                                        : kRec64Mixed * sizeof(double) + kRec32Mixed * sizeof(float);
}

}  // namespace

extern "C" int kf_fit_static(const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me,
                             const kf_field* fi, const kf_options* opt_in, const kf_outputs* out,
                             void* stream_v) {
  kf_options opt;
  if (opt_in) opt = *opt_in; else kf_default_options(&opt);
  if (!tr || !su || !me || !fi || !out) return KF_EINVAL;
  if (tr->n_tracks < 0 || me->n_states < 0 || su->n_surfaces < 1 || tr->max_states < 1) return KF_EINVAL;
  if (tr->n_tracks > 0 && (!tr->offsets || !tr->seed_params || !tr->seed_cov || !out->params || !out->cov ||
                           !out->chi2))
    return KF_EINVAL;
  if (me->n_states > 0 && (!me->surface_id || !me->loc || !me->cov || !me->is_hole)) return KF_EINVAL;
  if (!su->center || !su->rot || !su->x_over_x0) return KF_EINVAL;
  if (opt.precision != KF_PRECISION_FP64 && opt.precision != KF_PRECISION_MIXED) return KF_EUNSUPPORTED;
  if (!(opt.mass >= 0.0) || !(opt.h_max > 0.0) || opt.n_iter < 0 || opt.n_iter > 16) return KF_EINVAL;
  if (opt.block < 0 || (opt.block % 32) != 0 || opt.block > max_block(opt.precision == KF_PRECISION_MIXED, opt.min_blocks))
    return KF_EUNSUPPORTED;
  if (opt.schedule < KF_SCHEDULE_GRID || opt.schedule > KF_SCHEDULE_PERSISTENT) return KF_EUNSUPPORTED;
  if (opt.min_blocks < 0 || opt.min_blocks > 4) return KF_EUNSUPPORTED;
  if (opt.resident_warps < 0 || opt.resident_warps > 64) return KF_EINVAL;
  if (opt.wait_limit < 0 || (opt.test_wait_timeout != 0 && opt.test_wait_timeout != 1)) return KF_EINVAL;
  if (opt.team_warps > 1) return KF_EUNSUPPORTED;  // one thread per track only
  // the static block serves the baseline method only
  if (wants_variants(opt.smoother, opt.energy_loss, fi->map)) return KF_EUNSUPPORTED;
  // size limits of the static block
  if (su->n_surfaces > kMaxSurfaces) return KF_ESIZE;
  // one track's records (both precisions' parts, each 256-byte aligned) must fit
  const size_t per_track = rec_bytes(opt.precision) * (size_t)tr->max_states;
  if (per_track + 512 > kRecordBytes) return KF_ESIZE;
  if (tr->n_tracks == 0) return KF_SUCCESS;

  void* base = nullptr;
  cudaError_t e = static_block(&base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static block)");
  cudaStream_t stream = (cudaStream_t)stream_v;
  char* b = (char*)base;
  double* surf = (double*)b;
  int32_t* flag = (int32_t*)(b + kSurfBytes);
  char* rec = b + kSurfBytes + kFlagBytes;
  // tracks per launch
  size_t chunk = (kRecordBytes - 512) / per_track;
  if (chunk > (size_t)tr->n_tracks) chunk = (size_t)tr->n_tracks;
  const size_t n64 = opt.precision == KF_PRECISION_FP64 ? kRec64Fp64 : kRec64Mixed;
  const size_t bytes64 = (n64 * sizeof(double) * tr->max_states * chunk + 255) / 256 * 256;

  e = cudaMemsetAsync(flag, 0, 2 * sizeof(int32_t), stream);  // flag and work counter start at zero
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(static flag)");
  e = launch_pack_surfaces(su->n_surfaces, su->center, su->rot, su->x_over_x0, surf, stream);
  if (e != cudaSuccess) return cuda_fail(e, "pack_surfaces launch");
  FitParams p;
  memset(&p, 0, sizeof(p));
  p.resident_warps = opt.resident_warps;
  p.n_tracks_total = tr->n_tracks;
  p.max_states = tr->max_states;
  p.offsets = tr->offsets;
  p.seed_params = tr->seed_params;
  p.seed_cov = tr->seed_cov;
  p.n_surfaces = su->n_surfaces;
  p.surf = surf;
  p.n_states = me->n_states;
  p.surface_id = me->surface_id;
  p.loc = me->loc;
  p.cov = me->cov;
  p.is_hole = me->is_hole;
  for (int i = 0; i < 3; ++i) p.bfield[i] = fi->b[i];
  p.mass = opt.mass;
  p.h_max = opt.h_max;
  p.n_iter = opt.n_iter;
  p.out_params = out->params;
  p.out_cov = out->cov;
  p.out_chi2 = out->chi2;
  p.out_ndf = out->ndf;
  p.out_status = out->status;
  p.out_states = out->states;
  p.ws64 = (double*)rec;
  p.ws32 = opt.precision == KF_PRECISION_FP64 ? nullptr : (float*)(rec + bytes64);
  p.error_flag = flag;
  p.wait_limit = opt.wait_limit;
  p.skip_stage_copy = opt.test_wait_timeout;
  // persistent launches share one work counter, re-zeroed before each chunk
  const bool persistent = opt.schedule != KF_SCHEDULE_GRID;
  for (size_t t0 = 0; t0 < (size_t)tr->n_tracks; t0 += chunk) {
    p.track0 = (int32_t)t0;
    p.n_tracks = (int32_t)(((size_t)tr->n_tracks - t0) < chunk ? ((size_t)tr->n_tracks - t0) : chunk);
    p.work_counter = persistent ? flag + 1 : nullptr;
    if (persistent && t0 > 0) {
      e = cudaMemsetAsync(flag + 1, 0, sizeof(int32_t), stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(static counter)");
    }
    e = launch_fit(p, opt.precision, opt.block, opt.min_blocks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "fit launch");
  }
  return KF_SUCCESS;
}
