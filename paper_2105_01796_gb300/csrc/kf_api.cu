// kf_api.cu -- the C ABI declared in include/kf.h: argument validation,
// handle-owned workspace, chunking of large batches, host-buffer entry point.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/kf.h"
#include "kf_internal.h"

using namespace kfgb;

namespace {
thread_local char g_cuda_err[256] = "no CUDA error";
}

int kfgb::cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? KF_ENOMEM : KF_ECUDA;
}

struct kf_handle {
  int device = -1;
  // device workspace (per-state records) and the packed surface table
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* surf = nullptr;
  int surf_cap = 0;
  int32_t* error_flag = nullptr;
  // work counters (one per chunk launch) and the length-sort buffers
  int32_t* counters = nullptr;
  int counters_cap = 0;
  int32_t* order = nullptr;
  int64_t order_cap = 0;
  int32_t* hist = nullptr;
  int hist_cap = 0;
  // adjoint checkpoints
  double* ckpt = nullptr;
  size_t ckpt_bytes = 0;
  // autotuner cache: best launch options per batch shape
  struct Tuned {
    int32_t precision, n_tracks, max_states, n_surfaces, bz, variants;
    kf_options best;
    double ms;
  };
  Tuned tuned[16];
  int n_tuned = 0;
  // cached CUDA graph of the last captured fit and the call it replays
  cudaGraphExec_t graph_exec = nullptr;
  alignas(8) unsigned char graph_key[1024];
  int32_t graph_launches = 0;
  // device copies for kf_fit_host, and its streams and events (the
  // pipelined host path overlaps the copies of some chunks of tracks with
  // the fits of others, and lets consecutive fits overlap on two streams)
  static constexpr int kPipe = 8;
  void* dev_io = nullptr;
  size_t dev_io_bytes = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr, s_fit[kPipe - 1] = {};
  cudaEvent_t ev_in[kPipe] = {}, ev_fit[kPipe] = {}, ev_pack = nullptr;
  int32_t last_launches = 0;
};

namespace {


constexpr double kMuonMass = 0.1056583755;
constexpr int64_t kDefaultWorkspace = int64_t(32) << 30;

size_t record_bytes(int precision) {
  return precision == KF_PRECISION_FP64 ? kRec64Fp64 * sizeof(double)
                                        : kRec64Mixed * sizeof(double) + kRec32Mixed * sizeof(float);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// tracks per launch that fit the workspace cap
int64_t chunk_tracks(int64_t n_tracks, int32_t max_states, const kf_options& o) {
  const int64_t cap = o.workspace_bytes > 0 ? o.workspace_bytes : kDefaultWorkspace;
  const int64_t per_track = (int64_t)record_bytes(o.precision) * (max_states > 0 ? max_states : 1);
  int64_t c = cap / per_track;
  if (c < 1) c = 1;
  return c < n_tracks ? c : n_tracks;
}

int ensure_ws(kf_handle* h, size_t bytes) {
  if (h->ws_bytes >= bytes) return KF_SUCCESS;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
  h->ws_bytes = bytes;
  return KF_SUCCESS;
}

int ensure_surf(kf_handle* h, int n) {
  if (h->surf_cap >= n) return KF_SUCCESS;
  if (h->surf) cudaFree(h->surf);
  h->surf = nullptr;
  h->surf_cap = 0;
  cudaError_t e = cudaMalloc(&h->surf, (size_t)n * kSurfPacked * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(surfaces)");
  h->surf_cap = n;
  return KF_SUCCESS;
}

int validate(const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me, const kf_field* fi,
             const kf_options* opt, const kf_outputs* out) {
  if (!tr || !su || !me || !fi || !opt || !out) return KF_EINVAL;
  if (tr->n_tracks < 0 || su->n_surfaces < 1 || me->n_states < 0) return KF_EINVAL;
  if (tr->n_tracks > 0) {
    if (!tr->offsets || !tr->seed_params || !tr->seed_cov) return KF_EINVAL;
    if (!out->params || !out->cov || !out->chi2) return KF_EINVAL;
    if (tr->max_states < 1) return KF_EINVAL;
    if (me->n_states > 0 && (!me->surface_id || !me->loc || !me->cov || !me->is_hole)) return KF_EINVAL;
  }
  if (!su->center || !su->rot || !su->x_over_x0) return KF_EINVAL;
  if (su->n_surfaces > kMaxSurfaces) return KF_EUNSUPPORTED;
  if (opt->precision != KF_PRECISION_FP64 && opt->precision != KF_PRECISION_MIXED) return KF_EUNSUPPORTED;
  if (!(opt->mass >= 0.0) || !(opt->h_max > 0.0) || opt->n_iter < 0 || opt->n_iter > 16) return KF_EINVAL;
  if (opt->schedule < KF_SCHEDULE_AUTO || opt->schedule > KF_SCHEDULE_WAVES) return KF_EUNSUPPORTED;
  if (opt->min_blocks < 0 || opt->min_blocks > 4) return KF_EUNSUPPORTED;
  if (opt->block < 0 || (opt->block % 32) != 0 || opt->block > max_block(opt->precision == KF_PRECISION_MIXED, opt->min_blocks))
    return KF_EUNSUPPORTED;
  if (opt->resident_warps < 0 || opt->resident_warps > 64) return KF_EINVAL;
  if (opt->wait_limit < 0 || (opt->test_wait_timeout != 0 && opt->test_wait_timeout != 1)) return KF_EINVAL;
  if (opt->team_warps < 0 || opt->team_warps == 3 || opt->team_warps > 4) return KF_EINVAL;
  if (opt->team_warps > 1 && (opt->precision != KF_PRECISION_FP64 || wants_variants(opt->smoother, opt->energy_loss,
                                                                                     fi->map)))
    return KF_EUNSUPPORTED;
  for (int i = 0; i < 3; ++i)
    if (!(fi->b[i] == fi->b[i])) return KF_EINVAL;
  if (opt->smoother != KF_SMOOTHER_RTS && opt->smoother != KF_SMOOTHER_BACKWARD_FILTER) return KF_EUNSUPPORTED;
  if (opt->energy_loss != 0 && opt->energy_loss != 1) return KF_EINVAL;
  if (wants_variants(opt->smoother, opt->energy_loss, fi->map) && opt->precision != KF_PRECISION_FP64)
    return KF_EUNSUPPORTED;
  if (opt->smoother == KF_SMOOTHER_BACKWARD_FILTER && !(opt->bf_scale > 0.0 && opt->bf_scale < 1e300))
    return KF_EINVAL;
  if (opt->energy_loss) {
    const kf_material& m = opt->material;
    if (!(opt->mass > 0.0) || !(m.z_over_a > 0.0) || !(m.i_exc > 0.0) || !(m.x0_rho > 0.0)) return KF_EINVAL;
  }
  if (fi->map) {
    const kf_field_map& f = *fi->map;
    if (f.nx < 2 || f.ny < 2 || f.nz < 2 || !f.b) return KF_EINVAL;
    for (int i = 0; i < 3; ++i)
      if (!(f.spacing[i] > 0.0 && f.spacing[i] < 1e300) || !(f.origin[i] == f.origin[i])) return KF_EINVAL;
  }
  return KF_SUCCESS;
}

// silicon as tabulated by the PDG (atomic and nuclear properties): Z/A, I,
// X0 rho and the Sternheimer density-effect parameters
void silicon(kf_material* m) {
  m->z_over_a = 0.49848;
  m->i_exc = 173.0e-9;
  m->x0_rho = 21.82;
  m->sh_cbar = 4.4355;
  m->sh_x0 = 0.2015;
  m->sh_x1 = 2.8716;
  m->sh_a = 0.1492;
  m->sh_k = 3.2546;
  m->sh_delta0 = 0.14;
}

}  // namespace

extern "C" {

void kf_default_options(kf_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = KF_PRECISION_FP64;
  opt->mass = kMuonMass;
  opt->h_max = 50.0;
  opt->n_iter = 3;
  opt->block = 128;
  opt->workspace_bytes = 0;
  opt->schedule = KF_SCHEDULE_PERSISTENT;
  opt->min_blocks = 0;
  opt->use_graph = 0;
  opt->resident_warps = 0;
  opt->smoother = KF_SMOOTHER_RTS;
  opt->energy_loss = 0;
  opt->bf_scale = 1e4;
  silicon(&opt->material);
  opt->wait_limit = 0;
  opt->team_warps = 0;
  opt->test_wait_timeout = 0;
}

int kf_abi_version(void) { return KF_ABI_VERSION; }

int kf_selftest(int64_t n_patterns, uint64_t* counts) {
  if (!counts || n_patterns < 0) return KF_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 6 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(selftest)");
  e = cudaMemset(d, 0, 6 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_selftest(n_patterns, d, nullptr);
  if (e == cudaSuccess) e = launch_selftest_any(n_patterns, d + 5, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(counts, d, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "selftest");
  return KF_SUCCESS;
}

int kf_selftest_df(int64_t n_patterns, uint64_t* counts) {
  if (!counts || n_patterns < 0) return KF_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 5 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(selftest_df)");
  e = cudaMemset(d, 0, 5 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_selftest_df(n_patterns, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(counts, d, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "selftest_df");
  return KF_SUCCESS;
}

const char* kf_strerror(int code) {
  switch (code) {
    case KF_SUCCESS: return "success";
    case KF_EINVAL: return "invalid argument";
    case KF_ECUDA: return "CUDA error (see kf_last_cuda_error)";
    case KF_ENOMEM: return "out of memory";
    case KF_EUNSUPPORTED: return "unsupported option";
    case KF_EDEVICE: return "a device-side bounded wait timed out (its tracks have status KF_TRACK_TIMEOUT)";
    case KF_ESIZE: return "batch does not fit the fixed device block of kf_fit_static";
    default: return "unknown error";
  }
}

const char* kf_last_cuda_error(void) { return g_cuda_err; }

int kf_create(kf_handle** handle) {
  if (!handle) return KF_EINVAL;
  *handle = nullptr;
  kf_handle* h = new (std::nothrow) kf_handle();
  if (!h) return KF_ENOMEM;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDevice");
  }
  e = cudaMalloc(&h->error_flag, sizeof(int32_t));
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaMalloc(error flag)");
  }
  e = cudaMemset(h->error_flag, 0, sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaFree(h->error_flag);
    delete h;
    return cuda_fail(e, "cudaMemset");
  }
  *handle = h;
  return KF_SUCCESS;
}

void kf_destroy(kf_handle* h) {
  if (!h) return;
  if (h->ws) cudaFree(h->ws);
  if (h->surf) cudaFree(h->surf);
  if (h->error_flag) cudaFree(h->error_flag);
  if (h->dev_io) cudaFree(h->dev_io);
  if (h->counters) cudaFree(h->counters);
  if (h->order) cudaFree(h->order);
  if (h->hist) cudaFree(h->hist);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->ckpt) cudaFree(h->ckpt);
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  for (int i = 0; i < kf_handle::kPipe - 1; ++i)
    if (h->s_fit[i]) cudaStreamDestroy(h->s_fit[i]);
  for (int i = 0; i < kf_handle::kPipe; ++i) {
    if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
    if (h->ev_fit[i]) cudaEventDestroy(h->ev_fit[i]);
  }
  if (h->ev_pack) cudaEventDestroy(h->ev_pack);
  delete h;
}

int64_t kf_workspace_size(int32_t n_tracks, int32_t max_states, const kf_options* opt) {
  kf_options o;
  if (opt) o = *opt; else kf_default_options(&o);
  if (n_tracks <= 0 || max_states <= 0) return 0;
  const int64_t c = chunk_tracks(n_tracks, max_states, o);
  return (int64_t)record_bytes(o.precision) * max_states * c + 256;
}

int32_t kf_last_launch_count(const kf_handle* h) { return h ? h->last_launches : 0; }

}  // extern "C"

namespace {

// Everything kf_fit_ex computes before it queues work: chunking and the
// handle's buffers (allocations cannot happen inside a stream capture).
// schedules that take work from a global counter
inline bool uses_counter(int schedule) {
  return schedule == KF_SCHEDULE_PERSISTENT || schedule == KF_SCHEDULE_SORTED;
}

struct FitPlan {
  int64_t chunk;
  size_t bytes64;
  int n_chunks;
};

int prepare_fit(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const kf_options& opt, FitPlan* plan) {
  int rc;
  const int64_t chunk = chunk_tracks(tr->n_tracks, tr->max_states, opt);
  const size_t n64 = opt.precision == KF_PRECISION_FP64 ? kRec64Fp64 : kRec64Mixed;
  const size_t bytes64 = align_up(n64 * sizeof(double) * tr->max_states * chunk, 256);
  const size_t bytes32 =
      opt.precision == KF_PRECISION_FP64 ? 0 : align_up(kRec32Mixed * sizeof(float) * tr->max_states * chunk, 256);
  if ((rc = ensure_ws(h, bytes64 + bytes32))) return rc;
  if ((rc = ensure_surf(h, su->n_surfaces))) return rc;
  const int n_chunks = (int)((tr->n_tracks + chunk - 1) / chunk);
  if (uses_counter(opt.schedule) && h->counters_cap < n_chunks) {
    if (h->counters) cudaFree(h->counters);
    h->counters = nullptr;
    h->counters_cap = 0;
    cudaError_t e = cudaMalloc(&h->counters, sizeof(int32_t) * n_chunks);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(counters)");
    h->counters_cap = n_chunks;
  }
  if (opt.schedule == KF_SCHEDULE_SORTED) {
    if (h->order_cap < tr->n_tracks) {
      if (h->order) cudaFree(h->order);
      h->order = nullptr;
      h->order_cap = 0;
      cudaError_t e = cudaMalloc(&h->order, sizeof(int32_t) * (size_t)tr->n_tracks);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(order)");
      h->order_cap = tr->n_tracks;
    }
    if (h->hist_cap < tr->max_states + 2) {
      if (h->hist) cudaFree(h->hist);
      h->hist = nullptr;
      h->hist_cap = 0;
      cudaError_t e = cudaMalloc(&h->hist, sizeof(int32_t) * (size_t)(tr->max_states + 2));
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(hist)");
      h->hist_cap = tr->max_states + 2;
    }
  }
  plan->chunk = chunk;
  plan->bytes64 = bytes64;
  plan->n_chunks = n_chunks;
  return KF_SUCCESS;
}

// method-variant fields of the launch parameters
void fill_variants(FitParams* p, const kf_field* fi, const kf_options& opt) {
  p->smoother = opt.smoother;
  p->energy_loss = opt.energy_loss;
  p->bf_scale = opt.bf_scale;
  const kf_material& m = opt.material;
  const double mat[9] = {m.z_over_a, m.i_exc, m.x0_rho, m.sh_cbar, m.sh_x0, m.sh_x1, m.sh_a, m.sh_k, m.sh_delta0};
  for (int i = 0; i < 9; ++i) p->mat[i] = mat[i];
  if (fi->map) {
    const kf_field_map& f = *fi->map;
    p->map_n[0] = f.nx;
    p->map_n[1] = f.ny;
    p->map_n[2] = f.nz;
    for (int i = 0; i < 3; ++i) {
      p->map_origin[i] = f.origin[i];
      p->map_inv_spacing[i] = 1.0 / f.spacing[i];
    }
    p->map_b = f.b;
  }
}

// Queue the fit of tracks [t_begin, t_end) on `stream` (no allocation, no
// synchronisation).  pack: also pack the surface table first.  A partial
// range (the host entry's pipelined chunks) cannot use the length-sorted
// order, which spans the whole batch: it runs the persistent schedule.
// Fits of disjoint ranges that may run at the same time (on two streams)
// pass own_slice: each then uses its own work counter (counter_slot, reset
// by the caller) and the slice of the workspace at its first track (the
// plan must then hold the whole batch in one workspace chunk).
int enqueue_fit(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me,
                const kf_field* fi, const kf_options& opt_in, const kf_outputs* out, cudaStream_t stream,
                const FitPlan& plan, int* launches_out, int64_t t_begin = 0, int64_t t_end = -1,
                bool pack = true, bool own_slice = false, int counter_slot = 0) {
  if (t_end < 0) t_end = tr->n_tracks;
  kf_options opt = opt_in;
  if (opt.team_warps > 1) opt.schedule = KF_SCHEDULE_GRID;  // one CTA per 32 tracks
  const bool whole = t_begin == 0 && t_end == tr->n_tracks;
  if (!whole && opt.schedule == KF_SCHEDULE_SORTED) opt.schedule = KF_SCHEDULE_PERSISTENT;
  const int64_t chunk = plan.chunk;
  cudaError_t e = cudaSuccess;
  int launches = 0;
  if (pack) {
    // a new call: clear the flag a timed-out wait of an earlier call left
    e = cudaMemsetAsync(h->error_flag, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(error flag)");
    e = launch_pack_surfaces(su->n_surfaces, su->center, su->rot, su->x_over_x0, h->surf, stream);
    if (e != cudaSuccess) return cuda_fail(e, "pack_surfaces launch");
    launches = 1;
  }
  if (own_slice && plan.n_chunks != 1) return KF_EINVAL;
  if (uses_counter(opt.schedule) && !own_slice) {
    e = cudaMemsetAsync(h->counters, 0, sizeof(int32_t) * plan.n_chunks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
  }
  if (opt.schedule == KF_SCHEDULE_SORTED) {
    e = launch_length_order(tr->n_tracks, tr->max_states, tr->offsets, h->hist, h->order, stream);
    if (e != cudaSuccess) return cuda_fail(e, "length order launch");
    launches += 3;
  }
  FitParams p;
  memset(&p, 0, sizeof(p));
  p.n_tracks_total = tr->n_tracks;
  p.max_states = tr->max_states;
  p.offsets = tr->offsets;
  p.seed_params = tr->seed_params;
  p.seed_cov = tr->seed_cov;
  p.n_surfaces = su->n_surfaces;
  p.surf = h->surf;
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
  p.ws64 = (double*)h->ws;
  p.ws32 = opt.precision == KF_PRECISION_FP64 ? nullptr : (float*)((char*)h->ws + plan.bytes64);
  if (own_slice) {
    // records are [state][element][track] over the launch's own tracks, so
    // a range starting at track t_begin owns the slice from t_begin records on
    const size_t n64 = opt.precision == KF_PRECISION_FP64 ? kRec64Fp64 : kRec64Mixed;
    p.ws64 += n64 * (size_t)tr->max_states * (size_t)t_begin;
    if (p.ws32) p.ws32 += kRec32Mixed * (size_t)tr->max_states * (size_t)t_begin;
  }
  p.error_flag = h->error_flag;
  p.wait_limit = opt.wait_limit;
  p.skip_stage_copy = opt.test_wait_timeout;
  p.order = opt.schedule == KF_SCHEDULE_SORTED ? h->order : nullptr;
  p.resident_warps = opt.resident_warps;
  p.waves = opt.schedule == KF_SCHEDULE_WAVES;
  p.team_warps = opt.team_warps;
  const bool variants = wants_variants(opt.smoother, opt.energy_loss, fi->map);
  if (variants) fill_variants(&p, fi, opt);
  int c = 0;
  for (int64_t t0 = t_begin; t0 < t_end; t0 += chunk, ++c) {
    p.track0 = (int32_t)t0;
    p.n_tracks = (int32_t)((t_end - t0) < chunk ? (t_end - t0) : chunk);
    p.work_counter = uses_counter(opt.schedule) ? h->counters + counter_slot + c : nullptr;
    int l = 0;
    e = variants ? launch_fit_variants(p, opt.block, stream, &l)
                 : launch_fit(p, opt.precision, opt.block, opt.min_blocks, stream, &l);
    if (e != cudaSuccess) return cuda_fail(e, "fit launch");
    launches += l;
  }
  *launches_out = launches;
  return KF_SUCCESS;
}

// Everything that identifies a queued fit, for the graph cache.
struct GraphKey {
  kf_tracks tr;
  kf_surfaces su;
  kf_measurements me;
  kf_field fi;
  kf_options opt;
  kf_outputs out;
  kf_field_map map;  // the map the field points to (zero when none)
  void* stream;
  // the handle's buffers the graph's kernels point into
  const void* bufs[5];
};
static_assert(sizeof(GraphKey) <= 1024, "graph key storage");

// CTA sizes (in warps, 4..16) that split the ceil(n_tracks / 32) warp units
// of a batch into r nearly full waves of one CTA per SM, r = 1..4: a batch
// of a few waves loses less to a part-filled last wave than with the fixed
// CTA sizes. Writes up to 4 distinct values to w_out and returns how many.
int wave_filling_cta_warps(int64_t n_tracks, int nsm, int* w_out) {
  const int64_t U = (n_tracks + 31) / 32;
  int n = 0;
  for (int r = 1; r <= 4; ++r) {
    const int64_t w = (U + (int64_t)r * nsm - 1) / ((int64_t)r * nsm);
    if (w < 4 || w > 16) continue;
    if (n > 0 && w_out[n - 1] == (int)w) continue;
    w_out[n++] = (int)w;
  }
  return n;
}

GraphKey make_key(const kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me,
                  const kf_field* fi, const kf_options& opt, const kf_outputs* out, void* stream) {
  GraphKey k;
  memset(&k, 0, sizeof(k));  // padding bytes take part in the comparison
  k.tr = *tr;
  k.su = *su;
  k.me = *me;
  k.fi = *fi;
  k.opt = opt;
  k.out = *out;
  if (fi->map) k.map = *fi->map;
  k.stream = stream;
  k.bufs[0] = h->ws;
  k.bufs[1] = h->surf;
  k.bufs[2] = h->counters;
  k.bufs[3] = h->order;
  k.bufs[4] = h->hist;
  return k;
}

}  // namespace

extern "C" {

int kf_fit_ex(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me,
              const kf_field* fi, const kf_options* opt_in, const kf_outputs* out, void* stream_v) {
  if (!h) return KF_EINVAL;
  kf_options opt;
  if (opt_in) opt = *opt_in; else kf_default_options(&opt);
  int rc = validate(tr, su, me, fi, &opt, out);
  if (rc) return rc;
  h->last_launches = 0;
  if (tr->n_tracks == 0) return KF_SUCCESS;
  cudaStream_t stream = (cudaStream_t)stream_v;
  if (opt.schedule == KF_SCHEDULE_AUTO) {
    kf_options best;
    if ((rc = kf_autotune(h, tr, su, me, fi, &opt, out, stream_v, &best, nullptr))) return rc;
    opt.schedule = best.schedule;
    opt.block = best.block;
    opt.min_blocks = best.min_blocks;
    opt.resident_warps = best.resident_warps;
    opt.team_warps = best.team_warps;
  }
  FitPlan plan;
  if ((rc = prepare_fit(h, tr, su, opt, &plan))) return rc;
  if (!opt.use_graph) return enqueue_fit(h, tr, su, me, fi, opt, out, stream, plan, &h->last_launches);
  // CUDA graph: replay when every argument matches the captured call
  if (stream == nullptr) return KF_EUNSUPPORTED;  // the legacy stream cannot be captured
  GraphKey key = make_key(h, tr, su, me, fi, opt, out, stream_v);
  if (!h->graph_exec || memcmp(&key, h->graph_key, sizeof(key)) != 0) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    int launches = 0;
    rc = enqueue_fit(h, tr, su, me, fi, opt, out, stream, plan, &launches);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->graph_exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    memcpy(h->graph_key, &key, sizeof(key));
    h->graph_launches = launches;
  }
  cudaError_t e = cudaGraphLaunch(h->graph_exec, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  h->last_launches = h->graph_launches;
  return KF_SUCCESS;
}

int kf_autotune(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me,
                const kf_field* fi, const kf_options* base_in, const kf_outputs* out, void* stream_v,
                kf_options* best_out, double* best_ms) {
  if (!h || !best_out) return KF_EINVAL;
  kf_options base;
  if (base_in) base = *base_in; else kf_default_options(&base);
  base.schedule = KF_SCHEDULE_PERSISTENT;  // a valid placeholder for validation
  int rc = validate(tr, su, me, fi, &base, out);
  if (rc) return rc;
  const int bz = fi->b[0] == 0.0 && fi->b[1] == 0.0;
  const int variants = wants_variants(base.smoother, base.energy_loss, fi->map);
  for (int k = 0; k < h->n_tuned; ++k) {
    const kf_handle::Tuned& c = h->tuned[k];
    if (c.precision == base.precision && c.n_tracks == tr->n_tracks && c.max_states == tr->max_states &&
        c.n_surfaces == su->n_surfaces && c.bz == bz && c.variants == variants) {
      *best_out = base;
      best_out->schedule = c.best.schedule;
      best_out->block = c.best.block;
      best_out->min_blocks = c.best.min_blocks;
      best_out->resident_warps = c.best.resident_warps;
      best_out->team_warps = c.best.team_warps;
      if (best_ms) *best_ms = c.ms;
      return KF_SUCCESS;
    }
  }
  cudaStream_t stream = (cudaStream_t)stream_v;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    *best_out = base;  // no timing inside a capture: the default launch
    if (best_ms) *best_ms = -1.0;
    return KF_SUCCESS;
  }
  // candidate launch shapes: schedule x (threads per CTA, register variant).
  // Larger CTAs keep more warps in step (they start every unit together and
  // share instruction fetches), smaller ones leave a finer last wave on
  // small batches; then CTA sizes that split this batch into nearly full
  // waves, and the wave-split schedule for the large CTA sizes.
  const int schedules[3] = {KF_SCHEDULE_GRID, KF_SCHEDULE_PERSISTENT, KF_SCHEDULE_SORTED};
  const int shapes_fp64[4][2] = {{32, 0}, {64, 0}, {128, 0}, {256, 0}};
  const int shapes_mixed[11][2] = {{32, 0}, {64, 0}, {128, 0}, {256, 0}, {32, 3}, {64, 3},
                                   {128, 3}, {384, 3}, {128, 4}, {256, 4}, {512, 4}};
  const bool mixed = base.precision == KF_PRECISION_MIXED;
  const int n_shapes = mixed ? 11 : 4;
  kf_options cand[96];
  int n_cand = 0;
  for (int si = 0; si < 3; ++si)
    for (int bi = 0; bi < n_shapes; ++bi) {
      kf_options o = base;
      o.schedule = schedules[si];
      o.block = mixed ? shapes_mixed[bi][0] : shapes_fp64[bi][0];
      o.min_blocks = mixed ? shapes_mixed[bi][1] : shapes_fp64[bi][1];
      o.resident_warps = 0;
      o.team_warps = 0;
      o.use_graph = 0;
      cand[n_cand++] = o;
    }
  if (!mixed && !variants)
    for (int tw = 2; tw <= 4; tw += 2) {
      // each track shared by a team of warps (small batches)
      kf_options o = base;
      o.schedule = KF_SCHEDULE_GRID;
      o.block = 32 * tw;
      o.min_blocks = 0;
      o.resident_warps = 0;
      o.team_warps = tw;
      o.use_graph = 0;
      cand[n_cand++] = o;
    }
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0) {
      int ws[4];
      const int n_w = wave_filling_cta_warps(tr->n_tracks, nsm, ws);
      const int vars_mixed[3] = {0, 3, 4};
      for (int wi = 0; wi < n_w; ++wi)
        for (int si = 0; si < 2; ++si)
          for (int vi = 0; vi < (mixed ? 3 : 1); ++vi) {
            kf_options o = base;
            o.schedule = schedules[si];
            o.block = 32 * ws[wi];
            o.min_blocks = mixed ? vars_mixed[vi] : 0;
            if (o.block > max_block(mixed, o.min_blocks)) continue;
            o.resident_warps = 0;
            o.team_warps = 0;
            o.use_graph = 0;
            cand[n_cand++] = o;
          }
    }
  }
  {
    const int waves_fp64[3][2] = {{192, 0}, {224, 0}, {256, 0}};
    const int waves_mixed[7][2] = {{224, 0}, {256, 0}, {320, 3}, {352, 3}, {384, 3}, {448, 4}, {512, 4}};
    for (int bi = 0; bi < (mixed ? 7 : 3); ++bi) {
      kf_options o = base;
      o.schedule = KF_SCHEDULE_WAVES;
      o.block = mixed ? waves_mixed[bi][0] : waves_fp64[bi][0];
      o.min_blocks = mixed ? waves_mixed[bi][1] : waves_fp64[bi][1];
      o.resident_warps = 0;
      o.team_warps = 0;
      o.use_graph = 0;
      cand[n_cand++] = o;
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  }
  kf_options best = base;
  double best_t = 1e300;
  for (int ci = 0; ci < n_cand && rc == KF_SUCCESS; ++ci) {
    const kf_options& o = cand[ci];
    float times[3];
    for (int r = -1; r < 3 && rc == KF_SUCCESS; ++r) {  // one warm-up, three timed
      cudaEventRecord(e0, stream);
      rc = kf_fit_ex(h, tr, su, me, fi, &o, out, stream_v);
      cudaEventRecord(e1, stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) rc = cuda_fail(e, "autotune");
      if (r >= 0 && rc == KF_SUCCESS) cudaEventElapsedTime(&times[r], e0, e1);
    }
    if (rc) break;
    // median of three
    float a = times[0], b = times[1], c = times[2];
    const float med = a > b ? (b > c ? b : (a > c ? c : a)) : (a > c ? a : (b > c ? c : b));
    if (med < best_t) {
      best_t = med;
      best = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  best.use_graph = base_in ? base_in->use_graph : 0;
  kf_handle::Tuned& slot = h->tuned[h->n_tuned < 16 ? h->n_tuned++ : 15];
  slot.precision = base.precision;
  slot.n_tracks = tr->n_tracks;
  slot.max_states = tr->max_states;
  slot.n_surfaces = su->n_surfaces;
  slot.bz = bz;
  slot.variants = variants;
  slot.best = best;
  slot.ms = best_t;
  *best_out = best;
  if (best_ms) *best_ms = best_t;
  return KF_SUCCESS;
}

int kf_grad(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const double* align,
            const kf_measurements* me, const kf_field* fi, const kf_options* opt_in, const kf_grad_weights* wts,
            const kf_grad_outputs* go, void* stream_v) {
  if (!h || !go) return KF_EINVAL;
  kf_options opt;
  if (opt_in) {
    opt = *opt_in;
  } else {
    kf_default_options(&opt);
    opt.block = 0;  // the adjoint's own CTA size choice
  }
  opt.precision = KF_PRECISION_FP64;
  opt.schedule = KF_SCHEDULE_GRID;
  // the adjoint has its own register variants (up to 256 / 384 / 512
  // threads per CTA for min_blocks 1 / 3 / 4)
  const int grad_block = opt.block;
  if (grad_block < 0 || grad_block % 32 != 0 || grad_block > max_threads_of(opt.min_blocks)) return KF_EUNSUPPORTED;
  // team_warps 2: the pipelined form (two warps per 32 tracks); 1: one
  // thread per track; 0: the pipelined form while its two-warp teams fit in
  // one warp per SM sub-partition (a batch too small to fill the GPU)
  if (opt.team_warps != 0 && opt.team_warps != 1 && opt.team_warps != 2) return KF_EUNSUPPORTED;
  bool pipelined = opt.team_warps == 2;
  if (opt.team_warps == 0) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      pipelined = 2 * (((int64_t)tr->n_tracks + 31) / 32) <= 4 * (int64_t)nsm;
  }
  opt.team_warps = 0;
  opt.block = 0;
  kf_outputs dummy;
  memset(&dummy, 0, sizeof(dummy));
  double one = 0.0;  // non-null placeholders for the output checks of validate()
  dummy.params = dummy.cov = dummy.chi2 = &one;
  int rc = validate(tr, su, me, fi, &opt, &dummy);
  if (rc) return rc;
  // the adjoint differentiates the baseline method only
  if (wants_variants(opt.smoother, opt.energy_loss, fi->map)) return KF_EUNSUPPORTED;
  GradArgs a;
  memset(&a, 0, sizeof(a));
  a.align = align;
  if (wts) {
    a.dl_dchi2 = wts->dl_dchi2;
    a.dl_dparams = wts->dl_dparams;
    a.dl_dcov = wts->dl_dcov;
  }
  a.chi2 = go->chi2;
  a.params = go->params;
  a.cov = go->cov;
  a.grad_seed = go->grad_seed;
  a.grad_align = go->grad_align;
  cudaStream_t stream = (cudaStream_t)stream_v;
  if (a.grad_align) {
    cudaError_t e = cudaMemsetAsync(a.grad_align, 0, sizeof(double) * 6 * (size_t)su->n_surfaces, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(grad_align)");
  }
  h->last_launches = 0;
  if (tr->n_tracks == 0) return KF_SUCCESS;
  // scratch per track; batches whose scratch exceeds the workspace cap run
  // as several launches over consecutive track ranges
  const bool want = a.grad_seed || a.grad_align;
  const bool sm_adj = want && (a.dl_dparams || a.dl_dcov);
  const bool sm = sm_adj || a.params || a.cov;
  const size_t per_track = sizeof(double) * grad_scratch_doubles(tr->max_states, sm, sm_adj, pipelined);
  const int64_t cap = opt.workspace_bytes > 0 ? opt.workspace_bytes : kDefaultWorkspace;
  int64_t chunk = cap / (int64_t)per_track;
  if (chunk < 1) chunk = 1;
  if (chunk > tr->n_tracks) chunk = tr->n_tracks;
  // the alignment angles' cosines and sines ([6][S]) ahead of the tracks' scratch
  const size_t trig_bytes = align_up(sizeof(double) * 6 * (size_t)su->n_surfaces, 256);
  const size_t need = trig_bytes + per_track * (size_t)chunk;
  if (h->ckpt_bytes < need) {
    if (h->ckpt) cudaFree(h->ckpt);
    h->ckpt = nullptr;
    h->ckpt_bytes = 0;
    cudaError_t e = cudaMalloc(&h->ckpt, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(adjoint scratch)");
    h->ckpt_bytes = need;
  }
  if ((rc = ensure_surf(h, su->n_surfaces))) return rc;
  cudaError_t e = cudaMemsetAsync(h->error_flag, 0, sizeof(int32_t), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(error flag)");
  e = launch_pack_surfaces(su->n_surfaces, su->center, su->rot, su->x_over_x0, h->surf, stream);
  if (e != cudaSuccess) return cuda_fail(e, "pack_surfaces launch");
  int launches = 1;
  if (align) {
    a.align_cs = (const double*)h->ckpt;
    e = launch_align_trig(su->n_surfaces, align, (double*)h->ckpt, stream);
    if (e != cudaSuccess) return cuda_fail(e, "align trig launch");
    ++launches;
  }
  FitParams p;
  memset(&p, 0, sizeof(p));
  p.n_tracks_total = tr->n_tracks;
  p.max_states = tr->max_states;
  p.offsets = tr->offsets;
  p.seed_params = tr->seed_params;
  p.seed_cov = tr->seed_cov;
  p.n_surfaces = su->n_surfaces;
  p.surf = h->surf;
  p.n_states = me->n_states;
  p.surface_id = me->surface_id;
  p.loc = me->loc;
  p.cov = me->cov;
  p.is_hole = me->is_hole;
  for (int i = 0; i < 3; ++i) p.bfield[i] = fi->b[i];
  p.mass = opt.mass;
  p.h_max = opt.h_max;
  p.n_iter = opt.n_iter;
  p.error_flag = h->error_flag;
  p.wait_limit = opt.wait_limit;
  p.skip_stage_copy = opt.test_wait_timeout;
  for (int64_t t0 = 0; t0 < tr->n_tracks; t0 += chunk) {
    p.track0 = (int32_t)t0;
    p.n_tracks = (int32_t)((tr->n_tracks - t0) < chunk ? (tr->n_tracks - t0) : chunk);
    e = launch_grad(p, a, (double*)((char*)h->ckpt + trig_bytes), grad_block, opt.min_blocks, pipelined, stream);
    if (e != cudaSuccess) return cuda_fail(e, "grad launch");
    ++launches;
  }
  h->last_launches = launches;
  return KF_SUCCESS;
}

int kf_chi2_grad(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const double* align,
                 const kf_measurements* me, const kf_field* fi, const kf_options* opt_in, const double* dl_dchi2,
                 double* out_chi2, double* grad_seed, double* grad_align, void* stream_v) {
  kf_grad_weights w;
  memset(&w, 0, sizeof(w));
  w.dl_dchi2 = dl_dchi2;
  kf_grad_outputs o;
  memset(&o, 0, sizeof(o));
  o.chi2 = out_chi2;
  o.grad_seed = grad_seed;
  o.grad_align = grad_align;
  return kf_grad(h, tr, su, align, me, fi, opt_in, &w, &o, stream_v);
}

int kf_fit(const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me, const kf_field* fi,
           double* out_params, double* out_cov, double* out_chi2) {
  static std::mutex mu;
  static kf_handle* handles[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return KF_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (!handles[dev]) {
    int rc = kf_create(&handles[dev]);
    if (rc) return rc;
  }
  kf_outputs out;
  memset(&out, 0, sizeof(out));
  out.params = out_params;
  out.cov = out_cov;
  out.chi2 = out_chi2;
  int rc = kf_fit_ex(handles[dev], tr, su, me, fi, nullptr, &out, nullptr);
  if (rc) return rc;
  e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return KF_SUCCESS;
}

// streams and events of the pipelined host path, created on first use
static int ensure_host_streams(kf_handle* h) {
  if (h->ev_pack) return KF_SUCCESS;
  cudaError_t e = cudaSuccess;
  if (!h->s_in) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !h->s_out) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  for (int i = 0; i < kf_handle::kPipe - 1 && e == cudaSuccess; ++i)
    if (!h->s_fit[i]) e = cudaStreamCreateWithFlags(&h->s_fit[i], cudaStreamNonBlocking);
  for (int i = 0; i < kf_handle::kPipe && e == cudaSuccess; ++i) {
    if (!h->ev_in[i]) e = cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess && !h->ev_fit[i]) e = cudaEventCreateWithFlags(&h->ev_fit[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pack, cudaEventDisableTiming);
  return e == cudaSuccess ? KF_SUCCESS : cuda_fail(e, "host-path streams");
}

// copy columns [c0, c1) of a row-major [rows][ncol] array of `elem`-byte
// elements between host and device (same layout on both sides)
static cudaError_t copy_cols(void* dst, const void* src, size_t ncol, size_t elem, size_t rows, size_t c0,
                             size_t c1, cudaMemcpyKind kind, cudaStream_t s) {
  if (c1 <= c0 || rows == 0) return cudaSuccess;
  const size_t pitch = ncol * elem, off = c0 * elem;
  return cudaMemcpy2DAsync((char*)dst + off, pitch, (const char*)src + off, pitch, (c1 - c0) * elem, rows, kind, s);
}

int kf_fit_host(kf_handle* h, const kf_tracks* tr, const kf_surfaces* su, const kf_measurements* me,
                const kf_field* fi, const kf_options* opt, const kf_outputs* out, void* stream_v) {
  if (!h || !tr || !su || !me || !fi || !out) return KF_EINVAL;
  if (tr->n_tracks < 0 || me->n_states < 0 || su->n_surfaces < 1) return KF_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_v;
  const size_t T = (size_t)tr->n_tracks, S = (size_t)su->n_surfaces, M = (size_t)me->n_states;
  // device layout of the copies, 256-byte aligned pieces
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_off = take((T + 1) * 4), o_sp = take(6 * T * 8), o_sc = take(21 * T * 8);
  const size_t o_c = take(3 * S * 8), o_r = take(9 * S * 8), o_x = take(S * 8);
  const size_t o_sid = take(M * 4), o_loc = take(2 * M * 8), o_cov = take(3 * M * 8), o_h = take(M);
  const size_t o_p = take(6 * T * 8), o_pc = take(21 * T * 8), o_chi = take(T * 8), o_ndf = take(T * 4),
               o_st = take(T), o_states = take(out->states ? 6 * M * 8 : 0);
  size_t map_bytes = 0;
  if (fi->map) {
    const kf_field_map& f = *fi->map;
    if (f.nx < 2 || f.ny < 2 || f.nz < 2 || !f.b) return KF_EINVAL;
    map_bytes = (size_t)f.nx * (size_t)f.ny * (size_t)f.nz * 3 * sizeof(double);
  }
  const size_t o_map = take(map_bytes);
  if (h->dev_io_bytes < off) {
    if (h->dev_io) cudaFree(h->dev_io);
    h->dev_io = nullptr;
    h->dev_io_bytes = 0;
    cudaError_t e = cudaMalloc(&h->dev_io, off);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(io)");
    h->dev_io_bytes = off;
  }
  char* b = (char*)h->dev_io;
  kf_tracks dtr = *tr;
  dtr.offsets = (const int32_t*)(b + o_off);
  dtr.seed_params = (const double*)(b + o_sp);
  dtr.seed_cov = (const double*)(b + o_sc);
  kf_surfaces dsu = *su;
  dsu.center = (const double*)(b + o_c);
  dsu.rot = (const double*)(b + o_r);
  dsu.x_over_x0 = (const double*)(b + o_x);
  kf_measurements dme = *me;
  dme.surface_id = (const int32_t*)(b + o_sid);
  dme.loc = (const double*)(b + o_loc);
  dme.cov = (const double*)(b + o_cov);
  dme.is_hole = (const uint8_t*)(b + o_h);
  kf_outputs dout;
  dout.params = (double*)(b + o_p);
  dout.cov = (double*)(b + o_pc);
  dout.chi2 = (double*)(b + o_chi);
  dout.ndf = (int32_t*)(b + o_ndf);
  dout.status = (uint8_t*)(b + o_st);
  dout.states = out->states ? (double*)(b + o_states) : nullptr;
  kf_field dfi = *fi;
  kf_field_map dmap;
  if (fi->map) {
    dmap = *fi->map;
    dmap.b = (const double*)(b + o_map);
    dfi.map = &dmap;
  }
  kf_options o;
  if (opt) o = *opt; else kf_default_options(&o);
  struct Cp { size_t o; const void* src; size_t bytes; };
  // Large batches run as 2 to 8 chunks of at least 12.5k tracks: each
  // chunk's fit starts as soon as its inputs have arrived, on a stream of
  // its own (the caller's for chunk 0), so the fits of earlier chunks run
  // while later chunks' inputs travel and the CTAs of all of them share the
  // SMs; each chunk's outputs travel once its fit is done. (Not for a
  // schedule still to be tuned, a graph, or a small batch.)
  const bool pipelined = T >= 20000 && o.schedule != KF_SCHEDULE_AUTO && !o.use_graph && tr->offsets && out->params;
  if (!pipelined) {
    const Cp in[] = {{o_off, tr->offsets, (T + 1) * 4}, {o_sp, tr->seed_params, 6 * T * 8},
                     {o_sc, tr->seed_cov, 21 * T * 8},   {o_c, su->center, 3 * S * 8},
                     {o_r, su->rot, 9 * S * 8},          {o_x, su->x_over_x0, S * 8},
                     {o_sid, me->surface_id, M * 4},     {o_loc, me->loc, 2 * M * 8},
                     {o_cov, me->cov, 3 * M * 8},        {o_h, me->is_hole, M},
                     {o_map, fi->map ? fi->map->b : nullptr, map_bytes}};
    for (const Cp& c : in) {
      if (c.bytes == 0) continue;
      if (!c.src) return KF_EINVAL;
      cudaError_t e = cudaMemcpyAsync(b + c.o, c.src, c.bytes, cudaMemcpyHostToDevice, stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
    }
    int rc = kf_fit_ex(h, &dtr, &dsu, &dme, &dfi, opt, &dout, stream_v);
    if (rc) return rc;
    const Cp outs[] = {{o_p, out->params, 6 * T * 8}, {o_pc, out->cov, 21 * T * 8}, {o_chi, out->chi2, T * 8},
                       {o_ndf, out->ndf, T * 4},      {o_st, out->status, T},     {o_states, out->states, 6 * M * 8}};
    for (const Cp& c : outs) {
      if (!c.src || c.bytes == 0) continue;
      cudaError_t e = cudaMemcpyAsync((void*)c.src, b + c.o, c.bytes, cudaMemcpyDeviceToHost, stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
    }
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  } else {
    if (!tr->seed_params || !tr->seed_cov || !su->center || !su->rot || !su->x_over_x0 || !out->cov || !out->chi2)
      return KF_EINVAL;
    if (M > 0 && (!me->surface_id || !me->loc || !me->cov || !me->is_hole)) return KF_EINVAL;
    int rc = validate(&dtr, &dsu, &dme, &dfi, &o, &dout);
    if (rc) return rc;
    if ((rc = ensure_host_streams(h))) return rc;
    FitPlan plan;
    if ((rc = prepare_fit(h, &dtr, &dsu, o, &plan))) return rc;
    const int nch = (int)(T / 12500 < 2 ? 2 : (T / 12500 > (size_t)kf_handle::kPipe ? kf_handle::kPipe : T / 12500));
    // concurrent fits need their own workspace slices and work counters
    const bool concurrent = plan.n_chunks == 1;
    if (concurrent) {
      // the chunks' fits share the SMs, so no launch needs to fill them on
      // its own: plain grid launches of at most 128-thread CTAs pack them
      // best (measured on 100k tracks in 8 chunks: 2.16 ms end to end with
      // 128 threads, 2.22-2.33 ms with 224-384, 2.61 ms with 512)
      if (o.schedule == KF_SCHEDULE_WAVES) o.schedule = KF_SCHEDULE_GRID;
      if (o.block > 128) o.block = 128;
    }
    if (concurrent && uses_counter(o.schedule) && h->counters_cap < kf_handle::kPipe) {
      if (h->counters) cudaFree(h->counters);
      h->counters = nullptr;
      h->counters_cap = 0;
      cudaError_t ea = cudaMalloc(&h->counters, sizeof(int32_t) * kf_handle::kPipe);
      if (ea != cudaSuccess) return cuda_fail(ea, "cudaMalloc(counters)");
      h->counters_cap = kf_handle::kPipe;
    }
    size_t tcut[kf_handle::kPipe + 1], scut[kf_handle::kPipe + 1];
    for (int c = 0; c <= nch; ++c) {
      tcut[c] = T * (size_t)c / (size_t)nch;
      const int32_t v = tr->offsets[tcut[c]];
      if (v < 0 || (size_t)v > M) return KF_EINVAL;
      scut[c] = (size_t)v;
    }
    cudaError_t e = cudaSuccess;
    auto H2D = cudaMemcpyHostToDevice;
    auto D2H = cudaMemcpyDeviceToHost;
    int launches = 0;
    // Chunk by chunk, everything a chunk needs is queued before the next
    // chunk's copies, so the first fit is queued after a few calls: its
    // inputs (with the shared pieces ahead of chunk 0) on the copy stream,
    // its fit on its own stream once they are in, its outputs on the output
    // stream once the fit is done.
    for (int c = 0; c < nch; ++c) {
      const size_t t0 = tcut[c], t1 = tcut[c + 1], s0 = scut[c], s1 = scut[c + 1];
      cudaStream_t si = h->s_in;
      if (c == 0) {
        e = cudaMemcpyAsync(b + o_off, tr->offsets, (T + 1) * 4, H2D, si);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_c, su->center, 3 * S * 8, H2D, si);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_r, su->rot, 9 * S * 8, H2D, si);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_x, su->x_over_x0, S * 8, H2D, si);
        if (e == cudaSuccess && map_bytes) e = cudaMemcpyAsync(b + o_map, fi->map->b, map_bytes, H2D, si);
      }
      if (e == cudaSuccess) e = copy_cols(b + o_sp, tr->seed_params, T, 8, 6, t0, t1, H2D, si);
      if (e == cudaSuccess) e = copy_cols(b + o_sc, tr->seed_cov, T, 8, 21, t0, t1, H2D, si);
      if (e == cudaSuccess) e = copy_cols(b + o_sid, me->surface_id, M, 4, 1, s0, s1, H2D, si);
      if (e == cudaSuccess) e = copy_cols(b + o_loc, me->loc, M, 8, 2, s0, s1, H2D, si);
      if (e == cudaSuccess) e = copy_cols(b + o_cov, me->cov, M, 8, 3, s0, s1, H2D, si);
      if (e == cudaSuccess) e = copy_cols(b + o_h, me->is_hole, M, 1, 1, s0, s1, H2D, si);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[c], si);
      if (e != cudaSuccess) return cuda_fail(e, "host-path H2D");
      if (c == 0) {
        // the surface table (in chunk 0's copies) is packed once and the
        // work counters reset once, before any fit
        e = cudaStreamWaitEvent(stream, h->ev_in[0], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->error_flag, 0, sizeof(int32_t), stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        e = launch_pack_surfaces(dsu.n_surfaces, dsu.center, dsu.rot, dsu.x_over_x0, h->surf, stream);
        if (e != cudaSuccess) return cuda_fail(e, "pack_surfaces launch");
        launches = 1;
        if (concurrent && uses_counter(o.schedule)) {
          e = cudaMemsetAsync(h->counters, 0, sizeof(int32_t) * kf_handle::kPipe, stream);
          if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
        }
        e = cudaEventRecord(h->ev_pack, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
      }
      cudaStream_t fs = concurrent && c > 0 ? h->s_fit[c - 1] : stream;
      e = cudaStreamWaitEvent(fs, h->ev_in[c], 0);
      if (e == cudaSuccess && fs != stream) e = cudaStreamWaitEvent(fs, h->ev_pack, 0);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
      int l = 0;
      rc = enqueue_fit(h, &dtr, &dsu, &dme, &dfi, o, &dout, fs, plan, &l, (int64_t)t0, (int64_t)t1, false,
                       concurrent, concurrent ? c : 0);
      if (rc) return rc;
      launches += l;
      e = cudaEventRecord(h->ev_fit[c], fs);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
      cudaStream_t so = h->s_out;
      e = cudaStreamWaitEvent(so, h->ev_fit[c], 0);
      if (e == cudaSuccess) e = copy_cols(out->params, b + o_p, T, 8, 6, t0, t1, D2H, so);
      if (e == cudaSuccess) e = copy_cols(out->cov, b + o_pc, T, 8, 21, t0, t1, D2H, so);
      if (e == cudaSuccess) e = copy_cols(out->chi2, b + o_chi, T, 8, 1, t0, t1, D2H, so);
      if (e == cudaSuccess && out->ndf) e = copy_cols(out->ndf, b + o_ndf, T, 4, 1, t0, t1, D2H, so);
      if (e == cudaSuccess && out->status) e = copy_cols(out->status, b + o_st, T, 1, 1, t0, t1, D2H, so);
      if (e == cudaSuccess && out->states) e = copy_cols(out->states, b + o_states, M, 8, 6, s0, s1, D2H, so);
      if (e != cudaSuccess) break;
    }
    h->last_launches = launches;
    if (e != cudaSuccess) return cuda_fail(e, "host-path D2H");
    // the fit streams are done once the last output copy (which waited for
    // every fit) is
    e = cudaStreamSynchronize(h->s_out);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  }
  int32_t flag = 0;
  cudaError_t e = cudaMemcpy(&flag, h->error_flag, sizeof(flag), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(error flag)");
  if (flag) return KF_EDEVICE;
  return KF_SUCCESS;
}

}  // extern "C"
