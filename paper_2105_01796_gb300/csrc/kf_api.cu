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
  // device copies for kf_fit_host
  void* dev_io = nullptr;
  size_t dev_io_bytes = 0;
  int32_t last_launches = 0;
};

namespace {

thread_local char g_cuda_err[256] = "no CUDA error";

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? KF_ENOMEM : KF_ECUDA;
}

constexpr double kMuonMass = 0.1056583755;
constexpr int64_t kDefaultWorkspace = int64_t(4) << 30;

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
  cudaError_t e = cudaMalloc(&h->surf, (size_t)n * kSurfStride * sizeof(double));
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
  if (opt->block < 0 || opt->block > 128 || (opt->block % 32) != 0) return KF_EUNSUPPORTED;
  if (opt->schedule < KF_SCHEDULE_GRID || opt->schedule > KF_SCHEDULE_SORTED) return KF_EUNSUPPORTED;
  if (opt->min_blocks < 0 || opt->min_blocks > 4) return KF_EUNSUPPORTED;
  for (int i = 0; i < 3; ++i)
    if (!(fi->b[i] == fi->b[i])) return KF_EINVAL;
  return KF_SUCCESS;
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
}

int kf_abi_version(void) { return KF_ABI_VERSION; }

int kf_selftest(int64_t n_patterns, uint64_t* counts) {
  if (!counts || n_patterns < 0) return KF_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 5 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(selftest)");
  e = cudaMemset(d, 0, 5 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_selftest(n_patterns, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(counts, d, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "selftest");
  return KF_SUCCESS;
}

const char* kf_strerror(int code) {
  switch (code) {
    case KF_SUCCESS: return "success";
    case KF_EINVAL: return "invalid argument";
    case KF_ECUDA: return "CUDA error (see kf_last_cuda_error)";
    case KF_ENOMEM: return "out of memory";
    case KF_EUNSUPPORTED: return "unsupported option";
    case KF_EDEVICE: return "device-side wait timed out";
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
  const int64_t chunk = chunk_tracks(tr->n_tracks, tr->max_states, opt);
  const size_t n64 = opt.precision == KF_PRECISION_FP64 ? kRec64Fp64 : kRec64Mixed;
  const size_t bytes64 = align_up(n64 * sizeof(double) * tr->max_states * chunk, 256);
  const size_t bytes32 =
      opt.precision == KF_PRECISION_FP64 ? 0 : align_up(kRec32Mixed * sizeof(float) * tr->max_states * chunk, 256);
  if ((rc = ensure_ws(h, bytes64 + bytes32))) return rc;
  if ((rc = ensure_surf(h, su->n_surfaces))) return rc;
  const int n_chunks = (int)((tr->n_tracks + chunk - 1) / chunk);
  if (opt.schedule != KF_SCHEDULE_GRID && h->counters_cap < n_chunks) {
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
  cudaError_t e = launch_pack_surfaces(su->n_surfaces, su->center, su->rot, su->x_over_x0, h->surf, stream);
  if (e != cudaSuccess) return cuda_fail(e, "pack_surfaces launch");
  int launches = 1;
  if (opt.schedule != KF_SCHEDULE_GRID) {
    e = cudaMemsetAsync(h->counters, 0, sizeof(int32_t) * n_chunks, stream);
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
  p.ws32 = opt.precision == KF_PRECISION_FP64 ? nullptr : (float*)((char*)h->ws + bytes64);
  p.error_flag = h->error_flag;
  p.order = opt.schedule == KF_SCHEDULE_SORTED ? h->order : nullptr;
  int c = 0;
  for (int64_t t0 = 0; t0 < tr->n_tracks; t0 += chunk, ++c) {
    p.track0 = (int32_t)t0;
    p.n_tracks = (int32_t)((tr->n_tracks - t0) < chunk ? (tr->n_tracks - t0) : chunk);
    p.work_counter = opt.schedule == KF_SCHEDULE_GRID ? nullptr : h->counters + c;
    e = launch_fit(p, opt.precision, opt.block, opt.min_blocks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "fit launch");
    ++launches;
  }
  h->last_launches = launches;
  return KF_SUCCESS;
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
  if (h->dev_io_bytes < off) {
    if (h->dev_io) cudaFree(h->dev_io);
    h->dev_io = nullptr;
    h->dev_io_bytes = 0;
    cudaError_t e = cudaMalloc(&h->dev_io, off);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(io)");
    h->dev_io_bytes = off;
  }
  char* b = (char*)h->dev_io;
  struct Cp { size_t o; const void* src; size_t bytes; };
  const Cp in[] = {{o_off, tr->offsets, (T + 1) * 4}, {o_sp, tr->seed_params, 6 * T * 8},
                   {o_sc, tr->seed_cov, 21 * T * 8},   {o_c, su->center, 3 * S * 8},
                   {o_r, su->rot, 9 * S * 8},          {o_x, su->x_over_x0, S * 8},
                   {o_sid, me->surface_id, M * 4},     {o_loc, me->loc, 2 * M * 8},
                   {o_cov, me->cov, 3 * M * 8},        {o_h, me->is_hole, M}};
  for (const Cp& c : in) {
    if (c.bytes == 0) continue;
    if (!c.src) return KF_EINVAL;
    cudaError_t e = cudaMemcpyAsync(b + c.o, c.src, c.bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
  }
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
  int rc = kf_fit_ex(h, &dtr, &dsu, &dme, fi, opt, &dout, stream_v);
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
  int32_t flag = 0;
  e = cudaMemcpy(&flag, h->error_flag, sizeof(flag), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(error flag)");
  if (flag) return KF_EDEVICE;
  return KF_SUCCESS;
}

}  // extern "C"
