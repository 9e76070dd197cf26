"""GB300 (sm_103a) Kalman-filter track fitter -- Python binding of libkfgb.so.

A thin ctypes layer over the C ABI in ``include/kf.h``: it marshals pointers
and sizes and nothing else.  Every step of the fit runs in the library's CUDA
kernels; there is no CPU fallback.  If ``libkfgb.so`` has not been built the
calls raise instead of computing anything.

Names follow the C ABI: :func:`kf_fit`, :func:`kf_fit_ex`, :func:`kf_fit_host`,
:func:`kf_create`, :func:`kf_destroy`, :func:`kf_workspace_size`.
Device inputs are torch CUDA tensors (torch supplies device memory and the
stream); host inputs of :func:`kf_fit_host` are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkfgb.so")

KF_PRECISION_FP64 = 0
KF_PRECISION_MIXED = 1
KF_SCHEDULE_AUTO, KF_SCHEDULE_GRID, KF_SCHEDULE_PERSISTENT, KF_SCHEDULE_SORTED, KF_SCHEDULE_WAVES = -1, 0, 1, 2, 3
KF_SMOOTHER_RTS, KF_SMOOTHER_BACKWARD_FILTER = 0, 1
TRACK_STATUS = {0: "ok", 1: "no_intersection", 2: "non_spd", 3: "nonfinite", 4: "bad_input", 5: "timeout"}
MUON_MASS = 0.1056583755

# exported symbols of include/kf.h
EXPORTS = ("kf_default_options", "kf_create", "kf_destroy", "kf_fit", "kf_fit_ex",
           "kf_fit_host", "kf_workspace_size", "kf_last_launch_count", "kf_strerror",
           "kf_last_cuda_error", "kf_abi_version", "kf_selftest", "kf_selftest_df", "kf_fit_static",
           "kf_autotune", "kf_chi2_grad", "kf_grad")


class KfTracks(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_int32), ("max_states", ctypes.c_int32),
                ("offsets", ctypes.c_void_p), ("seed_params", ctypes.c_void_p),
                ("seed_cov", ctypes.c_void_p)]


class KfSurfaces(ctypes.Structure):
    _fields_ = [("n_surfaces", ctypes.c_int32), ("center", ctypes.c_void_p),
                ("rot", ctypes.c_void_p), ("x_over_x0", ctypes.c_void_p)]


class KfMeasurements(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_int64), ("surface_id", ctypes.c_void_p),
                ("loc", ctypes.c_void_p), ("cov", ctypes.c_void_p),
                ("is_hole", ctypes.c_void_p)]


class KfFieldMap(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("origin", ctypes.c_double * 3),
                ("spacing", ctypes.c_double * 3), ("b", ctypes.c_void_p)]


class KfField(ctypes.Structure):
    _fields_ = [("b", ctypes.c_double * 3), ("map", ctypes.c_void_p)]


class KfMaterial(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("z_over_a", "i_exc", "x0_rho", "sh_cbar", "sh_x0",
                                                 "sh_x1", "sh_a", "sh_k", "sh_delta0")]


class KfOutputs(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("cov", ctypes.c_void_p),
                ("chi2", ctypes.c_void_p), ("ndf", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("states", ctypes.c_void_p)]


class KfGradWeights(ctypes.Structure):
    _fields_ = [("dl_dchi2", ctypes.c_void_p), ("dl_dparams", ctypes.c_void_p),
                ("dl_dcov", ctypes.c_void_p)]


class KfGradOutputs(ctypes.Structure):
    _fields_ = [("chi2", ctypes.c_void_p), ("params", ctypes.c_void_p), ("cov", ctypes.c_void_p),
                ("grad_seed", ctypes.c_void_p), ("grad_align", ctypes.c_void_p)]


class KfOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("mass", ctypes.c_double),
                ("h_max", ctypes.c_double), ("n_iter", ctypes.c_int32),
                ("block", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("schedule", ctypes.c_int32), ("min_blocks", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("smoother", ctypes.c_int32),
                ("energy_loss", ctypes.c_int32), ("bf_scale", ctypes.c_double),
                ("material", KfMaterial), ("resident_warps", ctypes.c_int32),
                ("wait_limit", ctypes.c_int32), ("team_warps", ctypes.c_int32),
                ("test_wait_timeout", ctypes.c_int32)]


_lib = None


class KfError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Load libkfgb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise KfError("libkfgb.so is not built (run __graft_entry__.build()); "
                          "there is no CPU fallback")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.kf_default_options.argtypes = [ctypes.POINTER(KfOptions)]
        lib.kf_default_options.restype = None
        lib.kf_create.argtypes = [ctypes.POINTER(P)]
        lib.kf_create.restype = ctypes.c_int
        lib.kf_destroy.argtypes = [P]
        lib.kf_destroy.restype = None
        base = [ctypes.POINTER(KfTracks), ctypes.POINTER(KfSurfaces),
                ctypes.POINTER(KfMeasurements), ctypes.POINTER(KfField)]
        lib.kf_fit.argtypes = base + [P, P, P]
        lib.kf_fit.restype = ctypes.c_int
        lib.kf_fit_ex.argtypes = [P] + base + [ctypes.POINTER(KfOptions), ctypes.POINTER(KfOutputs), P]
        lib.kf_fit_ex.restype = ctypes.c_int
        lib.kf_fit_host.argtypes = lib.kf_fit_ex.argtypes
        lib.kf_fit_host.restype = ctypes.c_int
        lib.kf_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(KfOptions)]
        lib.kf_workspace_size.restype = ctypes.c_int64
        lib.kf_last_launch_count.argtypes = [P]
        lib.kf_last_launch_count.restype = ctypes.c_int32
        lib.kf_strerror.argtypes = [ctypes.c_int]
        lib.kf_strerror.restype = ctypes.c_char_p
        lib.kf_last_cuda_error.argtypes = []
        lib.kf_last_cuda_error.restype = ctypes.c_char_p
        lib.kf_abi_version.argtypes = []
        lib.kf_abi_version.restype = ctypes.c_int
        lib.kf_chi2_grad.argtypes = [P, ctypes.POINTER(KfTracks), ctypes.POINTER(KfSurfaces), P,
                                     ctypes.POINTER(KfMeasurements), ctypes.POINTER(KfField),
                                     ctypes.POINTER(KfOptions), P, P, P, P, P]
        lib.kf_chi2_grad.restype = ctypes.c_int
        lib.kf_grad.argtypes = [P, ctypes.POINTER(KfTracks), ctypes.POINTER(KfSurfaces), P,
                                ctypes.POINTER(KfMeasurements), ctypes.POINTER(KfField),
                                ctypes.POINTER(KfOptions), ctypes.POINTER(KfGradWeights),
                                ctypes.POINTER(KfGradOutputs), P]
        lib.kf_grad.restype = ctypes.c_int
        lib.kf_autotune.argtypes = [P] + base + [ctypes.POINTER(KfOptions), ctypes.POINTER(KfOutputs), P,
                                                 ctypes.POINTER(KfOptions), ctypes.POINTER(ctypes.c_double)]
        lib.kf_autotune.restype = ctypes.c_int
        lib.kf_fit_static.argtypes = base + [ctypes.POINTER(KfOptions), ctypes.POINTER(KfOutputs), P]
        lib.kf_fit_static.restype = ctypes.c_int
        lib.kf_selftest.argtypes = [ctypes.c_int64, ctypes.c_void_p]
        lib.kf_selftest.restype = ctypes.c_int
        lib.kf_selftest_df.argtypes = [ctypes.c_int64, ctypes.c_void_p]
        lib.kf_selftest_df.restype = ctypes.c_int
        _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        lib = load()
        msg = lib.kf_strerror(rc).decode()
        if rc == -2:
            msg += ": " + lib.kf_last_cuda_error().decode()
        raise KfError("kf error %d (%s)" % (rc, msg))


def kf_default_options(precision=KF_PRECISION_FP64, **kw) -> KfOptions:
    o = KfOptions()
    load().kf_default_options(ctypes.byref(o))
    o.precision = int(precision)
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


class Handle:
    """Owns a kf_handle (workspace + staging buffers on the current device)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().kf_create(ctypes.byref(h)))
        self.ptr = h

    def close(self):
        if self.ptr:
            load().kf_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_launch_count(self) -> int:
        return int(load().kf_last_launch_count(self.ptr))


def kf_create() -> Handle:
    return Handle()


def kf_destroy(h: Handle) -> None:
    h.close()


def kf_workspace_size(n_tracks, max_states, opt=None) -> int:
    return int(load().kf_workspace_size(int(n_tracks), int(max_states),
                                        ctypes.byref(opt) if opt is not None else None))


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _structs(ev, max_states):
    tr = KfTracks(int(ev["n_tracks"]), int(max_states), _ptr(ev["offsets"]),
                  _ptr(ev["seed_params"]), _ptr(ev["seed_cov"]))
    su = KfSurfaces(int(ev["center"].shape[1]), _ptr(ev["center"]), _ptr(ev["rot"]),
                    _ptr(ev["x_over_x0"]))
    me = KfMeasurements(int(ev["surface_id"].shape[0]), _ptr(ev["surface_id"]),
                        _ptr(ev["loc"]), _ptr(ev["cov"]), _ptr(ev["is_hole"]))
    fi = KfField((ctypes.c_double * 3)(*[float(b) for b in ev["bfield"]]), None)
    fm = ev.get("field_map")
    if fm is not None:
        b = fm["b"]
        nz, ny, nx = (int(v) for v in b.shape[:3])
        m = KfFieldMap(nx, ny, nz, 0, (ctypes.c_double * 3)(*[float(v) for v in fm["origin"]]),
                       (ctypes.c_double * 3)(*[float(v) for v in fm["spacing"]]), _ptr(b))
        fi.map = ctypes.cast(ctypes.pointer(m), ctypes.c_void_p)
        fi._map = m  # keeps the map struct alive with the field
    return tr, su, me, fi


def max_states_of(offsets) -> int:
    o = np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets)
    return int(np.max(np.diff(o))) if len(o) > 1 else 1


_HOST_DTYPES = {"offsets": np.int32, "seed_params": np.float64, "seed_cov": np.float64,
                "center": np.float64, "rot": np.float64, "x_over_x0": np.float64,
                "surface_id": np.int32, "loc": np.float64, "cov": np.float64,
                "is_hole": np.uint8}


def host_event(ev):
    """The event with every array field C-contiguous in the ABI's dtype."""
    out = dict(ev)
    for k, dt in _HOST_DTYPES.items():
        out[k] = np.ascontiguousarray(ev[k], dtype=dt)
    if ev.get("field_map") is not None:
        fm = dict(ev["field_map"])
        fm["b"] = np.ascontiguousarray(fm["b"], dtype=np.float64)
        out["field_map"] = fm
    return out


def event_to_device(ev, device="cuda"):
    """Copy the array fields of a synthetic event to torch tensors on device."""
    import torch
    out = dict(ev)
    for k, dt in _HOST_DTYPES.items():
        out[k] = torch.from_numpy(np.ascontiguousarray(ev[k], dtype=dt)).to(device)
    if ev.get("field_map") is not None:
        fm = dict(ev["field_map"])
        fm["b"] = torch.from_numpy(np.ascontiguousarray(fm["b"], dtype=np.float64)).to(device)
        out["field_map"] = fm
    out["max_states"] = max_states_of(ev["offsets"])
    return out


def alloc_outputs(n_tracks, n_states=None, device="cuda", with_states=False):
    import torch
    kw = dict(device=device)
    out = {"params": torch.empty((6, n_tracks), dtype=torch.float64, **kw),
           "cov": torch.empty((21, n_tracks), dtype=torch.float64, **kw),
           "chi2": torch.empty((n_tracks,), dtype=torch.float64, **kw),
           "ndf": torch.empty((n_tracks,), dtype=torch.int32, **kw),
           "status": torch.empty((n_tracks,), dtype=torch.uint8, **kw)}
    out["states"] = (torch.empty((6, n_states), dtype=torch.float64, **kw)
                     if with_states else None)
    return out


def kf_fit_ex(handle: Handle, dev_ev, out, opt: KfOptions | None = None, stream=None):
    """Queue one fit of a device-resident event on `stream` (a torch.cuda.Stream
    or a raw cudaStream_t integer; None = torch's current stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    tr, su, me, fi = _structs(dev_ev, dev_ev["max_states"])
    o = KfOutputs(_ptr(out["params"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out.get("ndf")),
                  _ptr(out.get("status")), _ptr(out.get("states")))
    _check(load().kf_fit_ex(handle.ptr, ctypes.byref(tr), ctypes.byref(su), ctypes.byref(me),
                            ctypes.byref(fi), ctypes.byref(opt) if opt is not None else None,
                            ctypes.byref(o), ctypes.c_void_p(int(stream))))
    return out


def kf_selftest(n_patterns=1 << 22):
    """Device self-check of the numeric helpers; returns the 6 mismatch counts."""
    counts = np.zeros(6, dtype=np.uint64)
    _check(load().kf_selftest(int(n_patterns), counts.ctypes.data_as(ctypes.c_void_p)))
    return [int(c) for c in counts]


def kf_selftest_df(n_patterns=1 << 22):
    """Device self-check of the mixed path's double-float arithmetic; returns
    the 4 counts of results beyond 2^-44 (sum, sum with a float, product,
    compensated dot product) and the count of patterns that a plain float
    sum already misses."""
    counts = np.zeros(5, dtype=np.uint64)
    _check(load().kf_selftest_df(int(n_patterns), counts.ctypes.data_as(ctypes.c_void_p)))
    return [int(c) for c in counts]


def kf_autotune(handle: Handle, dev_ev, out, opt: KfOptions | None = None, stream=None):
    """Time every launch shape on this batch; return (best options, median ms).
    The choice is cached in the handle per batch shape."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    tr, su, me, fi = _structs(dev_ev, dev_ev["max_states"])
    o = KfOutputs(_ptr(out["params"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out.get("ndf")),
                  _ptr(out.get("status")), _ptr(out.get("states")))
    best = KfOptions()
    ms = ctypes.c_double(0.0)
    _check(load().kf_autotune(handle.ptr, ctypes.byref(tr), ctypes.byref(su), ctypes.byref(me),
                              ctypes.byref(fi), ctypes.byref(opt) if opt is not None else None,
                              ctypes.byref(o), ctypes.c_void_p(int(stream)), ctypes.byref(best),
                              ctypes.byref(ms)))
    return best, ms.value


def kf_fit_static(dev_ev, out, opt: KfOptions | None = None, stream=None):
    """Fit without any device allocation: scratch lives in the library's fixed
    per-GPU block (for callers that cannot allocate: real-time loops, fixed
    memory budgets).  Same inputs, outputs and results as :func:`kf_fit_ex`; calls
    that overlap on the GPU share the block and must be serialised."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    tr, su, me, fi = _structs(dev_ev, dev_ev["max_states"])
    o = KfOutputs(_ptr(out["params"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out.get("ndf")),
                  _ptr(out.get("status")), _ptr(out.get("states")))
    _check(load().kf_fit_static(ctypes.byref(tr), ctypes.byref(su), ctypes.byref(me), ctypes.byref(fi),
                                ctypes.byref(opt) if opt is not None else None, ctypes.byref(o),
                                ctypes.c_void_p(int(stream))))
    return out


def kf_fit(dev_ev, out):
    """Default-option fit on the legacy default stream (synchronous)."""
    tr, su, me, fi = _structs(dev_ev, dev_ev["max_states"])
    _check(load().kf_fit(ctypes.byref(tr), ctypes.byref(su), ctypes.byref(me), ctypes.byref(fi),
                         _ptr(out["params"]), _ptr(out["cov"]), _ptr(out["chi2"])))
    return out


def kf_fit_host(handle: Handle, ev, opt: KfOptions | None = None, out=None, stream=None,
                with_states=False):
    """Fit a host-resident event (numpy arrays); copies happen inside the call."""
    T = int(ev["n_tracks"])
    M = int(ev["surface_id"].shape[0])
    if out is None:
        out = {"params": np.empty((6, T)), "cov": np.empty((21, T)), "chi2": np.empty(T),
               "ndf": np.empty(T, dtype=np.int32), "status": np.empty(T, dtype=np.uint8),
               "states": np.empty((6, M)) if with_states else None}
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ev = host_event(ev)
    ms = ev.get("max_states") or max_states_of(ev["offsets"])
    tr, su, me, fi = _structs(ev, ms)
    o = KfOutputs(_ptr(out["params"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out.get("ndf")),
                  _ptr(out.get("status")), _ptr(out.get("states")))
    _check(load().kf_fit_host(handle.ptr, ctypes.byref(tr), ctypes.byref(su), ctypes.byref(me),
                              ctypes.byref(fi), ctypes.byref(opt) if opt is not None else None,
                              ctypes.byref(o), ctypes.c_void_p(int(stream or 0))))
    return out


def kf_chi2_grad(handle: Handle, dev_ev, align=None, dl_dchi2=None, out_chi2=None, grad_seed=None,
                 grad_align=None, opt: KfOptions | None = None, stream=None):
    """chi2 per track and the gradient of sum_t w_t chi2_t (w = dl_dchi2, default
    1) with respect to the seeds (grad_seed [6][T]) and the per-surface
    alignment (grad_align [6][S]).  Device tensors; None outputs are skipped."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    tr, su, me, fi = _structs(dev_ev, dev_ev["max_states"])
    _check(load().kf_chi2_grad(handle.ptr, ctypes.byref(tr), ctypes.byref(su), _ptr(align), ctypes.byref(me),
                               ctypes.byref(fi), ctypes.byref(opt) if opt is not None else None,
                               _ptr(dl_dchi2), _ptr(out_chi2), _ptr(grad_seed), _ptr(grad_align),
                               ctypes.c_void_p(int(stream))))


def kf_grad(handle: Handle, dev_ev, align=None, dl_dchi2=None, dl_dparams=None, dl_dcov=None, out_chi2=None,
            out_params=None, out_cov=None, grad_seed=None, grad_align=None, opt: KfOptions | None = None,
            stream=None):
    """The adjoint of the whole fit (filter and smoother): chi2 [T], the
    smoothed state-0 parameters [6][T] and covariance [21][T] at this
    alignment, and the gradient of
    L = sum_t [w_t chi2_t + v_t . params_t + W_t . cov_t]
    (w = dl_dchi2, default 1; v = dl_dparams, W = dl_dcov, default 0) with
    respect to the seeds (grad_seed [6][T]) and the per-surface alignment
    (grad_align [6][S]).  Device tensors; None outputs are skipped."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    tr, su, me, fi = _structs(dev_ev, dev_ev["max_states"])
    w = KfGradWeights(_ptr(dl_dchi2), _ptr(dl_dparams), _ptr(dl_dcov))
    o = KfGradOutputs(_ptr(out_chi2), _ptr(out_params), _ptr(out_cov), _ptr(grad_seed), _ptr(grad_align))
    _check(load().kf_grad(handle.ptr, ctypes.byref(tr), ctypes.byref(su), _ptr(align), ctypes.byref(me),
                          ctypes.byref(fi), ctypes.byref(opt) if opt is not None else None, ctypes.byref(w),
                          ctypes.byref(o), ctypes.c_void_p(int(stream))))


def _chi2_function():
    import torch

    class KalmanChi2(torch.autograd.Function):
        """chi2 per track of the Kalman fit as a differentiable function of
        the seed parameters [6][T] and the surface alignment [6][S]; the
        backward pass is the library's adjoint kernel (kf_chi2_grad)."""

        @staticmethod
        def forward(ctx, seed_params, align, dev_ev, handle):
            ev = dict(dev_ev)
            ev["seed_params"] = seed_params.detach().contiguous()
            chi2 = torch.empty(int(ev["n_tracks"]), dtype=torch.float64, device=seed_params.device)
            kf_chi2_grad(handle, ev, align=align.detach().contiguous(), out_chi2=chi2)
            ctx.save_for_backward(seed_params.detach(), align.detach())
            ctx.ev = dev_ev
            ctx.handle = handle
            return chi2

        @staticmethod
        def backward(ctx, g):
            seed_params, align = ctx.saved_tensors
            ev = dict(ctx.ev)
            ev["seed_params"] = seed_params.contiguous()
            gs = torch.empty_like(seed_params) if ctx.needs_input_grad[0] else None
            ga = torch.empty_like(align) if ctx.needs_input_grad[1] else None
            kf_chi2_grad(ctx.handle, ev, align=align.contiguous(), dl_dchi2=g.contiguous().to(torch.float64),
                         grad_seed=gs, grad_align=ga)
            return gs, ga, None, None

    class KalmanFit(torch.autograd.Function):
        """The whole fit -- chi2 [T], smoothed state-0 parameters [6][T] and
        packed covariance [21][T] -- as a differentiable function of the seed
        parameters and the surface alignment; the backward pass is the
        library's adjoint of the filter and the smoother (kf_grad)."""

        @staticmethod
        def forward(ctx, seed_params, align, dev_ev, handle):
            ev = dict(dev_ev)
            ev["seed_params"] = seed_params.detach().contiguous()
            T = int(ev["n_tracks"])
            kw = dict(dtype=torch.float64, device=seed_params.device)
            chi2, params, cov = torch.empty(T, **kw), torch.empty((6, T), **kw), torch.empty((21, T), **kw)
            kf_grad(handle, ev, align=align.detach().contiguous(), out_chi2=chi2, out_params=params,
                    out_cov=cov)
            ctx.save_for_backward(seed_params.detach(), align.detach())
            ctx.ev = dev_ev
            ctx.handle = handle
            return chi2, params, cov

        @staticmethod
        def backward(ctx, g_chi2, g_params, g_cov):
            seed_params, align = ctx.saved_tensors
            ev = dict(ctx.ev)
            ev["seed_params"] = seed_params.contiguous()
            gs = torch.empty_like(seed_params) if ctx.needs_input_grad[0] else None
            ga = torch.empty_like(align) if ctx.needs_input_grad[1] else None
            f64 = lambda t: None if t is None else t.contiguous().to(torch.float64)
            w = f64(g_chi2) if g_chi2 is not None else torch.zeros(seed_params.shape[1], dtype=torch.float64,
                                                                   device=seed_params.device)
            kf_grad(ctx.handle, ev, align=align.contiguous(), dl_dchi2=w, dl_dparams=f64(g_params),
                    dl_dcov=f64(g_cov), grad_seed=gs, grad_align=ga)
            return gs, ga, None, None

    return KalmanChi2, KalmanFit


_CHI2_FN = None


def chi2_autograd(seed_params, align, dev_ev, handle):
    """Differentiable chi2 per track (torch.autograd), see KalmanChi2."""
    global _CHI2_FN
    if _CHI2_FN is None:
        _CHI2_FN = _chi2_function()
    return _CHI2_FN[0].apply(seed_params, align, dev_ev, handle)


def fit_autograd(seed_params, align, dev_ev, handle):
    """Differentiable (chi2 [T], params [6][T], cov [21][T]) of the whole fit
    (torch.autograd), see KalmanFit."""
    global _CHI2_FN
    if _CHI2_FN is None:
        _CHI2_FN = _chi2_function()
    return _CHI2_FN[1].apply(seed_params, align, dev_ev, handle)
