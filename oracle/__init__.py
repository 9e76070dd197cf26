"""Plain FP64 CPU oracle of the per-track Kalman fit (arXiv 2105.01796).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg load this module; the CUDA product path never
does.  The oracle is a small C library (``kf_oracle.c``) built with gcc by
:func:`build` and reached through ctypes.  It shares no code with the CUDA
path; the only thing both sides see is the synthetic input generator.

Parity status of each oracle function (what pins it) is listed in the
repository's design notes; every function here is pinned by a ``not gpu``
test in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_LIB = os.path.join(_HERE, "libkf_oracle.so")
_lib = None

OK, NO_INTERSECTION, NON_SPD, NONFINITE, BAD_INPUT = 0, 1, 2, 3, 4
MUON_MASS = 0.1056583755  # GeV
SMOOTHER_RTS, SMOOTHER_BACKWARD_FILTER = 0, 1


class FieldMap(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3),
                ("b", ctypes.c_void_p)]


class Material(ctypes.Structure):
    _fields_ = [("z_over_a", ctypes.c_double), ("i_exc", ctypes.c_double),
                ("x0_rho", ctypes.c_double), ("sh_cbar", ctypes.c_double),
                ("sh_x0", ctypes.c_double), ("sh_x1", ctypes.c_double),
                ("sh_a", ctypes.c_double), ("sh_k", ctypes.c_double),
                ("sh_delta0", ctypes.c_double)]


class Method(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("bf_scale", ctypes.c_double),
                ("energy_loss", ctypes.c_int), ("mat", Material),
                ("map", ctypes.c_void_p)]


def silicon() -> Material:
    """Silicon: Z/A, mean excitation energy, radiation length and the
    Sternheimer density-effect parameters as tabulated by the PDG (atomic
    and nuclear properties of materials)."""
    return Material(0.49848, 173.0e-9, 21.82, 4.4355, 0.2015, 2.8716, 0.1492, 3.2546, 0.14)


def field_map_struct(fm):
    """ctypes FieldMap for a map dict {origin[3], spacing[3], b[nz][ny][nx][3]};
    returns (struct, the contiguous value array that must stay alive)."""
    b = np.ascontiguousarray(fm["b"], dtype=np.float64)
    nz, ny, nx, three = b.shape
    assert three == 3
    st = FieldMap(nx, ny, nz, (ctypes.c_double * 3)(*[float(v) for v in fm["origin"]]),
                  (ctypes.c_double * 3)(*[float(v) for v in fm["spacing"]]),
                  b.ctypes.data_as(ctypes.c_void_p))
    return st, b


def method_struct(method=None, field_map=None):
    """Build the kfo_method for a dict {smoother: 'rts'|'backward',
    bf_scale, energy_loss, material} and an optional field-map dict.
    Returns (struct or None, objects to keep alive)."""
    if method is None and field_map is None:
        return None, []
    method = dict(method or {})
    keep = []
    m = Method()
    m.smoother = SMOOTHER_BACKWARD_FILTER if method.get("smoother", "rts") == "backward" else SMOOTHER_RTS
    m.bf_scale = float(method.get("bf_scale", 1e4))
    m.energy_loss = 1 if method.get("energy_loss", False) else 0
    m.mat = method.get("material") or silicon()
    if field_map is not None:
        fm, b = field_map_struct(field_map)
        keep += [fm, b]
        m.map = ctypes.cast(ctypes.pointer(fm), ctypes.c_void_p)
    else:
        m.map = None
    keep.append(m)
    return m, keep


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "kf_oracle.h"))
    ):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I, D, L = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.kfo_bound_to_free.argtypes = [P, P, P, P, P]
        lib.kfo_rkn_step.argtypes = [P, D, P, D, P]
        lib.kfo_propagate.argtypes = [P, P, P, P, D, D, I, P, P]
        lib.kfo_propagate.restype = I
        lib.kfo_transport.argtypes = [P, P, P, P, P, P, D, D, I, P, P, P]
        lib.kfo_transport.restype = I
        lib.kfo_highland.argtypes = [D, D, D, D]
        lib.kfo_highland.restype = D
        lib.kfo_update.argtypes = [P, P, P, P, P, P, P]
        lib.kfo_update.restype = I
        lib.kfo_rts_step.argtypes = [P] * 9
        lib.kfo_rts_step.restype = I
        lib.kfo_linear_fit.argtypes = [I] + [P] * 10
        lib.kfo_linear_fit.restype = I
        lib.kfo_fit_track.argtypes = [I, P, P, P, P, P, P, I, P, P, P, P, D, D, I] + [P] * 8
        lib.kfo_fit_track.restype = I
        lib.kfo_fit_batch.argtypes = [I, P, P, P, I, P, P, P, L, P, P, P, P, P, D, D, I,
                                      P, P, P, P, P, P, I, I, I]
        lib.kfo_fit_batch.restype = I
        lib.kfo_field_at.argtypes = [P, P, P, P]
        lib.kfo_rkn_step_field.argtypes = [P, D, P, P, D, P]
        lib.kfo_transport_field.argtypes = [P, P, P, P, P, P, P, D, D, I, P, P, P]
        lib.kfo_transport_field.restype = I
        lib.kfo_density_effect.argtypes = [D, P]
        lib.kfo_density_effect.restype = D
        lib.kfo_bethe.argtypes = [D, D, P]
        lib.kfo_bethe.restype = D
        lib.kfo_landau_xi.argtypes = [D, D, P]
        lib.kfo_landau_xi.restype = D
        lib.kfo_energy_loss.argtypes = [P, D, D, D, P, I, P, P]
        lib.kfo_energy_loss.restype = I
        lib.kfo_linear_fit_ex.argtypes = [I] + [P] * 7 + [I, D] + [P] * 3
        lib.kfo_linear_fit_ex.restype = I
        lib.kfo_fit_track_ex.argtypes = [I, P, P, P, P, P, P, I, P, P, P, P, D, D, I] + [P] * 9
        lib.kfo_fit_track_ex.restype = I
        lib.kfo_fit_batch_ex.argtypes = [I, P, P, P, I, P, P, P, L, P, P, P, P, P, D, D, I,
                                         P, P, P, P, P, P, P, I, I, I]
        lib.kfo_fit_batch_ex.restype = I
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def bound_to_free(c, R, x):
    c, R, x = _f64(c, 3), _f64(R, 9), _f64(x, 6)
    f = np.zeros(8)
    J = np.zeros((8, 6))
    _load().kfo_bound_to_free(_p(c), _p(R), _p(x), _p(f), _p(J))
    return f, J


def rkn_step(f, h, B, mass=MUON_MASS):
    f = _f64(f, 8).copy()
    D = np.eye(8)
    _load().kfo_rkn_step(_p(f), float(h), _p(_f64(B, 3)), float(mass), _p(D))
    return f, D


def propagate(f, c, R, B, mass=MUON_MASS, h_max=50.0, n_iter=3):
    f = _f64(f, 8).copy()
    D = np.zeros((8, 8))
    path = np.zeros(1)
    st = _load().kfo_propagate(_p(f), _p(_f64(c, 3)), _p(_f64(R, 9)), _p(_f64(B, 3)),
                               float(mass), float(h_max), int(n_iter), _p(D), _p(path))
    return st, f, D, float(path[0])


def transport(ca, Ra, x, cb, Rb, B, mass=MUON_MASS, h_max=50.0, n_iter=3):
    xo = np.zeros(6)
    F = np.zeros((6, 6))
    path = np.zeros(1)
    st = _load().kfo_transport(_p(_f64(ca, 3)), _p(_f64(Ra, 9)), _p(_f64(x, 6)),
                               _p(_f64(cb, 3)), _p(_f64(Rb, 9)), _p(_f64(B, 3)),
                               float(mass), float(h_max), int(n_iter), _p(xo), _p(F),
                               _p(path))
    return st, xo, F, float(path[0])


def field_at(B, r, field_map=None):
    out = np.zeros(3)
    if field_map is None:
        _load().kfo_field_at(_p(_f64(B, 3)), None, _p(_f64(r, 3)), _p(out))
    else:
        fm, keep = field_map_struct(field_map)
        _load().kfo_field_at(_p(_f64(B, 3)), ctypes.byref(fm), _p(_f64(r, 3)), _p(out))
    return out


def rkn_step_field(f, h, B, field_map, mass=MUON_MASS):
    f = _f64(f, 8).copy()
    D = np.eye(8)
    fm, keep = field_map_struct(field_map)
    _load().kfo_rkn_step_field(_p(f), float(h), _p(_f64(B, 3)), ctypes.byref(fm), float(mass), _p(D))
    return f, D


def transport_field(ca, Ra, x, cb, Rb, B, field_map, mass=MUON_MASS, h_max=50.0, n_iter=3):
    xo = np.zeros(6)
    F = np.zeros((6, 6))
    path = np.zeros(1)
    fm, keep = field_map_struct(field_map)
    st = _load().kfo_transport_field(_p(_f64(ca, 3)), _p(_f64(Ra, 9)), _p(_f64(x, 6)),
                                     _p(_f64(cb, 3)), _p(_f64(Rb, 9)), _p(_f64(B, 3)),
                                     ctypes.byref(fm), float(mass), float(h_max), int(n_iter),
                                     _p(xo), _p(F), _p(path))
    return st, xo, F, float(path[0])


def density_effect(bg, material=None):
    m = material or silicon()
    return _load().kfo_density_effect(float(bg), ctypes.byref(m))


def bethe(bg, mass=MUON_MASS, material=None):
    """Mean stopping power in GeV cm^2/g."""
    m = material or silicon()
    return _load().kfo_bethe(float(bg), float(mass), ctypes.byref(m))


def landau_xi(beta, thick, material=None):
    m = material or silicon()
    return _load().kfo_landau_xi(float(beta), float(thick), ctypes.byref(m))


def energy_loss(qop, xx0, cosinc, direction=1, mass=MUON_MASS, material=None):
    """Returns (status, new q/p, Jacobian factor, downstream q/p variance)."""
    m = material or silicon()
    q = np.array([float(qop)])
    jac = np.zeros(1)
    var = np.zeros(1)
    st = _load().kfo_energy_loss(_p(q), float(mass), float(xx0), float(cosinc), ctypes.byref(m),
                                 int(direction), _p(jac), _p(var))
    return st, float(q[0]), float(jac[0]), float(var[0])


def highland(qop, xx0, cosinc, mass=MUON_MASS):
    return _load().kfo_highland(float(qop), float(mass), float(xx0), float(cosinc))


def update(xp, Cp, m, V):
    xf = np.zeros(6)
    Cf = np.zeros((6, 6))
    chi2 = np.zeros(1)
    st = _load().kfo_update(_p(_f64(xp, 6)), _p(_f64(Cp, (6, 6))), _p(_f64(m, 2)),
                            _p(_f64(V, (2, 2))), _p(xf), _p(Cf), _p(chi2))
    return st, xf, Cf, float(chi2[0])


def rts_step(xf, Cf, xp1, Cp1, F1, xs1, Cs1):
    xs = np.zeros(6)
    Cs = np.zeros((6, 6))
    st = _load().kfo_rts_step(*[_p(_f64(a)) for a in (xf, Cf, xp1, Cp1, F1, xs1, Cs1)],
                              _p(xs), _p(Cs))
    return st, xs, Cs


def linear_fit(x0, C0, F, Q, m, V, hole, smoother="rts", bf_scale=1e4):
    n = len(hole)
    xs = np.zeros((n, 6))
    Cs = np.zeros((n, 6, 6))
    chi2 = np.zeros(n)
    hole = np.ascontiguousarray(hole, dtype=np.uint8)
    sm = SMOOTHER_BACKWARD_FILTER if smoother == "backward" else SMOOTHER_RTS
    st = _load().kfo_linear_fit_ex(n, _p(_f64(x0, 6)), _p(_f64(C0, (6, 6))),
                                   _p(_f64(F, (n, 6, 6))), _p(_f64(Q, (n, 6, 6))),
                                   _p(_f64(m, (n, 2))), _p(_f64(V, (n, 2, 2))), _p(hole),
                                   sm, float(bf_scale), _p(xs), _p(Cs), _p(chi2))
    return st, xs, Cs, chi2


def fit_track(ev, t, h_max=50.0, n_iter=3, mass=MUON_MASS, method=None):
    """Fit track ``t`` of a synthetic event; return every intermediate.
    ``method``: None (the baseline) or a dict of variants (see
    :func:`method_struct`); a field map is taken from ``ev['field_map']``."""
    o0, o1 = int(ev["offsets"][t]), int(ev["offsets"][t + 1])
    n = o1 - o0
    sid = np.ascontiguousarray(ev["surface_id"][o0:o1], dtype=np.int32)
    loc = _f64(ev["loc"][:, o0:o1].T)
    cov = _f64(ev["cov"][:, o0:o1].T)
    hole = np.ascontiguousarray(ev["is_hole"][o0:o1], dtype=np.uint8)
    seed = _f64(ev["seed_params"][:, t])
    C0 = unpack_sym(ev["seed_cov"][:, t])
    out = {k: np.zeros((n, 6)) for k in ("xp", "xf", "xs")}
    out.update({k: np.zeros((n, 6, 6)) for k in ("Cp", "Cf", "Cs", "F")})
    out["chi2"] = np.zeros(n)
    S = ev["center"].shape[1]
    center = _f64(ev["center"].T)
    rot = _f64(np.moveaxis(ev["rot"].reshape(9, S), 0, 1))
    meth, keep = method_struct(method, ev.get("field_map"))
    st = _load().kfo_fit_track_ex(
        n, _p(sid), _p(loc), _p(cov), _p(hole), _p(seed), _p(C0), S, _p(center),
        _p(rot), _p(_f64(ev["x_over_x0"])), _p(_f64(ev["bfield"], 3)), float(mass),
        float(h_max), int(n_iter), ctypes.byref(meth) if meth is not None else None,
        _p(out["xp"]), _p(out["Cp"]), _p(out["xf"]),
        _p(out["Cf"]), _p(out["xs"]), _p(out["Cs"]), _p(out["F"]), _p(out["chi2"]))
    out["status"] = st
    return out


def fit_batch(ev, h_max=50.0, n_iter=3, mass=MUON_MASS, t_begin=0, t_end=None,
              n_threads=None, with_states=False, method=None):
    """Fit tracks [t_begin, t_end) of a synthetic event (SoA boundary layout).
    ``method``: None (the baseline) or a dict of variants (see
    :func:`method_struct`); a field map is taken from ``ev['field_map']``.

    Returns the outputs for the full track range (entries outside the range
    are left NaN / zero).
    """
    T = int(ev["n_tracks"])
    M = int(ev["offsets"][-1])
    if t_end is None:
        t_end = T
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    S = ev["center"].shape[1]
    offsets = np.ascontiguousarray(ev["offsets"], dtype=np.int32)
    sid = np.ascontiguousarray(ev["surface_id"], dtype=np.int32)
    hole = np.ascontiguousarray(ev["is_hole"], dtype=np.uint8)
    center = _f64(ev["center"].T)
    rot = _f64(np.moveaxis(ev["rot"].reshape(9, S), 0, 1))
    seed = _f64(ev["seed_params"])
    seed_cov = _f64(ev["seed_cov"])
    loc = _f64(ev["loc"])
    cov = _f64(ev["cov"])
    out = {
        "params": np.full((6, T), np.nan),
        "cov": np.full((21, T), np.nan),
        "chi2": np.full(T, np.nan),
        "ndf": np.zeros(T, dtype=np.int32),
        "status": np.zeros(T, dtype=np.uint8),
    }
    states = np.full((6, M), np.nan) if with_states else None
    meth, keep = method_struct(method, ev.get("field_map"))
    rc = _load().kfo_fit_batch_ex(
        T, _p(offsets), _p(seed), _p(seed_cov), S, _p(center), _p(rot),
        _p(_f64(ev["x_over_x0"])), M, _p(sid), _p(loc), _p(cov), _p(hole),
        _p(_f64(ev["bfield"], 3)), float(mass), float(h_max), int(n_iter),
        ctypes.byref(meth) if meth is not None else None,
        _p(out["params"]), _p(out["cov"]), _p(out["chi2"]), _p(out["ndf"]),
        _p(out["status"]), _p(states), int(t_begin), int(t_end), int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected the batch arguments")
    if with_states:
        out["states"] = states
    return out


def unpack_sym(packed):
    """21 packed lower-triangle values -> dense symmetric 6x6."""
    C = np.zeros((6, 6))
    e = 0
    for i in range(6):
        for j in range(i + 1):
            C[i, j] = C[j, i] = packed[e]
            e += 1
    return C


def pack_sym(C):
    return np.array([C[i, j] for i in range(6) for j in range(i + 1)])


# ---------------------------------------------------------------------------
# alignment and the gradient of the summed chi2 (finite differences)
# ---------------------------------------------------------------------------

def apply_alignment(center, rot, align):
    """Aligned geometry: c' = c + R (du, dv, dn) and
    R' = R Ru(alpha) Rv(beta) Rn(gamma), rotations about the plane's own
    local axes u, v, n.  center [3][S], rot [9][S], align [6][S]."""
    center = np.asarray(center, dtype=np.float64)
    rot = np.asarray(rot, dtype=np.float64)
    S = center.shape[1]
    c2 = np.empty_like(center)
    r2 = np.empty_like(rot)
    for s in range(S):
        R = rot[:, s].reshape(3, 3)
        du, dv, dn, al, be, ga = [float(v) for v in align[:, s]]
        Ru = np.array([[1.0, 0.0, 0.0], [0.0, np.cos(al), -np.sin(al)], [0.0, np.sin(al), np.cos(al)]])
        Rv = np.array([[np.cos(be), 0.0, np.sin(be)], [0.0, 1.0, 0.0], [-np.sin(be), 0.0, np.cos(be)]])
        Rn = np.array([[np.cos(ga), -np.sin(ga), 0.0], [np.sin(ga), np.cos(ga), 0.0], [0.0, 0.0, 1.0]])
        c2[:, s] = center[:, s] + R @ np.array([du, dv, dn])
        r2[:, s] = (R @ Ru @ Rv @ Rn).ravel()
    return c2, r2


def chi2_per_track(ev, align=None, seed_params=None, **kw):
    """chi2 of every track with the geometry aligned by `align` [6][S]."""
    e = dict(ev)
    if align is not None:
        e["center"], e["rot"] = apply_alignment(ev["center"], ev["rot"], align)
    if seed_params is not None:
        e["seed_params"] = seed_params
    return fit_batch(e, **kw)["chi2"]


def objective_per_track(ev, align=None, seed_params=None, weights=None, dl_dparams=None, dl_dcov=None,
                        **kw):
    """Per-track objective of the fit with the geometry aligned by `align`:
    L_t = w_t chi2_t + sum_i v_it x_s0,it + sum_e W_et C_s0,et, where x_s0 and
    C_s0 (packed, 21) are the smoothed parameters and covariance of state 0
    (paper Sect. 2: the smoother's output), w = weights [T] (default 1),
    v = dl_dparams [6][T] and W = dl_dcov [21][T] (default 0).  Returns
    (L [T], |terms| [T]: the sum of the terms' magnitudes, the scale of L's
    rounding noise)."""
    e = dict(ev)
    if align is not None:
        e["center"], e["rot"] = apply_alignment(ev["center"], ev["rot"], align)
    if seed_params is not None:
        e["seed_params"] = seed_params
    r = fit_batch(e, **kw)
    T = int(ev["n_tracks"])
    w = np.ones(T) if weights is None else np.asarray(weights, dtype=np.float64)
    terms = [w * r["chi2"]]
    if dl_dparams is not None:
        terms += list(np.asarray(dl_dparams, dtype=np.float64) * r["params"])
    if dl_dcov is not None:
        terms += list(np.asarray(dl_dcov, dtype=np.float64) * r["cov"])
    terms = np.stack(terms)
    return terms.sum(axis=0), np.abs(terms).sum(axis=0)


def objective_gradient_fd(ev, align=None, weights=None, dl_dparams=None, dl_dcov=None, h_shift=1e-6,
                          h_rot=1e-6, h_seed=1e-6, n_threads=None):
    """Gradient of L = sum_t L_t (objective_per_track) with respect to the
    seed parameters and the per-surface alignment, by central finite
    differences of the oracle (the plain definition of the derivative).
    Returns (grad_seed [6][T], grad_align [6][S]).  Steps are in the
    parameters' units (mm, rad, GeV^-1, ns); the q/p step is relative to
    |q/p|."""
    T = int(ev["n_tracks"])
    S = ev["center"].shape[1]
    a0 = np.zeros((6, S)) if align is None else np.asarray(align, dtype=np.float64)
    seeds = np.asarray(ev["seed_params"], dtype=np.float64)
    kw = dict(weights=weights, dl_dparams=dl_dparams, dl_dcov=dl_dcov, n_threads=n_threads)
    gs = np.zeros((6, T))
    for i in range(6):
        hv = np.full(T, h_seed)
        if i == 4:
            hv = h_seed * np.abs(seeds[4])
        sp = seeds.copy(); sp[i] += hv
        sm = seeds.copy(); sm[i] -= hv
        lp, _ = objective_per_track(ev, a0, sp, **kw)
        lm, _ = objective_per_track(ev, a0, sm, **kw)
        gs[i] = (lp - lm) / (2 * hv)
    ga = np.zeros((6, S))
    for s in range(S):
        for e in range(6):
            h = h_shift if e < 3 else h_rot
            ap = a0.copy(); ap[e, s] += h
            am = a0.copy(); am[e, s] -= h
            lp, _ = objective_per_track(ev, ap, **kw)
            lm, _ = objective_per_track(ev, am, **kw)
            ga[e, s] = np.sum(lp - lm) / (2 * h)
    return gs, ga


def chi2_gradient_fd(ev, align=None, weights=None, h_shift=1e-6, h_rot=1e-6, h_seed=1e-6, n_threads=None):
    """Gradient of L = sum_t w_t chi2_t by central finite differences of the
    oracle (objective_gradient_fd without the smoother terms).  Returns
    (grad_seed [6][T], grad_align [6][S])."""
    return objective_gradient_fd(ev, align, weights, h_shift=h_shift, h_rot=h_rot, h_seed=h_seed,
                                 n_threads=n_threads)
