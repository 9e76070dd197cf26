"""Seeded synthetic track events shaped like the paper's telescope workloads.

This module only *simulates* inputs.  It holds none of the fit's arithmetic:
no Runge-Kutta-Nystrom stepping, no Jacobians, no Kalman update or smoother.
Truth trajectories are the closed-form helix of a unit charge in a constant
field along z, or, for a workload with a position-dependent field, a classical
fourth-order Runge-Kutta integration of the equations of motion written with
x as the independent variable (slopes dy/dx, dz/dx; 0.5 mm steps, every plane
reached exactly); multiple scattering is drawn with the Highland width at
every crossed plane; hits are Gaussian-smeared local positions.  Both the
CUDA path and the CPU oracle fit exactly these arrays.  A field-map workload
also returns the map (the analytic field sampled on a grid) that the fit
interpolates.

Stands in for the paper's Fatras single-muon samples (paper Sect. 5: a
telescope of planes perpendicular to x, constant 2 T field along z, single
muons, 50 um Gaussian smearing, truth-smeared seeds).

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea,
Flood 2014) applied to a key built from (seed, track, attempt, purpose,
index), so every track is reproducible on its own and independent of batch
size.  Normals use the Box-Muller transform.

Layout of the returned event (the library's structure-of-arrays boundary):
  offsets[T+1] int32, seed_params[6][T], seed_cov[21][T] (packed lower
  triangle), truth_params[6][T]; center[3][S], rot[9][S] (row-major R whose
  columns are u, v, n), x_over_x0[S]; surface_id[M] int32, loc[2][M],
  cov[3][M] (V00, V01, V11), is_hole[M] uint8, truth_states[6][M] (or None);
  bfield[3].
State 0 of every track is the reference plane x = 0 (surface 0), which has no
measurement and no material; the seed lives there.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

MUON_MASS = 0.1056583755  # GeV
_KAPPA = 2.99792458e-4  # GeV / (T mm)
_C = 299.792458  # mm / ns
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)

# purposes (stream ids) of the counter-based generator
_P_PHI, _P_THETA, _P_CHARGE, _P_MOM, _P_NHIT = 0, 1, 2, 3, 4
_P_SEED, _P_HIT, _P_MS, _P_HOLE = 5, 6, 7, 8


@dataclasses.dataclass(frozen=True)
class Workload:
    """A synthetic workload: geometry, field, kinematics and smearing."""
    name: str
    n_tracks: int
    plane_x: tuple            # x positions of the measurement planes (mm)
    x_over_x0: float          # material per plane (fraction of X0)
    bz: float                 # field along z (T)
    sigma: float              # hit resolution per axis (mm)
    p_range: tuple            # log-uniform momentum range (GeV)
    nhit_range: tuple | None = None   # planes crossed ~ U{lo..hi}; None = all
    hole_prob: float = 0.0    # probability that a crossed plane has no hit
    seed: int = 0
    phi_half: float = 0.3     # phi ~ U(-phi_half, phi_half)
    theta_half: float = 0.3   # theta ~ U(pi/2 - theta_half, pi/2 + theta_half)
    half_width: float = 500.0 # planes are 1 m x 1 m in the simulation
    min_cos_incidence: float = 0.1
    min_meas: int = 3         # resample tracks left with fewer measurements
    misalign: tuple | None = None  # (shift sigma mm, rotation sigma rad) of the
                                   # true planes; the event keeps the nominal
                                   # geometry and records align_true
    fringe: float = 0.0       # > 0: the field falls along x as
                              # Bz = bz (1 - fringe (x/1000)^2) with the
                              # matching Bx = -2 fringe bz x z / 1000^2
                              # (curl-free in the x-z plane); the fit gets it
                              # as a grid map
    map_step: float = 25.0    # grid spacing of that map along x (mm); twice
                              # that along y and z


def _planes(n, step):
    return tuple(step * (i + 1) for i in range(n))


# Workloads shaped like the paper's telescope (Sect. 5) at the sizes the
# benchmark and the parity tests use.
WORKLOADS = {
    "tel10_1k": Workload("tel10_1k", 1000, _planes(10, 30.0), 0.005, 2.0, 0.050,
                         (1.0, 10.0), seed=0),
    "tel30_100k": Workload("tel30_100k", 100_000, _planes(30, 25.0), 0.01, 2.0,
                           0.030, (0.5, 100.0), seed=1),
    "uneven30_1m": Workload("uneven30_1m", 1_000_000, _planes(30, 25.0), 0.01, 2.0,
                            0.050, (1.0, 50.0), nhit_range=(5, 30), hole_prob=0.05,
                            seed=2),
    "tel30_4m": Workload("tel30_4m", 4_000_000, _planes(30, 25.0), 0.01, 2.0, 0.050,
                         (1.0, 100.0), seed=4),
    "align20_100k": Workload("align20_100k", 100_000, _planes(20, 30.0), 0.005, 2.0, 0.050,
                             (1.0, 10.0), seed=3, misalign=(0.100, 0.001)),
    "fringe30_100k": Workload("fringe30_100k", 100_000, _planes(30, 25.0), 0.01, 2.0, 0.030,
                              (0.5, 100.0), seed=5, fringe=0.3),
}


def scaled(w: Workload, n_tracks: int, **kw) -> Workload:
    """The same workload with another track count (and optional overrides)."""
    return dataclasses.replace(w, n_tracks=int(n_tracks), **kw)


# ---------------------------------------------------------------------------
# counter-based random numbers
# ---------------------------------------------------------------------------

def _splitmix64(z):
    with np.errstate(over="ignore"):
        z = (z + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def _uniform(seed, tracks, attempt, purpose, index):
    """U(0,1) (open) for each track id; attempt may be an array."""
    t = np.asarray(tracks, dtype=np.uint64)
    a = np.asarray(attempt, dtype=np.uint64)
    stream = (a << np.uint64(32)) | np.uint64((purpose << 16) | index)
    k = _splitmix64(_splitmix64(np.uint64(seed) ^ _splitmix64(t)) ^ stream)
    return ((k >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def _normal(seed, tracks, attempt, purpose, index):
    u1 = _uniform(seed, tracks, attempt, purpose, 2 * index)
    u2 = _uniform(seed, tracks, attempt, purpose, 2 * index + 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# simulation
# ---------------------------------------------------------------------------

def _highland_width(qop, xx0, cos_inc, mass):
    """Highland/PDG projected scattering width for a unit charge."""
    p = 1.0 / np.abs(qop)
    beta2 = p * p / (p * p + mass * mass)
    eps = xx0 / np.abs(cos_inc)
    return 0.0136 / (np.sqrt(beta2) * p) * np.sqrt(eps) * (1.0 + 0.038 * np.log(eps / beta2))


_P_ALIGN = 9


def alignment_draw(w: Workload):
    """Per-surface misalignment (du, dv, dn, alpha, beta, gamma) of the true
    planes, [6][S]; surface 0 (the reference plane) stays nominal."""
    S = len(w.plane_x) + 1
    a = np.zeros((6, S))
    if w.misalign is None:
        return a
    ss, rs = w.misalign
    sid = np.arange(1, S, dtype=np.uint64)
    for e in range(6):
        a[e, 1:] = (ss if e < 3 else rs) * _normal(w.seed, sid, np.zeros(S - 1, dtype=np.uint64), _P_ALIGN, e)
    return a


def aligned_planes(center, rot, align):
    """Apply alignment: c' = c + R (du, dv, dn), R' = R Ru(alpha) Rv(beta) Rn(gamma)
    (rotations about the plane's local axes).  center [3][S], rot [9][S]."""
    S = center.shape[1]
    c2 = np.empty_like(center)
    r2 = np.empty_like(rot)
    for s in range(S):
        R = rot[:, s].reshape(3, 3)
        a = align[:, s]
        ca, sa, cb, sb, cg, sg = (np.cos(a[3]), np.sin(a[3]), np.cos(a[4]), np.sin(a[4]),
                                  np.cos(a[5]), np.sin(a[5]))
        Ru = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
        Rv = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
        Rn = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
        c2[:, s] = center[:, s] + R @ a[:3]
        r2[:, s] = (R @ Ru @ Rv @ Rn).ravel()
    return c2, r2


def _helix_at(x0, y0, z0, phi, st, ct, omega, s):
    """Position and azimuth after path s on the helix (stable as omega -> 0)."""
    half = 0.5 * omega * s
    small = np.abs(half) < 1e-9
    sinc = np.where(small, 1.0 - half * half / 6.0, np.sin(half) / np.where(small, 1.0, half))
    chord = s * sinc                                   # 2 sin(omega s / 2) / omega
    mid = phi - half
    x = x0 + st * chord * np.cos(mid)
    y = y0 + st * chord * np.sin(mid)
    z = z0 + s * ct
    return x, y, z, phi - omega * s


def fringe_field(w: Workload, x, y, z):
    """The analytic field of a fringe workload at (x, y, z) (arrays)."""
    L2 = 1000.0 ** 2
    bx = -2.0 * w.fringe * w.bz * x * z / L2
    by = np.zeros_like(x)
    bz = w.bz * (1.0 - w.fringe * x * x / L2)
    return bx, by, bz


def field_map_of(w: Workload) -> dict:
    """Grid map of the fringe field covering the telescope: x from -50 mm
    past the last plane, y and z over the plane size."""
    hx = w.map_step
    hy = 2.0 * w.map_step
    x0 = -50.0
    nx = int(math.ceil((max(w.plane_x) + 50.0 - x0) / hx)) + 1
    y0 = -w.half_width - hy
    ny = int(math.ceil(2 * (w.half_width + hy) / hy)) + 1
    gx = x0 + hx * np.arange(nx)
    gy = y0 + hy * np.arange(ny)
    gz = y0 + hy * np.arange(ny)
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    bx, by, bz = fringe_field(w, X, Y, Z)
    return {"origin": [x0, y0, y0], "spacing": [hx, hy, hy],
            "b": np.ascontiguousarray(np.stack([bx, by, bz], axis=-1))}


def _advance_in_x(w, y, z, ty, tz, t, qop, gam, x_from, x_to):
    """Classical RK4 in x of (y, z, ty, tz, t) with ty = dy/dx, tz = dz/dx:
    d(ty)/dx = (q/p) k N [tz Bx + ty tz By - (1 + ty^2) Bz],
    d(tz)/dx = (q/p) k N [(1 + tz^2) By - ty Bx - ty tz Bz],
    dt/dx = N gam, N = sqrt(1 + ty^2 + tz^2) (gam = dt/ds)."""
    nstep = max(1, int(math.ceil((x_to - x_from) / 0.5)))
    dx = (x_to - x_from) / nstep

    def deriv(x, s):
        yy, zz, a, b, _ = s
        bx, by, bz = fringe_field(w, np.full_like(yy, x), yy, zz)
        N = np.sqrt(1.0 + a * a + b * b)
        k = qop * _KAPPA * N
        return (a, b, k * (b * bx + a * b * by - (1.0 + a * a) * bz),
                k * ((1.0 + b * b) * by - a * bx - a * b * bz), N * gam)

    s = (y, z, ty, tz, t)
    x = x_from
    for _ in range(nstep):
        k1 = deriv(x, s)
        k2 = deriv(x + dx / 2, tuple(v + dx / 2 * d for v, d in zip(s, k1)))
        k3 = deriv(x + dx / 2, tuple(v + dx / 2 * d for v, d in zip(s, k2)))
        k4 = deriv(x + dx, tuple(v + dx * d for v, d in zip(s, k3)))
        s = tuple(v + dx / 6 * (a + 2 * b + 2 * c + d) for v, a, b, c, d in zip(s, k1, k2, k3, k4))
        x += dx
    return s


def _simulate_fringe(w: Workload, ids, attempt, mass):
    """_simulate for the fringe field: trajectories integrated in x."""
    n = len(ids)
    npl = len(w.plane_x)
    s = w.seed
    phi0 = -w.phi_half + 2 * w.phi_half * _uniform(s, ids, attempt, _P_PHI, 0)
    th0 = (math.pi / 2 - w.theta_half) + 2 * w.theta_half * _uniform(s, ids, attempt, _P_THETA, 0)
    q = np.where(_uniform(s, ids, attempt, _P_CHARGE, 0) < 0.5, -1.0, 1.0)
    lo, hi = math.log(w.p_range[0]), math.log(w.p_range[1])
    p = np.exp(lo + (hi - lo) * _uniform(s, ids, attempt, _P_MOM, 0))
    qop = q / p
    if w.nhit_range is None:
        nhit = np.full(n, npl, dtype=np.int64)
    else:
        a, b = w.nhit_range
        nhit = a + np.minimum((_uniform(s, ids, attempt, _P_NHIT, 0) * (b - a + 1)).astype(np.int64), b - a)
    gam = np.sqrt(1.0 + mass * mass * qop * qop) / _C
    ok = np.ones(n, dtype=bool)
    loc = np.zeros((2, npl, n)); meas = np.zeros((2, npl, n))
    leave = np.zeros((4, npl, n))
    hole = np.zeros((npl, n), dtype=bool)
    phi = phi0.copy(); th = th0.copy()
    y = np.zeros(n); z = np.zeros(n); t = np.zeros(n)
    x_prev = 0.0
    for j, xp in enumerate(w.plane_x):
        crossed = j < nhit
        ok &= np.abs(phi) < 1.2
        cphi = np.cos(np.clip(phi, -1.2, 1.2))
        ty = np.tan(np.clip(phi, -1.2, 1.2))
        tz = np.cos(th) / (np.sin(th) * cphi)
        y, z, ty, tz, t = _advance_in_x(w, y, z, ty, tz, t, qop, gam, x_prev, xp)
        N = np.sqrt(1.0 + ty * ty + tz * tz)
        phi1 = np.arctan2(ty, 1.0)
        th1 = np.arctan2(np.sqrt(1.0 + ty * ty), tz)
        cos_inc = 1.0 / N
        ok &= ~crossed | ((cos_inc > w.min_cos_incidence) & (np.abs(y) <= w.half_width)
                          & (np.abs(z) <= w.half_width))
        loc[0, j] = y; loc[1, j] = z
        meas[0, j] = y + w.sigma * _normal(s, ids, attempt, _P_HIT, 2 * j)
        meas[1, j] = z + w.sigma * _normal(s, ids, attempt, _P_HIT, 2 * j + 1)
        hole[j] = _uniform(s, ids, attempt, _P_HOLE, j) < w.hole_prob
        if w.x_over_x0 > 0:
            th0w = _highland_width(qop, w.x_over_x0, np.maximum(np.abs(cos_inc), 1e-3), mass)
            dphi = th0w / np.sin(th1) * _normal(s, ids, attempt, _P_MS, 2 * j)
            dth = th0w * _normal(s, ids, attempt, _P_MS, 2 * j + 1)
        else:
            dphi = dth = 0.0
        phi = phi1 + dphi
        th = th1 + dth
        leave[0, j] = phi; leave[1, j] = th; leave[2, j] = t
        x_prev = xp
    nmeas = np.sum(~hole & (np.arange(npl)[:, None] < nhit[None, :]), axis=0)
    ok &= nmeas >= w.min_meas
    return dict(phi0=phi0, th0=th0, qop=qop, nhit=nhit, loc=loc, meas=meas,
                leave=leave, hole=hole, ok=ok)


def _simulate(w: Workload, ids, attempt, mass):
    """Simulate tracks `ids` (attempt per track); return arrays + ok mask."""
    if w.fringe > 0:
        return _simulate_fringe(w, ids, attempt, mass)
    n = len(ids)
    npl = len(w.plane_x)
    s = w.seed
    phi0 = -w.phi_half + 2 * w.phi_half * _uniform(s, ids, attempt, _P_PHI, 0)
    th0 = (math.pi / 2 - w.theta_half) + 2 * w.theta_half * _uniform(s, ids, attempt, _P_THETA, 0)
    q = np.where(_uniform(s, ids, attempt, _P_CHARGE, 0) < 0.5, -1.0, 1.0)
    lo, hi = math.log(w.p_range[0]), math.log(w.p_range[1])
    p = np.exp(lo + (hi - lo) * _uniform(s, ids, attempt, _P_MOM, 0))
    qop = q / p
    if w.nhit_range is None:
        nhit = np.full(n, npl, dtype=np.int64)
    else:
        a, b = w.nhit_range
        nhit = a + np.minimum((_uniform(s, ids, attempt, _P_NHIT, 0) * (b - a + 1)).astype(np.int64), b - a)
    omega = qop * _KAPPA * w.bz  # turning rate: dphi/ds = -omega
    true_planes = None
    if w.misalign is not None:
        S = npl + 1
        c_nom = np.zeros((3, S)); c_nom[0, 1:] = np.asarray(w.plane_x)
        r_nom = np.repeat(np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]).reshape(9, 1), S, axis=1)
        c_true, r_true = aligned_planes(c_nom, r_nom, alignment_draw(w))
        true_planes = []
        for j in range(npl):
            R = r_true[:, j + 1].reshape(3, 3)
            true_planes.append((c_true[:, j + 1], R[:, 2], R[:, 0], R[:, 1]))
    gam = np.sqrt(1.0 + mass * mass * qop * qop) / _C  # dt/ds
    x0 = np.zeros(n); y0 = np.zeros(n); z0 = np.zeros(n); t0 = np.zeros(n)
    phi = phi0.copy(); th = th0.copy()
    ok = np.ones(n, dtype=bool)
    loc = np.zeros((2, npl, n)); meas = np.zeros((2, npl, n))
    leave = np.zeros((4, npl, n))  # phi, theta (leaving), t, unused
    hole = np.zeros((npl, n), dtype=bool)
    for j, xp in enumerate(w.plane_x):
        crossed = j < nhit
        st = np.sin(th)
        dx = xp - x0
        arg = np.sin(phi) - omega * dx / st
        ok &= ~crossed | (np.abs(arg) < 1.0)
        arg = np.clip(arg, -1.0, 1.0)
        psi = np.arcsin(arg)
        small = np.abs(omega) < 1e-12
        om_safe = np.where(small, 1.0, omega)
        # exact helix: path length and transverse displacement to the plane
        s_path = np.where(small, dx / (np.cos(phi) * st), (phi - psi) / om_safe)
        dy = np.where(small, dx * np.tan(phi),
                      -2.0 * st / om_safe * np.sin(0.5 * (psi + phi)) * np.sin(0.5 * (psi - phi)))
        y1 = y0 + dy
        z1 = z0 + s_path * np.cos(th)
        phi1 = np.where(small, phi, psi)
        cos_inc = np.cos(phi1) * st
        if true_planes is not None:
            # crossing of the true (shifted, rotated) plane: Newton on the
            # signed distance n'.(r(s) - c') along the helix
            cT, nT, uT, vT = true_planes[j]
            ct_ = np.cos(th)
            for _ in range(8):
                xh, yh, zh, ph = _helix_at(x0, y0, z0, phi, st, ct_, omega, s_path)
                g = nT[0] * (xh - cT[0]) + nT[1] * (yh - cT[1]) + nT[2] * (zh - cT[2])
                dg = nT[0] * st * np.cos(ph) + nT[1] * st * np.sin(ph) + nT[2] * ct_
                s_path = s_path - g / dg
            xh, yh, zh, ph = _helix_at(x0, y0, z0, phi, st, ct_, omega, s_path)
            dr = np.stack([xh - cT[0], yh - cT[1], zh - cT[2]])
            y1 = uT @ dr        # local coordinates on the true plane
            z1 = vT @ dr
            phi1 = ph
            cos_inc = nT[0] * st * np.cos(ph) + nT[1] * st * np.sin(ph) + nT[2] * ct_
            xt, yt, zt = xh, yh, zh
        t1 = t0 + s_path * gam
        ok &= ~crossed | ((cos_inc > w.min_cos_incidence) & (np.abs(y1) <= w.half_width)
                          & (np.abs(z1) <= w.half_width) & (s_path > 0))
        if true_planes is None:
            xt, yt, zt = np.full(n, xp, dtype=np.float64), y1, z1
        loc[0, j] = y1; loc[1, j] = z1
        meas[0, j] = y1 + w.sigma * _normal(s, ids, attempt, _P_HIT, 2 * j)
        meas[1, j] = z1 + w.sigma * _normal(s, ids, attempt, _P_HIT, 2 * j + 1)
        hole[j] = _uniform(s, ids, attempt, _P_HOLE, j) < w.hole_prob
        # multiple scattering in plane j, after the hit (state j leaves it)
        if w.x_over_x0 > 0:
            th0w = _highland_width(qop, w.x_over_x0, np.maximum(np.abs(cos_inc), 1e-3), mass)
            dphi = th0w / st * _normal(s, ids, attempt, _P_MS, 2 * j)
            dth = th0w * _normal(s, ids, attempt, _P_MS, 2 * j + 1)
        else:
            dphi = dth = 0.0
        phi = phi1 + dphi
        th = th + dth
        leave[0, j] = phi; leave[1, j] = th; leave[2, j] = t1
        x0 = xt; y0 = yt; z0 = zt; t0 = t1
    nmeas = np.sum(~hole & (np.arange(npl)[:, None] < nhit[None, :]), axis=0)
    ok &= nmeas >= w.min_meas
    return dict(phi0=phi0, th0=th0, qop=qop, nhit=nhit, loc=loc, meas=meas,
                leave=leave, hole=hole, ok=ok)


def _simulate_with_retries(w: Workload, ids, mass: float, max_attempts: int):
    """Simulate tracks `ids`, redrawing each rejected track with the next
    attempt number until it is accepted. Returns (sim, attempt, rejected)."""
    attempt = np.zeros(len(ids), dtype=np.uint64)
    sim = _simulate(w, ids, attempt, mass)
    rejected = 0
    for _ in range(max_attempts):
        bad = np.nonzero(~sim["ok"])[0]
        if bad.size == 0:
            break
        rejected += bad.size
        attempt[bad] += 1
        sub = _simulate(w, ids[bad], attempt[bad], mass)
        for k, v in sub.items():
            if isinstance(v, np.ndarray):
                sim[k][..., bad] = v
    else:
        raise RuntimeError("track simulation did not converge")
    return sim, attempt, rejected


def _simulate_tracks(w: Workload, ids, mass: float, max_attempts: int, with_truth_states: bool):
    """Simulate tracks `ids` and return per-track arrays plus the per-plane
    arrays of the crossed planes in state order (track by track, planes in
    order): a contiguous range of tracks maps to a contiguous range of
    states, so ranges simulated apart concatenate to the whole batch."""
    sim, attempt, rejected = _simulate_with_retries(w, ids, mass, max_attempts)
    npl = len(w.plane_x)
    nhit = sim["nhit"]
    crossed = np.arange(npl)[None, :] < nhit[:, None]       # [tracks, npl]

    def per_state(a):                                      # [npl, tracks] -> crossed states
        return np.ascontiguousarray(a.T)[crossed]

    hole = per_state(sim["hole"])
    out = dict(phi0=sim["phi0"], th0=sim["th0"], qop=sim["qop"], nhit=nhit, attempt=attempt,
               hole=hole, plane=np.broadcast_to(np.arange(npl, dtype=np.int32), crossed.shape)[crossed],
               m0=np.where(hole, 0.0, per_state(sim["meas"][0])),
               m1=np.where(hole, 0.0, per_state(sim["meas"][1])))
    if with_truth_states:
        out.update(l0=per_state(sim["loc"][0]), l1=per_state(sim["loc"][1]),
                   a0=per_state(sim["leave"][0]), a1=per_state(sim["leave"][1]),
                   a2=per_state(sim["leave"][2]))
    return out, rejected


def default_workers(n_tracks: int) -> int:
    """Threads make_event uses: one per 100k tracks, at most one per core."""
    return max(1, min(os.cpu_count() or 1, n_tracks // 100_000))


def make_event(w: Workload, mass: float = MUON_MASS, max_attempts: int = 200,
               workers: int | None = None, with_truth_states: bool = True) -> dict:
    """Simulate workload `w` and return the event dict (see module doc).

    Every draw is keyed by (seed, track, attempt, purpose), so the tracks can
    be simulated in contiguous ranges by `workers` threads with the same
    result as one thread (the work is whole-array numpy operations, which
    run outside the interpreter lock; threads, unlike worker processes, are
    safe after CUDA is initialised and need no main-module guard).
    `with_truth_states=False` leaves out the per-state truth (truth_states is
    then None), which large batches that are only fitted do not need.
    """
    T = w.n_tracks
    npl = len(w.plane_x)
    ids_all = np.arange(T, dtype=np.uint64)
    workers = default_workers(T) if workers is None else max(1, int(workers))
    if workers == 1 or T < 2 * workers:
        sim, rejected = _simulate_tracks(w, ids_all, mass, max_attempts, with_truth_states)
    else:
        from concurrent.futures import ThreadPoolExecutor
        cuts = [T * i // workers for i in range(workers + 1)]
        with ThreadPoolExecutor(workers) as pool:
            parts = list(pool.map(
                lambda i: _simulate_tracks(w, np.arange(cuts[i], cuts[i + 1], dtype=np.uint64), mass,
                                           max_attempts, with_truth_states), range(workers)))
        sim = {k: np.concatenate([pt[0][k] for pt in parts]) for k in parts[0][0]}
        rejected = sum(pt[1] for pt in parts)
        del parts
    attempt = sim["attempt"]

    nhit = sim["nhit"]
    nstates = nhit + 1
    offsets = np.zeros(T + 1, dtype=np.int64)
    np.cumsum(nstates, out=offsets[1:])
    M = int(offsets[-1])
    if M >= 2 ** 31:
        raise ValueError("too many states for int32 offsets")
    # track t holds its reference state, then planes 0..nhit[t]-1: the
    # crossed planes in state order fill exactly the states that are not a
    # track's first
    sel = np.ones(M, dtype=bool)
    sel[offsets[:-1]] = False
    surface_id = np.zeros(M, dtype=np.int32)
    loc = np.zeros((2, M)); cov = np.zeros((3, M)); is_hole = np.ones(M, dtype=np.uint8)
    surface_id[sel] = sim["plane"] + 1
    loc[0, sel] = sim["m0"]
    loc[1, sel] = sim["m1"]
    cov[0, sel] = w.sigma ** 2
    cov[2, sel] = w.sigma ** 2
    is_hole[sel] = sim["hole"].astype(np.uint8)
    truth_states = None
    if with_truth_states:
        truth_states = np.zeros((6, M))
        for r, k in enumerate(("l0", "l1", "a0", "a1")):
            truth_states[r, sel] = sim[k]
        truth_states[4, sel] = np.repeat(sim["qop"], nhit)
        truth_states[5, sel] = sim["a2"]
    # state 0: reference plane, no measurement
    s0 = offsets[:-1]
    surface_id[s0] = 0
    is_hole[s0] = 1
    cov[0, s0] = 1.0
    cov[2, s0] = 1.0
    truth = np.stack([np.zeros(T), np.zeros(T), sim["phi0"], sim["th0"], sim["qop"], np.zeros(T)])
    if truth_states is not None:
        truth_states[:, s0] = truth
    # seed: truth smeared with a consistent diagonal prior
    ids = ids_all
    sig_seed = np.stack([
        np.full(T, 10 * w.sigma), np.full(T, 10 * w.sigma),
        np.full(T, 10 * w.sigma / 100.0), np.full(T, 10 * w.sigma / 100.0),
        0.1 * np.abs(sim["qop"]), np.full(T, 1.0)])
    seed_params = truth + sig_seed * np.stack(
        [_normal(w.seed, ids, attempt, _P_SEED, i) for i in range(6)])
    seed_cov = np.zeros((21, T))
    for i in range(6):
        seed_cov[i * (i + 1) // 2 + i] = sig_seed[i] ** 2
    # geometry: surface 0 = reference plane at x = 0, then the telescope
    S = npl + 1
    center = np.zeros((3, S))
    center[0, 1:] = np.asarray(w.plane_x)
    Rn = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])  # u=y, v=z, n=x
    rot = np.repeat(Rn.reshape(9, 1), S, axis=1)
    x_over_x0 = np.full(S, w.x_over_x0)
    x_over_x0[0] = 0.0
    return dict(
        name=w.name, n_tracks=T, offsets=offsets.astype(np.int32),
        seed_params=seed_params, seed_cov=seed_cov, truth_params=truth,
        center=center, rot=rot, x_over_x0=x_over_x0,
        bfield=np.array([0.0, 0.0, w.bz]), surface_id=surface_id, loc=loc,
        cov=cov, is_hole=is_hole, truth_states=truth_states,
        sigma=w.sigma, rejected=rejected, align_true=alignment_draw(w),
        **({"field_map": field_map_of(w)} if w.fringe > 0 else {}),
    )


def subset(ev: dict, tracks) -> dict:
    """Event restricted to the given track indices (renumbered 0..k-1)."""
    tracks = np.asarray(tracks, dtype=np.int64)
    o = ev["offsets"].astype(np.int64)
    lens = o[tracks + 1] - o[tracks]
    new_off = np.zeros(len(tracks) + 1, dtype=np.int64)
    np.cumsum(lens, out=new_off[1:])
    idx = np.concatenate([np.arange(o[t], o[t + 1]) for t in tracks]) if len(tracks) else np.zeros(0, np.int64)
    out = dict(ev)
    out["n_tracks"] = len(tracks)
    out["offsets"] = new_off.astype(np.int32)
    for k in ("seed_params", "seed_cov", "truth_params"):
        out[k] = np.ascontiguousarray(ev[k][:, tracks])
    for k in ("loc", "cov", "truth_states"):
        if ev.get(k) is not None:
            out[k] = np.ascontiguousarray(ev[k][:, idx])
    for k in ("surface_id", "is_hole"):
        out[k] = np.ascontiguousarray(ev[k][idx])
    return out
