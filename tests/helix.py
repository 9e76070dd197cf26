"""Closed-form references used to pin the oracle (test helpers, numpy only).

* ``helix_to_plane``: exact trajectory of a unit charge in a constant field
  B = (0, 0, Bz) from a point to the plane x = x1.  With omega = kappa*Bz*q/p
  the azimuth turns as phi(s) = phi0 - omega*s, and
      x(s) = x0 + sin(theta)/omega * (sin(phi0) - sin(phi0 - omega*s))
      y(s) = y0 + sin(theta)/omega * (cos(phi0 - omega*s) - cos(phi0))
      z(s) = z0 + s*cos(theta),   t(s) = t0 + s*sqrt(1 + m^2 (q/p)^2)/c,
  so the crossing of x = x1 has sin(phi0 - omega*s) = sin(phi0) -
  omega*(x1 - x0)/sin(theta).
* ``lsq_fit``: Gauss-Newton least squares of a track model against the hits,
  with the seed as a Gaussian pseudo-measurement (the batch estimate that a
  linear Kalman filter + RTS smoother reproduces exactly).
"""
import math

import numpy as np

KAPPA = 2.99792458e-4
C_LIGHT = 299.792458
MUON_MASS = 0.1056583755


def helix_to_plane(x0, y0, z0, t0, phi, theta, qop, bz, x1, mass=MUON_MASS):
    """Return (y1, z1, t1, phi1, s) at the plane x = x1 (first crossing)."""
    st = math.sin(theta)
    omega = qop * KAPPA * bz
    dx = x1 - x0
    if abs(omega) < 1e-14:
        s = dx / (math.cos(phi) * st)
        y1 = y0 + dx * math.tan(phi)
        phi1 = phi
    else:
        arg = math.sin(phi) - omega * dx / st
        if abs(arg) >= 1.0:
            raise ValueError("no crossing")
        psi = math.asin(arg)
        s = (phi - psi) / omega
        y1 = y0 - 2.0 * st / omega * math.sin(0.5 * (psi + phi)) * math.sin(0.5 * (psi - phi))
        phi1 = psi
    z1 = z0 + s * math.cos(theta)
    t1 = t0 + s * math.sqrt(1.0 + mass * mass * qop * qop) / C_LIGHT
    return y1, z1, t1, phi1, s


def helix_bound_map(x, xa, xb, bz, mass=MUON_MASS):
    """Bound parameters on plane x = xa -> bound parameters on x = xb, for
    planes with u = y, v = z, n = x (no material)."""
    y1, z1, t1, phi1, _ = helix_to_plane(xa, x[0], x[1], x[5], x[2], x[3], x[4], bz, xb, mass)
    return np.array([y1, z1, phi1, x[3], x[4], t1])


def fd_jacobian(fun, x, rel=1e-6):
    x = np.asarray(x, dtype=float)
    f0 = fun(x)
    J = np.zeros((len(f0), len(x)))
    for i in range(len(x)):
        h = rel * max(1.0, abs(x[i]))
        e = np.zeros_like(x)
        e[i] = h
        J[:, i] = (fun(x + e) - fun(x - e)) / (2 * h)
    return J


def lsq_fit(model, m, sigma_m, x_seed, C_seed, iters=20):
    """Gauss-Newton: minimise |m - model(x)|^2/sigma^2 + (x - seed)^T C^-1 (x - seed).

    Returns the estimate and its covariance (inverse of the normal matrix)."""
    W0 = np.linalg.inv(C_seed)
    x = np.array(x_seed, dtype=float)
    A = None
    for _ in range(iters):
        f = model(x)
        J = fd_jacobian(model, x, rel=1e-7)
        A = J.T @ J / sigma_m ** 2 + W0
        b = J.T @ (m - f) / sigma_m ** 2 + W0 @ (x_seed - x)
        dx = np.linalg.solve(A, b)
        x = x + dx
        if np.all(np.abs(dx) < 1e-15 * (1 + np.abs(x))):
            break
    return x, np.linalg.inv(A)


def telescope_model(planes, bz, mass=MUON_MASS):
    """Hit positions (all y, then all z) on planes x = planes[k] for a track
    whose bound parameters are given on the reference plane x = 0."""
    def model(x):
        ys, zs = [], []
        xa, cur = 0.0, np.array(x, dtype=float)
        for xp in planes:
            cur = helix_bound_map(cur, xa, xp, bz, mass)
            xa = xp
            ys.append(cur[0])
            zs.append(cur[1])
        return np.array(ys + zs)
    return model
