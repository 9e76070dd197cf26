"""Error metrics of GPU results against the oracle.

Parameters: |dx_i| / max(|x_i,ref|, sqrt(C_ii,ref)) -- relative to the value,
floored at the parameter's own fitted uncertainty.  Covariances:
|dC_ij| / sqrt(C_ii,ref C_jj,ref) -- relative to the correlation scale.
"""
import numpy as np

DIAG = [i * (i + 1) // 2 + i for i in range(6)]
PAIRS = [(i, j) for i in range(6) for j in range(i + 1)]


def param_err(p, ref_p, ref_cov):
    sd = np.sqrt(np.abs(ref_cov[DIAG]))
    return np.abs(p - ref_p) / np.maximum(np.abs(ref_p), sd)


def cov_err(c, ref_cov):
    d = np.abs(ref_cov[DIAG])
    scale = np.stack([np.sqrt(d[i] * d[j]) for i, j in PAIRS])
    return np.abs(c - ref_cov) / scale


def chi2_err(c, ref):
    return np.abs(c - ref) / np.maximum(np.abs(ref), 1.0)


def state_sigmas(ev, **fit_kw):
    """Smoothed standard deviations of every state [6][M] from the oracle's
    per-track fits (the floor of the per-state parameter metric)."""
    import oracle
    o = np.asarray(ev["offsets"], dtype=np.int64)
    sd = np.full((6, int(o[-1])), np.nan)
    for t in range(int(ev["n_tracks"])):
        r = oracle.fit_track(ev, t, **fit_kw)
        if r["status"] == 0:
            sd[:, o[t]:o[t + 1]] = np.sqrt(np.abs(np.diagonal(r["Cs"], axis1=1, axis2=2))).T
    return sd


def states_err(g_states, r_states, sd):
    """|dx| / max(|x_ref|, sigma of that state) on every state."""
    return np.abs(g_states - r_states) / np.maximum(np.abs(r_states), sd)


# Element-wise check of gradients against central finite differences.  The
# oracle's objective L carries a relative rounding noise of about 1e-13: its
# chi2 terms are built from residuals m - x_p of ~50 um that are differences
# of positions of ~100 mm, so one rounding of a position is amplified ~2000x
# (measured on 100 tracks of the misaligned 20-plane telescope: central
# differences at steps h and 2h, h = 1e-6, differ by up to 6.5e-8 |L|, i.e.
# 6.5e-14 |L| / h).  A central difference with step h turns it into an
# absolute noise of about 1e-13 |L| / h in the derivative.  The floor is the
# derivative at which that noise is 1e-5 of it:
#   floor = 1e-13 |L| / h / 1e-5 = 1e-2 |L| (1e-6 / h),
# so |g - fd| <= 1e-5 max(|fd|, floor) holds each element to 1e-5 relative
# down to the size that finite differences can resolve at all.
FD_NOISE_REL = 1e-13


def fd_floor(l_abs, h, tol=1e-5):
    return FD_NOISE_REL * np.asarray(l_abs) / np.asarray(h) / tol


def seed_steps(seed_params, h=1e-6):
    """The FD steps of oracle.chi2_gradient_fd for the seeds [6][T] (the q/p
    step is relative)."""
    hs = np.full(np.shape(seed_params), h, dtype=np.float64)
    hs[4] = h * np.abs(np.asarray(seed_params)[4])
    return hs


def fd_floor_measured(fd_h, fd_2h, model_floor, tol=1e-5):
    """The floor with each element's measured finite-difference resolution:
    central differences at steps h and 2h differ by their noise (~1/h) and
    truncation (~h^2) errors, which bounds the step-h value's error within a
    factor of about two; an element is held to tol relative only above the
    size at which twice that spread is tol of it."""
    return np.maximum(model_floor, 2.0 * np.abs(np.asarray(fd_h) - np.asarray(fd_2h)) / tol)


def grad_err(g, fd, floor):
    """|g - fd| / max(|fd|, floor), element-wise."""
    return np.abs(np.asarray(g) - np.asarray(fd)) / np.maximum(np.abs(fd), floor)
