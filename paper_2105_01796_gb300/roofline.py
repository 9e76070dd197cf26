"""Algorithmic work of the fit, for roofline accounting.

Counts are floating-point operations (an FMA counts 2) of the arithmetic the
method requires in the structure-exploiting form the kernels use: symmetric
covariances stored as 21 values, H a projection onto (loc0, loc1), F with
its trivial q/p row and time column, a Cholesky solve instead of an inverse.
Transcendental calls (sin, cos, atan2, sqrt, log) count 1 each.

Per track with n states, m measured states and n-1 transitions:

  transition (propagation + Jacobian + covariance transport + noise)
      RKN4 step with its exact Jacobian, constant field along z:   RKN_STEP
      steps per transition: ceil(s0/h_max) + n_iter (4 in every workload)
      bound->free, path correction, free->bound, F assembly:       FRAME
      Bm = F Cf (150 FMA) and Cp = Bm F^T (sym., 105 FMA):          TRANSPORT
      Highland noise:                                              NOISE
  measured state
      S, det, gain K, x_f:                                         GAIN
      Joseph covariance update (expanded, 21 x 4 FMA + W 12 x 2):  JOSEPH
      chi2 = r^T S^-1 r:                                           CHI2
  smoother step (n-1 per track)
      Cholesky of Cp (35 FMA, 15 mul, 6 sqrt, 6 div):              CHOL
      six triangular-solve pairs for A^T = Cp^-1 Bm:               SOLVE
      x_s update (36 FMA + 12 add) and Cs = Cf + A dC A^T
      (dC 21 sub, A dC 216 FMA, (A dC) A^T 126 FMA, 21 add):       SMOOTH_UPD

The mixed path runs JOSEPH, CHI2, CHOL and SOLVE in FP64 and the rest in
FP32; the FP64 path runs everything in FP64.
"""

RKN_STEP = 2 * 3 * 3 * 9 + 2 * 3 * 7 + 2 * 3 * 9 + 16 + 20  # columns, q/p column, value, cross products, misc
FRAME = 12 + 4 + 2 * 5 * 10 + 2 * 5 * 6 + 10 + 13
TRANSPORT = 2 * (150 + 105)
NOISE = 12
GAIN = 3 + 3 + 4 + 2 * 12 + 2 * 12
JOSEPH = 2 * (12 * 2 + 21 * 4) + 3
CHI2 = 12
CHOL = 2 * 35 + 15 + 6 + 6
SOLVE = 6 * 2 * (2 * 15 + 6)
SMOOTH_UPD = 2 * 36 + 12 + 21 + 2 * 216 + 2 * 126 + 21


def flops_per_track(n_states, n_meas, steps_per_transition=4):
    """(fp64_flops, fp32_flops) per precision mode for one track."""
    tr = max(n_states - 1, 0)
    prop = tr * (steps_per_transition * RKN_STEP + FRAME + TRANSPORT + NOISE)
    upd_req = n_meas * (JOSEPH + CHI2)
    gain = n_meas * GAIN
    sm_req = tr * (CHOL + SOLVE)
    sm_rest = tr * SMOOTH_UPD
    fp64_path = {"fp64": prop + upd_req + gain + sm_req + sm_rest, "fp32": 0}
    mixed = {"fp64": upd_req + sm_req, "fp32": prop + gain + sm_rest}
    return {"fp64_path": fp64_path, "mixed": mixed}


def batch_flops(offsets, is_hole, precision, steps_per_transition=4):
    """Total (fp64, fp32) flops of one fit of a batch."""
    import numpy as np
    o = np.asarray(offsets, dtype=np.int64)
    n = np.diff(o)
    meas = (np.asarray(is_hole) == 0).astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(meas)])
    m = cs[o[1:]] - cs[o[:-1]]
    tr = np.maximum(n - 1, 0).sum()
    M = int(m.sum())
    prop = tr * (steps_per_transition * RKN_STEP + FRAME + TRANSPORT + NOISE)
    upd_req = M * (JOSEPH + CHI2)
    gain = M * GAIN
    sm_req = tr * (CHOL + SOLVE)
    sm_rest = tr * SMOOTH_UPD
    if precision == 0:
        return int(prop + upd_req + gain + sm_req + sm_rest), 0
    return int(upd_req + sm_req), int(prop + gain + sm_rest)


def algorithmic_bytes(n_tracks, n_states, precision):
    """Inputs read plus outputs written (the per-state record the smoother
    reads back is implementation traffic and is excluded)."""
    per_track = 4 + 6 * 8 + 21 * 8 + 6 * 8 + 21 * 8 + 8 + 4 + 1
    per_state = 4 + 2 * 8 + 3 * 8 + 1
    return int(n_tracks * per_track + n_states * per_state)
