"""Algorithmic work of the fit, for roofline accounting.

Counts are floating-point operations (an FMA counts 2; a square root,
reciprocal or transcendental call counts 1) of the arithmetic the method
needs in the structure-exploiting form the kernels use: covariances stored
as 21 values, H a projection onto (loc0, loc1), F with its trivial q/p row and
time column, constant field along z, solves instead of explicit inverses.

Per track: n states, n-1 transitions (state k-1 -> k), m measured states and
n-1 smoother steps.

FP64 path (everything in double precision):
  per transition
    RKN_STEP  one RKN4 step with its exact Jacobian columns (x4 per transition
              in every workload: one straight-line step + 3 Newton steps)
    FRAME     bound->free, plane distances, path correction, free->bound,
              assembly of F
    TRANSPORT Bm = F Cf (rows 0-3 and 5, five terms each) and Cp = Bm F^T
    NOISE     Highland width and the two variances
  per measured state
    GAIN      S, det, 1/det, residual, chi2, K, x_f
    JOSEPH    W = S K^T - H Cp (12 x 2 FMA) and Cf (21 x 4 FMA), S
  per smoother step
    CHOL      6x6 Cholesky (35 FMA, 15 mul, 6 rsqrt)
    SOLVE6    six forward/backward substitution pairs for Cp^-1 Bm
    RTS_UPD   xs update and Cs = Cf + A dC A^T

Mixed path: the double-precision part the method requires is
    per measured state   JOSEPH_64 + CHI2 (the Joseph update without its
                         second-order term K W, which is O(eps32 |Cp|) and
                         summed in FP32: JOSEPH_KW32)
    per smoother step    INV_COLS + NRANK   (the (phi, theta) columns of
                         Cp^-1 by a 4x4 LDL^T of the loc/q/p/t block, two
                         solves and the 2x2 Schur complement of the angle
                         block; N = Q - Q Cp^-1 Q)
and everything else runs in FP32 (counted as fp32 work).
"""

RKN_STEP = 58 + 3 * 56 + 50 + 3
FRAME = 22 + 4 * 15 + 14 + 100 + 100 + 9
TRANSPORT = 2 * 156 + 2 * 105
NOISE = 15
GAIN = 80
JOSEPH = 2 * 12 * 2 + 2 * 21 * 4 + 3
JOSEPH_KW32 = 2 * 21 * 2
JOSEPH_64 = JOSEPH - JOSEPH_KW32
CHI2 = 16
CHOL = 2 * 35 + 15 + 6
SOLVE6 = 6 * 2 * 36
SOLVE2 = 48 + 42
# 4x4 LDL^T (pivots 6 FMA, U 4 FMA, L 6 mul, 4 reciprocals), two solves
# (unit-lower 6 FMA, D^-1 4 mul, unit-upper 6 FMA each), Schur complement
# (12 FMA), its inverse (det 3, 1/det 1, 3 mul), off-block columns
# (8 x (FMA + mul)) -> flops
INV_COLS = (2 * 6 + 2 * 4 + 6 + 4) + 2 * (2 * 6 + 4 + 2 * 6) + 2 * 12 + 7 + 8 * 3
NRANK = 7
RTS_UPD = 84 + 21 + 2 * 216 + 2 * 126 + 21
# FP32 side of the mixed smoother: F^-1 (block form), gain A, xs, Cs
MIXED_SMOOTH_FP32 = 120 + 2 * 72 + 2 * 36 + 2 * 216 + 2 * 126 + 60


def _counts(offsets, is_hole):
    import numpy as np
    o = np.asarray(offsets, dtype=np.int64)
    n = np.diff(o)
    meas = (np.asarray(is_hole) == 0).astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(meas)])
    m = cs[o[1:]] - cs[o[:-1]]
    return int(np.maximum(n - 1, 0).sum()), int(m.sum())


def batch_flops(offsets, is_hole, precision, steps_per_transition=4):
    """(fp64_flops, fp32_flops) of one fit of a batch; precision 0 = FP64
    path, 1 = mixed path."""
    tr, M = _counts(offsets, is_hole)
    prop = tr * (steps_per_transition * RKN_STEP + FRAME + TRANSPORT + NOISE)
    if precision == 0:
        return prop + M * (GAIN + JOSEPH) + tr * (CHOL + SOLVE6 + RTS_UPD), 0
    f64 = M * (JOSEPH_64 + CHI2) + tr * (INV_COLS + NRANK)
    f32 = prop + M * (GAIN - CHI2 + JOSEPH_KW32) + tr * MIXED_SMOOTH_FP32
    return f64, f32


def algorithmic_bytes(offsets, is_hole):
    """Inputs read plus outputs written once (the per-state record the
    smoother reads back is implementation traffic and is excluded)."""
    import numpy as np
    T = len(offsets) - 1
    M = int(np.asarray(offsets)[-1])
    per_track = 4 + 6 * 8 + 21 * 8 + 6 * 8 + 21 * 8 + 8 + 4 + 1
    per_state = 4 + 2 * 8 + 3 * 8 + 1
    return T * per_track + M * per_state
