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
