"""Error metrics of the paper (test infrastructure only).

Eq. 12: normalised absolute error |S_lbm - S_ref| / max_theta S_ref.
Eq. 13: normalised RMS error sqrt(mean((S_lbm - S_ref)^2)) / max_theta S_ref.
"""
import numpy as np


def normalized_abs_error(s_lbm, s_ref):
    s_lbm, s_ref = np.asarray(s_lbm, float), np.asarray(s_ref, float)
    return np.abs(s_lbm - s_ref) / np.max(s_ref)


def normalized_rms(s_lbm, s_ref):
    s_lbm, s_ref = np.asarray(s_lbm, float), np.asarray(s_ref, float)
    return float(np.sqrt(np.mean((s_lbm - s_ref) ** 2)) / np.max(s_ref))


def rel_l2(a, b):
    """Relative L2 difference ||a - b|| / ||b|| (parity metric)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))
