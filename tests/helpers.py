"""Shared helpers for the GPU parity tests (no method arithmetic)."""
import numpy as np


def alpha_rel_err(y, y_ref, x, kappa_s, gamma):
    """Per-ray |dalpha| / max(|alpha_ref|, 1e-3 rms(alpha_ref)).

    alpha = diag(1-ks-g, 1-ks+g) x - y, so dalpha = -(y - y_ref)."""
    x = np.asarray(x).reshape(-1, 2)
    y = np.asarray(y).reshape(-1, 2)
    y_ref = np.asarray(y_ref).reshape(-1, 2)
    a = np.array([1 - kappa_s - gamma, 1 - kappa_s + gamma])
    al = a * x - y_ref
    mag = np.hypot(al[:, 0], al[:, 1])
    floor = 1e-3 * np.sqrt(np.mean(mag ** 2))
    return np.hypot(*(y - y_ref).T) / np.maximum(mag, floor)
