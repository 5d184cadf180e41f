"""Element-wise error measures shared by the GPU parity tests.

Besides the normwise relative error over a whole [T][d(.d)] array, every
parity test asserts an element-wise bound: at every (t, i) (and (t, i, j)),
|gpu - oracle| <= tol * (|oracle| + s), where s is the oracle's posterior
standard deviation of that entry (sqrt of the diagonal of the filtering or
smoothing covariance for a mean or a path; s_i s_j for a covariance entry).
An error confined to a few steps of a long array is then not diluted by the
rest of the array.

The worst values and the FP32 log-alpha errors / MH-decision mismatches seen
by the tests are collected in REPORT, printed at the end of the session
(tests/conftest.py) and written to the JSON file named by AUX_PARITY_REPORT.
"""
import numpy as np

REPORT = {"elementwise": {}, "log_alpha": {}}


def rel(a, b):
    """Normwise relative error ||a - b|| / ||b|| over the whole array."""
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def sd_of(P):
    """Posterior standard deviations [T][d] from covariances [T][d][d]."""
    return np.sqrt(np.maximum(np.einsum("...ii->...i", P), 0.0))


def scaled_max(gpu, ref, s):
    """max over entries of |gpu - ref| / (|ref| + s)."""
    return float(np.max(np.abs(gpu - ref) / (np.abs(ref) + s + 1e-300)))


def vec_err(gpu, ref, P):
    """Element-wise error of a mean or path [T][d] scaled by the posterior sd of P."""
    return scaled_max(gpu, ref, sd_of(P))


def mat_err(gpu, ref, P):
    """Element-wise error of covariances [T][d][d] scaled by s_i s_j."""
    s = sd_of(P)
    return scaled_max(gpu, ref, s[..., :, None] * s[..., None, :])


def note(kind, key, value):
    """Keep the worst value of `kind` seen under `key` for the session report."""
    d = REPORT["elementwise"].setdefault(kind, {})
    d[key] = max(d.get(key, 0.0), float(value))


def note_log_alpha(key, dla_values, mismatches, band):
    """FP32 log-alpha error distribution and MH-decision mismatches of a test."""
    a = np.asarray(dla_values, dtype=np.float64)
    if a.size == 0:
        return
    REPORT["log_alpha"][key] = dict(
        n=int(a.size), p50=float(np.percentile(a, 50)), p90=float(np.percentile(a, 90)),
        max=float(a.max()), decision_mismatches=int(mismatches), near_tie_band=float(band))
