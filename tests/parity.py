"""Parity helpers shared by the GPU tests.

Metric (per field, over interior cells of all leaves):
    err_v = max|a_v - b_v| / scale_v
with scale_v = max|b_v| for density and energy.  For a momentum component
the scale is max(max|b_v|, max rho c_s): round-off in the pressure part of
the momentum flux is ~eps p per update whatever the flow speed, so when the
momentum itself is tiny (a 1e-4 sound wave, a blast at rest outside its
centre) its own maximum would measure round-off of the O(1) pressure term,
not a difference in the method.  rho c_s is the momentum unit of the flow.
"""
import numpy as np

FIELDS = ("rho", "m1", "m2", "m3", "E")


def momentum_scale(ref: np.ndarray, gamma: float) -> float:
    r = np.asarray(ref, dtype=np.float64)
    rho = r[:, 0]
    ke = 0.5 * (r[:, 1] ** 2 + r[:, 2] ** 2 + r[:, 3] ** 2) / rho
    p = (gamma - 1.0) * (r[:, 4] - ke)
    return float(np.sqrt(np.maximum(gamma * p * rho, 0.0)).max())


def field_errors(gpu: np.ndarray, ref: np.ndarray, gamma: float = 5.0 / 3.0) -> np.ndarray:
    """[5] errors of a state [block, var, k, j, i] under the metric above."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    mscale = momentum_scale(r, gamma)
    out = np.zeros(5)
    for v in range(5):
        scale = max(np.abs(r[:, v]).max(), 1e-300)
        if v in (1, 2, 3):
            scale = max(scale, mscale)
        out[v] = np.abs(g[:, v] - r[:, v]).max() / scale
    return out


def plain_field_errors(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """[5] errors with every field scaled by its own maximum only."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    return np.array([np.abs(g[:, v] - r[:, v]).max() / max(np.abs(r[:, v]).max(), 1e-300)
                     for v in range(5)])


def describe(err) -> str:
    return ", ".join("%s=%.3g" % (f, e) for f, e in zip(FIELDS, err))
