"""Parity helpers shared by the GPU tests.

Two metrics, per field, over interior cells of all leaves:

plain   err_v = max|a_v - b_v| / max|b_v|           (every field by its own max)
scaled  err_v = max|a_v - b_v| / scale_v,  scale_v = max|b_v| for density and
        energy, max(max|b_v|, max rho c_s) for a momentum component.

They are the same for density and energy.  For momentum, round-off in the
pressure part of the momentum flux is ~eps p per update whatever the flow
speed, so when the momentum itself is tiny (a 1e-4 sound wave, a blast at rest
outside its centre) its own maximum measures round-off of the O(1) pressure
term, not a difference in the method; rho c_s is the momentum unit of the
flow.  The tests assert the scaled metric; every call also computes the plain
one, returns it on request and, when the environment variable PH_PARITY_LOG
names a file, appends both per test to it (JSON lines), so that a GPU run
records the plain momentum errors beside the asserted ones.
"""
import json
import os

import numpy as np

FIELDS = ("rho", "m1", "m2", "m3", "E")


def momentum_scale(ref: np.ndarray, gamma: float) -> float:
    r = np.asarray(ref, dtype=np.float64)
    rho = r[:, 0]
    ke = 0.5 * (r[:, 1] ** 2 + r[:, 2] ** 2 + r[:, 3] ** 2) / rho
    p = (gamma - 1.0) * (r[:, 4] - ke)
    return float(np.sqrt(np.maximum(gamma * p * rho, 0.0)).max())


def plain_field_errors(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """[5] errors with every field scaled by its own maximum only."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    return np.array([np.abs(g[:, v] - r[:, v]).max() / max(np.abs(r[:, v]).max(), 1e-300)
                     for v in range(5)])


def _record(scaled: np.ndarray, plain: np.ndarray) -> None:
    path = os.environ.get("PH_PARITY_LOG")
    if not path:
        return
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    with open(path, "a") as f:
        f.write(json.dumps({"test": test, "scaled": [float(x) for x in scaled],
                            "plain": [float(x) for x in plain]}) + "\n")


def field_errors(gpu: np.ndarray, ref: np.ndarray, gamma: float = 5.0 / 3.0,
                 with_plain: bool = False):
    """[5] scaled errors of a state [block, var, k, j, i] (and the plain
    ones as a second result when with_plain)."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    mscale = momentum_scale(r, gamma)
    plain = plain_field_errors(g, r)
    out = np.zeros(5)
    for v in range(5):
        scale = max(np.abs(r[:, v]).max(), 1e-300)
        if v in (1, 2, 3):
            scale = max(scale, mscale)
        out[v] = np.abs(g[:, v] - r[:, v]).max() / scale
    # density and energy: the scaled metric is the plain one
    assert out[0] == plain[0] and out[4] == plain[4]
    _record(out, plain)
    return (out, plain) if with_plain else out


def describe(err, plain=None) -> str:
    s = ", ".join("%s=%.3g" % (f, e) for f, e in zip(FIELDS, err))
    if plain is not None:
        s += " (plain: " + ", ".join("%s=%.3g" % (f, e) for f, e in zip(FIELDS, plain)) + ")"
    return s
