"""Shared helpers of the parity tests: the scaled error measure and patch
extraction for sampled full-size checks."""
import math

import numpy as np


def scales(params, water_height):
    """Natural scales used in the relative error: positions by the domain
    length, velocities by sqrt(|G| H), potentials by |G| H, accelerations by
    |G|, potential rates by C0^2 sqrt(|G| H) / h."""
    g = math.sqrt(sum(v * v for v in params["g"][: params["dim"]])) or 1.0
    H = water_height if water_height > 0 else 1.0
    h = params["h_over_dx"] * params["dx"]
    L = max(params["domain_max"][k] - params["domain_min"][k] for k in range(params["dim"]))
    return {"x": L, "u": math.sqrt(g * H), "phi": g * H, "dudt": g,
            "dphidt": params["c0"] ** 2 * math.sqrt(g * H) / h, "dushift": math.sqrt(g * H),
            "lambda": 1.0}


def scaled_err(a, b, scale):
    """max |a - b| / max(max |b|, scale)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    den = max(float(np.abs(b).max()), scale)
    return float(np.abs(a - b).max()) / den


def patch_indices(x, centres, radius):
    """Indices of particles within ``radius`` (per axis box) of any centre."""
    d, n = x.shape
    keep = np.zeros(n, dtype=bool)
    for c in centres.T:
        m = np.ones(n, dtype=bool)
        for k in range(d):
            m &= np.abs(x[k] - c[k]) <= radius
        keep |= m
    return np.nonzero(keep)[0]
