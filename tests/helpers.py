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
    """Indices (ascending) of particles within ``radius`` per axis (a box) of
    any centre. Particles are binned into cells of side ``radius`` once, so
    each centre only looks at the 3^d cells around it."""
    x = np.asarray(x, dtype=np.float64)
    centres = np.asarray(centres, dtype=np.float64).reshape(x.shape[0], -1)
    d, n = x.shape
    if n == 0 or centres.shape[1] == 0:
        return np.zeros(0, dtype=np.int64)
    lo = x.min(axis=1)
    cell = np.floor((x - lo[:, None]) / radius).astype(np.int64)
    ext = cell.max(axis=1) + 1
    key = np.zeros(n, dtype=np.int64)
    for k in reversed(range(d)):
        key = key * ext[k] + cell[k]
    order = np.argsort(key, kind="stable")
    skey = key[order]
    offsets = np.array(np.meshgrid(*[[-1, 0, 1]] * d, indexing="ij")).reshape(d, -1)
    found = []
    for c in centres.T:
        cc = np.floor((c - lo) / radius).astype(np.int64)
        for off in offsets.T:
            q = cc + off
            if np.any(q < 0) or np.any(q >= ext):
                continue
            kq = 0
            for k in reversed(range(d)):
                kq = kq * int(ext[k]) + int(q[k])
            a, b = np.searchsorted(skey, [kq, kq + 1])
            cand = order[a:b]
            m = np.ones(cand.size, dtype=bool)
            for k in range(d):
                m &= np.abs(x[k, cand] - c[k]) <= radius
            found.append(cand[m])
    if not found:
        return np.zeros(0, dtype=np.int64)
    return np.unique(np.concatenate(found))


def dynamic(scene, seed=5, amp=0.3, jitter=0.15):
    """A seeded non-equilibrium state of a scene: fluid positions jittered by
    ``jitter`` dx, normally distributed fluid velocities of deviation ``amp``
    m/s and potential noise of deviation 0.05 m^2/s^2."""
    from paper_2608_22269_gb300 import scenes as S
    s = S.jitter(scene, jitter, seed=seed)
    rng = np.random.default_rng(seed)
    f = s.type == 0
    s.u[:, f] = amp * rng.normal(size=(s.x.shape[0], int(f.sum())))
    s.phi[f] += 0.05 * rng.normal(size=int(f.sum()))
    return s


def sample_fluid(scene, k, seed=11, band=2.5):
    """About ``k`` distinct fluid particles, seeded: half from the band of
    ``band`` dx along the faces of the fluid's bounding box (walls, free
    surface, corners: where dummies and the TIC branch enter), half from the
    interior."""
    f = np.nonzero(scene.type == 0)[0]
    xf = scene.x[:, f]
    lo, hi = xf.min(axis=1), xf.max(axis=1)
    w = band * scene.params["dx"]
    near = np.zeros(f.size, dtype=bool)
    for a in range(xf.shape[0]):
        near |= (xf[a] - lo[a] < w) | (hi[a] - xf[a] < w)
    rng = np.random.default_rng(seed)
    pick = []
    for pool, m in ((f[near], k // 2), (f[~near], k - k // 2)):
        if pool.size:
            pick.append(rng.choice(pool, size=min(m, pool.size), replace=False))
    return np.unique(np.concatenate(pick)) if pick else np.zeros(0, dtype=np.int64)
