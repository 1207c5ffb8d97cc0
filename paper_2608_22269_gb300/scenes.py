"""Seeded synthetic scenes for the well-balanced WCSPH path.

This module builds inputs only: particle positions on a square (cubic)
lattice, particle types (0 fluid, 1 dummy wall particle), inward wall normals
for the dummies, and the initial state. It holds none of the method's
arithmetic; both the CUDA library and the CPU oracle consume its output.

Scene shapes follow the hydrostatic-tank, dam-break and sloshing workloads
of the paper's Section 4 (tanks filled on a lattice of spacing dx, three
layers of dummy particles behind slip walls). The paper's own experiments
need probe data and geometries that are not available; these scenes stand in
for them with the same structure.

Initial state: U = 0 and the hydrostatic potential of Eq. (eqSol) written
with the free surface at phi = 0, phi = G.x + |G| H, i.e. g (H - y) for
gravity -g along the vertical axis.

Arrays use structure-of-arrays layout: ``x[k, i]`` is component k of
particle i, float64, C-contiguous.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FLUID = 0
DUMMY = 1
BODY = 2  # wall particles of a rigid body translating with params["body_u"]


@dataclasses.dataclass
class Scene:
    params: dict
    x: np.ndarray        # (dim, n) float64
    u: np.ndarray        # (dim, n) float64
    phi: np.ndarray      # (n,) float64
    type: np.ndarray     # (n,) uint8
    normal: np.ndarray   # (dim, n) float64, zero for fluid
    name: str = ""
    water_height: float = 0.0

    @property
    def n(self) -> int:
        return int(self.phi.shape[0])

    @property
    def n_fluid(self) -> int:
        return int(np.count_nonzero(self.type == FLUID))

    @property
    def n_dummy(self) -> int:
        return int(np.count_nonzero(self.type == DUMMY))

    def copy(self) -> "Scene":
        return Scene(dict(self.params), self.x.copy(), self.u.copy(), self.phi.copy(),
                     self.type.copy(), self.normal.copy(), self.name, self.water_height)


def default_params(dim: int, dx: float, c0: float, **kw) -> dict:
    """Physical and numerical parameters; defaults are the paper's values
    (Sec. 4: rho0 = 1000, nu = 1e-4, |G| = 9.81, CFL = 0.2; Sec. 2.3:
    delta = 0.1, R = 0.2, n = 4, lambda threshold 0.75)."""
    g = [0.0, 0.0, 0.0]
    g[dim - 1] = -9.81
    p = dict(dim=dim, dx=dx, h_over_dx=1.3, rho0=1000.0, c0=c0, nu=1e-4, g=g, cfl=0.2,
             delta=0.1, pst_R=0.2, pst_n=4.0, tic_lambda=0.75,
             use_delta=0, use_pst=0, use_tic=0, use_visc=1,
             eos=0, tait_gamma=7.0,
             domain_min=[0.0, 0.0, 0.0], domain_max=[1.0, 1.0, 1.0],
             force_amp=[0.0, 0.0, 0.0], force_period=0.0, fixed_dt=0.0, scheme=0, art_alpha=0.02,
             wall_bc=0, body_u=[0.0, 0.0, 0.0])
    p.update(kw)
    return p


def _hydrostatic_phi(x: np.ndarray, dim: int, g: float, height: float) -> np.ndarray:
    return g * (height - x[dim - 1])


def _assemble(dim, fluid_pts, dummy_pts, dummy_nrm, params, height, name, g):
    x = np.ascontiguousarray(np.concatenate([fluid_pts, dummy_pts], axis=1), dtype=np.float64)
    n = x.shape[1]
    nf = fluid_pts.shape[1]
    typ = np.zeros(n, dtype=np.uint8)
    typ[nf:] = DUMMY
    normal = np.zeros((dim, n), dtype=np.float64)
    normal[:, nf:] = dummy_nrm
    u = np.zeros((dim, n), dtype=np.float64)
    phi = _hydrostatic_phi(x, dim, g, height)
    return Scene(params, x, u, np.ascontiguousarray(phi), typ, np.ascontiguousarray(normal),
                 name, height)


def _box_dummies(dim, counts, layers, top_count, closed_top=False):
    """Dummy lattice points of an open-top box with ``counts[k]`` lattice
    cells per axis (the vertical axis is the last; walls reach ``top_count``
    cells up; with ``closed_top`` a lid closes the box at that height). A
    solid lattice point is a dummy when its lattice distance to the open box
    is at most ``layers``; its normal points to the nearest open lattice
    point. Returns lattice indices (float) and unit normals."""
    pts, nrm = [], []
    ext = [np.arange(-layers, c + layers) for c in counts[:-1]]
    grids = np.meshgrid(*ext, indexing="ij")
    flat = [gr.reshape(-1) for gr in grids]
    for kv in range(-layers, top_count + (layers if closed_top else 0)):
        idx = flat + [np.full(flat[0].shape, kv)]
        off, sign = [], []
        for a, ia in enumerate(idx):
            below = ia < 0
            above = (ia >= counts[a]) if (a < dim - 1 or closed_top) else np.zeros_like(below)
            off.append(np.where(below, -ia, np.where(above, ia - (counts[a] - 1), 0)))
            sign.append(np.where(below, 1.0, -1.0))
        o = np.stack(off).astype(np.int64)
        d2 = (o * o).sum(axis=0)
        sel = (d2 > 0) & (d2 <= layers * layers)
        if not np.any(sel):
            continue
        v = (np.stack(sign) * o)[:, sel]
        v /= np.sqrt((v * v).sum(axis=0))
        pts.append(np.stack([ia[sel] for ia in idx]).astype(np.float64))
        nrm.append(v)
    return np.concatenate(pts, axis=1), np.concatenate(nrm, axis=1)


def box_tank(dim: int, size, dx: float, water, height: float, c0: float | None = None,
             layers: int = 3, name: str = "box", headroom: float = 0.25,
             closed_top: bool = False, **kw) -> Scene:
    """Box tank [0, size[0]] x ... with dummy walls (open top unless
    ``closed_top``); ``water`` is a callable on lattice coordinates (tuple of
    arrays, metres) returning the fluid mask, ``height`` the free-surface
    height used for the initial hydrostatic potential."""
    g = 9.81
    if c0 is None:
        c0 = 10.0 * math.sqrt(g * height)
    counts = [int(round(s / dx)) for s in size]
    axes = [(np.arange(c) + 0.5) * dx for c in counts]
    grids = np.meshgrid(*axes, indexing="ij")
    mask = water(tuple(grids))
    fluid = np.stack([gr[mask] for gr in grids]).astype(np.float64)
    dpts, dnrm = _box_dummies(dim, counts, layers, counts[-1], closed_top)
    dpts = (dpts + 0.5) * dx
    margin = layers * dx + 2.0 * dx
    dmin = [-margin] * dim + [0.0] * (3 - dim)
    dmax = [s + margin for s in size] + [1.0] * (3 - dim)
    dmax[dim - 1] = size[-1] * (1.0 + headroom) + (margin if closed_top else 0.0)
    params = default_params(dim, dx, c0, domain_min=dmin, domain_max=dmax, **kw)
    return _assemble(dim, fluid, dpts, dnrm, params, height, name, g)


def hydrostatic_tank_2d(dx=0.01, width=1.0, depth=0.5, wall=0.6, eos=1, lid=False,
                        **kw) -> Scene:
    """2D flat-bottom hydrostatic tank: water width x depth (5,000 fluid
    particles at dx = 0.01), walls ``wall`` high, three dummy layers; Tait
    EOS (gamma = 7) by default with c0 = 10 sqrt(g H). With ``lid`` the tank
    is closed by dummy particles at the water surface (no free surface)."""
    if lid:
        wall = depth
    return box_tank(2, (width, wall), dx, lambda g_: g_[1] < depth, depth, eos=eos,
                    closed_top=lid, name="hydrostatic_tank_2d" + ("_lid" if lid else ""), **kw)


def topography_tank_2d(kind: str, dx=0.002, width=2.0, depth=0.5, wall=0.6, bump=0.1,
                       bump_width=0.2, sigma=0.05, layers=3, water_column=None,
                       c0=None, **kw) -> Scene:
    """2D basin over bottom topography: ``kind`` in {"flat", "rect", "tri",
    "gauss"}: a rectangular step of height ``bump`` and width ``bump_width``,
    a triangular bump of that height and base, or a Gaussian bump
    bump * exp(-(x - x_c)^2 / (2 sigma^2)), all centred at x_c = width/2.
    ``water_column=(w, h)`` makes a dam-break column at the left wall
    instead of a filled basin. Dummies are the solid lattice points within
    three lattice spacings of the open region; their normal points to the
    nearest open lattice point (ties averaged)."""
    g = 9.81
    xc = 0.5 * width

    def bottom(xs):
        if kind == "flat":
            return np.zeros_like(xs)
        if kind == "rect":
            return np.where(np.abs(xs - xc) <= 0.5 * bump_width, bump, 0.0)
        if kind == "tri":
            return np.maximum(bump * (1.0 - np.abs(xs - xc) / (0.5 * bump_width)), 0.0)
        if kind == "gauss":
            return bump * np.exp(-((xs - xc) ** 2) / (2.0 * sigma * sigma))
        raise ValueError(kind)

    nx, ny = int(round(width / dx)), int(round(wall / dx))
    ii = np.arange(-layers, nx + layers)
    jj = np.arange(-layers, ny)
    I, J = np.meshgrid(ii, jj, indexing="ij")
    X, Y = (I + 0.5) * dx, (J + 0.5) * dx
    solid = (I < 0) | (I >= nx) | (J < 0) | (Y < bottom(X))
    openm = ~solid
    pad = layers
    op = np.pad(openm, pad, constant_values=False)
    best = np.full(openm.shape, np.inf)
    vsum = np.zeros((2,) + openm.shape)
    offs = [(a, b) for a in range(-layers, layers + 1) for b in range(-layers, layers + 1)
            if 0 < a * a + b * b <= layers * layers]
    for a, b in offs:
        sh = op[pad + a: pad + a + openm.shape[0], pad + b: pad + b + openm.shape[1]]
        d2 = float(a * a + b * b)
        better = sh & (d2 < best)
        tie = sh & (d2 == best)
        r = math.sqrt(d2)
        for k, comp in enumerate((a / r, b / r)):
            vsum[k] = np.where(better, comp, np.where(tie, vsum[k] + comp, vsum[k]))
        best = np.where(better, d2, best)
    dummy = solid & np.isfinite(best)
    if water_column is None:
        height = depth
        water = openm & (Y < depth)
    else:
        cw, ch = water_column
        height = ch
        water = openm & (Y < ch) & (X < cw)
    fluid = np.stack([X[water], Y[water]]).astype(np.float64)
    dpts = np.stack([X[dummy], Y[dummy]]).astype(np.float64)
    v = vsum[:, dummy]
    v /= np.sqrt((v * v).sum(axis=0))
    if c0 is None:
        c0 = 10.0 * math.sqrt(g * height)
    margin = layers * dx + 2.0 * dx
    params = default_params(2, dx, c0, domain_min=[-margin, -margin, 0.0],
                            domain_max=[width + margin, wall * 1.25, 1.0], **kw)
    name = f"topography_{kind}" if water_column is None else "dam_break_2d"
    return _assemble(2, fluid, dpts, v, params, height, name, g)


def dam_break_2d(dx=0.002, width=2.0, wall=0.6, column=(0.6, 0.3), **kw) -> Scene:
    """2D dam break: water column released from rest at the left wall of a
    flat basin (45,000 fluid particles at dx = 0.002); delta-SPH, shifting and
    TIC on."""
    kw.setdefault("use_delta", 1)
    kw.setdefault("use_pst", 1)
    kw.setdefault("use_tic", 1)
    return topography_tank_2d("flat", dx=dx, width=width, wall=wall, water_column=column, **kw)


def dam_break_3d(dx=0.0084, box=(3.2, 1.0, 1.0), column=(1.2, 1.0, 0.6), **kw) -> Scene:
    """3D dam break: water column (1.2 x 1.0 x 0.6 m) at one end of a
    3.2 x 1.0 x 1.0 m box; delta-SPH, shifting and TIC on. At dx = 0.0084
    the column holds 143 x 119 x 71 = 1,208,207 fluid particles."""
    kw.setdefault("use_delta", 1)
    kw.setdefault("use_pst", 1)
    kw.setdefault("use_tic", 1)
    cw, cd, ch = column

    def water(g_):
        return (g_[0] < cw) & (g_[1] < cd) & (g_[2] < ch)

    return box_tank(3, box, dx, water, ch, name="dam_break_3d", **kw)


def sloshing_3d(dx=0.00769, tank=(4.0, 2.0, 2.0), depth=1.0, amp=0.01, period=1.5, **kw) -> Scene:
    """3D sloshing tank with horizontal harmonic forcing: tank displacement
    amp * sin(2 pi t / period) along x, water depth ``depth``; delta-SPH,
    shifting and TIC on."""
    kw.setdefault("use_delta", 1)
    kw.setdefault("use_pst", 1)
    kw.setdefault("use_tic", 1)
    return box_tank(3, tank, dx, lambda g_: g_[2] < depth, depth, name="sloshing_3d",
                    force_amp=[amp, 0.0, 0.0], force_period=period, **kw)


def moving_body(dim: int = 2, dx: float = 0.01, tank=(1.0, 0.6), depth: float = 0.4,
                body=(0.12, 0.12), center=(0.3, 0.2), body_u=(0.5, 0.0), **kw) -> Scene:
    """A rigid rectangular (box-shaped in 3D) body of wall particles (type
    BODY) translating with the prescribed velocity ``body_u`` through a tank
    of water at rest: the tank of ``box_tank`` with the water up to ``depth``,
    the body a solid block of lattice points (the fluid there removed), each
    body particle's normal pointing out of the block towards its nearest face
    (averaged over equally near faces). ``tank``, ``body``, ``center`` and
    ``body_u`` have ``dim`` entries; the vertical axis is the last."""
    tank, body, center, body_u = (tuple(v[:dim]) for v in (tank, body, center, body_u))
    sc = box_tank(dim, tank, dx, lambda g_: g_[dim - 1] < depth, depth, name="moving_body",
                  body_u=list(body_u) + [0.0] * (3 - dim), **kw)
    lo = np.array([c - b / 2 for c, b in zip(center, body)])[:, None]
    hi = np.array([c + b / 2 for c, b in zip(center, body)])[:, None]
    inside = np.all((sc.x >= lo) & (sc.x <= hi), axis=0)
    in_fluid = inside & (sc.type == FLUID)
    keep = ~inside | (sc.type != FLUID)
    bx = sc.x[:, in_fluid]
    # outward normal: towards the nearest face(s) of the block
    dist = np.concatenate([bx - lo, hi - bx])  # 2 dim rows: distance to each face
    dmin = dist.min(axis=0)
    near = np.isclose(dist, dmin[None, :], rtol=0, atol=1e-9 * dx)
    sign = np.concatenate([-np.ones((dim, 1)), np.ones((dim, 1))])
    nrm = np.zeros((dim, bx.shape[1]))
    for k in range(2 * dim):
        nrm[k % dim] += np.where(near[k], sign[k, 0], 0.0)
    nrm /= np.sqrt((nrm * nrm).sum(axis=0))[None, :]
    x = np.concatenate([sc.x[:, keep], bx], axis=1)
    typ = np.concatenate([sc.type[keep], np.full(bx.shape[1], BODY, dtype=np.uint8)])
    normal = np.concatenate([sc.normal[:, keep], nrm], axis=1)
    u = np.zeros_like(x)
    u[:, typ == BODY] = np.asarray(body_u, dtype=np.float64)[:, None]
    phi = np.concatenate([sc.phi[keep], _hydrostatic_phi(bx, dim, 9.81, depth)])
    return Scene(sc.params, np.ascontiguousarray(x), u, np.ascontiguousarray(phi), typ,
                 np.ascontiguousarray(normal), "moving_body", depth)


def jitter(scene: Scene, amount: float, seed: int = 2026, fluid_only: bool = True) -> Scene:
    """Uniform random displacement of up to ``amount`` * dx per axis."""
    s = scene.copy()
    rng = np.random.default_rng(seed)
    dx = s.params["dx"]
    d = rng.uniform(-amount * dx, amount * dx, size=s.x.shape)
    if fluid_only:
        d[:, s.type != FLUID] = 0.0
    s.x = np.ascontiguousarray(s.x + d)
    return s


def random_box(n: int, dim: int, side: float, dx: float, seed: int = 2026,
               on_faces: bool = True) -> Scene:
    """Uniform random points in a cube, all fluid, for neighbour tests; with
    ``on_faces`` some coordinates are snapped exactly onto cell faces and
    some pairs are placed at exactly r = 2h along an axis."""
    rng = np.random.default_rng(seed)
    p = default_params(dim, dx, 20.0, domain_min=[0.0] * 3, domain_max=[side] * dim + [1.0] * (3 - dim))
    x = rng.uniform(0.0, side, size=(dim, n))
    if on_faces:
        R = 2.0 * p["h_over_dx"] * dx
        k = max(1, n // 10)
        cells = np.floor(x[:, :k] / R)
        x[:, :k] = np.minimum(cells * R, side)
        m = max(1, n // 20)
        src = rng.integers(0, n, size=m)
        dst = rng.integers(0, n, size=m)
        x[:, dst] = x[:, src]
        x[0, dst] = np.minimum(x[0, src] + R, side)
    x = np.ascontiguousarray(x)
    z = np.zeros((dim, n))
    return Scene(p, x, z.copy(), np.zeros(n), np.zeros(n, dtype=np.uint8), z.copy(),
                 "random_box", 0.0)


def lattice_cloud(dim: int, n_side: int, dx: float = 0.01, jitter_amount: float = 0.0,
                  seed: int = 2026, c0: float = 20.0, **kw) -> Scene:
    """All-fluid square (cubic) lattice of n_side^dim particles with no walls
    and zero gravity, optionally jittered, for operator tests."""
    ax = (np.arange(n_side) + 0.5) * dx
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    x = np.stack([g_.reshape(-1) for g_ in grids]).astype(np.float64)
    if jitter_amount > 0:
        rng = np.random.default_rng(seed)
        x = x + rng.uniform(-jitter_amount * dx, jitter_amount * dx, size=x.shape)
    n = x.shape[1]
    side = n_side * dx
    kw.setdefault("g", [0.0, 0.0, 0.0])
    p = default_params(dim, dx, c0, domain_min=[-dx] * dim + [0.0] * (3 - dim),
                       domain_max=[side + dx] * dim + [1.0] * (3 - dim), **kw)
    z = np.zeros((dim, n))
    return Scene(p, np.ascontiguousarray(x), z.copy(), np.zeros(n), np.zeros(n, dtype=np.uint8),
                 z.copy(), "lattice_cloud", 0.0)
