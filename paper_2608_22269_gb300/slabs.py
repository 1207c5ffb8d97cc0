"""Slab decomposition of the well-balanced WCSPH step over several ranks.

The paper leaves multi-GPU runs to future work (Conclusions); this module is
the decomposition of one particle set into slabs of whole neighbour-build
cells (cell size R = 2h) along one axis, one slab per rank, with the
per-stage exchange the method needs and nothing more:

  step start   each rank sends to each neighbouring rank its particles in
               the two cells next to their common face (ghosts: fluid, wall
               and body particles with x, U, phi, mass, type, normal). Two
               cells, because a wall particle within 2h of an owned particle
               takes its potential from its nearest fluid particle, which
               can lie up to 2h further out (Sec. 2.4, Eq. phiBn).
               U_max over the owned fluid particles: allreduce max.
  stage 1      on owned + ghosts, at the step's start time, the time step
               from the global U_max (the same on every rank).
  exchange     each owner sends the stage-1 state (x, U, phi) of the ghosts
               it sent; the receivers overwrite them. U_max of stage 2:
               allreduce max.
  stage 2      the owned particles keep their results; ghosts are dropped.
  migration    owned particles whose cell left the slab go to the rank that
               owns it (a neighbour: a particle moves far less than a cell
               per step).

A subdomain lists its particles in ascending global id, so that the ties of
the nearest-fluid search of the wall update (smallest id wins) resolve as in
the single domain. The compute backend runs the stages (GpuBackend: the CUDA
library's wbsph_stage and wbsph_update_particles); the communicator moves
the ghosts and migrants and reduces U_max (TorchComm: torch.distributed
send/recv and all_reduce, gloo on CPU tensors or NCCL on device tensors).
"""
from __future__ import annotations

import math

import numpy as np

FLUID = 0


def slab_bounds(params, x, nranks, axis, min_cells=2):
    """Cell indices b_0 = 0 < b_1 < ... < b_W = N of the slabs along `axis`
    (rank r owns cells [b_r, b_{r+1})), balanced by the particle counts of
    the scene and at least `min_cells` cells wide each (a slab never narrower
    than the ghost band, so ghosts come from the neighbouring ranks only)."""
    R = 2.0 * params["h_over_dx"] * params["dx"]
    lo, hi = params["domain_min"][axis], params["domain_max"][axis]
    ncell = int(math.floor((hi - lo) / R)) + 1
    if ncell < min_cells * nranks:
        raise ValueError(f"{ncell} cells along axis {axis} cannot hold {nranks} slabs of {min_cells} cells")
    c = np.clip(np.floor((x[axis] - lo) / R).astype(np.int64), 0, ncell - 1)
    cum = np.cumsum(np.bincount(c, minlength=ncell))
    b = [0]
    for r in range(1, nranks):
        cut = int(np.searchsorted(cum, cum[-1] * r / nranks)) + 1
        cut = max(cut, b[-1] + min_cells)
        cut = min(cut, ncell - min_cells * (nranks - r))
        b.append(cut)
    b.append(ncell)
    return np.array(b, dtype=np.int64)


class Slab:
    """The particles a rank owns and the stepping of its slab.

    scene: the full initial scene (every rank builds the same one; each keeps
    its slab); comm: rank, size, exchange(left, right) and allreduce_max;
    backend: load, stage, get, update, dt (see GpuBackend)."""

    def __init__(self, scene, comm, backend, axis=None, ghost_cells=2):
        self.params = dict(scene.params)
        self.dim = int(self.params["dim"])
        self.comm = comm
        self.backend = backend
        if axis is None:
            ext = [self.params["domain_max"][k] - self.params["domain_min"][k] for k in range(self.dim)]
            axis = int(np.argmax(ext))
        self.axis = axis
        self.R = 2.0 * self.params["h_over_dx"] * self.params["dx"]
        self.ghost_cells = int(ghost_cells)
        self.bounds = slab_bounds(self.params, scene.x, comm.size, axis, self.ghost_cells)
        self.ncell = int(self.bounds[-1])
        own = self._owner(scene.x) == comm.rank
        gid = np.nonzero(own)[0]
        self.state = {"gid": gid.astype(np.int64), "x": scene.x[:, own].copy(), "u": scene.u[:, own].copy(),
                      "phi": scene.phi[own].copy(), "type": scene.type[own].copy(),
                      "normal": scene.normal[:, own].copy()}
        self.t = 0.0
        self.steps = 0

    # -- geometry --------------------------------------------------------------------------
    def _cell(self, x):
        lo = self.params["domain_min"][self.axis]
        return np.clip(np.floor((x[self.axis] - lo) / self.R).astype(np.int64), 0, self.ncell - 1)

    def _owner(self, x):
        return np.searchsorted(self.bounds, self._cell(x), side="right") - 1

    # -- packing of particle records ------------------------------------------------------------
    def _pack(self, sel):
        s = self.state
        d = self.dim
        rec = np.empty((sel.size, 3 + 3 * d), dtype=np.float64)
        rec[:, 0] = s["gid"][sel]
        rec[:, 1:1 + d] = s["x"][:, sel].T
        rec[:, 1 + d:1 + 2 * d] = s["u"][:, sel].T
        rec[:, 1 + 2 * d] = s["phi"][sel]
        rec[:, 2 + 2 * d] = s["type"][sel]
        rec[:, 3 + 2 * d:] = s["normal"][:, sel].T
        m = np.empty((sel.size, 1))
        m[:, 0] = s["mass"][sel]
        return np.hstack([rec, m])

    def _unpack(self, rec):
        d = self.dim
        return {"gid": rec[:, 0].astype(np.int64), "x": np.ascontiguousarray(rec[:, 1:1 + d].T),
                "u": np.ascontiguousarray(rec[:, 1 + d:1 + 2 * d].T), "phi": rec[:, 1 + 2 * d].copy(),
                "type": rec[:, 2 + 2 * d].astype(np.uint8),
                "normal": np.ascontiguousarray(rec[:, 3 + 2 * d:3 + 3 * d].T), "mass": rec[:, 3 + 3 * d].copy()}

    @staticmethod
    def _concat(parts):
        out = {}
        for k in parts[0]:
            arrs = [p[k] for p in parts]
            out[k] = np.concatenate(arrs, axis=-1) if arrs[0].ndim == 2 else np.concatenate(arrs)
        return out

    def _umax(self, u, typ):
        f = typ == FLUID
        local = float(np.sqrt((u[:, f] ** 2).sum(0).max())) if f.any() else 0.0
        return self.comm.allreduce_max(local)

    # -- one SSP-RK2 step -------------------------------------------------------------------------
    def step(self):
        s = self.state
        r, W = self.comm.rank, self.comm.size
        if s.get("mass") is None:
            self.backend.load(s["x"], s["u"], s["phi"], None, s["type"], s["normal"])
            s["mass"] = self.backend.get("mass")
        # ghosts: the owned particles within ghost_cells cells of a shared
        # face, by coordinate with a margin of 1e-9 cells, so that rounding of
        # the cell index cannot drop one that is needed
        lo = self.params["domain_min"][self.axis]
        xa = s["x"][self.axis]
        margin = 1e-9 * self.R
        to_left = (np.nonzero(xa < lo + (self.bounds[r] + self.ghost_cells) * self.R + margin)[0] if r > 0
                   else np.zeros(0, np.int64))
        to_right = (np.nonzero(xa >= lo + (self.bounds[r + 1] - self.ghost_cells) * self.R - margin)[0] if r < W - 1
                    else np.zeros(0, np.int64))
        gl, gr = self.comm.exchange(self._pack(to_left), self._pack(to_right))
        gl = gl if gl is not None else np.zeros((0, 4 + 3 * self.dim))
        gr = gr if gr is not None else np.zeros((0, 4 + 3 * self.dim))
        own = {k: s[k] for k in ("gid", "x", "u", "phi", "type", "normal", "mass")}
        allp = self._concat([own, self._unpack(gl), self._unpack(gr)])
        order = np.argsort(allp["gid"], kind="stable")          # ascending global id
        sub = {k: (v[:, order] if v.ndim == 2 else v[order]) for k, v in allp.items()}
        pos = np.empty(order.size, dtype=np.int64)
        pos[order] = np.arange(order.size)                      # concatenated index -> subdomain index
        n_own = s["gid"].size
        n_gl = gl.shape[0]
        own_pos = pos[:n_own]
        ghost_left_pos = pos[n_own:n_own + n_gl]
        ghost_right_pos = pos[n_own + n_gl:]
        self.backend.load(sub["x"], sub["u"], sub["phi"], sub["mass"], sub["type"], sub["normal"])
        # stage 1
        self.backend.stage(1, self.t, 0.0, self._umax(s["u"], s["type"]))
        dt = self.backend.dt()
        x1, u1, phi1 = self.backend.get("x"), self.backend.get("u"), self.backend.get("phi")
        # the ghosts' stage-1 state from their owners
        sl = own_pos[to_left]
        sr = own_pos[to_right]
        pack1 = lambda idx: np.hstack([x1[:, idx].T, u1[:, idx].T, phi1[idx][:, None]])  # noqa: E731
        rl, rr = self.comm.exchange(pack1(sl), pack1(sr))
        d = self.dim
        upd_ids, upd = [], []
        for ids, rec in ((ghost_left_pos, rl), (ghost_right_pos, rr)):
            if rec is not None and len(rec):
                upd_ids.append(ids)
                upd.append(rec)
        if upd:
            rec = np.vstack(upd)
            self.backend.update(np.concatenate(upd_ids), np.ascontiguousarray(rec[:, :d].T),
                                np.ascontiguousarray(rec[:, d:2 * d].T), rec[:, 2 * d].copy())
        u1_own = u1[:, own_pos]
        self.backend.stage(2, self.t, 0.0, self._umax(u1_own, s["type"]))
        x2, u2, phi2 = self.backend.get("x"), self.backend.get("u"), self.backend.get("phi")
        s["x"], s["u"], s["phi"] = x2[:, own_pos], u2[:, own_pos], phi2[own_pos]
        self.t += dt
        self.steps += 1
        # migration to the neighbouring slabs
        dest = self._owner(s["x"])
        if np.any(np.abs(dest - r) > 1):
            raise RuntimeError("a particle moved further than one slab in one step")
        ml, mr = np.nonzero(dest == r - 1)[0], np.nonzero(dest == r + 1)[0]
        il, ir = self.comm.exchange(self._pack(ml), self._pack(mr))
        keep = dest == r
        kept = {k: (v[:, keep] if v.ndim == 2 else v[keep]) for k, v in s.items()}
        arrived = [self._unpack(a) for a in (il, ir) if a is not None and len(a)]
        self.state = self._concat([kept] + arrived) if arrived else kept
        return dt

    def owned(self):
        """(gid, x, u, phi, type) of the owned particles."""
        s = self.state
        return s["gid"], s["x"], s["u"], s["phi"], s["type"]


class GpuBackend:
    """The CUDA library as the compute of a slab (one handle per rank)."""

    def __init__(self, params, water_height=0.0, device=0):
        from . import wbsph
        self.sim = wbsph.Sim(params, water_height=water_height, device=device)

    def load(self, x, u, phi, mass, typ, normal):
        self.sim.set_particles(x, u, phi, typ, normal, mass)

    def stage(self, stage, t, dt, umax):
        self.sim.stage(stage, t, dt, umax)

    def get(self, field):
        return self.sim.get(field)

    def update(self, ids, x, u, phi):
        self.sim.update_particles(ids, x, u, phi)

    def dt(self):
        return self.sim.stats()["dt"]

    def close(self):
        self.sim.close()


class TorchComm:
    """Neighbour exchange and U_max reduction over torch.distributed (the
    default group): gloo moves CPU tensors, NCCL device tensors."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()
        self.device = device if device is not None else torch.device("cpu")

    def _t(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(self.device)

    def exchange(self, to_left, to_right):
        """Send to_left to rank - 1 and to_right to rank + 1 (2-D float64
        arrays of records); return what those neighbours sent here."""
        torch, dist = self.torch, self.dist
        nbrs = [(self.rank - 1, to_left), (self.rank + 1, to_right)]
        nbrs = [(q, a) for q, a in nbrs if 0 <= q < self.size]
        shapes = {}
        reqs = []
        for q, a in nbrs:  # record counts and widths first
            a = np.zeros((0, 1)) if a is None else a
            reqs.append(dist.isend(self._t(np.array(a.shape, dtype=np.float64)), q))
            shapes[q] = torch.zeros(2, dtype=torch.float64, device=self.device)
            reqs.append(dist.irecv(shapes[q], q))
        for rq in reqs:
            rq.wait()
        reqs, bufs = [], {}
        for q, a in nbrs:
            a = np.zeros((0, 1)) if a is None else a
            if a.size:
                reqs.append(dist.isend(self._t(a), q))
            m, w = (int(v) for v in shapes[q].cpu().tolist())
            bufs[q] = torch.zeros((m, w), dtype=torch.float64, device=self.device)
            if m * w:
                reqs.append(dist.irecv(bufs[q], q))
        for rq in reqs:
            rq.wait()
        got = {q: bufs[q].cpu().numpy() for q in bufs}
        return got.get(self.rank - 1), got.get(self.rank + 1)

    def allreduce_max(self, v):
        t = self.torch.tensor([float(v)], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())
