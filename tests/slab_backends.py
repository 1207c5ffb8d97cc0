"""Test-side pieces of the slab decomposition: the oracle as a slab's compute
backend, and an in-process communicator over threads (ranks as threads of
one process, for tests that keep every rank in one interpreter)."""
import threading

import numpy as np

from oracle import oracle as O

FLUID, BODY = 0, 2


class OracleBackend:
    """One SSP-RK2 stage of a subdomain on the oracle (Sec. 2.3): the rates
    of oracle.stage_rates with the global U_max, the time step of the
    three-condition rule from the global U_max, and the stage updates of the
    oracle's full step written out for one stage at a time."""

    def __init__(self, params):
        self.p = dict(params)
        self.d = int(params["dim"])

    def load(self, x, u, phi, mass, typ, normal):
        self.x, self.u, self.phi = (np.array(a, dtype=np.float64) for a in (x, u, phi))
        self.type = np.array(typ, dtype=np.uint8)
        self.normal = np.array(normal, dtype=np.float64)
        self.m = O.mass(self.p, self.phi) if mass is None else np.array(mass, dtype=np.float64)

    def stage(self, stage, t, dt, umax):
        d = self.d
        if stage == 1:
            if dt > 0:
                self._dt = dt
            else:  # the rule on one fluid particle moving at the global U_max
                one = np.zeros((d, 1))
                one[0, 0] = umax
                self._dt = O.time_step(self.p, one, np.zeros(1, np.uint8))
            self.x0, self.u0, self.p0 = self.x.copy(), self.u.copy(), self.phi.copy()
        dt = self._dt
        r = O.stage_rates(self.p, self.x, self.u, self.phi, self.m, self.type, self.normal,
                          t if stage == 1 else t + dt, umax=umax)
        self.u, self.phi = r["u"], r["phi"]            # walls after their update
        fl, bd = self.type == FLUID, self.type == BODY
        bu = np.asarray(self.p.get("body_u", [0.0, 0.0, 0.0])[:d], dtype=np.float64)[:, None]
        ra, rp, rs = r["dudt"], r["dphidt"], r["dushift"]
        if stage == 1:
            self.x[:, bd] = self.x0[:, bd] + dt * bu
            self.x[:, fl] = self.x0[:, fl] + dt * (self.u0[:, fl] + rs[:, fl])
            self.u[:, fl] = self.u0[:, fl] + dt * ra[:, fl]
            self.phi[fl] = self.p0[fl] + dt * rp[fl]
        else:
            self.x[:, bd] = 0.5 * self.x0[:, bd] + 0.5 * (self.x[:, bd] + dt * bu)
            x1, u1 = self.x[:, fl], self.u[:, fl]
            self.x[:, fl] = 0.5 * self.x0[:, fl] + 0.5 * (x1 + dt * (u1 + rs[:, fl]))
            self.u[:, fl] = 0.5 * self.u0[:, fl] + 0.5 * (u1 + dt * ra[:, fl])
            self.phi[fl] = 0.5 * self.p0[fl] + 0.5 * (self.phi[fl] + dt * rp[fl])

    def get(self, field):
        return {"x": self.x, "u": self.u, "phi": self.phi, "mass": self.m}[field].copy()

    def update(self, ids, x, u, phi):
        # the argument contract of the library's wbsph_update_particles, so
        # the slab driver's ghost refresh is held to it on CPU ranks too
        from paper_2608_22269_gb300.wbsph import check_update_args
        ids, x, u, phi = check_update_args(ids, x, u, phi, self.x.shape[0], self.x.shape[1])
        ids = ids.astype(np.int64)
        self.x[:, ids], self.u[:, ids], self.phi[ids] = x, u, phi

    def dt(self):
        return self._dt


class ThreadComm:
    """Communicator of one rank among `size` threads sharing a ThreadHub."""

    def __init__(self, hub, rank):
        self.hub, self.rank, self.size = hub, rank, hub.size

    def exchange(self, to_left, to_right):
        hub, r = self.hub, self.rank
        if r > 0:
            hub.put(r, r - 1, to_left)
        if r < self.size - 1:
            hub.put(r, r + 1, to_right)
        left = hub.get(r - 1, r) if r > 0 else None
        right = hub.get(r + 1, r) if r < self.size - 1 else None
        return left, right

    def allreduce_max(self, v):
        return self.hub.allreduce_max(self.rank, v)


class ThreadHub:
    def __init__(self, size, timeout=600.0):
        self.size, self.timeout = size, timeout
        self.cv = threading.Condition()
        self.box = {}
        self.vals = {}
        self.rounds = [0] * size
        self.failed = False

    def put(self, src, dst, a):
        with self.cv:
            self.box.setdefault((src, dst), []).append(None if a is None else np.array(a, copy=True))
            self.cv.notify_all()

    def get(self, src, dst):
        with self.cv:
            if not self.cv.wait_for(lambda: self.failed or self.box.get((src, dst)), timeout=self.timeout):
                raise TimeoutError(f"no message from rank {src} to rank {dst}")
            if self.failed:
                raise RuntimeError("another rank failed")
            return self.box[(src, dst)].pop(0)

    def allreduce_max(self, rank, v):
        k = self.rounds[rank]
        self.rounds[rank] += 1
        with self.cv:
            self.vals.setdefault(k, []).append(float(v))
            self.cv.notify_all()
            if not self.cv.wait_for(lambda: self.failed or len(self.vals[k]) == self.size,
                                    timeout=self.timeout):
                raise TimeoutError("allreduce incomplete")
            if self.failed:
                raise RuntimeError("another rank failed")
            return max(self.vals[k])


def run_threads(size, body):
    """Run body(rank, comm) for every rank in its own thread; re-raise the
    first failure; return the per-rank results."""
    hub = ThreadHub(size)
    out, err = [None] * size, []

    def go(r):
        try:
            out[r] = body(r, ThreadComm(hub, r))
        except BaseException as e:  # noqa: BLE001
            err.append(e)
            with hub.cv:
                hub.failed = True
                hub.cv.notify_all()

    ts = [threading.Thread(target=go, args=(r,)) for r in range(size)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if err:
        raise err[0]
    return out


def combine(parts, n, dim):
    """Fields of every particle in global order from the ranks' owned sets
    [(gid, x, u, phi, type), ...]; each particle owned exactly once."""
    x = np.full((dim, n), np.nan)
    u = np.full((dim, n), np.nan)
    phi = np.full(n, np.nan)
    seen = np.zeros(n, dtype=np.int64)
    for gid, xs, us, ps, _ in parts:
        seen[gid] += 1
        x[:, gid], u[:, gid], phi[gid] = xs, us, ps
    assert np.all(seen == 1), "a particle is owned by no rank or by several"
    return x, u, phi
