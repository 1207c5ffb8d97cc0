"""Training and evaluation driver of the learned surrogate (BF16 message passing).

Trajectories of the plain FP64 method (CUDA path) provide the training states;
the network is trained on the GPU by the library's own forward/backward
kernels (wbsph_surrogate_train_step), its targets being the plain rates of
each state. Rollouts replace the pair pass by the network inside the same
SSP-RK2 step and re-anchor with a plain FP64 step every `anchor_every` steps
(wbsph_step_surrogate), which also measures the surrogate's acceleration
error against the plain one on the anchor state.

Scenes: 2D dam breaks in a 2.0 x 1.0 m basin, column width and height drawn
(seeded) from [0.3, 0.8] x [0.2, 0.5] m, dx = sqrt(w h / n_target); in 3D,
dam breaks in the 1.6 x 0.5 x 0.5 m box (the 3D dam break halved along every
axis) at its dx = 0.0084 m, column length and height from the same draws
with the height mapped to [0.2, 0.35] m.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import scenes as S
from . import wbsph


def column_sizes(n: int, seed: int = 7):
    rng = np.random.default_rng(seed)
    return [(float(rng.uniform(0.3, 0.8)), float(rng.uniform(0.2, 0.5))) for _ in range(n)]


def dam_scene_3d(w: float, h: float, dx: float = 0.0084):
    """3D dam break in the 1.6 x 0.5 x 0.5 m box: a column w long, 0.5 m wide
    and 0.2 + (h - 0.2) / 2 m high (h from the 2D draws)."""
    return S.dam_break_3d(dx=dx, box=(1.6, 0.5, 0.5), column=(w, 0.5, 0.2 + 0.5 * (h - 0.2)))


def dam_scene(w: float, h: float, n_target: int, width: float = 2.0, wall: float = 1.0):
    dx = math.sqrt(w * h / n_target)
    return S.dam_break_2d(dx=dx, width=width, wall=wall, column=(w, h))


def generate(n_traj=40, n_target=50_000, t_end=0.2, frames=20, seed=7, log=print, concurrent=8, scene_fn=None):
    """Plain FP64 trajectories; returns a list of (scene, [(x, u, phi), ...]).

    Each trajectory advances in chunks of 20 steps and records a frame at
    the first chunk end past each of the frame times t_end (f + 1) / frames.
    A 50k-particle step leaves most of the GPU idle, so `concurrent`
    trajectories run at once, each on its own stream, advanced in lockstep
    (the frames are the same as one at a time). scene_fn(w, h) builds a
    scene from a column draw (default: the 2D dam break with n_target fluid
    particles)."""
    if scene_fn is None:
        scene_fn = lambda w, h: dam_scene(w, h, n_target)  # noqa: E731
    sizes = column_sizes(n_traj, seed)
    data = [None] * n_traj
    t0 = time.time()
    for b0 in range(0, n_traj, concurrent):
        batch = []
        for k in range(b0, min(b0 + concurrent, n_traj)):
            sc = scene_fn(*sizes[k])
            sim = wbsph.Sim(sc.params, water_height=sc.water_height)
            sim.set_scene(sc)
            batch.append({"k": k, "sc": sc, "sim": sim, "states": []})
        live = list(batch)
        while live:
            for b in live:
                b["sim"].step(20)  # enqueued on the trajectory's own stream
            for b in live:
                if b["sim"].stats()["t"] >= t_end * (len(b["states"]) + 1) / frames:
                    b["states"].append((b["sim"].get("x"), b["sim"].get("u"), b["sim"].get("phi")))
            done = [b for b in live if len(b["states"]) == frames]
            live = [b for b in live if len(b["states"]) < frames]
            for b in done:
                sc, sim = b["sc"], b["sim"]
                data[b["k"]] = (sc, b["states"])
                nsteps = sim.stats()["steps"]
                sim.close()
                if log:
                    w, h = sizes[b["k"]]
                    log(f"trajectory {b['k']}: column {w:.2f} x {h:.2f}, n_fluid {sc.n_fluid}, "
                        f"steps {nsteps}, elapsed {time.time() - t0:.1f} s")
    return data


def _load_state(sim, sc, st):
    x, u, phi = st
    sim.set_particles(x, u, phi, sc.type, sc.normal)


def hydrostatic_potential(params, x, water_height):
    """phi_hs(x) = G.x + |G| H: the split of the potential that the network's
    inputs use (the constant body force G of the scene)."""
    d = int(params["dim"])
    g = np.asarray(params["g"][:d], dtype=np.float64)
    return g @ np.asarray(x)[:d] + np.linalg.norm(g) * water_height


def normalisation(data, samples=20, seed=0):
    """Means and standard deviations of the node inputs (U, rho/rho0 - 1,
    phi'), the scales of the edge inputs (RMS over edges of the velocity and
    potential differences), and the means and deviations of the plain rates
    (DU/Dt, Dphi/Dt), over sampled frames. Returns (node_mean, node_std,
    edge_std, out_mean, out_std)."""
    rng = np.random.default_rng(seed)
    feats, outs, du, dp = [], [], [], []
    for _ in range(samples):
        sc, states = data[rng.integers(len(data))]
        st = states[rng.integers(len(states))]
        sim = wbsph.Sim(sc.params, water_height=sc.water_height)
        _load_state(sim, sc, st)
        sim.eval_rates()
        f = sc.type == 0
        rho = sim.get("rho")
        u, phi = sim.get("u"), sim.get("phi")          # wall particles after their update
        phip = phi - hydrostatic_potential(sc.params, st[0], sc.water_height)
        feats.append(np.r_[u[:, f], (rho[f] / sc.params["rho0"] - 1.0)[None], phip[None, f]])
        outs.append(np.r_[sim.get("dudt")[:, f], sim.get("dphidt")[None, f]])
        row, col = sim.neighbors()
        recv = np.repeat(np.arange(sc.n), np.diff(row))
        keep = f[recv]
        recv, send = recv[keep], col[keep].astype(np.int64)
        du.append((u[:, send] - u[:, recv]).ravel())
        dp.append(phip[send] - phip[recv])
        sim.close()
    F = np.concatenate(feats, axis=1)
    O = np.concatenate(outs, axis=1)
    fs = np.maximum(F.std(1), 1e-6)
    os_ = np.maximum(O.std(1), 1e-6)
    es = np.array([max(float(np.sqrt(np.mean(np.concatenate(du) ** 2))), 1e-6),
                   max(float(np.sqrt(np.mean(np.concatenate(dp) ** 2))), 1e-6)])
    return F.mean(1), fs, es, O.mean(1), os_


def train(sur: "wbsph.Surrogate", data, iters=2000, lr=1e-3, seed=1, log=print, log_every=200):
    """Adam with cosine decay over random frames; returns the loss history."""
    rng = np.random.default_rng(seed)
    sims = {}
    hist = []
    t0 = time.time()
    for it in range(iters):
        k = int(rng.integers(len(data)))
        sc, states = data[k]
        if k not in sims:
            sims[k] = wbsph.Sim(sc.params, water_height=sc.water_height)
        sim = sims[k]
        _load_state(sim, sc, states[int(rng.integers(len(states)))])
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        loss = sur.train_step(sim, lr_t)
        hist.append(loss)
        if log and (it % log_every == 0 or it == iters - 1):
            log(f"iter {it}: loss {np.mean(hist[-log_every:]):.4e} lr {lr_t:.2e} ({time.time() - t0:.1f} s)")
    for s in sims.values():
        s.close()
    return hist


def gravity_only_params(dim, out_mean, out_std, g):
    """Parameters of a network whose output is exactly (G, 0) for every
    particle: all weights zero, decoder bias set to the normalised gravity."""
    from_flat = np.zeros(wbsph_num_params(dim), dtype=np.float32)
    tgt = np.r_[np.asarray(g[:dim], dtype=np.float64), 0.0]
    b2 = ((tgt - out_mean) / out_std).astype(np.float32)
    from_flat[-(dim + 1):] = b2
    return from_flat


def block_dims(dim, hidden=64, layers=3):
    """(name, inputs, outputs) of the parameter blocks in their flat order:
    node encoder, (edge MLP, node MLP) per layer, decoder."""
    fn, fe, fo = dim + 3, 2 * dim + 2, dim + 1
    blocks = [("enc", fn, hidden)]
    for _ in range(layers):  # the edge MLP reads the edge inputs, h_i and the sender's first 32 features
        blocks += [("edge", fe + hidden + 32, hidden), ("node", 2 * hidden, hidden)]
    blocks.append(("dec", hidden, fo))
    return blocks


def wbsph_num_params(dim, hidden=64, layers=3):
    return sum(i * hidden + hidden + hidden * o + o for _, i, o in block_dims(dim, hidden, layers))


def comparison_step(sc):
    """A fixed time step for rollout comparisons: CFL dx / (C0 + 2 sqrt(g H)),
    the adaptive step of the method once the dam-break front runs at its
    shallow-water speed 2 sqrt(g H) (so it stays stable for the whole run)."""
    p = sc.params
    g = float(np.linalg.norm(np.asarray(p["g"][: p["dim"]])))
    return p["cfl"] * p["dx"] / (p["c0"] + 2.0 * math.sqrt(g * sc.water_height))


def _fixed(sc, dt):
    s2 = sc.copy()
    s2.params = dict(sc.params, fixed_dt=float(dt))
    return s2


def _pos_rms(a, b, sc):
    f = sc.type == 0
    return float(np.sqrt(((a[:, f] - b[:, f]) ** 2).sum(0).mean()) / sc.params["dx"])


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def rollout_error(sc, sur, nsteps, anchor_every=10, tau=0.1, dt=None, ref_x=None):
    """Run the plain FP64 rollout (unless its final positions ref_x are given)
    and a surrogate rollout from the same state, both with the fixed step dt
    when given; return position RMS / dx, the anchor statistics and the wall
    times."""
    if dt is not None:
        sc = _fixed(sc, dt)
    out = {}
    if ref_x is None:
        ref = wbsph.Sim(sc.params, water_height=sc.water_height)
        ref.set_scene(sc)
        _, out["wall_plain_s"] = _timed(lambda: (ref.step(nsteps), ref.sync()))
        ref_x = ref.get("x")
        ref.close()
    sim = wbsph.Sim(sc.params, water_height=sc.water_height)
    sim.set_scene(sc)
    stats, out["wall_surrogate_s"] = _timed(lambda: sur.step(sim, nsteps, anchor_every=anchor_every, tau=tau))
    out["pos_rms_over_dx"] = _pos_rms(ref_x, sim.get("x"), sc)
    out["anchors"] = stats
    sim.close()
    return out


def _checkpointed(sc, advance, checkpoints):
    """Positions of a rollout at the checkpoint step counts; advance(sim, k)
    runs k more steps. A run that fails (non-finite state) gives None from
    there on."""
    sim = wbsph.Sim(sc.params, water_height=sc.water_height)
    sim.set_scene(sc)
    out, done, failed = [], 0, None
    for c in checkpoints:
        if failed is None:
            try:
                advance(sim, c - done)
                done = c
                x = sim.get("x")
                if not np.all(np.isfinite(x)):
                    raise wbsph.WbsphError(-6, "non-finite positions")
                out.append(x)
                continue
            except wbsph.WbsphError as exc:
                failed = f"step <= {c}: {exc}"
        out.append(None)
    sim.close()
    return out, failed


def gain_report(held, sur, norm, steps=400, anchor_every=10, seed=7, log=print, every=50):
    """What the trained network gains over the method without it, on a
    held-out scene, every rollout with the same fixed step and the same
    anchoring (a plain FP64 step every anchor_every steps, starting with the
    first; no fallback). Position RMS / dx against the plain FP64 rollout at
    every `every` steps up to `steps`, for:
      trained    the trained network;
      frozen     control A: the rates of the last plain step, replayed;
      gravity    control B: a network predicting (G, 0);
      untrained  the initial weights;
      coarse     the plain FP64 method alone with its step enlarged so that it
                 spends the trained rollout's wall-clock time on the same
                 physical time (equal wall clock; compared at the end).
    A rollout that leaves the finite range is recorded as diverged (inf)."""
    dim = held.params["dim"]
    dt = comparison_step(held)
    sc = _fixed(held, dt)
    cps = list(range(every, steps + 1, every))
    inf = float("inf")
    rep = {"steps": steps, "dt": dt, "anchor_every": anchor_every, "checkpoints": cps}
    # wall clock of the plain and the trained rollouts (after a warm-up of each)
    for warm in range(2):
        ref = wbsph.Sim(sc.params, water_height=sc.water_height)
        ref.set_scene(sc)
        _, t_plain = _timed(lambda: (ref.step(steps if warm else 2), ref.sync()))
        ref_end = ref.get("x")
        ref.close()
        sim = wbsph.Sim(sc.params, water_height=sc.water_height)
        sim.set_scene(sc)
        sur.set_mode(wbsph.SURROGATE_NETWORK)
        _, t_sur = _timed(lambda: sur.step(sim, steps if warm else 2, anchor_every=anchor_every, tau=inf))
        sim.close()
    rep["wall_plain_s"], rep["wall_trained_s"] = t_plain, t_sur
    ref_x, _ = _checkpointed(sc, lambda s, k: (s.step(k), s.sync()), cps)

    def errors(xs):
        return [_pos_rms(r, x, sc) if x is not None else inf for r, x in zip(ref_x, xs)]

    def run(net, mode=wbsph.SURROGATE_NETWORK):
        net.set_mode(mode)
        xs, failed = _checkpointed(sc, lambda s, k: net.step(s, k, anchor_every=anchor_every, tau=inf), cps)
        net.set_mode(wbsph.SURROGATE_NETWORK)
        e = errors(xs)
        return {"pos_rms_over_dx": e[-1], "history": e, "diverged": failed}

    rep["trained"] = run(sur)
    rep["frozen"] = run(sur, wbsph.SURROGATE_FROZEN)
    grav = wbsph.Surrogate(dim)
    grav.set_params(gravity_only_params(dim, norm[3], norm[4], held.params["g"]))
    grav.set_normalization(*norm)
    rep["gravity"] = run(grav)
    grav.close()
    untrained = wbsph.Surrogate(dim)
    untrained.set_params(init_params(dim, seed=seed))
    untrained.set_normalization(*norm)
    rep["untrained"] = run(untrained)
    untrained.close()
    speedup = t_plain / t_sur
    m = max(1, int(round(steps / speedup)))
    xc, failed = _checkpointed(_fixed(sc, steps * dt / m), lambda s, k: (s.step(k), s.sync()), [m])
    rep["coarse"] = {"pos_rms_over_dx": _pos_rms(ref_end, xc[0], sc) if xc[0] is not None else inf,
                     "steps": m, "dt": steps * dt / m, "cfl": sc.params["cfl"] * steps / m,
                     "speedup_of_trained": speedup, "diverged": failed}
    if log:
        log("gain: " + ", ".join(f"{k} {rep[k]['pos_rms_over_dx']:.4f}" for k in
                                 ("trained", "frozen", "gravity", "untrained", "coarse")))
    return rep


def save(path, sur, norm, meta):
    np.savez(path, params=sur.get_params(), node_mean=norm[0], node_std=norm[1], edge_std=norm[2],
             out_mean=norm[3], out_std=norm[4], meta=np.frombuffer(str(meta).encode(), dtype=np.uint8))


def load(path, dim=2):
    """Network and normalisation (node_mean, node_std, edge_std, out_mean,
    out_std) from a file written by save()."""
    z = np.load(path)
    sur = wbsph.Surrogate(dim)
    sur.set_params(z["params"])
    norm = (z["node_mean"], z["node_std"], z["edge_std"], z["out_mean"], z["out_std"])
    sur.set_normalization(*norm)
    return sur, norm


def main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description="train the BF16 surrogate on plain FP64 trajectories")
    ap.add_argument("--out", required=True, help="output .npz with parameters and normalisation")
    ap.add_argument("--report", default=None, help="JSON report path")
    ap.add_argument("--trajectories", type=int, default=200)
    ap.add_argument("--particles", type=int, default=50_000)
    ap.add_argument("--t-end", type=float, default=0.4)
    ap.add_argument("--frames", type=int, default=40)
    ap.add_argument("--iters", type=int, default=30000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--eval-steps", type=int, default=400)
    ap.add_argument("--concurrent", type=int, default=16, help="trajectories generated at once")
    ap.add_argument("--dim", type=int, default=2, choices=(2, 3))
    ap.add_argument("--dx3", type=float, default=0.0084, help="particle spacing of the 3D scenes")
    ap.add_argument("--eval-only", default=None, help="skip training: evaluate the weights in this file")
    args = ap.parse_args(argv)
    dim = args.dim
    if dim == 2:
        scene_fn = lambda w, h: dam_scene(w, h, args.particles)  # noqa: E731
    else:
        scene_fn = lambda w, h: dam_scene_3d(w, h, args.dx3)  # noqa: E731
    if args.eval_only:
        sur, norm = load(args.eval_only, dim)
        rep = gain_report(scene_fn(0.55, 0.35), sur, norm, args.eval_steps, seed=args.seed)
        print(json.dumps(rep))
        if args.report:
            with open(args.report, "w") as fh:
                json.dump(rep, fh, indent=1)
        return
    t0 = time.time()
    data = generate(args.trajectories, args.particles, args.t_end, args.frames, args.seed,
                    concurrent=args.concurrent, scene_fn=scene_fn)
    t_gen = time.time() - t0
    norm = normalisation(data)
    print("normalisation", [np.round(np.asarray(v), 5).tolist() for v in norm], flush=True)
    sur = wbsph.Surrogate(dim)
    theta0 = init_params(dim, seed=args.seed)
    sur.set_params(theta0)
    sur.set_normalization(*norm)
    t0 = time.time()
    hist = train(sur, data, iters=args.iters, lr=args.lr, seed=args.seed)
    t_train = time.time() - t0
    meta = dict(dim=dim, trajectories=args.trajectories, particles=args.particles, dx3=args.dx3, t_end=args.t_end,
                frames=args.frames, iters=args.iters, lr=args.lr, seed=args.seed)
    save(args.out, sur, norm, meta)
    # gain test on a held-out column, same anchoring for every variant
    held = scene_fn(0.55, 0.35)
    rep = {"meta": meta, "gen_s": t_gen, "train_s": t_train,
           "loss_first": float(np.mean(hist[:50])), "loss_last": float(np.mean(hist[-50:])),
           "gain": gain_report(held, sur, norm, args.eval_steps, seed=args.seed)}
    print(json.dumps(rep))
    if args.report:
        with open(args.report, "w") as fh:
            json.dump(rep, fh, indent=1)


def init_params_2d(seed=0, hidden=64, layers=3):
    """init_params in 2D."""
    return init_params(2, seed, hidden, layers)


def init_params(dim, seed=0, hidden=64, layers=3):
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases; the output layers of
    the processor MLPs scaled by 0.1 (small residual updates at the start),
    the edge MLP's by a further 1/8 (its outputs are summed over the
    receiver's neighbours)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, i, o in block_dims(dim, hidden, layers):
        s1, s2 = 1.0 / math.sqrt(i), 1.0 / math.sqrt(hidden)
        if name in ("edge", "node"):
            s2 *= 0.1
        if name == "edge":
            s2 /= 8.0
        parts += [rng.uniform(-s1, s1, i * hidden), np.zeros(hidden), rng.uniform(-s2, s2, hidden * o),
                  np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


if __name__ == "__main__":
    main()
