"""What the trained surrogate gains over the method without it.

On a held-out 2D dam-break column (0.55 x 0.35 m; the training columns are
seeded draws from [0.3, 0.8] x [0.2, 0.5] m), anchored rollouts (a plain FP64
step every 10 steps, no fallback) with the committed trained weights stay
closer to the plain FP64 rollout than the same rollouts with the untrained
initial weights or with a network that predicts gravity alone."""
import os

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2608_22269_gb300", "data", "surrogate_2d.npz")


def test_trained_surrogate_beats_untrained_and_gravity_only():
    from paper_2608_22269_gb300 import surrogate as SG
    from paper_2608_22269_gb300 import wbsph
    sur, norm = SG.load(WEIGHTS, 2)
    held = SG.dam_scene(0.55, 0.35, 50_000)
    inf = float("inf")
    steps = 400
    err = {"trained": SG.rollout_error(held, sur, steps, tau=inf)["pos_rms_over_dx"]}
    grav = wbsph.Surrogate(2)
    grav.set_params(SG.gravity_only_params(2, norm[2], norm[3], held.params["g"]))
    grav.set_normalization(*norm)
    err["gravity_only"] = SG.rollout_error(held, grav, steps, tau=inf)["pos_rms_over_dx"]
    untrained = wbsph.Surrogate(2)
    untrained.set_params(SG.init_params_2d(seed=7))
    untrained.set_normalization(*norm)
    err["untrained"] = SG.rollout_error(held, untrained, steps, tau=inf)["pos_rms_over_dx"]
    print("position RMS / dx after", steps, "steps:", err)
    assert err["trained"] < 0.8 * err["untrained"]
    assert err["trained"] < 0.8 * err["gravity_only"]
    for s in (sur, grav, untrained):
        s.close()


def test_trained_3d_surrogate_beats_untrained_and_gravity_only():
    """The same comparison in 3D: a held-out dam-break column (0.55 m long,
    0.275 m high) in the half-size box at dx = 0.0126 m, 200 steps, anchors
    every 10 steps, with the committed 3D weights (trained on 24 columns in
    that box)."""
    from paper_2608_22269_gb300 import surrogate as SG
    from paper_2608_22269_gb300 import wbsph
    sur, norm = SG.load(os.path.join(ROOT, "paper_2608_22269_gb300", "data", "surrogate_3d.npz"), 3)
    held = SG.dam_scene_3d(0.55, 0.35, 0.0126)
    inf = float("inf")
    steps = 200
    err = {"trained": SG.rollout_error(held, sur, steps, tau=inf)["pos_rms_over_dx"]}
    grav = wbsph.Surrogate(3)
    grav.set_params(SG.gravity_only_params(3, norm[2], norm[3], held.params["g"]))
    grav.set_normalization(*norm)
    err["gravity_only"] = SG.rollout_error(held, grav, steps, tau=inf)["pos_rms_over_dx"]
    untrained = wbsph.Surrogate(3)
    untrained.set_params(SG.init_params(3, seed=7))
    untrained.set_normalization(*norm)
    err["untrained"] = SG.rollout_error(held, untrained, steps, tau=inf)["pos_rms_over_dx"]
    print("3D position RMS / dx after", steps, "steps:", err)
    assert err["trained"] < 0.8 * err["untrained"]
    assert err["trained"] < 0.8 * err["gravity_only"]
    for s in (sur, grav, untrained):
        s.close()
