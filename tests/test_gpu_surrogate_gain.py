"""What the trained surrogate gains over the method without it.

Rollouts from a held-out dam-break column (0.55 m wide, 0.35 m high in 2D;
the training columns are seeded draws from [0.3, 0.8] x [0.2, 0.5] m), all
with the same fixed time step and the same anchoring: a plain FP64 step
every 10 steps, starting with the first, and no fallback. The position RMS
error against the plain FP64 rollout, every 50 steps, is compared for:
  - the committed trained weights;
  - control A: the rates of the last plain step, replayed until the next
    anchor (the frozen-rates mode of the library);
  - control B: a network that predicts gravity alone;
  - the untrained initial weights.
The plain method with its step enlarged to the trained rollout's wall-clock
time (equal wall clock) is reported beside them (gain_report)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check(rep, label):
    err = {k: rep[k]["pos_rms_over_dx"] for k in ("trained", "frozen", "gravity", "untrained", "coarse")}
    print(label, "position RMS / dx after", rep["steps"], "steps:", err)
    print(label, "histories:", {k: np.round(rep[k]["history"], 4).tolist() for k in ("trained", "frozen")},
          "frozen diverged:", rep["frozen"]["diverged"])
    print(label, "equal wall clock:", rep["coarse"])
    assert np.isfinite(err["trained"]) and rep["trained"]["diverged"] is None
    assert err["trained"] < 0.8 * err["untrained"]
    assert err["trained"] < 0.8 * err["gravity"]
    assert err["trained"] < err["frozen"]          # control A (inf where it diverged)


def test_trained_surrogate_beats_the_controls_2d():
    from paper_2608_22269_gb300 import surrogate as SG
    sur, norm = SG.load(os.path.join(ROOT, "paper_2608_22269_gb300", "data", "surrogate_2d.npz"), 2)
    rep = SG.gain_report(SG.dam_scene(0.55, 0.35, 50_000), sur, norm, steps=400, seed=7, log=None)
    _check(rep, "2D")
    sur.close()


def test_trained_surrogate_beats_the_controls_3d():
    """The same comparison in 3D: a held-out column in the half-size box of
    the 3D dam break at dx = 0.0126 m, 200 steps, with the committed 3D
    weights (trained on columns in that box)."""
    from paper_2608_22269_gb300 import surrogate as SG
    sur, norm = SG.load(os.path.join(ROOT, "paper_2608_22269_gb300", "data", "surrogate_3d.npz"), 3)
    rep = SG.gain_report(SG.dam_scene_3d(0.55, 0.35, 0.0126), sur, norm, steps=200, seed=7, log=None)
    _check(rep, "3D")
    sur.close()
