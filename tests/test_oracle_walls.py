"""Pins of the oracle's wall options (Sec. 2.4): the no-slip velocity of
Eq. (velBn), the slip condition against a moving wall, the viscous
interaction with wall particles under no-slip, and bodies of wall particles
translating with a prescribed velocity."""
import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S


def _nearest_fluid(x, typ, i, two_h):
    f = np.nonzero(typ == 0)[0]
    d2 = ((x[:, f] - x[:, i:i + 1]) ** 2).sum(0)
    k = np.argmin(d2)
    return f[k] if d2[k] <= two_h ** 2 else -1


@pytest.mark.parametrize("wall_bc", [0, 1])
def test_wall_velocities_by_definition(wall_bc):
    """Every wall particle next to the water: with no-slip, U_d = 2 U_w - U_f
    (Eq. velBn); with slip, U_d keeps U_f's tangential part and takes U_w's
    normal part (U_w = 0 for fixed walls, body_u for the body); f its
    nearest fluid particle."""
    sc = S.jitter(S.moving_body(2, body_u=(0.4, -0.1)), 0.1, seed=3)
    p = dict(sc.params, wall_bc=wall_bc)
    rng = np.random.default_rng(2)
    f = sc.type == 0
    u = sc.u.copy()
    u[:, f] = rng.normal(scale=0.3, size=(2, f.sum()))
    uo, _ = oracle.dummy_update(p, sc.x, u, sc.phi, sc.type, sc.normal)
    two_h = 2 * p["h_over_dx"] * p["dx"]
    checked = 0
    for i in np.nonzero(sc.type != 0)[0]:
        j = _nearest_fluid(sc.x, sc.type, i, two_h)
        if j < 0:
            continue
        uw = np.array(p["body_u"][:2]) if sc.type[i] == 2 else np.zeros(2)
        if wall_bc == 1:
            want = 2 * uw - u[:, j]
            assert np.allclose(uo[:, i], want, rtol=0, atol=1e-15)
        else:
            n = sc.normal[:, i]
            assert abs((uo[:, i] - uw) @ n) <= 1e-15
            t = np.array([-n[1], n[0]])
            assert abs(uo[:, i] @ t - u[:, j] @ t) <= 1e-15
        checked += 1
    assert checked > 100


def test_no_slip_viscosity_drags_the_water_next_to_a_wall():
    """Uniform water velocity along a fixed wall: with slip walls the viscous
    sum over fluid neighbours vanishes; with no-slip walls the wall particles
    (U_d = -U_f) enter it and the viscous acceleration of the water next to
    the wall opposes the flow."""
    sc = S.hydrostatic_tank_2d(dx=0.02, eos=0)
    f = sc.type == 0
    u = sc.u.copy()
    u[0, f] = 0.2
    m = oracle.mass(sc.params, sc.phi)
    out = {}
    for bc in (0, 1):
        p = dict(sc.params, wall_bc=bc, use_delta=0, use_pst=0, use_tic=1, nu=1e-2)
        p0 = dict(p, use_visc=0)
        r = oracle.stage_rates(p, sc.x, u, sc.phi, m, sc.type, sc.normal)
        r0 = oracle.stage_rates(p0, sc.x, u, sc.phi, m, sc.type, sc.normal)
        out[bc] = r["dudt"][0, f] - r0["dudt"][0, f]  # the viscous part
    bottom = f & (sc.x[1] < 1.5 * sc.params["dx"])
    interior = f & (sc.x[1] > 0.1) & (sc.x[1] < 0.3) & (sc.x[0] > 0.2) & (sc.x[0] < 0.8)
    assert np.abs(out[0]).max() <= 1e-12
    assert np.all(out[1][bottom[f]] < 0.0)
    assert np.abs(out[1][interior[f]]).max() <= 1e-12


def test_body_translates_with_the_prescribed_velocity():
    """After 30 SSP-RK2 steps every body particle sits at x0 + body_u t (to
    rounding) while the fixed walls stay put."""
    sc = S.moving_body(2, body_u=(0.5, 0.1))
    st = oracle.State(sc).step(30)
    b = sc.type == 2
    want = sc.x[:, b] + np.array([0.5, 0.1])[:, None] * st.t
    assert np.abs(st.x[:, b] - want).max() <= 1e-13
    w = sc.type == 1
    assert np.array_equal(st.x[:, w], sc.x[:, w])


def test_body_speed_bounds_the_time_step():
    sc = S.moving_body(2, body_u=(30.0, 0.0))
    dt = oracle.time_step(sc.params, sc.u, sc.type)
    p = sc.params
    assert dt == pytest.approx(p["cfl"] * p["dx"] / (p["c0"] + 30.0), rel=1e-15)
