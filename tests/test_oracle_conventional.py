"""Pins of the oracle's conventional WCSPH foil (Sec. 2.1: Eq. nslag with the
printed operators, linear EOS of Eq. eos-water, artificial viscosity).

The foil has no implementation to compare against either, so it is pinned
by what its definition fixes: the pressure and artificial-viscosity pair
terms are equal and opposite (total momentum changes only by gravity), a
two-particle case assembled by hand from the kernel values, and the
property that makes it the foil: unlike the well-balanced scheme it does
not hold a hydrostatic tank at rest.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S


def _conventional(params, **kw):
    return dict(params, scheme=1, use_delta=0, use_pst=0, use_tic=0, **kw)


@pytest.mark.parametrize("dim,n_side", [(2, 24), (3, 9)])
def test_pressure_and_artificial_viscosity_conserve_momentum(dim, n_side):
    """sum_i m_i (DU_i/Dt - G) = 0 for an all-fluid cloud with random
    potentials and velocities (viscosity off): the pressure term
    -V_i sum (p_i + p_j) grad_i W_ij V_j and the artificial viscosity
    -m_i sum m_j Pi_ij grad_i W_ij are antisymmetric in i and j."""
    sc = S.lattice_cloud(dim, n_side, 0.01, jitter_amount=0.2, seed=4, g=[0.0, -9.81, 0.0][:3])
    p = _conventional(sc.params, nu=0.0, use_visc=0, art_alpha=0.5)
    rng = np.random.default_rng(5)
    phi = rng.normal(scale=2.0, size=sc.n)
    u = rng.normal(scale=0.5, size=(dim, sc.n))
    m = oracle.mass(p, phi)
    r = oracle.stage_rates(p, sc.x, u, phi, m, sc.type, sc.normal)
    G = np.asarray(p["g"][:dim])[:, None]
    f = m[None, :] * (r["dudt"] - G)
    assert np.all(np.abs(f.sum(1)) <= 1e-13 * np.abs(f).sum(1))
    assert np.all(r["dushift"] == 0.0)


def test_two_particles_by_hand():
    """Two fluid particles 0.6 h apart on the x axis, closing at 1 m/s: the
    pressure, artificial-viscosity, viscous and continuity terms of particle
    0, assembled from the kernel derivative and the EOS by hand."""
    p = S.default_params(2, 0.01, 20.0, domain_min=[0.0, 0.0, 0.0], domain_max=[1.0, 1.0, 1.0],
                         g=[0.0, -9.81, 0.0])
    p = _conventional(p, nu=1e-3, use_visc=1, art_alpha=0.1)
    h = p["h_over_dx"] * p["dx"]
    d = 0.6 * h
    x = np.array([[0.5, 0.5 + d], [0.5, 0.5]])
    u = np.array([[0.5, -0.5], [0.0, 0.0]])
    phi = np.array([3.0, 1.0])
    m = np.array([0.1, 0.12])
    r = oracle.stage_rates(p, x, u, phi, m, np.zeros(2, np.uint8), np.zeros((2, 2)))
    _, dw = oracle.kernel(p, np.array([d]))
    dwdr = float(dw[0])
    c0, rho0 = p["c0"], p["rho0"]
    rho = rho0 * np.exp(phi / c0 ** 2)
    pres = c0 ** 2 * (rho - rho0)
    V = m / rho
    gw0 = dwdr * (x[0, 0] - x[0, 1]) / d  # x component of grad_0 W_01 (the y component is zero)
    uijxij = (u[0, 0] - u[0, 1]) * (x[0, 0] - x[0, 1])  # -1 m/s times d: closing
    pi01 = -p["art_alpha"] * h * c0 * uijxij / (0.5 * (rho[0] + rho[1]) * (d * d + 0.01 * h * h))
    lap = (u[0, 1] - u[0, 0]) * ((x[0, 1] - x[0, 0]) * gw0) / (d * d) * V[1]
    ax = -(pres[0] + pres[1]) * gw0 * V[1] / rho[0] - m[1] * pi01 * gw0 + 2 * p["nu"] * lap
    dphi = -c0 ** 2 * (u[0, 1] - u[0, 0]) * gw0 * V[1]
    assert math.isclose(r["dudt"][0, 0], ax, rel_tol=1e-13)
    assert math.isclose(r["dudt"][1, 0], -9.81, rel_tol=1e-15)
    assert math.isclose(r["dphidt"][0], dphi, rel_tol=1e-13)


def test_conventional_tank_is_not_well_balanced():
    """The same 2D hydrostatic tank at rest (linear EOS, stabilisers off, 60
    steps): the well-balanced scheme keeps the spurious velocity at rounding
    level, the conventional one does not (the contrast of Sec. 4.1)."""
    sc = S.hydrostatic_tank_2d(dx=0.02, eos=0)
    wb = oracle.State(sc).step(60)
    conv_scene = sc.copy()
    conv_scene.params = _conventional(sc.params)
    conv = oracle.State(conv_scene).step(60)
    l2_wb, _ = wb.l2_velocity()
    l2_conv, _ = conv.l2_velocity()
    print("L2 spurious velocity: well-balanced", l2_wb, "conventional", l2_conv)
    assert l2_wb <= 1e-12
    assert l2_conv >= 1e-5


def test_conventional_scheme_takes_no_stabilisers():
    p = dict(S.default_params(2, 0.01, 20.0), scheme=1, use_delta=1)
    with pytest.raises(Exception):
        oracle.stage_rates(p, np.zeros((2, 1)), np.zeros((2, 1)), np.zeros(1), np.ones(1),
                           np.zeros(1, np.uint8), np.zeros((2, 1)))
