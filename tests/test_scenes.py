"""The synthetic workloads that stand in for the paper's scenes.

The benchmark quotes particle counts in its `config`; these tests build each
workload with the benchmark's own constructors and check the counts it
quotes, and check the structure every scene shares: fluid on the lattice
inside the water region, three layers of dummy particles outside the open
region with unit normals pointing into it, fluid at rest with the
hydrostatic potential phi = G.x + |G| H (Eq. eqSol), and the domain holding
every particle. The 17.6M-particle sloshing tank is not built here (about
2 GB of host memory); its lattice is the same code as the smaller boxes.
"""
import re

import numpy as np
import pytest

import bench
from paper_2608_22269_gb300 import scenes as S


def _quoted(text):
    """(fluid, dummy) counts quoted as 'N fluid + M dummy' in a description."""
    m = re.search(r"([\d,]+) fluid \+ ([\d,]+) dummy", text)
    assert m, text
    return int(m.group(1).replace(",", "")), int(m.group(2).replace(",", ""))


@pytest.mark.parametrize("key,which", [("dam3d", "make"), ("dam3d", "sample"), ("dam3d_s", "make")])
def test_benchmark_workloads_have_the_quoted_counts(key, which):
    wl = bench.WORKLOADS[key]
    text = wl["desc"] if which == "make" else wl["sample_desc"]
    nf, nd = _quoted(text)
    sc = wl[which]()
    assert sc.n_fluid == nf
    assert sc.n - sc.n_fluid == nd


def _check_structure(sc, water, open_box, layers=3):
    p = sc.params
    dim, dx = p["dim"], p["dx"]
    f = sc.type == 0
    w = ~f
    # fluid: lattice sites (i + 1/2) dx inside the water region, at rest
    assert np.all(water(sc.x[:, f]))
    frac = sc.x[:, f] / dx - 0.5
    assert np.abs(frac - np.rint(frac)).max() < 1e-9
    assert np.all(sc.u == 0.0)
    # hydrostatic potential phi = G.x + |G| H
    G = np.asarray(p["g"][:dim])
    phi_hs = G @ sc.x[:, f] + np.linalg.norm(G) * sc.water_height
    assert np.abs(sc.phi[f] - phi_hs).max() <= 1e-12
    # dummies: outside the open box, within `layers` spacings of it
    lo, hi = np.zeros(dim), np.asarray(open_box, dtype=float)
    xd = sc.x[:, w]
    inside = np.all((xd > lo[:, None]) & (xd < hi[:, None]), axis=0)
    assert not inside.any()
    out = np.maximum(lo[:, None] - xd, xd - hi[:, None]).max(axis=0)
    assert out.max() <= layers * dx
    # unit normals pointing into the open region (toward the box)
    n = sc.normal[:, w]
    assert np.allclose(np.linalg.norm(n, axis=0), 1.0, atol=1e-12)
    centre = hi / 2.0
    assert np.all(np.einsum("ij,ij->j", n, centre[:, None] - xd) > 0.0)
    # every particle inside the neighbour grid's domain
    dmin = np.asarray(p["domain_min"][:dim])[:, None]
    dmax = np.asarray(p["domain_max"][:dim])[:, None]
    assert np.all((sc.x >= dmin) & (sc.x <= dmax))


def test_3d_dam_break_structure():
    box, col = (3.2, 1.0, 1.0), (1.2, 1.0, 0.6)
    sc = S.dam_break_3d(dx=0.04, box=box, column=col)
    _check_structure(sc, lambda x: (x[0] < col[0]) & (x[1] < col[1]) & (x[2] < col[2]), box)
    assert sc.water_height == col[2]


def test_2d_dam_break_structure():
    sc = S.dam_break_2d(dx=0.01, width=2.0, wall=0.6, column=(0.6, 0.3))
    _check_structure(sc, lambda x: (x[0] < 0.6) & (x[1] < 0.3), (2.0, 0.6))


def test_3d_sloshing_tank_structure():
    sc = S.sloshing_3d(dx=0.1, tank=(4.0, 2.0, 2.0), depth=1.0)
    _check_structure(sc, lambda x: x[2] < 1.0, (4.0, 2.0, 2.0))
    assert sc.params["force_period"] == 1.5 and sc.params["force_amp"][0] == 0.01
