"""Pins of the diagnostics oracle (oracle/diagnostics.py) on fields whose answers are known by
construction: plateau means and exact bulk-cell counts of a sharp slab, the equivalent radius
of a sharp disk, and a zero iso-fugacity residual at the flash's phase states."""
import math

import numpy as np
import pytest

from conftest import read_table
from oracle import diagnostics as dg
from oracle import thermo as th


def _c3_nc5():
    t = {r[0]: th.Component(r[0], r[2], r[1], r[3], r[4]) for r in read_table("table1_components.txt")}
    lb, ts, ps = th.lattice_components([t["C3"], t["nC5"]])
    return lb, ts, ps


def test_sharp_slab_plateaus_and_bulk_counts():
    lb, _, _ = _c3_nc5()
    ny, nx, lo, hi = 6, 100, 30, 70                   # liquid in columns [30, 70)
    rho = np.empty((2, ny, nx))
    rl, rv = [1.3, 6.1], [0.4, 0.2]
    for c in range(2):
        rho[c] = rv[c]
        rho[c][:, lo:hi] = rl[c]
    p = np.full((ny, nx), 0.05)
    p[:, lo:hi] = 0.07
    d = dg.bulk_diagnostics(lb, [[0, 0], [0, 0]], 0.9 * lb[0].Tc, 1.0, rho, p, erode=8)
    assert d["threshold"] == pytest.approx(0.5 * (sum(rl) + sum(rv)))
    assert d["n_l"] == (hi - lo - 2 * 8) * ny          # cells 9+ columns inside the liquid
    assert d["n_v"] == (nx - (hi - lo) - 2 * 8) * ny
    assert d["liquid_cells"] == (hi - lo) * ny
    assert np.allclose(d["rho_l"], rl, rtol=1e-15) and np.allclose(d["rho_v"], rv, rtol=1e-15)
    assert d["p_l"] == pytest.approx(0.07, rel=1e-15) and d["dp"] == pytest.approx(0.02, rel=1e-12)
    M = np.array([k.M for k in lb])
    x = (np.array(rl) / M) / (np.array(rl) / M).sum()
    assert np.allclose(d["x"], x, rtol=1e-15)


def test_sharp_disk_equivalent_radius():
    lb, _, _ = _c3_nc5()
    n, R0 = 128, 20.0
    yy, xx = np.mgrid[0:n, 0:n] + 0.5
    inside = (xx - n / 2) ** 2 + (yy - n / 2) ** 2 < R0 * R0
    rho = np.stack([np.where(inside, 1.3, 0.4), np.where(inside, 6.1, 0.2)])
    p = np.where(inside, 0.07, 0.05)
    d = dg.bulk_diagnostics(lb, [[0, 0], [0, 0]], 0.9 * lb[0].Tc, 1.0, rho, p, erode=8)
    assert d["liquid_cells"] == int(inside.sum())
    assert d["radius"] == pytest.approx(R0, rel=0.01)
    assert d["n_l"] > 0 and d["n_v"] > 0


def test_residual_vanishes_at_the_flash_phase_states():
    """Two plateaus at the flash's liquid and vapour states (Section 4.2 state at 200 psia),
    pressures from the EOS at those densities (Eq. MCPengRobinson): the fugacities match."""
    lb, ts, ps = _c3_nc5()
    T, P = 666.06 * ts, 200.0 * ps
    kij = [[0.0, 0.0], [0.0, 0.0]]
    fr = th.flash(lb, kij, T, P, [0.4, 0.6])
    rl, rv, nl, nv = th.phase_partial_densities(lb, T, P, 1.0, fr)
    ny, nx = 4, 80
    rho = np.empty((2, ny, nx))
    for c in range(2):
        rho[c] = rv[c]
        rho[c][:, 20:60] = rl[c]
    M = [k.M for k in lb]
    pl = th.pressure(lb, kij, T, 1.0, [rl[0] / M[0], rl[1] / M[1]])
    pv = th.pressure(lb, kij, T, 1.0, [rv[0] / M[0], rv[1] / M[1]])
    assert pl == pytest.approx(P, rel=1e-9) and pv == pytest.approx(P, rel=1e-9)
    p = np.full((ny, nx), pv)
    p[:, 20:60] = pl
    d = dg.bulk_diagnostics(lb, kij, T, 1.0, rho, p, erode=8)
    assert d["residual"] < 1e-16
    assert np.allclose(d["x"], fr.x, rtol=1e-9) and np.allclose(d["y"], fr.y, rtol=1e-9)
