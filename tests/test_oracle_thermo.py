"""Pins of the phase-equilibrium oracle (oracle/thermo.py) against values the paper prints and
against thermodynamic identities that do not depend on the oracle's own formulas."""
import math

import numpy as np
import pytest

from conftest import read_table
from oracle import thermo as th

R_FIELD = 10.7316  # psia ft^3 / (lbmol degR)


def _table1():
    return {r[0]: th.Component(r[0], r[2], r[1], r[3], r[4]) for r in read_table("table1_components.txt")}


def _c3_nc5():
    t = _table1()
    return [t["C3"], t["nC5"]]


KIJ0 = [[0.0, 0.0], [0.0, 0.0]]
T_TABLE2 = 666.06
Z_TABLE2 = [0.4, 0.6]


@pytest.mark.parametrize("row", [r for r in read_table("table2_c3_nc5.txt") if r[2] is not None and r[1] is not None])
def test_flash_reproduces_table2(row):
    """Table 2: every two-phase row (Z, x, y, the four partial densities and gamma_1)."""
    p, zl, zv, x1, y1, r1l, r2l, r1v, r2v, g1 = row
    comps = _c3_nc5()
    fr = th.flash(comps, KIJ0, T_TABLE2, p, Z_TABLE2)
    assert not fr.trivial
    assert fr.residual < 1e-20  # Eq. error at the converged flash
    assert fr.Zl == pytest.approx(zl, rel=5e-4)
    assert fr.Zv == pytest.approx(zv, rel=5e-4)
    assert fr.x[0] == pytest.approx(x1, rel=5e-4)
    assert fr.y[0] == pytest.approx(y1, rel=5e-4)
    rl, rv, _, _ = th.phase_partial_densities(comps, T_TABLE2, p, R_FIELD, fr)
    # densities are printed to 3 decimals (half-digit 5e-4) and sit up to 5e-4 relative from
    # the flash, about what a gas constant of 10.73 instead of 10.7316 gives
    for got, want in zip(list(rl) + list(rv), [r1l, r2l, r1v, r2v]):
        assert abs(got - want) <= 5e-4 + 6e-4 * want
    g, h = th.gamma_coefficients(rl, rv, fr.K)
    assert h == 1
    assert g[1] == 1.0
    assert g[0] == pytest.approx(g1, abs=1e-4)
    # the second form of Eq. gamma, from molar densities and K values
    nl, nv = p / (fr.Zl * R_FIELD * T_TABLE2), p / (fr.Zv * R_FIELD * T_TABLE2)
    alt = (math.log(nl / nv) - math.log(fr.K[0])) / (math.log(nl / nv) - math.log(fr.K[1]))
    assert alt == pytest.approx(g[0], rel=1e-12)


def test_bubble_and_dew_rows_of_table2():
    """Table 2 first and last rows: liquid Z at the bubble point (x = z) and vapour Z at the
    dew point (y = z); the negative flash puts V = 0 and V = 1 there."""
    comps = _c3_nc5()
    zl, _ = th.phase_state(comps, KIJ0, T_TABLE2, 246.0, Z_TABLE2, which="l")
    zv, _ = th.phase_state(comps, KIJ0, T_TABLE2, 127.9, Z_TABLE2, which="v")
    assert zl == pytest.approx(0.06877, rel=5e-4)
    assert zv == pytest.approx(0.83699, rel=5e-4)
    fb = th.flash(comps, KIJ0, T_TABLE2, 246.0, Z_TABLE2)
    fd = th.flash(comps, KIJ0, T_TABLE2, 127.9, Z_TABLE2)
    assert abs(fb.V) < 5e-3
    assert abs(fd.V - 1.0) < 5e-3


def test_maxwell_pure_saturation():
    """Section 4.1: a = 2/49, b = 2/21, omega = 0.344, T = 0.9 T_c gives rho_l = 5.90796 and
    rho_v = 0.58007 by the Maxwell rule."""
    a, b, omega, tr, rl, rv = read_table("maxwell_pr.txt")[0]
    Tc = (th.OMEGA_B / th.OMEGA_A) * (a / b)
    pc = th.OMEGA_B * Tc / b
    comp = th.Component("pure", Tc, pc, omega, 1.0)
    assert th.a_b(comp, 1.0)[0] == pytest.approx(a, rel=1e-14)
    assert th.a_b(comp, 1.0)[1] == pytest.approx(b, rel=1e-14)
    p, nl, nv = th.pure_saturation(comp, tr * Tc)
    assert nl == pytest.approx(rl, rel=1e-4)
    assert nv == pytest.approx(rv, rel=1e-4)


def test_maxwell_equal_area_independently():
    """The saturation pair satisfies the equal-area rule, checked by quadrature of the
    isotherm p(v) in specific volume (scipy), independent of ln phi."""
    from scipy.integrate import quad
    a, b, omega, tr = 2 / 49, 2 / 21, 0.344, 0.9
    Tc = (th.OMEGA_B / th.OMEGA_A) * (a / b)
    comp = th.Component("pure", Tc, th.OMEGA_B * Tc / b, omega, 1.0)
    T = tr * Tc
    p, nl, nv = th.pure_saturation(comp, T)
    pv = lambda v: th.pressure([comp], [[0.0]], T, 1.0, [1.0 / v])
    area, _ = quad(lambda v: pv(v) - p, 1 / nl, 1 / nv, limit=400, epsabs=1e-13, epsrel=1e-12)
    assert abs(area) < 1e-9 * p * (1 / nv - 1 / nl)
    assert pv(1 / nl) == pytest.approx(p, rel=1e-9)
    assert pv(1 / nv) == pytest.approx(p, rel=1e-9)


def test_ln_phi_is_partial_molar_of_mixture_residual_gibbs():
    """ln phi_i = d(n g_R)/dn_i at fixed T, p with g_R = Z - 1 - ln(Z - B) - A/(2 sqrt2 B)
    ln[(Z + (1+sqrt2)B)/(Z + (1-sqrt2)B)] the residual Gibbs energy of the mixture: a finite
    difference of the mixture quantity pins Eq. fugacitycoeff2 term by term."""
    comps = _c3_nc5()
    kij = [[0.0, 0.03], [0.03, 0.0]]
    T, p = 666.06, 200.0
    s2 = math.sqrt(2)

    def nG(nvec, which):
        n = sum(nvec)
        c = [v / n for v in nvec]
        _, _, _, A, B = th.coefficients(comps, kij, T, p, c)
        r = th.z_roots(A, B)
        Z = r[0] if which == "l" else r[-1]
        g = Z - 1 - math.log(Z - B) - A / (2 * s2 * B) * math.log((Z + (1 + s2) * B) / (Z + (1 - s2) * B))
        return n * g

    for which, c in (("l", [0.3, 0.7]), ("v", [0.65, 0.35])):
        _, lp = th.phase_state(comps, kij, T, p, c, which=which)
        h = 1e-6
        for i in range(2):
            up = list(c); up[i] += h
            dn = list(c); dn[i] -= h
            fd = (nG(up, which) - nG(dn, which)) / (2 * h)
            assert fd == pytest.approx(lp[i], rel=1e-6, abs=1e-8)


def test_cubic_roots_satisfy_the_eos():
    """Each selected Z gives back the pressure through Eq. MCPengRobinson at n = p/(Z R T)."""
    comps = _c3_nc5()
    for p in (140.0, 200.0, 240.0):
        fr = th.flash(comps, KIJ0, T_TABLE2, p, Z_TABLE2)
        for Z, c in ((fr.Zl, fr.x), (fr.Zv, fr.y)):
            n = p / (Z * R_FIELD * T_TABLE2)
            got = th.pressure(comps, KIJ0, T_TABLE2, R_FIELD, [n * ci for ci in c])
            assert got == pytest.approx(p, rel=1e-10)


def test_gibbs_selection_switches_at_saturation():
    """Eq. solutionselection: for a pure fluid dG = 0 exactly at saturation; above it the liquid
    root is chosen, below it the vapour root."""
    Tc = (th.OMEGA_B / th.OMEGA_A) * (th.A1_LB / th.B1_LB)
    comp = th.Component("pure", Tc, th.OMEGA_B * Tc / th.B1_LB, 0.344, 1.0)
    T = 0.9 * Tc
    p, _, _ = th.pure_saturation(comp, T)
    for fac, want in ((1.02, "l"), (0.98, "v")):
        _, _, _, A, B = th.coefficients([comp], [[0.0]], T, p * fac, [1.0])
        r = th.z_roots(A, B)
        assert len(r) == 3
        z = th.select_root(r, A, B)
        assert z == (r[0] if want == "l" else r[-1])
    _, _, _, A, B = th.coefficients([comp], [[0.0]], T, p, [1.0])
    r = th.z_roots(A, B)
    assert abs(th.gibbs_dG(r[0], r[-1], A, B)) < 1e-9


def test_ideal_gas_limit():
    """A, B -> 0 (low pressure, high temperature): Z -> 1 and ln phi -> 0."""
    comps = _c3_nc5()
    Z, lp = th.phase_state(comps, KIJ0, 3000.0, 1e-3, [0.5, 0.5])
    assert Z == pytest.approx(1.0, abs=1e-6)
    assert max(abs(v) for v in lp) < 1e-6


def test_lattice_units_scaling():
    """a_1 = 2/49, b_1 = 2/21, R = 1 fix T_c1 = (Omega_b/Omega_a)(a_1/b_1) = 0.0729220 and
    p_c1 = Omega_b T_c1 / b_1 = 0.0595700; reduced quantities are unchanged, so the flash in
    lattice units returns the same Z, x, y as in field units."""
    comps = _c3_nc5()
    lb, ts, ps = th.lattice_components(comps)
    assert lb[0].Tc == pytest.approx(0.0729220, rel=1e-6)
    assert lb[0].pc == pytest.approx(0.0595700, rel=1e-6)
    assert th.a_b(lb[0], 1.0)[0] == pytest.approx(2 / 49, rel=1e-12)
    assert th.a_b(lb[0], 1.0)[1] == pytest.approx(2 / 21, rel=1e-12)
    assert lb[0].M == 1.0
    f1 = th.flash(comps, KIJ0, T_TABLE2, 200.0, Z_TABLE2)
    f2 = th.flash(lb, KIJ0, T_TABLE2 * ts, 200.0 * ps, Z_TABLE2)
    assert f2.Zl == pytest.approx(f1.Zl, rel=1e-9)
    assert f2.Zv == pytest.approx(f1.Zv, rel=1e-9)
    assert f2.x[0] == pytest.approx(f1.x[0], rel=1e-9)


def test_residual_vanishes_only_at_equilibrium():
    """Eq. error is zero at the flash solution and positive for perturbed phase compositions."""
    comps = _c3_nc5()
    fr = th.flash(comps, KIJ0, T_TABLE2, 200.0, Z_TABLE2)
    fl, _ = th.fugacities(comps, KIJ0, T_TABLE2, 200.0, fr.x)
    fv, _ = th.fugacities(comps, KIJ0, T_TABLE2, 200.0, fr.y)
    assert th.iso_fugacity_residual(fl, fv) < 1e-20
    x2 = [fr.x[0] * 1.05, 1 - fr.x[0] * 1.05]
    fl2, _ = th.fugacities(comps, KIJ0, T_TABLE2, 200.0, x2)
    assert th.iso_fugacity_residual(fl2, fv) > 1e-4


def test_gamma_identical_components_is_one():
    """Two copies of one component: both have the same K, so Eq. gamma gives gamma = 1."""
    rl, rv = [3.0, 2.0], [0.3, 0.2]  # same phase-density ratio, as for identical components
    g, _ = th.gamma_coefficients(rl, rv, [0.1, 0.1])
    assert g == pytest.approx([1.0, 1.0])


def test_workload_cases_are_flash_consistent(cases):
    """The stored workload constants satisfy iso-fugacity at their (T, p) in lattice units."""
    for key in ("c1", "c2", "c3", "c5"):
        c = cases[key]
        comps = [th.Component(d["name"], d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]
        fl, _ = th.fugacities(comps, c["kij"], c["T"], c["p"], c["x"])
        fv, _ = th.fugacities(comps, c["kij"], c["T"], c["p"], c["y"])
        assert th.iso_fugacity_residual(fl, fv) < 1e-16
        assert min(c["gamma"]) > 0 and max(c["gamma"]) == 1.0
