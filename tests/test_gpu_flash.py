"""lbm_flash (the batched GPU flash of Section 3.2) against the FP64 oracle flash and against
Table 2 of the paper."""
import json
import os

import numpy as np
import pytest

from conftest import GOLDEN, read_table
from oracle import thermo as th

pytestmark = pytest.mark.gpu

R_FIELD = 10.7316  # psia ft^3 / (lbmol degR), the field units of Table 2
T_TABLE2 = 666.06
Z_TABLE2 = [0.4, 0.6]


def _table1():
    return {r[0]: (r[2], r[1], r[3], r[4]) for r in read_table("table1_components.txt")}


@pytest.fixture(scope="module")
def sweep():
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        return json.load(fh)["c4"]


def test_flash_matches_oracle_on_the_sweep_cases(sweep):
    """All 512 flash-sweep cases (C1/nC4, 0.75-0.95 T_pc, C1 feed 0.1-0.6; lattice units)
    against the oracle flash written into the case file: phase compositions, roots, K,
    vapour fraction, phase densities and gamma."""
    from paper_1909_12390_gb300 import lbm
    cs = sweep["cases"]
    comps = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in cs[0]["components"]]
    for c in cs:
        assert [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]] == comps
    T = np.array([c["T"] for c in cs])
    p = np.array([c["p"] for c in cs])
    z = np.array([c["z"] for c in cs])
    kij = np.array([c["kij"] for c in cs])
    r = lbm.flash(comps, T, p, z, kij, R=1.0)
    assert np.all(r["status"] == lbm.FLASH_TWO_PHASE)
    assert np.all(r["residual"] < 1e-20)

    def rel(a, b):
        return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))

    assert rel(r["x"], [c["x"] for c in cs]) < 1e-10
    assert rel(r["y"], [c["y"] for c in cs]) < 1e-10
    assert rel(r["Zl"], [c["Zl"] for c in cs]) < 1e-10
    assert rel(r["Zv"], [c["Zv"] for c in cs]) < 1e-10
    assert rel(r["K"], [c["K"] for c in cs]) < 1e-10
    assert float(np.max(np.abs(r["V"] - np.array([c["V"] for c in cs])))) < 1e-10
    assert rel(r["rho_l"], [c["rho_l"] for c in cs]) < 1e-10
    assert rel(r["rho_v"], [c["rho_v"] for c in cs]) < 1e-10
    assert rel(r["gamma"], [c["gamma"] for c in cs]) < 1e-9


@pytest.mark.parametrize("row", [r for r in read_table("table2_c3_nc5.txt") if r[2] is not None and r[1] is not None])
def test_flash_reproduces_table2(row):
    """Table 2 (40 % C3 / 60 % nC5 at T_c,C3, field units): the two-phase rows' Z, x, y,
    partial densities and gamma_1, within the table's printed precision."""
    from paper_1909_12390_gb300 import lbm
    t = _table1()
    comps = [t["C3"], t["nC5"]]
    pr, zl, zv, x1, y1, r1l, r2l, r1v, r2v, g1 = row
    r = lbm.flash(comps, [T_TABLE2], [pr], [Z_TABLE2], R=R_FIELD)
    assert r["status"][0] == lbm.FLASH_TWO_PHASE
    assert r["Zl"][0] == pytest.approx(zl, rel=5e-4)
    assert r["Zv"][0] == pytest.approx(zv, rel=5e-4)
    assert r["x"][0, 0] == pytest.approx(x1, rel=5e-4)
    assert r["y"][0, 0] == pytest.approx(y1, rel=5e-4)
    # printed to 3 decimals; the table's own rounding (x, Z) adds up to ~1e-3 relative
    for got, want in ((r["rho_l"][0, 0], r1l), (r["rho_l"][0, 1], r2l), (r["rho_v"][0, 0], r1v),
                      (r["rho_v"][0, 1], r2v)):
        assert got == pytest.approx(want, abs=5e-4 + 6e-4 * want)
    assert r["gamma"][0, 0] == pytest.approx(g1, abs=1e-4)


def test_flash_single_phase_and_agreement_with_oracle_flags():
    """Far above the two-phase window the flash is single phase (status 1), as the oracle's
    trivial flag says; inside it both give two phases with the same vapour fraction."""
    from paper_1909_12390_gb300 import lbm
    t = _table1()
    comps = [t["C3"], t["nC5"]]
    pcs = [2000.0, 200.0, 40.0]
    r = lbm.flash(comps, [T_TABLE2] * 3, pcs, [Z_TABLE2] * 3, R=R_FIELD)
    for k, pr in enumerate(pcs):
        fr = th.flash([th.Component("a", *comps[0]), th.Component("b", *comps[1])], [[0.0, 0.0], [0.0, 0.0]],
                      T_TABLE2, pr, Z_TABLE2)
        assert (r["status"][k] == lbm.FLASH_SINGLE) == fr.trivial, pr
        if not fr.trivial:
            assert r["V"][k] == pytest.approx(fr.V, abs=1e-10)


def test_flash_with_binary_interaction_matches_oracle():
    """Non-zero zeta_12 (the adjoint workload's target value 0.02 and 0.1) on C1/nC4 in
    lattice units, against the oracle flash."""
    from paper_1909_12390_gb300 import lbm
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        c = json.load(fh)["c4"]["cases"][17]
    comps = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]
    for zeta in (0.02, 0.1):
        kij = [[0.0, zeta], [zeta, 0.0]]
        fr = th.flash([th.Component("a", *comps[0]), th.Component("b", *comps[1])], kij, c["T"], c["p"], c["z"])
        r = lbm.flash(comps, [c["T"]], [c["p"]], [c["z"]], [kij], R=1.0)
        assert r["status"][0] == (lbm.FLASH_SINGLE if fr.trivial else lbm.FLASH_TWO_PHASE)
        if not fr.trivial:
            assert np.allclose(r["x"][0], fr.x, rtol=1e-10, atol=0)
            assert np.allclose(r["y"][0], fr.y, rtol=1e-10, atol=0)
            assert r["Zl"][0] == pytest.approx(fr.Zl, rel=1e-10)
            assert r["Zv"][0] == pytest.approx(fr.Zv, rel=1e-10)
