"""Two-phase diagnostics of a lattice state (plain numpy, FP64): the checks of Sections 4.2
and 4.3 of Peng, Ayala & Ayala, arXiv:1909.12390.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke(), bench.py's cpu_baseline /
reference leg and the case-writing scripts beside the golden files may import this module.
It shares no code with the CUDA library.

What it computes:
  * the contour level of the total density rho = sum_s rho_s: a given level, else
    (max + min) / 2 (the rho = (rho_l + rho_v) / 2 contour of Section 4.3);
  * the bulk phases: cells whose whole (2e + 1)^D box (periodic) lies above (liquid) or below
    (vapour) the level -- farther than e cells from the contour in the L-infinity norm
    (reading: the paper measures bulk values away from the interface, e = 8);
  * their mean component densities and EOS pressures, molar compositions x / y, and the
    iso-fugacity residual of Eq. error with ln phi_i of Eq. fugacitycoeff2 at Z = p/(n R T);
  * the liquid cell count, the equivalent radius (sqrt(V / pi) in 2-D, cbrt(3 V / (4 pi)) in
    3-D) and the pressure jump p_l - p_v of Laplace's law (Section 4.3).
"""
from __future__ import annotations

import math

import numpy as np

from . import thermo as th


def erode_masks(liq: np.ndarray, e: int):
    """(all-liquid, any-liquid) over the periodic L-infinity box of half-width e."""
    all_l = liq.copy()
    any_l = liq.copy()
    for axis in range(liq.ndim):
        n = liq.shape[axis]
        w = min(e, n)
        a2 = np.ones_like(all_l)
        b2 = np.zeros_like(any_l)
        for d in range(-w, w + 1):
            a2 &= np.roll(all_l, d, axis=axis)
            b2 |= np.roll(any_l, d, axis=axis)
        all_l, any_l = a2, b2
    return all_l, any_l


def bulk_diagnostics(comps, kij, T, R, rho: np.ndarray, p: np.ndarray, erode: int = 8, threshold: float = 0.0):
    """comps: thermo.Component list (lattice units), rho: (nc, *grid) cell-volume densities,
    p: (*grid) EOS pressure. Returns a dict with the quantities of the module docstring."""
    nc = rho.shape[0]
    tot = rho.sum(axis=0)
    thr = threshold if threshold > 0 else 0.5 * (float(tot.max()) + float(tot.min()))
    liq = tot > thr
    all_l, any_l = erode_masks(liq, erode)
    bl, bv = all_l, ~any_l
    out = dict(threshold=thr, rho_max=float(tot.max()), rho_min=float(tot.min()),
               n_l=int(bl.sum()), n_v=int(bv.sum()), liquid_cells=int(liq.sum()))
    M = np.array([k.M for k in comps])
    rl = np.array([rho[c][bl].mean() if bl.any() else math.nan for c in range(nc)])
    rv = np.array([rho[c][bv].mean() if bv.any() else math.nan for c in range(nc)])
    pl = float(p[bl].mean()) if bl.any() else math.nan
    pv = float(p[bv].mean()) if bv.any() else math.nan
    nl, nv = rl / M, rv / M
    x, y = nl / nl.sum(), nv / nv.sum()
    res = math.nan
    if bl.any() and bv.any():
        lp = []
        for c, n, pp in ((x, nl.sum(), pl), (y, nv.sum(), pv)):
            _, Bi, Aij, A, B = th.coefficients(comps, kij, T, pp, list(c))
            Z = pp / (n * R * T)
            lp.append(th.ln_phi(Z, A, B, Aij, Bi, list(c)))
        res = sum((math.exp(a - b) * xi * pl / (yi * pv) - 1.0) ** 2 for a, b, xi, yi in zip(lp[0], lp[1], x, y))
    D = rho.ndim - 1
    V = float(liq.sum())
    out.update(rho_l=rl, rho_v=rv, p_l=pl, p_v=pv, x=x, y=y, residual=res,
               radius=math.sqrt(V / math.pi) if D == 2 else (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0),
               dp=pl - pv)
    return out
