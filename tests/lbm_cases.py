"""Test helpers: build the oracle problem and the CUDA lattice of one workload from the
constants in tests/golden/cases.json, and their shared seeded initial fields."""
import numpy as np

import lbm_inputs
import oracle

PREC = {"fp64": 0, "fp32s": 1}
COLL = {"bgk": 0, "mrt": 1}


def comps_of(c):
    return [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]


def oracle_case(c, shape, collision=None, s=None, **over):
    k = comps_of(c)
    coll = COLL[c.get("collision", "bgk")] if collision is None else collision
    rates = s if s is not None else c.get("mrt_s")
    args = dict(Q=9 if len(shape) == 2 else 19, shape=tuple(shape), Tc=[x[0] for x in k],
                pc=[x[1] for x in k], omega=[x[2] for x in k], M=[x[3] for x in k], T=c["T"],
                tau=c.get("tau", 0.8), gamma=list(c["gamma"]), kij=c["kij"], beta=c.get("beta", 1.0),
                G=c["G"], collision=coll, s=rates if coll else None)
    args.update(over)
    return oracle.Case(**args)


def gpu_lattice(c, shape, precision, collision=None, s=None, **over):
    from paper_1909_12390_gb300 import lbm
    coll = COLL[c.get("collision", "bgk")] if collision is None else collision
    rates = s if s is not None else c.get("mrt_s")
    kw = dict(T=c["T"], tau=c.get("tau", 0.8), gamma=list(c["gamma"]),
              kij=np.array(c["kij"], dtype=float), beta=c.get("beta", 1.0), G=c["G"],
              collision=coll, mrt_rates=rates if coll else None, precision=precision)
    kw.update(over)
    return lbm.Lattice(tuple(shape), comps_of(c), **kw)


def initial_rho(c, shape):
    """The workload's initial component densities on grid `shape` (x first)."""
    grid = tuple(reversed(shape))
    ini = c["init"]
    if ini["kind"] == "slab":
        axis = {"x": len(grid) - 1, "y": len(grid) - 2, "z": 0}[ini["axis"]]
        return lbm_inputs.slab_fields(grid, c["rho_l"], c["rho_v"], ini["lo"], ini["hi"],
                                      ini["width"], ini.get("noise", 0.0), ini.get("seed", 0), axis=axis)
    return lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], ini["radius"], ini["width"])


def random_rho(c, grid, seed):
    """Densities drawn between the vapour and liquid values of each component."""
    u = lbm_inputs.uniform01(seed, int(np.prod(grid)) * len(c["rho_l"])).reshape((len(c["rho_l"]),) + tuple(grid))
    lo = np.array(c["rho_v"]).reshape((-1,) + (1,) * len(grid))
    hi = np.array(c["rho_l"]).reshape((-1,) + (1,) * len(grid))
    return lo + (hi - lo) * u


def _erode(liq, e):
    """(all-liquid, any-liquid) over the periodic L-infinity box of half-width e."""
    all_l, any_l = liq.copy(), liq.copy()
    for axis in range(liq.ndim):
        a2, b2 = np.ones_like(all_l), np.zeros_like(any_l)
        for d in range(-e, e + 1):
            a2 &= np.roll(all_l, d, axis=axis)
            b2 |= np.roll(any_l, d, axis=axis)
        all_l, any_l = a2, b2
    return all_l, any_l


def bulk_masks(rho, erode=8):
    """Bulk liquid and vapour cells of a state: farther than `erode` cells (L-infinity) from the
    (max + min) / 2 contour of the total density."""
    tot = rho.sum(axis=0)
    liq = tot > 0.5 * (tot.max() + tot.min())
    all_l, any_l = _erode(liq, erode)
    return all_l, ~any_l


def composition_profile_loss(rho, target, M, erode=8):
    """The adjoint workload's loss and its gradient with respect to rho (numpy, FP64):
    L = sum_i (x_i - x_i^T)^2 + sum_i (y_i - y_i^T)^2 + mean_x (rho(x) - rho^T(x))^2, with x, y the
    molar compositions of the mean bulk liquid / vapour partial densities (each state its own
    bulk masks) and rho the total density. The masks are piecewise constant in rho, so the
    gradient treats them as fixed."""
    M = np.asarray(M, dtype=float)
    nc = rho.shape[0]
    shp = (nc,) + (1,) * (rho.ndim - 1)

    def comp(r, mask):
        rbar = np.array([r[c][mask].mean() for c in range(nc)])
        n = rbar / M
        return n / n.sum(), n.sum(), int(mask.sum())

    bl, bv = bulk_masks(rho, erode)
    tl, tv = bulk_masks(target, erode)
    x, nl, Nl = comp(rho, bl)
    y, nv, Nv = comp(rho, bv)
    xT, _, _ = comp(target, tl)
    yT, _, _ = comp(target, tv)
    tot, totT = rho.sum(0), target.sum(0)
    N = tot.size
    L = float(np.sum((x - xT) ** 2) + np.sum((y - yT) ** 2) + np.mean((tot - totT) ** 2))
    g = np.broadcast_to(2.0 * (tot - totT) / N, rho.shape).copy()
    for comp_, ref, n, cnt, mask in ((x, xT, nl, Nl, bl), (y, yT, nv, Nv, bv)):
        # d comp_i / d rho_c(site) = (delta_ic - comp_i) / (n M_c cnt) on the bulk cells
        w = 2.0 * (comp_ - ref)
        for c in range(nc):
            dc = (w[c] - np.dot(w, comp_)) / (n * M[c] * cnt)
            g[c][mask] += dc
    return L, g
