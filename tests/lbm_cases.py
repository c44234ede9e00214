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
