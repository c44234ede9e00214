"""Writes tests/golden/long_runs.npz: FP64 oracle results of the full-length 2-D workloads, at
sampled sites, for the GPU parity tests at the stated step counts.

  * droplet (D2Q9 MRT, 3 components, 512^2, 20000 steps): densities of every component at the
    sampled sites, and the per-component mass.
  * adjoint droplet (D2Q9 BGK, 2 components, 256^2, 3000 steps, zeta_12 = 0): densities at the
    sampled sites, and dL/dzeta_12, dL/ds of the loss L = sum w rho^2 / 2 (w from SplitMix64,
    seed 99) by forward-mode dual numbers.

Every number comes from oracle/ (the FP64 CPU oracle) and the seeded input module.
Run:  OMP_NUM_THREADS=<cores> python tests/golden/make_long_runs.py [droplet] [adjoint]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import lbm_inputs  # noqa: E402
import oracle  # noqa: E402
from lbm_cases import initial_rho, oracle_case  # noqa: E402

OUT = os.path.join(HERE, "long_runs.npz")


def sample_sites(shape, n, seed):
    """n distinct site indices (y, x) of a 2-D grid, SplitMix64 draws plus the centre and a corner."""
    nx, ny = shape
    u = lbm_inputs.uniform01(seed, 2 * n)
    ys = np.minimum((u[:n] * ny).astype(int), ny - 1)
    xs = np.minimum((u[n:] * nx).astype(int), nx - 1)
    ys = np.concatenate([[ny // 2, 0], ys])
    xs = np.concatenate([[nx // 2, 0], xs])
    return ys, xs


def main():
    with open(os.path.join(HERE, "cases.json")) as fh:
        cases = json.load(fh)
    which = set(sys.argv[1:]) or {"droplet", "adjoint"}
    data = dict(np.load(OUT)) if os.path.exists(OUT) else {}
    if "droplet" in which:
        c = cases["c2"]
        shape = tuple(c["shape"])
        case = oracle_case(c, shape)
        rho0 = initial_rho(c, shape)
        t0 = time.time()
        f = oracle.step(case, oracle.equilibrium(case, rho0), c["steps"])
        rho = oracle.fields(case, f).rho
        ys, xs = sample_sites(shape, 4096, 2024)
        data["droplet_sites"] = np.stack([ys, xs])
        data["droplet_rho"] = rho[:, ys, xs]
        data["droplet_mass"] = oracle.mass(f)
        data["droplet_steps"] = np.array(c["steps"])
        print("droplet done in %.0f s" % (time.time() - t0), flush=True)
    if "adjoint" in which:
        c = cases["c5"]
        shape = tuple(c["shape"])
        grid = tuple(reversed(shape))
        rho0 = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], c["init"]["radius"], 4.0)
        w = lbm_inputs.uniform01(99, rho0.size).reshape(rho0.shape)
        g = np.array(c["gamma"])
        oc = oracle_case(dict(c, Q=9), shape, collision=0, kij=[[0.0, 0.0], [0.0, 0.0]], gamma=list(g))
        f0 = oracle.equilibrium(oc, rho0)
        df0 = np.zeros((2,) + f0.shape)
        dk = np.zeros((2, 2, 2))
        dk[0, 0, 1] = dk[0, 1, 0] = 1.0
        dg = np.zeros((2, 2))
        dg[1, 0] = g[0]
        t0 = time.time()
        f, df = oracle.step_dual(oc, f0, df0, dk, dg, c["steps"])
        rho = f.sum(axis=1)
        drho = df.sum(axis=2)
        gl = w * rho
        ys, xs = sample_sites(shape, 2048, 2025)
        data["adjoint_sites"] = np.stack([ys, xs])
        data["adjoint_rho"] = rho[:, ys, xs]
        data["adjoint_loss"] = np.array(0.5 * np.sum(w * rho * rho))
        data["adjoint_dk12"] = np.array(np.sum(gl * drho[0]))
        data["adjoint_ds"] = np.array(np.sum(gl * drho[1]))
        data["adjoint_steps"] = np.array(c["steps"])
        print("adjoint done in %.0f s: dL/dk12 %.10e dL/ds %.10e" % (time.time() - t0, data["adjoint_dk12"],
                                                                      data["adjoint_ds"]), flush=True)
    np.savez_compressed(OUT, **data)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
