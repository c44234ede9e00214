"""Writes tests/golden/long_runs.npz: FP64 oracle results of the full-length 2-D workloads, at
sampled sites, for the GPU parity tests at the stated step counts.

  * droplet (D2Q9 MRT, 3 components, 512^2, 20000 steps): densities of every component at the
    sampled sites, and the per-component mass.
  * adjoint droplet (D2Q9 BGK, 2 components, 256^2, 3000 steps, zeta_12 = 0): densities at the
    sampled sites, and dL/dzeta_12, dL/ds of the loss L = sum w rho^2 / 2 (w from SplitMix64,
    seed 99) by forward-mode dual numbers.
  * adjoint workload loss ("adjoint_loss"): the same run and its dual derivatives, with the loss
    the workload states: squared errors of the bulk liquid / vapour molar compositions and
    mean squared error of the total density profile against a target run at zeta_12 = 0.02
    (tests/lbm_cases.composition_profile_loss); dL/dzeta_12, dL/ds at zeta_12 = 0, s = 1.
  * slab (D2Q9 BGK FP64, 2 components, 64^2, 2000 steps): the densities of every site and the
    per-component mass.
  * sweep (the batched flash sweep, D2Q9 BGK, 2 components, 10000 steps): the densities of
    every site of cases 0, 137 and 411.
  * sphere (D3Q19 MRT, 3 components, FP64, 5000 steps) on a 96^3 box with R = 18, the
    256^3 / R = 48 workload's liquid fraction and constants at the size the host cores can step
    5000 times: densities at sampled sites (z, y, x) and the per-component mass.

Every number comes from oracle/ (the FP64 CPU oracle) and the seeded input module.
Run:  OMP_NUM_THREADS=<cores> python tests/golden/make_long_runs.py [droplet] [adjoint] [adjoint_loss] [slab]
        [sweep] [sphere]
(with no argument: droplet and adjoint)
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
from lbm_cases import composition_profile_loss, initial_rho, oracle_case  # noqa: E402

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
    if "adjoint_loss" in which:
        c = cases["c5"]
        shape = tuple(c["shape"])
        grid = tuple(reversed(shape))
        rho0 = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], c["init"]["radius"], 4.0)
        g = np.array(c["gamma"])
        kt = float(c["target_k12"])
        t0 = time.time()
        tc = oracle_case(dict(c, Q=9), shape, collision=0, kij=[[0.0, kt], [kt, 0.0]], gamma=list(g))
        target = oracle.step(tc, oracle.equilibrium(tc, rho0), c["steps"]).sum(axis=1)
        oc = oracle_case(dict(c, Q=9), shape, collision=0, kij=[[0.0, 0.0], [0.0, 0.0]], gamma=list(g))
        f0 = oracle.equilibrium(oc, rho0)
        dk = np.zeros((2, 2, 2))
        dk[0, 0, 1] = dk[0, 1, 0] = 1.0
        dg = np.zeros((2, 2))
        dg[1, 0] = g[0]
        f, df = oracle.step_dual(oc, f0, np.zeros((2,) + f0.shape), dk, dg, c["steps"])
        rho = f.sum(axis=1)
        drho = df.sum(axis=2)
        M = [d["M"] for d in c["components"]]
        L, gl = composition_profile_loss(rho, target, M)
        ys, xs = sample_sites(shape, 2048, 2026)
        data["loss_target_sites"] = np.stack([ys, xs])
        data["loss_target_rho"] = target[:, ys, xs]
        data["loss_value"] = np.array(L)
        data["loss_dk12"] = np.array(np.sum(gl * drho[0]))
        data["loss_ds"] = np.array(np.sum(gl * drho[1]))
        data["loss_steps"] = np.array(c["steps"])
        print("adjoint loss done in %.0f s: L %.6e dL/dk12 %.10e dL/ds %.10e" % (
            time.time() - t0, L, data["loss_dk12"], data["loss_ds"]), flush=True)
    if "slab" in which:
        c = cases["c1"]
        shape = tuple(c["shape"])
        case = oracle_case(c, shape)
        f = oracle.step(case, oracle.equilibrium(case, initial_rho(c, shape)), c["steps"])
        data["slab_rho"] = oracle.fields(case, f).rho
        data["slab_mass"] = oracle.mass(f)
        data["slab_steps"] = np.array(c["steps"])
        print("slab done", flush=True)
    if "sweep" in which:
        sw = cases["c4"]
        picked = [0, 137, 411]
        for i in picked:
            c = dict(sw["cases"][i], tau=sw["tau"], beta=sw["beta"], Q=9)
            shape = tuple(c["shape"])
            case = oracle_case(c, shape, collision=0)
            f = oracle.step(case, oracle.equilibrium(case, initial_rho(c, shape)), sw["steps"])
            data["sweep_rho_%d" % i] = oracle.fields(case, f).rho
        data["sweep_cases"] = np.array(picked)
        data["sweep_steps"] = np.array(sw["steps"])
        print("sweep done", flush=True)
    if "sphere" in which:
        c = cases["c3"]
        n, R = 96, 18.0
        shape = (n, n, n)
        case = oracle_case(c, shape)
        rho0 = initial_rho(dict(c, init=dict(c["init"], radius=R)), shape)
        t0 = time.time()
        f = oracle.step(case, oracle.equilibrium(case, rho0), c["steps"])
        rho = oracle.fields(case, f).rho
        u = lbm_inputs.uniform01(2027, 3 * 4096)
        zs, ys, xs = (np.minimum((u[k * 4096:(k + 1) * 4096] * n).astype(int), n - 1) for k in range(3))
        line = np.arange(n)
        zs = np.concatenate([[n // 2, 0], np.full(n, n // 2), zs])
        ys = np.concatenate([[n // 2, 0], np.full(n, n // 2), ys])
        xs = np.concatenate([[n // 2, 0], line, xs])
        data["sphere_shape"] = np.array(shape)
        data["sphere_radius"] = np.array(R)
        data["sphere_sites"] = np.stack([zs, ys, xs])
        data["sphere_rho"] = rho[:, zs, ys, xs]
        data["sphere_mass"] = oracle.mass(f)
        data["sphere_steps"] = np.array(c["steps"])
        print("sphere done in %.0f s" % (time.time() - t0), flush=True)
    np.savez_compressed(OUT, **data)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
