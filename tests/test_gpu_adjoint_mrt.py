"""The hand-written adjoint with the MRT collision (lbm_record / lbm_adjoint on an LBM_MRT
lattice) against the FP64 oracle's MRT step differentiated by forward-mode dual numbers, and
against central finite differences. The MRT relaxation K = w I + M^T Lam M is symmetric for the
orthogonal moment basis, so the adjoint's collision part relaxes the adjoint populations with
the same K; these tests pin that reading, the Guo term's (I - K / 2) and every other part of the
reverse step on D2Q9 (fused reverse kernel, ragged tiles included) and D3Q19."""
import json
import os

import numpy as np
import pytest

import lbm_inputs
import oracle
from conftest import GOLDEN
from lbm_cases import comps_of, oracle_case

pytestmark = pytest.mark.gpu

FP64, FP32S = 0, 1


@pytest.fixture(scope="module")
def cases():
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        return json.load(fh)


def _mixture(cases, Q):
    """The adjoint workload's binary mixture with the D2Q9 MRT rates (Q = 9), or the 3-component
    sphere mixture with its D3Q19 rates (Q = 19)."""
    if Q == 9:
        return dict(cases["c5"], mrt_s=cases["c2"]["mrt_s"])
    return cases["c3"]


def _setup(c, shape):
    grid = tuple(reversed(shape))
    rho0 = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], min(shape) / 3.0, 3.0,
                                  center=[g / 2 - 0.35 for g in grid])
    w = lbm_inputs.uniform01(99, rho0.size).reshape(rho0.shape)
    return rho0, w


def _loss_grad(rho, w):
    """L = sum w rho^2 / 2 -> dL/drho = w rho."""
    return 0.5 * float(np.sum(w * rho * rho)), w * rho


def _kij(nc, k12):
    k = np.zeros((nc, nc))
    k[0, 1] = k[1, 0] = k12
    return k


def _gpu_run(c, shape, rho0, precision, k12, s, steps, K):
    from paper_1909_12390_gb300 import lbm
    nc = len(c["gamma"])
    g = np.array(c["gamma"], dtype=float)
    g[0] *= s
    lat = lbm.Lattice(shape, comps_of(c), T=c["T"], tau=c["tau"], gamma=g, kij=_kij(nc, k12), beta=c["beta"],
                      G=c["G"], collision=lbm.MRT, mrt_rates=c["mrt_s"], precision=precision)
    lat.init(rho0)
    lat.record(steps, K)
    return lat


def _oracle_grads(c, shape, rho0, w, k12, s, steps):
    """Loss, dL/dzeta_12 and dL/ds (gamma_0 = s gamma0_0) from the oracle's MRT step in dual
    numbers."""
    nc = len(c["gamma"])
    g0 = np.array(c["gamma"], dtype=float)
    g = g0.copy()
    g[0] *= s
    oc = oracle_case(dict(c, Q=9 if len(shape) == 2 else 19), shape, collision=1, s=c["mrt_s"],
                     kij=_kij(nc, k12).tolist(), gamma=list(g))
    f0 = oracle.equilibrium(oc, rho0)
    df0 = np.zeros((2,) + f0.shape)
    dk = np.zeros((2, nc, nc))
    dk[0, 0, 1] = dk[0, 1, 0] = 1.0          # direction 0: d/dzeta_12
    dg = np.zeros((2, nc))
    dg[1, 0] = g0[0]                          # direction 1: d/ds
    f, df = oracle.step_dual(oc, f0, df0, dk, dg, steps)
    rho = f.sum(axis=1)
    drho = df.sum(axis=2)
    L, gl = _loss_grad(rho, w)
    return L, float(np.sum(gl * drho[0])), float(np.sum(gl * drho[1])), rho


@pytest.mark.parametrize("Q,shape,steps,K", [(9, (32, 24), 40, 7), (9, (37, 13), 30, 30), (9, (12, 6), 20, 6),
                                             (19, (10, 8, 6), 12, 5)])
def test_mrt_adjoint_fp64_matches_oracle_duals(cases, Q, shape, steps, K):
    c = _mixture(cases, Q)
    rho0, w = _setup(c, shape)
    k12, s = 0.01, 1.1
    lat = _gpu_run(c, shape, rho0, FP64, k12, s, steps, K)
    rho = lat.fields(u=False, p=False, psi=False)["rho"]
    _, gl = _loss_grad(rho, w)
    dk, dgam, _ = lat.adjoint(gl)
    lat.close()
    Lo, ok12, os_, rho_o = _oracle_grads(c, shape, rho0, w, k12, s, steps)
    assert np.max(np.abs(rho - rho_o) / rho_o) < 1e-11
    dk12 = dk[0, 1] + dk[1, 0]
    ds = dgam[0] * c["gamma"][0]
    print("MRT Q%d %s: dL/dk12 %.12e (oracle %.12e)  dL/ds %.12e (oracle %.12e)" % (Q, shape, dk12, ok12, ds, os_))
    assert dk12 == pytest.approx(ok12, rel=1e-8)
    assert ds == pytest.approx(os_, rel=1e-8)


@pytest.mark.parametrize("Q,shape", [(9, (32, 24)), (19, (10, 8, 6))])
def test_mrt_adjoint_initial_density_gradient_matches_central_differences(cases, Q, shape):
    """dL/drho(0) along one seeded direction against central differences with h = 1e-5 (FP64)."""
    c = _mixture(cases, Q)
    rho0, w = _setup(c, shape)
    k12, s, h, steps = 0.02, 1.0, 1e-5, 20

    def L_of(r0):
        lt = _gpu_run(c, shape, r0, FP64, k12, s, steps, steps)
        v_ = _loss_grad(lt.fields(u=False, p=False, psi=False)["rho"], w)[0]
        lt.close()
        return v_

    lat = _gpu_run(c, shape, rho0, FP64, k12, s, steps, 6)
    _, gl = _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)
    _, _, d0 = lat.adjoint(gl)
    lat.close()
    v = lbm_inputs.uniform01(7, rho0.size).reshape(rho0.shape) - 0.5
    fd = (L_of(rho0 + h * v) - L_of(rho0 - h * v)) / (2 * h)
    assert float(np.sum(d0 * v)) == pytest.approx(fd, rel=1e-6)


def test_mrt_adjoint_fp32_matches_fp64_oracle(cases):
    """FP32-shifted storage, 150 steps in segments of 55, against the FP64 oracle's duals."""
    c = _mixture(cases, 9)
    shape = (64, 48)
    rho0, w = _setup(c, shape)
    k12, s, steps = 0.0, 1.0, 150
    lat = _gpu_run(c, shape, rho0, FP32S, k12, s, steps, 55)
    _, gl = _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)
    dk, dgam, _ = lat.adjoint(gl)
    lat.close()
    Lo, ok12, os_, _ = _oracle_grads(c, shape, rho0, w, k12, s, steps)
    print("MRT fp32: dL/dk12 %.6e (oracle %.6e)  dL/ds %.6e (oracle %.6e)"
          % (dk[0, 1] + dk[1, 0], ok12, dgam[0] * c["gamma"][0], os_))
    assert dk[0, 1] + dk[1, 0] == pytest.approx(ok12, rel=2e-3)
    assert dgam[0] * c["gamma"][0] == pytest.approx(os_, rel=2e-3)


def test_mrt_autograd_function_matches_oracle_duals(cases):
    """LatticeRun with the MRT collision: dL/dzeta_12 and dL/ds through torch's backward equal
    the oracle's MRT dual numbers (FP64)."""
    import torch
    from paper_1909_12390_gb300 import lbm
    from paper_1909_12390_gb300.autograd import LatticeRun
    c = _mixture(cases, 9)
    shape, steps, k12 = (32, 24), 24, 0.01
    rho0, w = _setup(c, shape)
    spec = dict(shape=shape, components=comps_of(c), T=c["T"], tau=c["tau"], gamma=c["gamma"], beta=c["beta"],
                G=c["G"], collision=lbm.MRT, mrt_rates=c["mrt_s"], precision=FP64, rho0=rho0, steps=steps,
                checkpoint_every=8)
    zeta = torch.tensor(k12, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    rho = LatticeRun.apply(zeta, s, spec)
    loss = 0.5 * (torch.from_numpy(w) * rho * rho).sum()
    loss.backward()
    Lo, ok12, os_, _ = _oracle_grads(c, shape, rho0, w, k12, 1.0, steps)
    assert float(loss) == pytest.approx(Lo, rel=1e-11)
    assert float(zeta.grad) == pytest.approx(ok12, rel=1e-8)
    assert float(s.grad) == pytest.approx(os_, rel=1e-8)
