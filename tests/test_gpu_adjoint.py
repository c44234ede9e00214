"""The hand-written adjoint (lbm_record / lbm_adjoint) against the FP64 oracle differentiated
by forward-mode dual numbers, against central finite differences, and its torch
autograd.Function."""
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
def case5():
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        return json.load(fh)["c5"]


def _setup(c, shape, radius):
    grid = tuple(reversed(shape))
    rho0 = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], radius, 4.0,
                                  center=[g / 2 - 0.35 for g in grid])
    w = lbm_inputs.uniform01(99, rho0.size).reshape(rho0.shape)
    return rho0, w


def _loss_grad(rho, w):
    """L = sum w rho^2 / 2 -> dL/drho = w rho."""
    return 0.5 * float(np.sum(w * rho * rho)), w * rho


def _gpu_run(c, shape, rho0, precision, k12, s, steps, K):
    from paper_1909_12390_gb300 import lbm
    g = np.array(c["gamma"]) * np.array([s, 1.0])
    kij = np.array([[0.0, k12], [k12, 0.0]])
    lat = lbm.Lattice(shape, comps_of(c), T=c["T"], tau=c["tau"], gamma=g, kij=kij, beta=c["beta"],
                      G=c["G"], precision=precision)
    lat.init(rho0)
    lat.record(steps, K)
    return lat, g


def _oracle_grads(c, shape, rho0, w, k12, steps, s=1.0):
    g0 = np.array(c["gamma"])
    g = g0 * np.array([s, 1.0])
    oc = oracle_case(dict(c, Q=9), shape, collision=0, kij=[[0.0, k12], [k12, 0.0]], gamma=list(g))
    f0 = oracle.equilibrium(oc, rho0)
    df0 = np.zeros((2,) + f0.shape)
    dk = np.zeros((2, 2, 2))
    dk[0, 0, 1] = dk[0, 1, 0] = 1.0          # direction 0: d/dk12
    dg = np.zeros((2, 2))
    dg[1, 0] = g0[0]                          # direction 1: d/ds, gamma_0 = s g0_0
    f, df = oracle.step_dual(oc, f0, df0, dk, dg, steps)
    rho = f.sum(axis=1)
    drho = df.sum(axis=2)
    L, gl = _loss_grad(rho, w)
    return L, float(np.sum(gl * drho[0])), float(np.sum(gl * drho[1])), rho


@pytest.mark.parametrize("K,s", [(7, 1.0), (1, 1.0), (60, 1.0), (7, 1.3)])
def test_adjoint_fp64_matches_oracle_duals(case5, K, s):
    c = case5
    shape = (32, 24)
    steps = 60
    rho0, w = _setup(c, shape, 6.0)
    k12 = 0.01
    lat, g = _gpu_run(c, shape, rho0, FP64, k12, s, steps, K)
    rho = lat.fields(u=False, p=False, psi=False)["rho"]
    L, gl = _loss_grad(rho, w)
    dk, dgam, d0 = lat.adjoint(gl)
    dk12 = dk[0, 1] + dk[1, 0]
    ds = dgam[0] * c["gamma"][0]  # gamma_0 = s gamma0_0
    Lo, ok12, os_, rho_o = _oracle_grads(c, shape, rho0, w, k12, steps, s)
    assert np.max(np.abs(rho - rho_o) / rho_o) < 1e-11
    print("K=%d dL/dk12 %.12e (oracle %.12e)  dL/ds %.12e (oracle %.12e)" % (K, dk12, ok12, ds, os_))
    assert dk12 == pytest.approx(ok12, rel=1e-8)
    assert ds == pytest.approx(os_, rel=1e-8)


def test_adjoint_fp64_matches_central_differences(case5):
    """Central differences with h = 1e-5 on the FP64 path for zeta_12, s and one initial
    density direction."""
    c = case5
    shape = (32, 24)
    steps = 40
    rho0, w = _setup(c, shape, 6.0)
    k12, s, h = 0.02, 1.0, 1e-5

    def L_of(k, sc, r0):
        lat, _ = _gpu_run(c, shape, r0, FP64, k, sc, steps, steps)
        return _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)[0]

    lat, g = _gpu_run(c, shape, rho0, FP64, k12, s, steps, 9)
    _, gl = _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)
    dk, dgam, d0 = lat.adjoint(gl)
    fd_k = (L_of(k12 + h, s, rho0) - L_of(k12 - h, s, rho0)) / (2 * h)
    fd_s = (L_of(k12, s + h, rho0) - L_of(k12, s - h, rho0)) / (2 * h)
    v = lbm_inputs.uniform01(7, rho0.size).reshape(rho0.shape) - 0.5
    fd_r = (L_of(k12, s, rho0 + h * v) - L_of(k12, s, rho0 - h * v)) / (2 * h)
    assert dk[0, 1] + dk[1, 0] == pytest.approx(fd_k, rel=1e-6)
    assert dgam[0] * g[0] == pytest.approx(fd_s, rel=1e-6)
    assert float(np.sum(d0 * v)) == pytest.approx(fd_r, rel=1e-6)


def test_adjoint_fp32_matches_fp64_oracle(case5):
    c = case5
    shape = (64, 48)
    steps = 150
    rho0, w = _setup(c, shape, 12.0)
    k12 = 0.0
    lat, g = _gpu_run(c, shape, rho0, FP32S, k12, 1.0, steps, 55)
    _, gl = _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)
    dk, dgam, _ = lat.adjoint(gl)
    Lo, ok12, os_, _ = _oracle_grads(c, shape, rho0, w, k12, steps)
    print("fp32: dL/dk12 %.6e (oracle %.6e)  dL/ds %.6e (oracle %.6e)" % (dk[0, 1] + dk[1, 0], ok12, dgam[0] * g[0], os_))
    assert dk[0, 1] + dk[1, 0] == pytest.approx(ok12, rel=2e-3)
    assert dgam[0] * g[0] == pytest.approx(os_, rel=2e-3)


@pytest.mark.parametrize("s0", [1.0, 1.3])
def test_autograd_function_gradients(case5, s0):
    """torch.autograd.Function wrapper: its gradients equal the oracle's dual numbers, also at
    a split-factor scale s != 1 (dL/ds = sum_k dL/dgamma_k gamma0_k, not s times that)."""
    import torch
    from paper_1909_12390_gb300 import lbm
    from paper_1909_12390_gb300.autograd import LatticeRun
    c = case5
    shape = (32, 24)
    rho0, w = _setup(c, shape, 6.0)
    spec = dict(shape=shape, components=comps_of(c), T=c["T"], tau=c["tau"], gamma=c["gamma"],
                beta=c["beta"], G=c["G"], steps=30, checkpoint_every=8, rho0=rho0, precision=lbm.FP64,
                pair=(0, 1), least_volatile=1)
    zeta = torch.tensor(0.01, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(s0, dtype=torch.float64, requires_grad=True)
    rho = LatticeRun.apply(zeta, s, spec)
    loss = 0.5 * (torch.from_numpy(w) * rho * rho).sum()
    loss.backward()
    _, ok12, os_, _ = _oracle_grads(c, shape, rho0, w, 0.01, 30, s0)
    assert zeta.grad.item() == pytest.approx(ok12, rel=1e-8)
    assert s.grad.item() == pytest.approx(os_, rel=1e-8)


def test_adjoint_full_workload_against_stored_duals(case5):
    """The adjoint workload at full size: D2Q9 BGK binary droplet 256^2, FP32 forward with the
    FP64 EOS, 3000 steps, checkpoints every 55 steps; dL/dzeta_12 and dL/ds against the FP64
    oracle differentiated by dual numbers (tests/golden/make_long_runs.py). Prints the cost of
    the backward pass relative to the forward run."""
    import time
    p = os.path.join(GOLDEN, "long_runs.npz")
    ref = dict(np.load(p)) if os.path.exists(p) else {}
    if "adjoint_dk12" not in ref:
        pytest.skip("long_runs.npz has no adjoint reference")
    c = case5
    shape = tuple(c["shape"])
    grid = tuple(reversed(shape))
    rho0 = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], c["init"]["radius"], 4.0)
    w = lbm_inputs.uniform01(99, rho0.size).reshape(rho0.shape)
    from paper_1909_12390_gb300 import lbm
    g = np.array(c["gamma"])
    lat = lbm.Lattice(shape, comps_of(c), T=c["T"], tau=c["tau"], gamma=g, kij=np.zeros((2, 2)), beta=c["beta"],
                      G=c["G"], precision=FP32S)
    lat.init(rho0)
    lat.step(1)  # warm-up
    lat.init(rho0)
    t0 = time.perf_counter()
    lat.step(int(ref["adjoint_steps"]))
    t_plain = time.perf_counter() - t0
    lat.init(rho0)
    t0 = time.perf_counter()
    lat.record(int(ref["adjoint_steps"]), c["checkpoint_every"])
    t_fwd = time.perf_counter() - t0
    rho = lat.fields(u=False, p=False, psi=False)["rho"]
    ys, xs = ref["adjoint_sites"]
    assert float(np.max(np.abs(rho[:, ys, xs] - ref["adjoint_rho"]) / ref["adjoint_rho"].sum(0))) < 2e-4
    t0 = time.perf_counter()
    dk, dg, _ = lat.adjoint(w * rho)
    t_adj = time.perf_counter() - t0
    dk12, ds = dk[0, 1] + dk[1, 0], dg[0] * g[0]
    print("adjoint workload: dL/dk12 %.6e (oracle %.6e), dL/ds %.6e (oracle %.6e); forward %.3f s, "
          "recorded forward %.3f s, backward %.3f s (%.2f x the forward)"
          % (dk12, ref["adjoint_dk12"], ds, ref["adjoint_ds"], t_plain, t_fwd, t_adj, t_adj / t_plain))
    assert dk12 == pytest.approx(float(ref["adjoint_dk12"]), rel=5e-3)
    assert ds == pytest.approx(float(ref["adjoint_ds"]), rel=5e-3)


def test_workload_loss_gradient_against_oracle_duals(case5):
    """The adjoint workload as stated: D2Q9 BGK binary droplet 256^2, FP32 forward with the FP64
    EOS, 3000 steps, checkpoints every 55 steps; loss = squared errors of the bulk liquid and
    vapour molar compositions plus the mean squared error of the density profile against a
    target run at zeta_12 = 0.02 (paper_1909_12390_gb300.losses); gradient with respect to
    zeta_12 and the split-factor scale s at zeta_12 = 0, s = 1 through LatticeRun, against the
    FP64 oracle's dual numbers with the oracle's own target run (tests/golden/make_long_runs.py).
    The loss compares two states that differ only through zeta_12, so its terms are differences
    of nearly equal quantities (|x - x^T| ~ 1e-3) and carry the FP32 state error (~1e-5 of the
    densities) magnified about a hundredfold: tolerance 2e-2. Prints the cost of the recorded
    forward run and the backward pass relative to a plain forward run."""
    import time

    import torch
    p = os.path.join(GOLDEN, "long_runs.npz")
    ref = dict(np.load(p)) if os.path.exists(p) else {}
    if "loss_dk12" not in ref:
        pytest.skip("long_runs.npz has no workload-loss reference")
    from paper_1909_12390_gb300 import lbm
    from paper_1909_12390_gb300.autograd import LatticeRun
    from paper_1909_12390_gb300.losses import composition_profile_loss
    c = case5
    shape = tuple(c["shape"])
    grid = tuple(reversed(shape))
    rho0 = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], c["init"]["radius"], 4.0)
    steps, K = int(ref["loss_steps"]), c["checkpoint_every"]
    kt = float(c["target_k12"])
    tgt = lbm.Lattice(shape, comps_of(c), T=c["T"], tau=c["tau"], gamma=c["gamma"],
                      kij=np.array([[0.0, kt], [kt, 0.0]]), beta=c["beta"], G=c["G"], precision=FP32S)
    tgt.init(rho0)
    tgt.step(1)
    tgt.init(rho0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tgt.step(steps)
    t_plain = time.perf_counter() - t0
    target = tgt.fields(u=False, p=False, psi=False)["rho"]
    tgt.close()
    ys, xs = ref["loss_target_sites"]
    assert float(np.max(np.abs(target[:, ys, xs] - ref["loss_target_rho"]) / ref["loss_target_rho"].sum(0))) < 2e-4
    spec = dict(shape=shape, components=comps_of(c), T=c["T"], tau=c["tau"], gamma=c["gamma"], beta=c["beta"],
                G=c["G"], steps=steps, checkpoint_every=K, rho0=rho0, precision=lbm.FP32_SHIFTED, pair=(0, 1),
                least_volatile=int(c["least_volatile"]))
    zeta = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    t0 = time.perf_counter()
    rho = LatticeRun.apply(zeta, s, spec)
    t_rec = time.perf_counter() - t0
    L = composition_profile_loss(rho, torch.from_numpy(target), [d["M"] for d in c["components"]])
    t0 = time.perf_counter()
    L.backward()
    t_back = time.perf_counter() - t0
    print("workload loss: L %.6e (oracle %.6e); dL/dk12 %.6e (oracle %.6e); dL/ds %.6e (oracle %.6e); "
          "forward %.3f s, recorded forward %.3f s, backward %.3f s: (record + backward) / forward = %.2f"
          % (float(L.detach()), float(ref["loss_value"]), zeta.grad.item(), float(ref["loss_dk12"]), s.grad.item(),
             float(ref["loss_ds"]), t_plain, t_rec, t_back, (t_rec + t_back) / t_plain))
    assert float(L.detach()) == pytest.approx(float(ref["loss_value"]), rel=2e-2)
    assert zeta.grad.item() == pytest.approx(float(ref["loss_dk12"]), rel=2e-2)
    assert s.grad.item() == pytest.approx(float(ref["loss_ds"]), rel=2e-2)


@pytest.mark.parametrize("precision", [FP64, FP32S])
@pytest.mark.parametrize("K,snaps", [(60, 1), (60, 2), (60, 3), (60, 7), (20, 2), (25, 4)])
def test_revolve_checkpointing_equals_full_storage(case5, precision, K, snaps):
    """Revolve-style binomial checkpointing with few state slots recomputes the states it
    needs; they are bit-identical to the recorded ones, so every gradient equals the
    full-storage schedule's bit for bit (60 steps: one segment of 60, three of 20, or 25 + 25 +
    10 with a short last segment)."""
    c = case5
    shape = (32, 24)
    steps = 60
    rho0, w = _setup(c, shape, 6.0)
    out = []
    for mem in (0, snaps):
        lat, g = _gpu_run(c, shape, rho0, precision, 0.01, 1.3, steps, K)
        lat.set_adjoint_memory(mem)
        _, gl = _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)
        out.append(lat.adjoint(gl))
        lat.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [FP64, FP32S])
def test_overlapped_replay_equals_serial_order(case5, precision):
    """The replay of the next segment runs on its own stream beside the current segment's
    reverse sweep (a second set of state slots); the serial order, used when that set cannot
    be allocated, gives the same gradients bit for bit (60 steps in three segments of 20 and
    in 25 + 25 + 10)."""
    c = case5
    shape = (32, 24)
    rho0, w = _setup(c, shape, 6.0)
    for K in (20, 25):
        out = []
        for on in (True, False):
            lat, g = _gpu_run(c, shape, rho0, precision, 0.01, 1.3, 60, K)
            lat.test_adjoint_overlap(on)
            _, gl = _loss_grad(lat.fields(u=False, p=False, psi=False)["rho"], w)
            out.append(lat.adjoint(gl))
            lat.close()
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [(37, 13), (12, 6), (45, 9)])
def test_adjoint_ragged_grids_match_oracle(case5, shape):
    """Grids that are no multiple of the fused reverse kernel's 32 x 8 tiles (ragged last tiles,
    and a grid smaller than one tile, whose halo wraps onto the tile itself): dL/dzeta_12 and
    dL/ds against the oracle's dual numbers, dL/drho(0) along one direction against central
    differences (FP64 path, K = 7: segments of 7 and a short last one)."""
    c = case5
    steps, K, k12, s, h = 30, 7, 0.01, 1.0, 1e-5
    rho0, w = _setup(c, shape, min(shape) / 3.0)
    lat, g = _gpu_run(c, shape, rho0, FP64, k12, s, steps, K)
    rho = lat.fields(u=False, p=False, psi=False)["rho"]
    _, gl = _loss_grad(rho, w)
    dk, dgam, d0 = lat.adjoint(gl)
    lat.close()
    Lo, ok12, os_, rho_o = _oracle_grads(c, shape, rho0, w, k12, steps, s)
    assert np.max(np.abs(rho - rho_o) / rho_o) < 1e-11
    assert dk[0, 1] + dk[1, 0] == pytest.approx(ok12, rel=1e-8)
    assert dgam[0] * c["gamma"][0] == pytest.approx(os_, rel=1e-8)

    def L_of(r0):
        lt, _ = _gpu_run(c, shape, r0, FP64, k12, s, steps, steps)
        v_ = _loss_grad(lt.fields(u=False, p=False, psi=False)["rho"], w)[0]
        lt.close()
        return v_

    v = lbm_inputs.uniform01(11, rho0.size).reshape(rho0.shape) - 0.5
    fd = (L_of(rho0 + h * v) - L_of(rho0 - h * v)) / (2 * h)
    assert float(np.sum(d0 * v)) == pytest.approx(fd, rel=1e-6)
