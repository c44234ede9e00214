"""Benchmark of the multi-component pseudo-potential LB step on one GB300.

Workload: the 3-component (C1/C3/nC5) D3Q19 MRT sphere on a 256^3 periodic grid with FP32
populations stored shifted and an FP64 EOS (constants from tests/golden/cases.json, seeded
synthetic initial fields from lbm_inputs). One "step" is one full time step of the lattice:
pseudo-potential pass + force / split / collide / in-place stream pass.

Prints one JSON line. `value` is component-MLUPS (sites x components x steps / s) over the
device-timed region with the populations resident in HBM; `e2e` is the same metric through
the C ABI with host buffers (lbm_init from host densities, the steps, lbm_fields back to host
densities) inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the oracle (FP64 CPU, the test oracle) is timed on the host cores on a
bounded sample of the same workload; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "component-MLUPS (D3Q19 MRT, FP32-shifted populations, FP64 EOS)"
PATH_NAMES = {1: "two-kernel", 2: "fused", 3: "trailing", 4: "queue"}
# what the FP32-shifted path computes in which precision
EOS_PRECISION = ("FP64: the EOS sums B, A2, the numerator and denominator of p (their cancellation); "
                 "FP32: n_i = rho_i / M_i, the quotient p = pD / Dd, psi = sqrt(psi^2), moments, force, collision; "
                 "mass (S7): compensated FP32 sums per thread reduced in FP64")
UNIT = "MLUPS/component"
WORKLOAD = "sphere_d3q19_fp32s_mrt: 3 components C1/C3/nC5, 256^3 periodic, droplet R=48"


def load_case(key="c3"):
    with open(os.path.join(ROOT, "tests", "golden", "cases.json")) as fh:
        return json.load(fh)[key]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha():
    """Hash of what defines the benchmarked kernels (k_psi, k_collide, k_fused3, k_trail3 of the
    D3Q19 FP32-shifted MRT unit): their headers, the unit and the build flags."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1909_12390_gb300")
    files = [os.path.join("csrc", f) for f in ("lbm_core.cuh", "lbm_kernels.cuh", "lbm_fused3.cuh", "lbm_trail3.cuh",
                                               "lbm_trailq.cuh",
                                               "lbm_ops.h", "lbm_d3q19_f32s_mrt.cu")] + ["build.py"]
    for fn in files:
        with open(os.path.join(pkg, fn), "rb") as fh:
            h.update(fn.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel sources; otherwise None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(kernel_name)
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def init_fields(c):
    import lbm_inputs
    grid = tuple(reversed(c["shape"]))
    return lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], c["init"]["radius"], c["init"]["width"])


def lattice_for(c, precision):
    from paper_1909_12390_gb300 import lbm
    comps = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]
    return lbm.Lattice(tuple(c["shape"]), comps, T=c["T"], tau=c["tau"], gamma=c["gamma"],
                       kij=np.array(c["kij"], dtype=float), beta=c["beta"], G=c["G"],
                       collision=lbm.MRT if c["collision"] == "mrt" else lbm.BGK,
                       mrt_rates=c.get("mrt_s"), precision=precision)


def _oracle_sample(c, n):
    import lbm_inputs
    import oracle
    k = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]
    case = oracle.Case(Q=19, shape=(n, n, n), Tc=[x[0] for x in k], pc=[x[1] for x in k],
                       omega=[x[2] for x in k], M=[x[3] for x in k], T=c["T"], tau=c["tau"],
                       gamma=c["gamma"], kij=c["kij"], beta=c["beta"], G=c["G"], collision=1,
                       s=c["mrt_s"])
    rho = lbm_inputs.ball_fields((n, n, n), c["rho_l"], c["rho_v"], 48.0 * n / 256, c["init"]["width"])
    return case, oracle.equilibrium(case, rho), rho


def cpu_baseline(c, target_s=12.0, n=64):
    """The oracle as it stands on the host cores: D3Q19 MRT steps of a periodic n^3 sample of
    the workload (same constants, droplet radius scaled with the box), timed until about
    target_s of CPU work. Returns the baseline entry and the sample's end state (case, initial
    densities, steps taken, final populations)."""
    import oracle
    case, f, rho0 = _oracle_sample(c, n)
    f = oracle.step(case, f, 1)  # warm-up (thread pool, pages)
    steps, t0 = 0, time.perf_counter()
    while True:
        f = oracle.step(case, f, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el > target_s:
            break
    val = n ** 3 * case.nc * steps / el / 1e6
    return ({"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
             "sample": "%d steps of a periodic %d^3 D3Q19 MRT FP64 sample of the workload (3 components)"
                       % (steps, n)}, (case, rho0, steps + 1, f))


def accuracy(c, sample):
    """Error of the FP32-shifted and FP64 paths against the oracle on the baseline's sample:
    the same initial densities and step count on the GPU, max over sites and components of
    |rho_s - rho_s,oracle| / sum_s rho_s,oracle."""
    import oracle
    from paper_1909_12390_gb300 import lbm
    case, rho0, steps, f = sample
    ro = oracle.fields(case, f).rho
    n = rho0.shape[-1]
    cs = dict(c, shape=[n, n, n])
    out = {"measure": "max over sites and components of |rho_s - rho_s,oracle| / sum_s rho_s,oracle",
           "sample": "periodic %d^3 sample of the workload after %d steps (the cpu_baseline run)" % (n, steps)}
    for name, prec in (("fp32s", lbm.FP32_SHIFTED), ("fp64", lbm.FP64)):
        g = lattice_for(cs, prec)
        g.init(rho0)
        g.step(steps)
        rg = g.fields(u=False, p=False, psi=False)["rho"]
        g.close()
        out[name] = float(np.max(np.abs(rg - ro) / ro.sum(0)))
    out["tolerance"] = {"fp32s": 2e-4, "fp64": 1e-10}
    return out


def run_reference(args, rank):
    """Reference arm: the oracle on the host cores, one oracle step of a periodic 32^3 sample
    of the workload per benchmark step."""
    if rank != 0:
        return
    import oracle
    c = load_case()
    n = 32
    case, f, _ = _oracle_sample(c, n)
    f = oracle.step(case, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.step(case, f, args.steps)
    el = time.perf_counter() - t0
    val = n ** 3 * case.nc * args.steps / el / 1e6
    sample = "periodic %d^3 D3Q19 MRT FP64 sample of the workload per step (3 components)" % n
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference", "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (the job's time is its slowest replica's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(sites, components, steps, world, ms):
    """Whole-job component-MLUPS of `world` replicas of `sites` sites each over `ms` ms."""
    return sites * components * steps * world / (ms / 1e3) / 1e6


def flash_variant(reps=5):
    """lbm_flash over the 512 cases of the flash sweep (the state that sets each case up),
    host clock around the C-ABI call (host structs, copies and the kernel), best of reps."""
    from paper_1909_12390_gb300 import lbm
    with open(os.path.join(ROOT, "tests", "golden", "cases.json")) as fh:
        cs = json.load(fh)["c4"]["cases"]
    comps = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in cs[0]["components"]]
    T = [c["T"] for c in cs]
    p = [c["p"] for c in cs]
    z = [c["z"] for c in cs]
    kij = [c["kij"] for c in cs]
    best, r = None, None
    for _ in range(reps):
        t0 = time.perf_counter()
        r = lbm.flash(comps, T, p, z, kij)
        el = time.perf_counter() - t0
        best = el if best is None else min(best, el)
    return {"cases": len(cs), "ms_per_call": best * 1e3, "flashes_per_s": len(cs) / best,
            "iterations_max": int(np.max(r["iterations"])), "two_phase": int(np.sum(r["status"] == 0))}


def case_fields(c):
    """Initial component densities of a workload of tests/golden/cases.json (its slab or
    droplet recipe), grid (nz,) ny, nx."""
    import lbm_inputs
    grid = tuple(reversed(c["shape"]))
    ini = c["init"]
    if ini["kind"] == "slab":
        axis = {"x": len(grid) - 1, "y": len(grid) - 2, "z": 0}[ini["axis"]]
        return lbm_inputs.slab_fields(grid, c["rho_l"], c["rho_v"], ini["lo"], ini["hi"], ini["width"],
                                      ini.get("noise", 0.0), ini.get("seed", 0), axis=axis)
    return lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], ini["radius"], ini["width"])


def l2_variants(stream, steps=2000):
    """The workloads whose populations fit in L2 (129 MB), reported in MLUPS and algorithmic
    bytes per site update rather than as a fraction of HBM bandwidth: the FP64 BGK slab (64^2),
    the FP32-shifted MRT droplet (512^2) and the FP32-shifted BGK adjoint droplet (256^2), each
    on the library's automatic path, CUDA-event timed over `steps` steps after 20 warm-up steps
    (no L2 flush: these states are L2-resident by size)."""
    import torch

    from paper_1909_12390_gb300 import lbm
    out = {}
    for key in ("c1", "c2", "c5"):
        c = load_case(key)
        fp64 = c["precision"] == "fp64"
        g = lattice_for(c, lbm.FP64 if fp64 else lbm.FP32_SHIFTED)
        g.init(case_fields(c))
        g.step(20)
        g.set_stream(stream.cuda_stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        path = PATH_NAMES[g.path]
        g.close()
        nc, n = len(c["components"]), int(np.prod(c["shape"]))
        q = 19 if len(c["shape"]) == 3 else 9
        bps = 2 * q * nc * (8 if fp64 else 4)
        out[key] = {"workload": c["name"], "value": n * nc / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                    "steps": steps, "path": path, "alg_bytes_per_site_update": bps,
                    "footprint_mb": n * q * nc * (8 if fp64 else 4) / 1e6}
    return out


def batched_variant(stream, steps=10000):
    """The batched flash sweep (512 independent D2Q9 BGK binary slabs of 64-256 x 8 sites,
    FP32-shifted, one block per case in shared memory) timed over its stated 10000 steps after
    the autotuner picked block sizes."""
    import torch

    import lbm_inputs
    from paper_1909_12390_gb300 import lbm
    with open(os.path.join(ROOT, "tests", "golden", "cases.json")) as fh:
        sw = json.load(fh)["c4"]
    specs, rhos = _sweep_specs(sw)
    b = lbm.Batch(specs, precision=lbm.FP32_SHIFTED)
    b.init(rhos)
    report = b.tune(20)
    b.step(100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    el = time.perf_counter() - t0
    sites = sum(s["shape"][0] * s["shape"][1] for s in specs)
    b.close()
    return {"value": sites * 2 * steps / el / 1e6, "unit": UNIT, "cases": len(specs), "sites": sites,
            "steps": steps, "ms_per_step": el / steps * 1e3, "timing": "host clock around lbm_batch_step",
            "tune": report}


def _load_refs():
    p = os.path.join(ROOT, "tests", "golden", "long_runs.npz")
    return dict(np.load(p)) if os.path.exists(p) else {}


def config_checks():
    """Every workload at its stated step count on the library's automatic path against the
    stored FP64 oracle runs (tests/golden/long_runs.npz, written by the committed script beside
    it from oracle/ only). Error measure: max over the compared sites and components of
    |rho_s - rho_s,oracle| / sum_s rho_s,oracle (FP64: / rho_s,oracle)."""
    from paper_1909_12390_gb300 import lbm
    ref = _load_refs()
    out = {}

    def err(got, want, fp64):
        return float(np.max(np.abs(got - want) / (want if fp64 else want.sum(0))))

    def run(c, shape, precision, steps, rho0):
        g = lattice_for(dict(c, shape=list(shape)), precision)
        g.init(rho0)
        t0 = time.perf_counter()
        g.step(steps)
        el = time.perf_counter() - t0
        rho = g.fields(u=False, p=False, psi=False)["rho"]
        m = g.mass()
        path = PATH_NAMES[g.path]
        g.close()
        return rho, m, el, path

    if "slab_rho" in ref:
        c = load_case("c1")
        rho, m, el, path = run(c, c["shape"], lbm.FP64, int(ref["slab_steps"]), case_fields(c))
        out["c1_slab"] = {"steps": int(ref["slab_steps"]), "err": err(rho, ref["slab_rho"], True), "tolerance": 1e-10,
                          "compared": "every site", "mass_rel_err": float(np.max(np.abs(m / ref["slab_mass"] - 1))),
                          "path": path, "host_s": el}
    if "droplet_rho" in ref:
        c = load_case("c2")
        rho, m, el, path = run(c, c["shape"], lbm.FP32_SHIFTED, int(ref["droplet_steps"]), case_fields(c))
        ys, xs = ref["droplet_sites"]
        out["c2_droplet"] = {"steps": int(ref["droplet_steps"]), "err": err(rho[:, ys, xs], ref["droplet_rho"], False),
                             "tolerance": 2e-4, "compared": "%d sampled sites" % len(ys),
                             "mass_rel_err": float(np.max(np.abs(m / ref["droplet_mass"] - 1))), "path": path,
                             "host_s": el}
    if "sphere_rho" in ref:
        c = load_case("c3")
        shape = [int(v) for v in ref["sphere_shape"]]
        cc = dict(c, shape=shape, init=dict(c["init"], radius=float(ref["sphere_radius"])))
        rho, m, el, path = run(cc, shape, lbm.FP32_SHIFTED, int(ref["sphere_steps"]), init_fields(cc))
        zs, ys, xs = ref["sphere_sites"]
        out["c3_sphere"] = {"steps": int(ref["sphere_steps"]), "grid": shape, "radius": float(ref["sphere_radius"]),
                            "err": err(rho[:, zs, ys, xs], ref["sphere_rho"], False), "tolerance": 2e-4,
                            "compared": "%d sampled sites" % len(zs),
                            "mass_rel_err": float(np.max(np.abs(m / ref["sphere_mass"] - 1))), "path": path,
                            "host_s": el,
                            "note": "the 256^3 workload's mixture, state and liquid fraction on the box the oracle "
                                    "can step 5000 times"}
    if "sweep_cases" in ref:
        with open(os.path.join(ROOT, "tests", "golden", "cases.json")) as fh:
            sw = json.load(fh)["c4"]
        specs, rhos = _sweep_specs(sw)
        b = lbm.Batch(specs, precision=lbm.FP32_SHIFTED)
        b.init(rhos)
        b.tune(20)
        b.init(rhos)
        t0 = time.perf_counter()
        b.step(int(ref["sweep_steps"]))
        el = time.perf_counter() - t0
        got = b.rho()
        b.close()
        e = max(err(got[i], ref["sweep_rho_%d" % i], False) for i in ref["sweep_cases"])
        out["c4_sweep"] = {"steps": int(ref["sweep_steps"]), "err": e, "tolerance": 2e-4,
                           "compared": "every site of cases %s" % list(map(int, ref["sweep_cases"])),
                           "cases": len(specs), "host_s": el}
    if "adjoint_rho" in ref:
        c = load_case("c5")
        grid = tuple(reversed(c["shape"]))
        rho0 = init_fields_ball(c, grid)
        rho, m, el, path = run(c, c["shape"], lbm.FP32_SHIFTED, int(ref["adjoint_steps"]), rho0)
        ys, xs = ref["adjoint_sites"]
        out["c5_adjoint_droplet"] = {"steps": int(ref["adjoint_steps"]),
                                     "err": err(rho[:, ys, xs], ref["adjoint_rho"], False), "tolerance": 2e-4,
                                     "compared": "%d sampled sites (the forward run of the adjoint workload)" % len(ys),
                                     "path": path, "host_s": el}
    return out


def init_fields_ball(c, grid):
    import lbm_inputs
    return lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], c["init"]["radius"], 4.0)


def _sweep_specs(sw):
    import lbm_inputs
    specs, rhos = [], []
    for c in sw["cases"]:
        nx, ny = c["shape"]
        ini = c["init"]
        rhos.append(lbm_inputs.slab_fields((ny, nx), c["rho_l"], c["rho_v"], ini["lo"], ini["hi"], ini["width"],
                                           ini["noise"], ini["seed"], axis=1))
        specs.append(dict(shape=c["shape"], components=[(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]],
                          T=c["T"], tau=sw["tau"], gamma=c["gamma"], kij=np.array(c["kij"]), beta=sw["beta"], G=c["G"]))
    return specs, rhos


def adjoint_variant():
    """The adjoint workload as stated (D2Q9 BGK binary droplet 256^2, FP32 forward, FP64 EOS,
    3000 steps, checkpoints every 55 steps, loss on the bulk compositions and the density
    profile against a target run at zeta_12 = 0.02; gradient with respect to zeta_12 and the
    split-factor scale at zeta_12 = 0, s = 1) through LatticeRun and loss.backward(), host clock
    around each call (each synchronises), after one untimed evaluation. Reports (recorded forward + backward) / plain forward
    and the gradients against the FP64 oracle's dual numbers (stored run)."""
    import torch

    from paper_1909_12390_gb300 import lbm
    from paper_1909_12390_gb300.autograd import LatticeRun
    from paper_1909_12390_gb300.losses import composition_profile_loss
    c = load_case("c5")
    ref = _load_refs()
    shape = tuple(c["shape"])
    rho0 = init_fields_ball(c, tuple(reversed(shape)))
    comps = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]
    kt = float(c["target_k12"])
    g = lbm.Lattice(shape, comps, T=c["T"], tau=c["tau"], gamma=c["gamma"], kij=np.array([[0.0, kt], [kt, 0.0]]),
                    beta=c["beta"], G=c["G"], precision=lbm.FP32_SHIFTED)
    g.init(rho0)
    g.step(10)
    g.init(rho0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(c["steps"])
    t_fwd = time.perf_counter() - t0
    target = g.fields(u=False, p=False, psi=False)["rho"]
    g.close()
    spec = dict(shape=shape, components=comps, T=c["T"], tau=c["tau"], gamma=c["gamma"], beta=c["beta"], G=c["G"],
                steps=c["steps"], checkpoint_every=c["checkpoint_every"], rho0=rho0, precision=lbm.FP32_SHIFTED,
                pair=(0, 1), least_volatile=int(c["least_volatile"]))
    M = [d["M"] for d in c["components"]]
    # one untimed gradient evaluation first, as the forward run above had its warm-up steps:
    # the first adjoint call of a process loads its kernels (lazy module loading)
    zw = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    sw = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    composition_profile_loss(LatticeRun.apply(zw, sw, spec), torch.from_numpy(target), M).backward()
    zeta = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    t0 = time.perf_counter()
    rho = LatticeRun.apply(zeta, s, spec)
    t_rec = time.perf_counter() - t0
    L = composition_profile_loss(rho, torch.from_numpy(target), M)
    t0 = time.perf_counter()
    L.backward()
    t_back = time.perf_counter() - t0
    out = {"steps": c["steps"], "checkpoint_every": c["checkpoint_every"], "forward_s": t_fwd,
           "recorded_forward_s": t_rec, "backward_s": t_back, "cost_vs_forward": (t_rec + t_back) / t_fwd,
           "target": 3.0, "loss": float(L.detach()), "dL_dk12": zeta.grad.item(), "dL_ds": s.grad.item(),
           "timing": "host clock around lbm_step / LatticeRun.apply / loss.backward (each synchronises), "
                     "after one untimed gradient evaluation"}
    if "loss_dk12" in ref:
        out["oracle"] = {"loss": float(ref["loss_value"]), "dL_dk12": float(ref["loss_dk12"]),
                         "dL_ds": float(ref["loss_ds"])}
        out["rel_err"] = {"dL_dk12": abs(zeta.grad.item() / float(ref["loss_dk12"]) - 1),
                          "dL_ds": abs(s.grad.item() / float(ref["loss_ds"]) - 1)}
    return out


def cpu_baselines(budget_s=2.5):
    """The oracle as it stands on the host cores for each workload, on one core and on all of
    them: a bounded sample of each (stated), steps timed until about budget_s per setting."""
    import lbm_inputs
    import oracle
    cores = oracle.threads()
    out = {}

    def timed(case, f):
        f = oracle.step(case, f, 1)
        n, t0 = 0, time.perf_counter()
        while True:
            f = oracle.step(case, f, 1)
            n += 1
            el = time.perf_counter() - t0
            if el > budget_s:
                return case.nsites * case.nc * n / el / 1e6, n

    def case_of(c, shape, Q):
        k = [(d["Tc"], d["pc"], d["omega"], d["M"]) for d in c["components"]]
        coll = 1 if c.get("collision") == "mrt" else 0
        return oracle.Case(Q=Q, shape=tuple(shape), Tc=[x[0] for x in k], pc=[x[1] for x in k],
                           omega=[x[2] for x in k], M=[x[3] for x in k], T=c["T"], tau=c["tau"], gamma=c["gamma"],
                           kij=c["kij"], beta=c["beta"], G=c["G"], collision=coll,
                           s=c.get("mrt_s") if coll else None)

    samples = []
    c1 = load_case("c1")
    samples.append(("c1_slab", c1, c1["shape"], 9, case_fields(c1), "the full 64^2 FP64 BGK slab"))
    c2 = load_case("c2")
    r2 = c2["init"]["radius"] / 4
    g2 = (128, 128)
    samples.append(("c2_droplet", c2, [128, 128], 9,
                    lbm_inputs.ball_fields(g2, c2["rho_l"], c2["rho_v"], r2, 4.0),
                    "128^2 box of the MRT droplet (radius scaled by 1/4)"))
    c3 = load_case("c3")
    samples.append(("c3_sphere", c3, [32, 32, 32], 19,
                    lbm_inputs.ball_fields((32, 32, 32), c3["rho_l"], c3["rho_v"], 6.0, 4.0),
                    "32^3 box of the MRT sphere (radius scaled by 1/8)"))
    with open(os.path.join(ROOT, "tests", "golden", "cases.json")) as fh:
        sw = json.load(fh)["c4"]
    specs, rhos = _sweep_specs(sw)
    c4 = dict(sw["cases"][0], tau=sw["tau"], beta=sw["beta"], collision="bgk")
    samples.append(("c4_sweep", c4, c4["shape"], 9, rhos[0], "sweep case 0 (%dx%d, BGK)" % tuple(c4["shape"])))
    c5 = load_case("c5")
    samples.append(("c5_adjoint_droplet", c5, c5["shape"], 9, init_fields_ball(c5, tuple(reversed(c5["shape"]))),
                    "the full 256^2 BGK droplet (forward step)"))
    for name, c, shape, Q, rho, what in samples:
        case = case_of(c, shape, Q)
        f = oracle.equilibrium(case, rho)
        row = {"sample": what, "unit": UNIT}
        for label, n in (("one_core", 1), ("all_cores", cores)):
            oracle.set_threads(n)
            v, steps = timed(case, f)
            row[label] = {"value": v, "cores": n, "steps": steps}
        out[name] = row
    oracle.set_threads(cores)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--path", default="auto", choices=["auto", "fused", "two", "trailing", "queue"],
                    help="step path of the timed run (default: the library's choice)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-workload error check against the stored oracle runs")
    ap.add_argument("--grid", type=int, default=0,
                    help="cube edge of a smaller case of the same workload (profiling); 0 = 256")
    ap.add_argument("--fp64", action="store_true",
                    help="time FP64 storage instead of FP32-shifted (profiling the FP64 path)")
    ap.add_argument("--nz", type=int, default=0,
                    help="z extent of a shorter case with the same planes (profiling); 0 = cube")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1909_12390_gb300 import lbm
    c = load_case()
    if args.grid:
        c = dict(c, shape=[args.grid] * 3, init=dict(c["init"], radius=48.0 * args.grid / 256))
    if args.nz:
        sh = c["shape"]
        c = dict(c, shape=[sh[0], sh[1], args.nz],
                 init=dict(c["init"], radius=min(c["init"]["radius"], args.nz / 3.0)))
    nc = len(c["components"])
    N = int(np.prod(c["shape"]))
    rho0 = init_fields(c)

    gpu = lattice_for(c, lbm.FP64 if args.fp64 else lbm.FP32_SHIFTED)
    if args.path != "auto":
        gpu.set_path({"fused": lbm.PATH_FUSED, "two": lbm.PATH_TWO_KERNEL, "trailing": lbm.PATH_TRAILING,
                      "queue": lbm.PATH_QUEUE}[args.path])
    gpu.init(rho0)
    gpu.step(args.warmup)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    gpu.set_stream(stream.cuda_stream)
    gpu.profile(True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        gpu.step(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
    ms_total = start.elapsed_time(stop)
    path = gpu.path
    psi_ms, psi_n = gpu.profile_read(0)
    col_ms, col_n = gpu.profile_read(1)
    fus_ms, fus_n = gpu.profile_read(2)
    gpu.profile(False)
    mass_end = gpu.mass()
    # S7, the per-component mass reduction (lbm_mass reads every population once), timed
    # over 10 calls on the same stream; each call ends with a 3-double read-back
    a7 = torch.cuda.Event(enable_timing=True)
    b7 = torch.cuda.Event(enable_timing=True)
    a7.record(stream)
    for _ in range(10):
        gpu.mass()
    b7.record(stream)
    torch.cuda.synchronize()
    ms7 = a7.elapsed_time(b7) / 10
    s7_bytes = N * 19 * nc * 4
    t_max = max_over_ranks(ms_total, dist, "cuda")
    ms_step = t_max / args.steps
    value = job_value(N, nc, args.steps, world, t_max)

    # roofline of the dominant kernel: algorithmic bytes are one read and one write of every
    # FP32 population, 2 * 19 * nc * 4 B per site (the fused kernel and the collide pass each
    # move exactly that; psi traffic is not counted)
    peak, peak_kind = peaks()
    alg_site = 2 * 19 * nc * (8 if args.fp64 else 4)
    if path in (lbm.PATH_TRAILING, lbm.PATH_QUEUE):
        kname, kavg = "k_trail3" if path == lbm.PATH_TRAILING else "k_trailq", fus_ms / max(fus_n, 1)
        kinds = {kname: kavg}
        if psi_n:
            kinds["k_psi (first step of the call)"] = psi_ms / psi_n
    elif path == lbm.PATH_FUSED:
        kname = "k_fused3" if gpu.fused_kind == lbm.FUSED_PLANES else "k_fused"
        kavg = fus_ms / max(fus_n, 1)
        kinds = {kname: kavg}
    else:
        kname, kavg = "k_collide", col_ms / max(col_n, 1)
        kinds = {"k_psi": psi_ms / max(psi_n, 1), "k_collide": kavg}
    achieved = N * alg_site / (kavg / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ncu_traffic(kname),
            "kernel": "%s<19,%d,FP32S,MRT>" % (kname, nc), "peak_kind": peak_kind,
            "alg_bytes_per_launch": N * alg_site,
            "step_frac": (N * alg_site / (ms_step / 1e3) / 1e9) / peak,
            "kernels_ms_avg": kinds, "path": PATH_NAMES[path]}

    # end to end through the C ABI with pinned host buffers: the densities go in, the steps
    # run, the densities come back
    gpu.set_stream(0)
    rho_in = torch.empty(rho0.shape, dtype=torch.float64, pin_memory=True).numpy()
    rho_in[...] = rho0
    rho_out = torch.empty((nc,) + tuple(reversed(c["shape"])), dtype=torch.float64, pin_memory=True).numpy()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    gpu.init(rho_in)
    gpu.step(args.steps)
    gpu.fields_into(rho=rho_out)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": N * nc * args.steps / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(rho0.nbytes / args.steps),
           "d2h_bytes_per_step": int(rho_out.nbytes / args.steps),
           "note": "lbm_init from pinned host densities + steps + lbm_fields to pinned host densities"}
    gpu.close()

    variants = {}
    if not args.no_variants and rank == 0:
        # plain FP64 storage on the same workload (the FP64 EOS is the same code)
        g64 = lattice_for(c, lbm.FP64)
        g64.init(rho0)
        g64.step(3)
        k64 = 20
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        g64.set_stream(stream.cuda_stream)
        a.record(stream)
        g64.step(k64)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / k64
        g64.close()
        variants["fp64"] = {"value": N * nc / (ms64 / 1e3) / 1e6, "ms_per_step": ms64,
                            "hbm_frac_of_step": (N * 2 * 19 * nc * 8 / (ms64 / 1e3) / 1e9) / peak}
        variants["fp32s"] = {"value": value, "ms_per_step": ms_step, "path": roof["path"]}
        # the same workload on the other step paths
        for other in (lbm.PATH_TWO_KERNEL, lbm.PATH_QUEUE, lbm.PATH_TRAILING, lbm.PATH_FUSED):
            if other == path:
                continue
            g2 = lattice_for(c, lbm.FP32_SHIFTED)
            try:
                g2.set_path(other)
            except lbm.LBMError:
                g2.close()
                continue
            g2.init(rho0)
            g2.step(3)
            g2.set_stream(stream.cuda_stream)
            a.record(stream)
            g2.step(50)
            b.record(stream)
            torch.cuda.synchronize()
            ms2 = a.elapsed_time(b) / 50
            variants["fp32s_" + PATH_NAMES[other].replace("-", "_")] = {
                "value": N * nc / (ms2 / 1e3) / 1e6, "ms_per_step": ms2,
                "hbm_frac_of_step": (N * alg_site / (ms2 / 1e3) / 1e9) / peak}
            g2.close()
        variants["batched"] = batched_variant(stream)
        variants["l2_resident"] = l2_variants(stream)
        variants["flash"] = flash_variant()
        variants["adjoint"] = adjoint_variant()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "precision": EOS_PRECISION, "data": "synthetic",
           "config": {"workload": WORKLOAD, "lattice": "D3Q19", "grid": c["shape"], "components": nc,
                      "collision": "mrt", "precision": "fp32-shifted", "parallelism": "replicas" if world > 1 else "single",
                      "l2": "inputs larger than L2 (%.2f GB populations)" % (N * 19 * nc * 4 / 1e9)},
           "e2e": e2e, "roofline": roof, "gpu_launches": psi_n + col_n + fus_n,
           "mass_reduction": {"ms_per_call": ms7, "bytes": s7_bytes,
                              "achieved_gbs": s7_bytes / (ms7 / 1e3) / 1e9,
                              "frac": s7_bytes / (ms7 / 1e3) / 1e9 / peak,
                              "note": "lbm_mass (S7) outside the timed step, 10 calls"},
           "clocks": clk.summary(), "site_mlups": value / nc,
           "mass_drift": float(np.max(np.abs(mass_end / (rho0.reshape(nc, -1).sum(1)) - 1)))}
    if variants:
        out["variants"] = variants
    if rank == 0 and not args.no_configs:
        out["configs_vs_oracle"] = config_checks()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"], sample = cpu_baseline(c)
        out["err_vs_oracle"] = accuracy(c, sample)
        out["cpu_baselines"] = cpu_baselines()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
