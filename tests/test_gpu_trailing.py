"""The one-pass steps whose psi of the next step trails the collisions (LBM_PATH_TRAILING: one
persistent launch per step, psi of the next step computed from the just-written populations a
few planes behind the collision; LBM_PATH_QUEUE: the same two kinds of work as tasks taken from
a ticket counter) against the two-kernel step, bit for bit, and against the FP64 oracle; their
failure semantics and their bounded waits."""
import json
import os

import numpy as np
import pytest

import lbm_inputs
import oracle
from conftest import GOLDEN
from lbm_cases import gpu_lattice, initial_rho, oracle_case, random_rho

pytestmark = pytest.mark.gpu

FP64, FP32S = 0, 1


@pytest.fixture(scope="module")
def cases():
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        return json.load(fh)


@pytest.fixture(params=["trailing", "queue"])
def trail_path(request):
    from paper_1909_12390_gb300 import lbm
    return {"trailing": lbm.PATH_TRAILING, "queue": lbm.PATH_QUEUE}[request.param]


def _pair(c, shape, precision, collision, rates, path, **kw):
    from paper_1909_12390_gb300 import lbm
    a = gpu_lattice(c, shape, precision, collision=collision, s=rates, **kw)
    b = gpu_lattice(c, shape, precision, collision=collision, s=rates, **kw)
    a.set_path(path)
    b.set_path(lbm.PATH_TWO_KERNEL)
    assert a.path == path and b.path == lbm.PATH_TWO_KERNEL
    return a, b


def _ball(c, shape):
    grid = tuple(reversed(shape))
    return lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], min(shape) / 3.0, 3.0,
                                  center=[g / 2 - 0.7 for g in grid])


# small grids give few CTAs with ranges shorter than a row (up to 16 neighbour CTAs); ragged
# sizes give ranges that start mid-row; nz from 3 (the shortest march) up
@pytest.mark.parametrize("shape", [(16, 12, 10), (40, 36, 33), (64, 16, 16), (96, 64, 24), (33, 17, 5),
                                   (24, 24, 3)])
@pytest.mark.parametrize("precision", [FP64, FP32S])
@pytest.mark.parametrize("collision", [0, 1])
def test_trailing_equals_two_kernel_bitwise(cases, shape, precision, collision, trail_path):
    """The collision is the same per-site code and psi of the next step is computed from the
    same slots in the same order, so every population agrees bit for bit after any number of
    steps, over several lbm_step calls (psi carried over between calls) and both parities."""
    c = cases["c3"]
    a, b = _pair(c, shape, precision, collision, c["mrt_s"], trail_path)
    rho = _ball(c, shape)
    a.init(rho)
    b.init(rho)
    for n in (1, 2, 7, 3):
        a.step(n)
        b.step(n)
        assert a.time == b.time
        assert np.array_equal(a.save()[0], b.save()[0])
    a.close()
    b.close()


@pytest.mark.parametrize("nc", [1, 2, 4])
def test_trailing_equals_two_kernel_other_component_counts(cases, nc, trail_path):
    from test_gpu_parity import _mixture
    c = _mixture(cases, nc)
    shape = (48, 20, 12)
    a, b = _pair(c, shape, FP32S, 1, cases["c3"]["mrt_s"], trail_path)
    rho = random_rho(c, tuple(reversed(shape)), seed=3 + nc)
    a.init(rho)
    b.init(rho)
    a.step(9)
    b.step(9)
    assert np.array_equal(a.save()[0], b.save()[0])


def test_trailing_long_run_with_graph_replay_and_state_changes(cases, trail_path):
    """130 steps (two captured 64-step graphs and direct launches), then a restore of an earlier
    state and a re-initialisation: psi is recomputed whenever the state changed outside the
    trailing step."""
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"]
    shape = (64, 40, 20)
    a, b = _pair(c, shape, FP32S, 1, c["mrt_s"], trail_path)
    rho = _ball(c, shape)
    a.init(rho)
    b.init(rho)
    a.step(5)
    b.step(5)
    saved, t = b.save()
    a.step(130)
    b.step(130)
    assert np.array_equal(a.save()[0], b.save()[0])
    a.restore(saved, t)
    b.restore(saved, t)
    a.step(4)
    b.step(4)
    assert np.array_equal(a.save()[0], b.save()[0])
    a.set_path(lbm.PATH_TWO_KERNEL)
    a.step(1)
    a.set_path(trail_path)
    b.step(1)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.save()[0], b.save()[0])
    a.init(rho)
    b.init(rho)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.save()[0], b.save()[0])


def test_trailing_matches_oracle(cases, trail_path):
    c = cases["c3"]
    shape = (20, 18, 16)
    rates = c["mrt_s"]
    from paper_1909_12390_gb300 import lbm
    for precision, tol in ((FP64, 1e-12), (FP32S, 2e-4)):
        ocase = oracle_case(c, shape, collision=1, s=rates)
        gpu = gpu_lattice(c, shape, precision, collision=1, s=rates)
        gpu.set_path(trail_path)
        rho = random_rho(c, ocase.grid, seed=9)
        gpu.init(rho)
        f = oracle.equilibrium(ocase, rho)
        gpu.step(6)
        f = oracle.step(ocase, f, 6)
        ro = oracle.fields(ocase, f).rho
        rg = gpu.fields()["rho"]
        assert float(np.max(np.abs(rg - ro) / ro.sum(0))) < tol
        gpu.close()


def test_trailing_failure_reports_the_same_step_as_the_two_kernel_path(cases, trail_path):
    """A momentum kick planted at one site (the density there unchanged) makes the step after
    it leave the EOS's domain. The trailing step finds that in its psi stage for the next step;
    both paths report the same status at the same step index, with the same populations (the
    state before the failing step)."""
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"]
    shape = (32, 24, 12)
    a, b = _pair(c, shape, FP64, 0, None, trail_path)
    rho = _ball(c, shape)
    a.init(rho)
    b.init(rho)
    a.step(4)
    b.step(4)
    raw, t = b.save()
    f = raw.view(np.float64).reshape(3, 19, -1).copy()
    site = 5 * 32 * 24 + 7 * 32 + 11
    f[2, 1, site] += 1e3
    f[2, 2, site] -= 1e3
    kicked = f.reshape(-1).view(np.uint8)
    a.restore(kicked, t)
    b.restore(kicked, t)
    errs = []
    for g in (a, b):
        with pytest.raises(lbm.LBMError) as ei:
            g.step(6)
        errs.append((ei.value.status, g.time))
    assert errs[0] == errs[1], errs
    assert errs[0][0] in (lbm.ERR_PSI_DOMAIN, lbm.ERR_NONFINITE)
    assert errs[0][1] > t  # the kick's own step completes; a later one fails
    assert np.array_equal(a.save()[0], b.save()[0])
    # the context recovers after a new state
    a.init(rho)
    b.init(rho)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.save()[0], b.save()[0])


def test_trailing_silent_cta_times_out_and_context_recovers(cases, trail_path):
    """A CTA (trailing path) or a chunk's collision tasks (queue path) that never publish their
    progress make the bounded waits of the psi work that needs them run out: the step returns
    LBM_ERR_TIMEOUT within seconds, the GPU stays usable, and after lbm_init the context steps
    normally again."""
    import time
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"]
    shape = (64, 16, 16)
    rho = initial_rho(dict(c, init=dict(kind="ball", radius=5.0, width=4.0)), shape)
    gpu = gpu_lattice(c, shape, FP32S)
    gpu.set_path(trail_path)
    gpu.init(rho)
    gpu.step(2)
    gpu.test_silence_block(1)
    t0 = time.time()
    with pytest.raises(lbm.LBMError) as ei:
        gpu.step(1)
    assert ei.value.status == lbm.ERR_TIMEOUT
    assert time.time() - t0 < 30
    gpu.test_silence_block(-1)
    gpu.init(rho)
    gpu.step(3)
    ref = gpu_lattice(c, shape, FP32S)
    ref.set_path(lbm.PATH_TWO_KERNEL)
    ref.init(rho)
    ref.step(3)
    assert np.array_equal(gpu.get_f(), ref.get_f())


@pytest.mark.parametrize("shape", [(30, 8, 2), (30, 8)])
def test_trailing_rejected_when_the_grid_does_not_fit(cases, shape, trail_path):
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"] if len(shape) == 3 else cases["c2"]
    gpu = gpu_lattice(c, shape, FP32S)
    with pytest.raises(lbm.LBMError) as ei:
        gpu.set_path(trail_path)
    assert ei.value.status == lbm.ERR_ARG
    assert gpu.path == lbm.PATH_TWO_KERNEL
    gpu.close()
