"""The fused single-kernel step (one persistent cooperative launch per step, psi exchanged
between tile columns through release/acquire progress flags) against the two-kernel step and
the FP64 oracle, and its bounded waits."""
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


def _pair(c, shape, precision, collision, rates):
    from paper_1909_12390_gb300 import lbm
    a = gpu_lattice(c, shape, precision, collision=collision, s=rates)
    b = gpu_lattice(c, shape, precision, collision=collision, s=rates)
    a.set_path(lbm.PATH_FUSED)
    b.set_path(lbm.PATH_TWO_KERNEL)
    assert a.path == lbm.PATH_FUSED and b.path == lbm.PATH_TWO_KERNEL
    return a, b


# grids that tile: D3Q19 tiles are 32 x 8 (x, y), D2Q9 tiles are 128 (x); the marched axis
# is cut into chunks of at least two groups of 4 planes: (32, 8, 8) and (128, 8) are one chunk,
# (64, 16, 16) two, (32, 16, 24) three, (256, 24) three, (128, 64) eight
@pytest.mark.parametrize("shape", [(32, 8, 8), (64, 16, 12), (64, 16, 16), (32, 16, 24), (128, 8), (256, 12),
                                   (256, 24), (128, 64)])
@pytest.mark.parametrize("precision", [FP64, FP32S])
@pytest.mark.parametrize("collision", [0, 1])
def test_fused_equals_two_kernel_bitwise(cases, shape, precision, collision):
    """Both paths run the same per-site code in the same order, so every population agrees
    bit for bit after any number of steps (both parities, several chunks)."""
    c = cases["c3"] if len(shape) == 3 else cases["c2"]
    a, b = _pair(c, shape, precision, collision, c["mrt_s"])
    grid = tuple(reversed(shape))
    rho = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], min(shape) / 3.0, 3.0,
                                 center=[g / 2 - 0.7 for g in grid])
    a.init(rho)
    b.init(rho)
    for n in (1, 2, 7):
        a.step(n)
        b.step(n)
        assert a.time == b.time
        assert np.array_equal(a.get_f(), b.get_f())


@pytest.mark.parametrize("shape,nc", [((64, 16, 8), 3), ((32, 8, 12), 2), ((256, 8), 3), ((128, 12), 4)])
def test_fused_matches_oracle(cases, shape, nc):
    c = dict(cases["c3"])
    if nc != 3:
        from test_gpu_parity import _mixture
        c = _mixture(cases, nc)
    rates = cases["c3"]["mrt_s"] if len(shape) == 3 else cases["c2"]["mrt_s"]
    from paper_1909_12390_gb300 import lbm
    for precision, tol in ((FP64, 1e-12), (FP32S, 2e-4)):
        ocase = oracle_case(c, shape, collision=1, s=rates, tau=0.8, beta=1.9)
        gpu = gpu_lattice(c, shape, precision, collision=1, s=rates, tau=0.8, beta=1.9)
        gpu.set_path(lbm.PATH_FUSED)
        rho = random_rho(c, ocase.grid, seed=7)
        gpu.init(rho)
        f = oracle.equilibrium(ocase, rho)
        gpu.step(5)
        f = oracle.step(ocase, f, 5)
        ro = oracle.fields(ocase, f).rho
        rg = gpu.fields()["rho"]
        assert float(np.max(np.abs(rg - ro) / ro.sum(0))) < tol
        gpu.close()


def test_benchmark_grid_paths(cases):
    """The 256^3 sphere: the automatic path is the two-kernel step (the faster on GB300); the
    fused path, when asked for, is the plane-range form."""
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"]
    gpu = gpu_lattice(c, tuple(c["shape"]), FP32S)
    assert gpu.path == lbm.PATH_TWO_KERNEL and gpu.fused_kind == 0
    gpu.set_path(lbm.PATH_FUSED)
    assert gpu.path == lbm.PATH_FUSED
    assert gpu.fused_kind == lbm.FUSED_PLANES
    gpu.set_path(lbm.PATH_AUTO)
    assert gpu.path == lbm.PATH_TWO_KERNEL
    gpu.close()


@pytest.mark.parametrize("shape", [(30, 8, 2), (30, 8)])
def test_fused_rejected_when_the_grid_does_not_fit(cases, shape):
    """D3Q19 needs at least 3 planes (the plane-range kernel keeps the first and last plane's
    psi apart); D2Q9 needs rows that split into 128-site tiles."""
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"] if len(shape) == 3 else cases["c2"]
    gpu = gpu_lattice(c, shape, FP32S)
    assert gpu.path == lbm.PATH_TWO_KERNEL
    with pytest.raises(lbm.LBMError) as ei:
        gpu.set_path(lbm.PATH_FUSED)
    assert ei.value.status == lbm.ERR_ARG
    gpu.close()


def test_silent_block_times_out_and_context_recovers(cases):
    """A block that never publishes its progress makes its neighbours' bounded waits run out:
    the step returns LBM_ERR_TIMEOUT within seconds, the GPU stays usable, and after lbm_init
    the context steps normally again."""
    import time
    from paper_1909_12390_gb300 import lbm
    c = cases["c3"]
    shape = (64, 16, 16)
    rho = initial_rho(dict(c, init=dict(kind="ball", radius=5.0, width=4.0)), shape)
    gpu = gpu_lattice(c, shape, FP32S)
    gpu.set_path(lbm.PATH_FUSED)
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
