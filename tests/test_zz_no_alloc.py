"""lbm_step_static, the allocation-free step, against the context step (lbm_create /
lbm_step) through the C ABI.

Some callers cannot let a library allocate device memory (their own pool allocator owns the
GPU's memory, or an allocation would synchronise the device at the wrong moment). For them
lbm_step_static advances caller-owned device populations with its scratch in a fixed static
device array. This test gives it the populations of a context (the test, as the caller,
owns that device buffer), advances both by the same steps twice in a row and compares the
populations. This file is collected last so that a failing run has already run every other
test; it also passes on its own in a fresh process.
"""
import json
import os

import numpy as np
import pytest

from conftest import GOLDEN
from lbm_cases import comps_of, initial_rho

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        return json.load(fh)


def _setup(c, precision, shape=(96, 64), **over):
    from paper_1909_12390_gb300 import lbm

    rho = initial_rho(dict(c, init=dict(kind="ball", radius=18.0, width=4.0)), shape)
    rho_ref = rho.reshape(len(c["rho_l"]), -1).mean(axis=1)
    kw = dict(gamma=c["gamma"], kij=np.array(c["kij"]), beta=c["beta"], G=c["G"], collision=lbm.MRT,
              mrt_rates=c["mrt_s"], precision=precision, rho_ref=rho_ref)
    kw.update(over)
    ctx = lbm.Lattice(shape, comps_of(c), T=c["T"], tau=c["tau"], **kw)
    ctx.set_path(lbm.PATH_TWO_KERNEL)
    ctx.init(rho)
    return ctx, kw


@pytest.mark.parametrize("precision", [0, 1])
def test_static_step_matches_context_step_twice(cases, precision):
    """Both sides launch the same kernels in the same order, so the populations agree bit for
    bit after each of two calls in a row; the step index returned is t0 + completed steps."""
    import torch

    from paper_1909_12390_gb300 import lbm

    c = cases["c2"]
    shape = (96, 64)
    ctx, kw = _setup(c, precision, shape)
    raw, t = ctx.save()
    assert t == 0
    dev = torch.empty(raw.size, dtype=torch.uint8, device="cuda")
    dev.copy_(torch.from_numpy(raw))
    torch.cuda.synchronize()
    t_static = 0
    for _ in range(2):
        ctx.step(7)
        t_static = lbm.step_static(shape, comps_of(c), c["T"], c["tau"], dev.data_ptr(), t_static, 7, **kw)
        assert t_static == ctx.time
        assert np.array_equal(dev.cpu().numpy(), ctx.save()[0])
    ctx.close()


def test_static_step_allocates_nothing_once_warm(cases):
    """After one warm-up call of the variant (which may load the library's device code), further
    calls leave the device's free memory unchanged."""
    import torch

    from paper_1909_12390_gb300 import lbm

    c = cases["c2"]
    shape = (96, 64)
    ctx, kw = _setup(c, 1, shape)
    raw, _ = ctx.save()
    ctx.close()
    dev = torch.from_numpy(raw).cuda()
    t = lbm.step_static(shape, comps_of(c), c["T"], c["tau"], dev.data_ptr(), 0, 3, **kw)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        t = lbm.step_static(shape, comps_of(c), c["T"], c["tau"], dev.data_ptr(), t, 5, **kw)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert t == 18
    assert free1 == free0


def test_static_step_failure_stops_at_the_failing_step(cases):
    """A state outside the EOS's domain (G > 0 makes psi^2 negative) and a planted NaN are
    reported as statuses; the step index stays at t0 and the populations keep the state before
    the failing step. A following call on a valid state succeeds (each call resets the status
    word it shares with earlier calls)."""
    import torch

    from paper_1909_12390_gb300 import lbm

    c = cases["c2"]
    shape = (96, 64)
    ctx, kw = _setup(c, 0, shape)
    ctx.step(4)
    raw, t0 = ctx.save()
    ctx.close()
    assert t0 == 4
    dev = torch.from_numpy(raw).cuda()
    bad = dict(kw, G=1.0)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_static(shape, comps_of(c), c["T"], c["tau"], dev.data_ptr(), t0, 5, **bad)
    assert ei.value.status == lbm.ERR_PSI_DOMAIN
    assert ei.value.time == t0
    assert np.array_equal(dev.cpu().numpy(), raw)
    nan = raw.copy()
    nan.view(np.float64)[12345] = np.nan
    devn = torch.from_numpy(nan).cuda()
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_static(shape, comps_of(c), c["T"], c["tau"], devn.data_ptr(), t0, 5, **kw)
    assert ei.value.status == lbm.ERR_NONFINITE
    assert ei.value.time == t0
    assert np.array_equal(devn.cpu().numpy().view(np.float64), nan.view(np.float64), equal_nan=True)
    assert lbm.step_static(shape, comps_of(c), c["T"], c["tau"], dev.data_ptr(), t0, 5, **kw) == t0 + 5


def test_static_step_rejects_grids_above_its_maximum(cases):
    from paper_1909_12390_gb300 import lbm

    c = cases["c2"]
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_static((2048, 1024), comps_of(c), c["T"], c["tau"], 1 << 20, 0, 1, gamma=c["gamma"])
    assert ei.value.status == lbm.ERR_ARG
    assert "LBM_STATIC_MAX_SITES" in str(ei.value)
