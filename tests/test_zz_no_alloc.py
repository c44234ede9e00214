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


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-4)])
def test_static_step_matches_context_step_twice(cases, precision, tol):
    import torch

    from paper_1909_12390_gb300 import lbm

    c = cases["c2"]
    shape = (96, 64)
    rho = initial_rho(dict(c, init=dict(kind="ball", radius=18.0, width=4.0)), shape)
    rho_ref = rho.reshape(len(c["rho_l"]), -1).mean(axis=1)
    kw = dict(gamma=c["gamma"], kij=np.array(c["kij"]), beta=c["beta"], G=c["G"], collision=lbm.MRT,
              mrt_rates=c["mrt_s"], precision=precision, rho_ref=rho_ref)
    ctx = lbm.Lattice(shape, comps_of(c), T=c["T"], tau=c["tau"], **kw)
    ctx.set_path(lbm.PATH_TWO_KERNEL)
    ctx.init(rho)
    raw, t = ctx.save()
    assert t == 0
    dev = torch.empty(raw.size, dtype=torch.uint8, device="cuda")
    dev.copy_(torch.from_numpy(raw))
    torch.cuda.synchronize()
    dt = np.float64 if precision == 0 else np.float32
    t_static = 0
    for _ in range(2):
        ctx.step(7)
        t_static = lbm.step_static(shape, comps_of(c), c["T"], c["tau"], dev.data_ptr(), t_static, 7, **kw)
        assert t_static == ctx.time
        want = ctx.save()[0].view(dt).astype(np.float64)
        got = dev.cpu().numpy().view(dt).astype(np.float64)
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want)) <= tol * scale
    ctx.close()


def test_static_step_rejects_grids_above_its_maximum(cases):
    from paper_1909_12390_gb300 import lbm

    c = cases["c2"]
    with pytest.raises(lbm.LBMError) as ei:
        lbm.step_static((2048, 1024), comps_of(c), c["T"], c["tau"], 1 << 20, 0, 1, gamma=c["gamma"])
    assert ei.value.status == lbm.ERR_ARG
    assert "LBM_STATIC_MAX_SITES" in str(ei.value)
