"""Host logic of the torch.autograd.Function wrapper (no GPU): how the split-factor scale s
maps onto the volatility coefficients, and the choice of the least volatile component."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1909_12390_gb300.autograd import _gamma, _kij  # noqa: E402


def test_scale_leaves_the_least_volatile_coefficient_and_keeps_the_unscaled_one():
    g, g0, h = _gamma({"gamma": [0.09, 1.0]}, 1.3)
    assert h == 1
    assert np.allclose(g, [0.09 * 1.3, 1.0]) and np.allclose(g0, [0.09, 1.0])
    g, g0, h = _gamma({"gamma": [0.5, 0.7, 0.2], "least_volatile": 2}, 2.0)
    assert h == 2 and np.allclose(g, [1.0, 1.4, 0.2]) and np.allclose(g0, [0.5, 0.7, 0.2])


@pytest.mark.parametrize("gamma", [[0.5, 0.7], [1.0, 1.0]])
def test_ambiguous_least_volatile_component_is_an_error(gamma):
    with pytest.raises(ValueError):
        _gamma({"gamma": gamma}, 1.0)


def test_pair_coefficient_is_set_symmetrically():
    k = _kij({"components": [0, 0, 0], "pair": (0, 2)}, 0.02)
    assert k[0, 2] == k[2, 0] == 0.02 and np.count_nonzero(k) == 2


def test_workload_loss_gradient_matches_the_closed_form():
    """The torch loss of the adjoint workload (losses.composition_profile_loss) and its autograd
    gradient against the test helpers' numpy closed form (lbm_cases.composition_profile_loss),
    written independently, on a droplet and a shifted target."""
    import json
    import os

    import torch

    import lbm_inputs
    from conftest import GOLDEN
    from lbm_cases import composition_profile_loss as np_loss
    from paper_1909_12390_gb300.losses import composition_profile_loss

    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        c = json.load(fh)["c5"]
    grid = (40, 48)
    rho = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], 12.0, 4.0)
    tgt = lbm_inputs.ball_fields(grid, c["rho_l"], c["rho_v"], 12.5, 4.0) * np.array([1.01, 0.99]).reshape(2, 1, 1)
    M = [d["M"] for d in c["components"]]
    L0, g0 = np_loss(rho, tgt, M)
    r = torch.tensor(rho, requires_grad=True)
    L = composition_profile_loss(r, torch.tensor(tgt), M)
    L.backward()
    assert float(L) == pytest.approx(L0, rel=1e-12)
    assert np.max(np.abs(r.grad.numpy() - g0)) < 1e-12 * np.max(np.abs(g0))
