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
