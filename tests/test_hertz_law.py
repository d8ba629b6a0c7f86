"""The bonded-layer correction used by the sphere-indentation check
reproduces its published incompressible series."""
import pytest

from gpu_util import bonded_layer_factor


def test_bonded_layer_factor_incompressible_limit():
    # the published nu = 1/2 series
    chi = 0.3
    assert bonded_layer_factor(chi, 0.5) == pytest.approx(
        1 + 1.133 * chi + 1.283 * chi ** 2 + 0.769 * chi ** 3 + 0.0975 * chi ** 4, rel=1e-3)
