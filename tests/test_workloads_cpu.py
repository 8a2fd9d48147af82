"""The workload table's host-side pieces: weights, grids and fields for every configuration."""
import numpy as np
import pytest

from paper_2010_04868_gb300 import workloads as W


@pytest.mark.parametrize("name", [n for n in W.CONFIGS if n not in ("batch3d", "life", "lcs")])
def test_config_weights_match_the_stencil(name):
    dim, shape = W.CONFIGS[name][0], W.CONFIGS[name][1]
    k = W.k_points(dim, shape, W.RADIUS.get(name, 1))
    assert len(W.config_weights(name)) == k


@pytest.mark.parametrize("name", sorted(W.FIELD))
def test_config_field_on_its_own_and_on_smaller_extents(name):
    dim, shape = W.CONFIGS[name][0], W.CONFIGS[name][1]
    k = W.k_points(dim, shape, W.RADIUS.get(name, 1))
    small = (5,) * dim
    f = W.config_field(name, small)
    assert f.shape == (k,) + small
    assert np.all(f > 0) and np.allclose(f.sum(axis=0), 1.0, atol=1e-14)
