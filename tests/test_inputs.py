"""The seeded synthetic density recipes (no GPU): determinism, shapes and
the properties each recipe states."""
import numpy as np
import pytest

from paper_2011_07099_gb300 import inputs


def test_recipes_are_seeded_and_deterministic():
    a = inputs.config_density(0, n=16, field=3)
    b = inputs.config_density(0, n=16, field=3)
    c = inputs.config_density(0, n=16, field=4)
    assert a.dtype == np.float32 and a.shape == (16, 16, 16) and a.flags.c_contiguous
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_lognormal_mean_and_positivity():
    rho = inputs.lognormal(32, sigma=0.5, seed=1, amp=0.5, background=1.0).astype(np.float64)
    # exp(sigma g - sigma^2 / 2) has mean 1 for a unit-variance g
    assert rho.min() > 1.0
    assert abs(rho.mean() - 1.5) < 0.05


def test_gaussian_field_is_unit_variance_and_mean_free():
    g = inputs.gaussian_field(32, np.random.Generator(np.random.PCG64(7)))
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12


def test_plummer_clump_masses_add_up_to_the_background_mass():
    n, bg = 32, 1.0
    rho = inputs.plummer(n, n_clumps=8, seed=3, background=bg).astype(np.float64)
    # background n^3 bg plus clumps whose masses add up to the same amount
    assert rho.sum() == pytest.approx(2.0 * bg * n ** 3, rel=1e-5)
    assert rho.min() >= bg * (1 - 1e-6)


def test_point_source_has_unit_mass():
    rho = inputs.point(16, cell=(1, 2, 3)).astype(np.float64)
    assert rho.sum() / 16 ** 3 == pytest.approx(1.0)
    assert rho[1, 2, 3] == 16 ** 3 and np.count_nonzero(rho) == 1


def test_device_recipe_matches_the_host_recipe_on_cpu():
    torch = pytest.importorskip("torch")
    host = inputs.lognormal(16, sigma=0.5, seed=9)
    dev = inputs.lognormal(16, sigma=0.5, seed=9, device=torch.device("cpu")).numpy()
    np.testing.assert_allclose(dev, host, rtol=1e-5)
