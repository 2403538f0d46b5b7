"""The downhill simplex of the a_k fit (host logic, no GPU)."""
import numpy as np

from paper_2011_07099_gb300 import fit


def test_simplex_finds_the_minimum_of_a_quadratic():
    c = np.array([0.3, -1.2])
    x, fx, ev = fit.nelder_mead(lambda x: float(np.sum((x - c) ** 2 * np.array([1.0, 10.0]))), [0.0, 0.0], 0.5,
                                xtol=1e-9, ftol=1e-18, max_iter=500)
    np.testing.assert_allclose(x, c, atol=1e-7)
    assert fx < 1e-13 and ev < 500


def test_simplex_on_rosenbrock_and_in_one_dimension():
    rosen = lambda x: float((1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2)
    x, fx, _ = fit.nelder_mead(rosen, [-1.2, 1.0], 0.1, xtol=1e-10, ftol=1e-20, max_iter=2000)
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-6)
    # one parameter (the a_1 fit): a non-smooth (L_MAX-like) objective too
    x, fx, _ = fit.nelder_mead(lambda a: abs(a[0] + 0.12) + 1.0, [-0.125], 0.01, xtol=1e-9, ftol=0.0)
    assert abs(x[0] + 0.12) < 1e-8


def test_gk_mesh_helper_equals_the_explicit_inverse_dft():
    # the G_K mesh handed to fmm_plan_set_green_mesh (FFT on the host here)
    # against the oracle's explicit inverse-DFT sum of eq. gfk
    import torch
    from oracle import pm
    from paper_2011_07099_gb300 import ablation
    N = 8
    K = ablation.g_k_mesh(N, torch.device("cpu")).numpy().reshape(4, N, N, N)
    kern, grad = pm.g_k_real_space(N)
    np.testing.assert_allclose(K[0], kern, atol=1e-13)
    np.testing.assert_allclose(K[1:], -np.moveaxis(grad, -1, 0), atol=1e-13)
