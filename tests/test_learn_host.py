"""Host-side pieces of the learned-correction trainer (no GPU)."""
import numpy as np


def test_gk_training_target_equals_the_oracle_spectral_pm():
    # the PM(G_K) target of the trainer, computed with torch FFTs (here on
    # the CPU), against the oracle's spectral PM with G_K (eq. gfk)
    import torch
    from oracle import pm
    from paper_2011_07099_gb300 import inputs, learn
    N = 16
    rho = inputs.lognormal(N, sigma=0.5, seed=3)
    phi, g = learn.pm_target_gk(torch.from_numpy(rho), N)
    kphi, kg = pm.pm_gk(pm.masses(rho.astype(np.float64)))
    assert np.abs(phi.numpy() - kphi).max() <= 1e-6 * np.abs(kphi).max()
    assert np.abs(g.numpy() - kg).max() <= 1e-6 * np.abs(kg).max()
