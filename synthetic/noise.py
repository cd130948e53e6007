"""Gaussian draws for synthetic measurement noise (Section 6.3).

The paper adds 10 % additive Gaussian white noise with independent values for
the real and imaginary parts; the workloads here use a relative level eta.
"""

import numpy as np


def noise_draws(shape, seed=1234):
    """Two independent N(0, 1) arrays (real and imaginary parts), PCG64."""
    rng = np.random.default_rng(seed)
    xi1 = rng.standard_normal(shape)
    xi2 = rng.standard_normal(shape)
    return xi1, xi2


def add_noise(S, eta=0.01, seed=1234):
    """S_mes = S + eta |S| (xi1 + i xi2) / sqrt(2), entry by entry."""
    S = np.asarray(S, dtype=np.complex128)
    xi1, xi2 = noise_draws(S.shape, seed)
    return S + eta * np.abs(S) * (xi1 + 1j * xi2) / np.sqrt(2.0)
