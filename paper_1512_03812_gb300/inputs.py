"""Seeded synthetic inputs for the Schwinger-model HMC.

This module holds random-number draws only, none of the method's
arithmetic, so that the CUDA path and the CPU oracle can be fed identical
inputs.  Every array is float64 (complex128 for spinors) in the flat
site-major layout used throughout: site n = x + L t, and per site either
two link components (mu = x, t) or two spin components.

Distributions
-------------
* link angles q_mu(n): uniform in [-pi, pi)       (hot start)
* momenta p_mu(n):     N(0, 1) per link           (H has 1/2 sum p^2)
* noise eta(n, s):     Re, Im ~ N(0, 1/2)         (density ~ exp(-eta^dag eta))
* Metropolis uniforms: U[0, 1)
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def hot_links(L: int, T: int, seed: int) -> np.ndarray:
    """Angles q, shape (L*T, 2), uniform in [-pi, pi)."""
    return _rng(seed, 1).uniform(-np.pi, np.pi, size=(L * T, 2))


def momenta(L: int, T: int, seed: int) -> np.ndarray:
    """Momenta p, shape (L*T, 2), standard normal."""
    return _rng(seed, 2).standard_normal((L * T, 2))


def noise(L: int, T: int, seed: int) -> np.ndarray:
    """Gaussian spinor eta, shape (L*T, 2) complex, Re and Im ~ N(0, 1/2)."""
    g = _rng(seed, 3).standard_normal((L * T, 2, 2)) * np.sqrt(0.5)
    return g[..., 0] + 1j * g[..., 1]


def spinor(L: int, T: int, seed: int) -> np.ndarray:
    """A generic complex test spinor, shape (L*T, 2), Re and Im ~ N(0, 1)."""
    g = _rng(seed, 4).standard_normal((L * T, 2, 2))
    return g[..., 0] + 1j * g[..., 1]


def link_field(L: int, T: int, seed: int) -> np.ndarray:
    """A generic real link field (e.g. a direction v), shape (L*T, 2)."""
    return _rng(seed, 5).standard_normal((L * T, 2))


def uniforms(n: int, seed: int) -> np.ndarray:
    """n Metropolis uniforms in [0, 1)."""
    return _rng(seed, 6).uniform(0.0, 1.0, size=n)


def chain_sides(n: int, seed: int, sides=(16, 32, 48, 64, 128)) -> np.ndarray:
    """Square lattice sides for a batch of n independent chains, drawn
    uniformly from ``sides``."""
    return _rng(seed, 7).choice(np.asarray(sides), size=n)


def chain_couplings(n: int, seed: int, betas=(1.0, 2.0, 4.0), kappa=(0.20, 0.26)):
    """Per-chain beta (from ``betas``) and hopping parameter kappa
    (uniform in ``kappa``) for a batch of n chains."""
    r = _rng(seed, 8)
    return r.choice(np.asarray(betas), size=n), r.uniform(kappa[0], kappa[1], size=n)
