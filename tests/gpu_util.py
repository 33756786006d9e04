"""Helpers for the GPU parity tests: ragged batches of seeded inputs, fed
identically to the CUDA path (through the C ABI) and to the CPU oracle."""
from __future__ import annotations

import numpy as np

from oracle import schwinger as sw
from paper_1512_03812_gb300 import inputs as I


class Batch:
    def __init__(self, dims, betas=2.0, kappas=0.24, seed=0):
        import torch

        import paper_1512_03812_gb300 as P

        self.dims = list(dims)
        n = len(self.dims)
        self.betas = np.broadcast_to(np.asarray(betas, float), (n,)).copy()
        self.kappas = np.broadcast_to(np.asarray(kappas, float), (n,)).copy()
        self.m0 = np.array([sw.kappa_to_m0(k) for k in self.kappas])
        self.lat = P.Lattice([d[0] for d in self.dims], [d[1] for d in self.dims], self.betas,
                             self.m0)
        self.olat = [sw.Lattice(L, T, b, m) for (L, T), b, m in zip(self.dims, self.betas, self.m0)]
        self.off = self.lat.offsets
        self.seed = seed
        self.torch = torch

    # numpy batch arrays (concatenated chains) -------------------------------
    def gen(self, fn, salt):
        return np.concatenate([fn(L, T, self.seed * 1000 + 17 * c + salt)
                               for c, (L, T) in enumerate(self.dims)])

    def q(self, salt=1):
        return self.gen(I.hot_links, salt)

    def p(self, salt=2):
        return self.gen(I.momenta, salt)

    def eta(self, salt=3):
        return self.gen(I.noise, salt)

    def spinor(self, salt=4):
        return self.gen(I.spinor, salt)

    def v(self, salt=5):
        return self.gen(I.link_field, salt)

    def dev(self, a, dtype=None):
        t = self.torch.tensor(np.ascontiguousarray(a), device="cuda")
        return t if dtype is None else t.to(dtype)

    def chain(self, a, c):
        """Chain c of a batch array, reshaped to the oracle's (T, L, ...)."""
        L, T = self.dims[c]
        if hasattr(a, "cpu"):
            a = a.cpu().numpy()
        return a[self.off[c]:self.off[c + 1]].reshape(T, L, *a.shape[1:])


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(1e-300, np.abs(b).max()))
