"""The action S(U) as a torch.autograd.Function on a 128 x 128 lattice,
beta = 4.0, kappa = 0.25: backward against central finite differences
(step 1e-6, FP64) on 64 random links and against the oracle's force;
double backward against finite differences of the force and against the
exact force-gradient term; the shifted-force approximation against the
exact term."""
import math

import numpy as np
import pytest

from oracle import schwinger as sw
from paper_1512_03812_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = T = 128
BETA, KAPPA = 4.0, 0.25


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    P.build()
    m0 = sw.kappa_to_m0(KAPPA)
    lat = P.Lattice(L, T, BETA, m0)
    q0 = I.hot_links(L, T, 31)
    eta = I.noise(L, T, 32)
    q = torch.tensor(q0, device="cuda")
    U64, _ = lat.links(q)
    phi = lat.apply_D(U64, torch.tensor(eta, device="cuda"), dagger=True)
    idx = np.random.default_rng(33).choice(L * T * 2, size=64, replace=False)
    return P, torch, lat, q0, eta, q, phi, idx, P.CG(tol=1e-13, maxit=50000)


def test_backward_matches_finite_differences(env):
    P, torch, lat, q0, eta, q, phi, idx, cg = env
    from paper_1512_03812_gb300.autograd import action
    qq = q.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(action(qq, phi, lat, "full", cg).sum(), qq)
    g = g.detach().cpu().numpy().ravel()
    eps = 1e-6
    fd = []
    for i in idx:
        qp = q.clone().view(-1)
        qm = q.clone().view(-1)
        qp[i] += eps
        qm[i] -= eps
        Sp = float(action(qp.view(-1, 2), phi, lat, "full", cg))
        Sm = float(action(qm.view(-1, 2), phi, lat, "full", cg))
        fd.append((Sp - Sm) / (2 * eps))
    fd = np.array(fd)
    # FD error ~ |S| eps_machine / eps + O(eps^2): about 1e-6 absolute here
    assert np.abs(g[idx] - fd).max() < 2e-5 * max(1.0, np.abs(fd).max()), np.abs(g[idx] - fd).max()


def test_backward_matches_oracle_force(env):
    P, torch, lat, q0, eta, q, phi, idx, cg = env
    from paper_1512_03812_gb300.autograd import action
    qq = q.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(action(qq, phi, lat, "full", cg).sum(), qq)
    olat = sw.Lattice(L, T, BETA, sw.kappa_to_m0(KAPPA))
    U = sw.links(q0.reshape(T, L, 2))
    ph = sw.apply_D(olat, U, eta.reshape(T, L, 2), dagger=True)
    F = sw.force(olat, U, ph, sw.Solver(tol=1e-13))
    gg = g.cpu().numpy().reshape(T, L, 2)
    assert np.abs(gg - F).max() < 1e-10 * np.abs(F).max()


def test_double_backward_is_hessian_vector_product(env):
    P, torch, lat, q0, eta, q, phi, idx, cg = env
    from paper_1512_03812_gb300.autograd import action
    v = torch.tensor(I.link_field(L, T, 34), device="cuda")
    qq = q.clone().requires_grad_(True)
    (F,) = torch.autograd.grad(action(qq, phi, lat, "full", cg).sum(), qq, create_graph=True)
    (Hv,) = torch.autograd.grad((F * v).sum(), qq, retain_graph=True)
    eps = 1e-5
    Fp = lat.force(q + eps * v, phi, "full", cg)
    Fm = lat.force(q - eps * v, phi, "full", cg)
    fd = (Fp - Fm) / (2 * eps)
    err = float((Hv - fd).abs().max() / fd.abs().max())
    assert err < 1e-6, err
    # at v = F the double backward gives C / 2 (Eq. force_gradient)
    (Hf,) = torch.autograd.grad((F * F.detach()).sum(), qq)
    C = lat.force_gradient(q, phi, "full", cg)
    assert float((2 * Hf - C).abs().max() / C.abs().max()) < 1e-10


def test_shifted_force_approximates_exact_force_gradient(env):
    P, torch, lat, q0, eta, q, phi, idx, cg = env
    F = lat.force(q, phi, "full", cg)
    C = lat.force_gradient(q, phi, "full", cg)
    errs = []
    for h in (0.1, 0.05):
        Fs = lat.fg_shifted_force(q, phi, h, "full", cg)
        errs.append(float((Fs - (F - h * h / 48 * C)).abs().max()))
    # F(q - h^2/24 F) - (F - h^2/48 C) = O(h^4)
    assert 3.3 < math.log2(errs[0] / errs[1]) < 4.7, errs
