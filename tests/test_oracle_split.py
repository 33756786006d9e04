"""Pins of the oracle's determinant split over two masses and of the
three-level schemes (the paper's outlook, Conclusions: the fermion
determinant factorised so that the action has more than two parts).

The split is exact algebra, so it is pinned exactly on tiny lattices with
dense matrices; the forces by finite differences of the actions; the
force-gradient term of the ratio part by finite differences of |F_r|^2; the
schemes by reversibility, the order of Delta H in h and their inversion
counts.  All CPU."""
import math

import numpy as np
import pytest

from oracle import integrators as ig
from oracle import schwinger as sw
from paper_1512_03812_gb300 import inputs as I


def field(a, L, T):
    return a.reshape(T, L, *a.shape[1:])


def setup(L=4, T=4, beta=2.0, kappa=0.2, dm=0.3, seed=1):
    lat = sw.Lattice(L, T, beta=beta, m0=sw.kappa_to_m0(kappa))
    lat_h = sw.heavy_lattice(lat, dm)
    q = field(I.hot_links(L, T, seed), L, T)
    U = sw.links(q)
    eta_r = field(I.noise(L, T, seed + 1), L, T)
    eta_h = field(I.noise(L, T, seed + 2), L, T)
    phi_r, phi_h = sw.heatbath_split(lat, lat_h, U, eta_r, eta_h, sw.Solver(1e-14))
    return lat, lat_h, q, phi_r, phi_h, eta_r, eta_h


def _fd_grad(fun, q, eps=1e-5):
    g = np.zeros_like(q)
    for i in np.ndindex(q.shape):
        e = np.zeros_like(q)
        e[i] = eps
        g[i] = (fun(q + e) - fun(q - e)) / (2 * eps)
    return g


@pytest.mark.parametrize("L,T", [(2, 2), (2, 3)])
def test_split_reproduces_the_determinant_and_the_ratio_kernel(L, T):
    """det(D^dag D) = det(D_h^dag D_h) det(W^dag W), W = D D_h^{-1}, and the
    kernel of S_r (built column by column through ratio_action's operators)
    is (W^dag W)^{-1} = D_h (D^dag D)^{-1} D_h^dag, from dense matrices."""
    lat = sw.Lattice(L, T, beta=1.0, m0=sw.kappa_to_m0(0.24))
    lat_h = sw.heavy_lattice(lat, 0.4)
    U = sw.links(field(I.hot_links(L, T, 31), L, T))
    D, Dh = sw.dense_D(lat, U), sw.dense_D(lat_h, U)
    W = D @ np.linalg.inv(Dh)
    lhs = np.linalg.det(D.conj().T @ D)
    rhs = np.linalg.det(Dh.conj().T @ Dh) * np.linalg.det(W.conj().T @ W)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    n = 2 * L * T
    solver = sw.Solver(1e-15)
    K = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        psi = sw.apply_D(lat_h, U, e.reshape(T, L, 2), dagger=True)
        X = solver.DdagD_inv(lat, U, psi)
        K[:, j] = sw.apply_D(lat_h, U, X).reshape(-1)
    assert np.abs(K - np.linalg.inv(W.conj().T @ W)).max() < 1e-10 * np.abs(K).max()
    # and S_r is the quadratic form of that kernel
    phi = field(I.spinor(L, T, 32), L, T)
    S = sw.ratio_action(lat, lat_h, U, phi, solver)
    assert abs(S - np.vdot(phi.reshape(-1), K @ phi.reshape(-1)).real) < 1e-10 * abs(S)


def test_ratio_part_is_trivial_at_equal_masses():
    """dm = 0: D_h = D, so S_r = phi^dag phi whatever the links and F_r = 0."""
    lat, _, q, phi_r, _, _, _ = setup()
    same = sw.heavy_lattice(lat, 0.0)
    U = sw.links(q)
    solver = sw.Solver(1e-14)
    assert abs(sw.ratio_action(lat, same, U, phi_r, solver) - np.vdot(phi_r, phi_r).real) < 1e-10
    assert np.abs(sw.ratio_force(lat, same, U, phi_r, solver)).max() < 1e-10


def test_split_heatbath_gives_the_noise_norms():
    """phi_r = W^dag eta_r and phi_h = D_h^dag eta_h: S_r = eta_r^dag eta_r
    and S_h = eta_h^dag eta_h at the start of a trajectory."""
    lat, lat_h, q, phi_r, phi_h, eta_r, eta_h = setup(4, 6)
    U = sw.links(q)
    s = sw.Solver(1e-14)
    Sr = sw.ratio_action(lat, lat_h, U, phi_r, s)
    Sh = sw.fermion_action(lat_h, U, phi_h, s)
    assert abs(Sr - np.vdot(eta_r, eta_r).real) < 1e-10 * Sr
    assert abs(Sh - np.vdot(eta_h, eta_h).real) < 1e-10 * Sh


def test_ratio_and_heavy_forces_are_gradients_of_their_actions():
    lat, lat_h, q, phi_r, phi_h, _, _ = setup()
    s = sw.Solver(1e-14)
    Fr = sw.ratio_force(lat, lat_h, sw.links(q), phi_r, s)
    g = _fd_grad(lambda qq: sw.ratio_action(lat, lat_h, sw.links(qq), phi_r, s), q)
    assert np.abs(Fr - g).max() < 1e-7 * max(1, np.abs(Fr).max())
    Fh = sw.fermion_force(lat_h, sw.links(q), phi_h, s)
    g = _fd_grad(lambda qq: sw.fermion_action(lat_h, sw.links(qq), phi_h, s), q)
    assert np.abs(Fh - g).max() < 1e-7 * max(1, np.abs(Fh).max())


def test_ratio_force_gradient_is_gradient_of_its_force_norm():
    """C_r = grad |F_r|^2 (the force-gradient term of the ratio part alone)."""
    lat, lat_h, q, phi_r, _, _, _ = setup()
    s = sw.Solver(1e-14)
    F, C = sw.ratio_force_and_gradient(lat, lat_h, sw.links(q), phi_r, s)
    g = _fd_grad(lambda qq: np.sum(sw.ratio_force(lat, lat_h, sw.links(qq), phi_r, s) ** 2), q)
    assert np.abs(C - g).max() < 1e-6 * np.abs(C).max()


def test_split_actions_are_gauge_invariant():
    L, T = 4, 6
    lat, lat_h, q, phi_r, phi_h, _, _ = setup(L, T)
    s = sw.Solver(1e-14)
    alpha = np.random.default_rng(7).uniform(-np.pi, np.pi, (T, L))
    qg = q + np.stack([alpha - sw.shift(alpha, 0, 1), alpha - sw.shift(alpha, 1, 1)], axis=-1)
    g = np.exp(1j * alpha)[..., None]
    U, Ug = sw.links(q), sw.links(qg)
    assert abs(sw.ratio_action(lat, lat_h, U, phi_r, s)
               - sw.ratio_action(lat, lat_h, Ug, g * phi_r, s)) < 1e-9
    assert abs(sw.fermion_action(lat_h, U, phi_h, s)
               - sw.fermion_action(lat_h, Ug, g * phi_h, s)) < 1e-9
    assert np.abs(sw.ratio_force(lat, lat_h, U, phi_r, s)
                  - sw.ratio_force(lat, lat_h, Ug, g * phi_r, s)).max() < 1e-9


def _state(seed=2, tol=1e-14, dm=0.3):
    lat, lat_h, q, phi_r, phi_h, _, _ = setup(dm=dm)
    p = field(I.momenta(lat.L, lat.T, seed), lat.L, lat.T)
    return ig.State(lat, q.copy(), p, phi_r, sw.Solver(tol), lat_h, phi_h)


def _H(st):
    return sw.hamiltonian_split(st.lat, st.lat_h, st.q, st.p, st.phi, st.phi_h, st.solver)


@pytest.mark.parametrize("scheme,fg", [("nested3_leapfrog", "exact"),
                                       ("adapted_nested3_fg", "exact"),
                                       ("adapted_nested3_fg", "shifted")])
def test_three_level_reversibility(scheme, fg):
    st = _state()
    q0, p0 = st.q.copy(), st.p.copy()
    ig.md_trajectory(st, scheme, 0.6, 3, M=2, fg=fg, M2=2)
    st.p = -st.p
    ig.md_trajectory(st, scheme, 0.6, 3, M=2, fg=fg, M2=2)
    assert np.abs(st.q - q0).max() < 1e-10
    assert np.abs(st.p + p0).max() < 1e-10


def _dH_slope(scheme, M2, fg="exact", ns=(4, 8), tau=0.5):
    errs = []
    for n in ns:
        st = _state(tol=1e-11)
        H0 = _H(st)
        ig.md_trajectory(st, scheme, tau, n, M=1, fg=fg, M2=M2)
        errs.append(abs(_H(st) - H0))
    return math.log(errs[0] / errs[1]) / math.log(ns[1] / ns[0])


@pytest.mark.parametrize("scheme,M2,fg,order", [
    ("nested3_leapfrog", 2, "exact", 2),
    ("adapted_nested3_fg", 1, "exact", 2),
    # fourth order once the leapfrog levels' errors O((h/M2)^2) are negligible
    # against O(h^4) over the step sizes compared: M2 = 400 here (measured
    # local slopes 4.27, 4.04, 3.91 from n = 3 to 6; n = 3, 4 compared)
    ("adapted_nested3_fg", 400, "exact", 4),
])
def test_three_level_delta_H_order(scheme, M2, fg, order):
    s = _dH_slope(scheme, M2, fg, ns=(3, 4) if M2 > 100 else (4, 8))
    assert abs(s - order) < 0.6, s


def test_shifted_ratio_force_matches_its_force_gradient_to_fourth_order():
    """F_r(q - (h^2/24) F_r(q)) = F_r - (h^2/48) C_r + O(h^4): the shifted
    kick of the ratio part replaces the exact one to the order the scheme
    needs (so the shifted three-level scheme keeps the exact one's order)."""
    lat, lat_h, q, phi_r, _, _, _ = setup()
    s = sw.Solver(1e-14)
    F, C = sw.ratio_force_and_gradient(lat, lat_h, sw.links(q), phi_r, s)
    errs = []
    for h in (0.2, 0.1):
        Fs = sw.ratio_force(lat, lat_h, sw.links(q - (h * h / 24.0) * F), phi_r, s)
        errs.append(np.abs(Fs - (F - h * h / 48.0 * C)).max())
    assert 3.5 < math.log2(errs[0] / errs[1]) < 4.5, errs


@pytest.mark.parametrize("scheme,fg,light,heavy_per_M2", [
    ("nested3_leapfrog", "exact", 4, 4),
    ("adapted_nested3_fg", "exact", 8, 8),
    ("adapted_nested3_fg", "shifted", 8, 8),
])
def test_three_level_inversions_per_step(scheme, fg, light, heavy_per_M2):
    """Per step: 2 inversions per force of a part (one solve of D^dag D),
    2 more for the exact C of the ratio part (the Z-solve), the same 2 for
    the second force of the shifted form; the ratio part's solves are of
    the light operator, the heavy part's of D_h."""
    for M2 in (1, 3):
        st = _state(tol=1e-8)
        ig.SCHEMES[scheme](st, 0.1, M=2, M2=M2, fg=fg)
        by = st.solver.inversions_by_m0
        assert by.get(st.lat.m0, 0) == light
        assert by.get(st.lat_h.m0, 0) == heavy_per_M2 * M2


def test_split_hmc_accepts_by_delta_H_and_matches_its_parts():
    """One HMC update with the split action: H at the start is K + S_G +
    eta_r^dag eta_r + eta_h^dag eta_h (the heatbath identity), Delta H is
    small at a small step, and sf_start='noise' gives the same trajectory."""
    lat, lat_h, q, _, _, eta_r, eta_h = setup()
    p = field(I.momenta(4, 4, 9), 4, 4)
    eta = np.stack([eta_r, eta_h])
    s = sw.Solver(1e-14)
    r = ig.hmc_trajectory(lat, q, p, eta, 0.5, "adapted_nested3_fg", 0.5, 4, M=2, M2=2,
                          solver=s, dm=0.3)
    H0 = (sw.kinetic(p) + sw.gauge_action(lat, sw.links(q)) + np.vdot(eta_r, eta_r).real
          + np.vdot(eta_h, eta_h).real)
    assert abs(r.H0 - H0) < 1e-10 * abs(H0)
    assert abs(r.dH) < 0.05 and r.accepted
    r2 = ig.hmc_trajectory(lat, q, p, eta, 0.5, "adapted_nested3_fg", 0.5, 4, M=2, M2=2,
                           solver=s, dm=0.3, sf_start="noise")
    assert np.abs(r2.q_md - r.q_md).max() < 1e-12
    assert abs(r2.dH - r.dH) < 1e-9
