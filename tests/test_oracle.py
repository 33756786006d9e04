"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form, a brute-force construction, finite differences, an invariance,
or a number printed in the paper.  All CPU, small lattices.
"""
import math
import os

import numpy as np
import pytest

from oracle import integrators as ig
from oracle import schwinger as sw
from paper_1512_03812_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def field(a, L, T):
    return a.reshape(T, L, *a.shape[1:])


def setup(L=4, T=6, beta=1.3, kappa=0.22, seed=1):
    lat = sw.Lattice(L, T, beta=beta, m0=sw.kappa_to_m0(kappa))
    q = field(I.hot_links(L, T, seed), L, T)
    eta = field(I.noise(L, T, seed + 1), L, T)
    phi = sw.apply_D(lat, sw.links(q), eta, dagger=True)
    return lat, q, phi


# ------------------------------------------------------------ operator D ----

@pytest.mark.parametrize("L,T", [(2, 2), (3, 5), (4, 6), (1, 4)])
def test_D_matches_dense_matrix_entry_by_entry(L, T):
    lat, q, _ = setup(L, T)
    U = sw.links(q)
    D = sw.dense_D(lat, U)
    psi = field(I.spinor(L, T, 7), L, T)
    assert np.allclose(sw.apply_D(lat, U, psi).ravel(), D @ psi.ravel(), atol=1e-13)
    assert np.allclose(sw.apply_D(lat, U, psi, dagger=True).ravel(),
                       D.conj().T @ psi.ravel(), atol=1e-13)


def _free_eigs(L, T, m0, a=(0.0, 0.0)):
    """Closed-form spectrum of D at U_mu = exp(i a_mu):
    m0 + sum(1 - cos k) +- i sqrt(sum sin^2 k), k_x = 2 pi j / L + a_x,
    k_t = 2 pi (j + 1/2) / T + a_t (antiperiodic in time)."""
    out = []
    for jx in range(L):
        for jt in range(T):
            k = (2 * np.pi * jx / L + a[0], 2 * np.pi * (jt + 0.5) / T + a[1])
            re = m0 + sum(1 - np.cos(kk) for kk in k)
            im = np.sqrt(sum(np.sin(kk) ** 2 for kk in k))
            out += [re + 1j * im, re - 1j * im]
    return np.array(out)


def _same_multiset(a, b, tol=1e-10):
    a = list(a)
    for z in b:
        j = int(np.argmin(np.abs(np.array(a) - z)))
        if abs(a[j] - z) > tol:
            return False
        a.pop(j)
    return True


@pytest.mark.parametrize("L,T,m0", [(4, 4, 0.1), (6, 4, -0.3), (5, 3, 0.5)])
def test_free_field_spectrum(L, T, m0):
    lat = sw.Lattice(L, T, beta=1.0, m0=m0)
    U = np.ones((T, L, 2), dtype=complex)
    assert _same_multiset(np.linalg.eigvals(sw.dense_D(lat, U)), _free_eigs(L, T, m0))


def test_constant_background_shifts_momenta():
    L, T, m0, a = 4, 6, 0.2, (0.3, -0.7)
    lat = sw.Lattice(L, T, beta=1.0, m0=m0)
    q = np.empty((T, L, 2))
    q[..., 0], q[..., 1] = a
    ev = np.linalg.eigvals(sw.dense_D(lat, sw.links(q)))
    assert _same_multiset(ev, _free_eigs(L, T, m0, a))


def test_pure_gauge_background_has_free_spectrum():
    L, T, m0 = 4, 6, 0.2
    lat = sw.Lattice(L, T, beta=1.0, m0=m0)
    alpha = np.random.default_rng(3).uniform(-np.pi, np.pi, (T, L))
    q = np.stack([alpha - sw.shift(alpha, 0, 1), alpha - sw.shift(alpha, 1, 1)], axis=-1)
    ev = np.linalg.eigvals(sw.dense_D(lat, sw.links(q)))
    assert _same_multiset(ev, _free_eigs(L, T, m0))


def test_gamma5_hermiticity():
    lat, q, _ = setup(5, 4)
    U = sw.links(q)
    x = field(I.spinor(5, 4, 11), 5, 4)
    y = field(I.spinor(5, 4, 12), 5, 4)
    s3 = lambda v: v @ sw.SIGMA3.T
    # sigma_3 D sigma_3 = D^dag
    assert np.allclose(s3(sw.apply_D(lat, U, s3(x))), sw.apply_D(lat, U, x, dagger=True), atol=1e-13)
    # <y, D^dag x> = <D y, x>
    assert abs(np.vdot(y, sw.apply_D(lat, U, x, True)) - np.vdot(sw.apply_D(lat, U, y), x)) < 1e-12


def test_cg_matches_dense_solve_and_true_residual():
    lat, q, phi = setup(4, 4, kappa=0.24)
    U = sw.links(q)
    D = sw.dense_D(lat, U)
    solver = sw.Solver(tol=1e-12)
    x = solver.cg(lat, U, phi)
    xd = np.linalg.solve(D.conj().T @ D, phi.ravel())
    assert np.allclose(x.ravel(), xd, atol=1e-9 * np.abs(xd).max())
    r = phi - sw.apply_DdagD(lat, U, x)
    assert np.linalg.norm(r) <= 2e-12 * np.linalg.norm(phi)


# ------------------------------------------------------- actions, forces ----

def _fd_grad(fun, q, eps=1e-5, idx=None):
    idx = list(np.ndindex(q.shape)) if idx is None else idx
    g = np.zeros_like(q)
    for i in idx:
        e = np.zeros_like(q)
        e[i] = eps
        g[i] = (fun(q + e) - fun(q - e)) / (2 * eps)
    return g, idx


def test_gauge_action_closed_form():
    # S_G = beta sum (1 - cos theta), theta = q1(n) + q2(n+1) - q1(n+2) - q2(n)
    lat, q, _ = setup(5, 3)
    th = q[..., 0] + sw.shift(q[..., 1], 0, 1) - sw.shift(q[..., 0], 1, 1) - q[..., 1]
    assert abs(sw.gauge_action(lat, sw.links(q)) - lat.beta * np.sum(1 - np.cos(th))) < 1e-12


def test_gauge_force_is_gradient_of_gauge_action():
    lat, q, _ = setup(4, 5)
    F = sw.gauge_force(lat, sw.links(q))
    g, _ = _fd_grad(lambda qq: sw.gauge_action(lat, sw.links(qq)), q)
    assert np.abs(F - g).max() < 1e-8 * max(1, np.abs(F).max())


def test_fermion_force_is_gradient_of_fermion_action():
    lat, q, phi = setup(4, 4)
    solver = sw.Solver(tol=1e-14)
    f = sw.fermion_force(lat, sw.links(q), phi, solver)
    g, _ = _fd_grad(lambda qq: sw.fermion_action(lat, sw.links(qq), phi, solver), q)
    assert np.abs(f - g).max() < 1e-7 * max(1, np.abs(f).max())


def test_fermion_action_at_heatbath_equals_noise_norm():
    # phi = D^dag eta  =>  phi^dag (D^dag D)^{-1} phi = eta^dag eta
    L, T = 4, 6
    lat, q, _ = setup(L, T)
    eta = field(I.noise(L, T, 5), L, T)
    phi = sw.apply_D(lat, sw.links(q), eta, dagger=True)
    S = sw.fermion_action(lat, sw.links(q), phi, sw.Solver(tol=1e-14))
    assert abs(S - np.vdot(eta, eta).real) < 1e-10 * S


def test_gauge_invariance():
    L, T = 4, 6
    lat, q, phi = setup(L, T)
    solver = sw.Solver(tol=1e-14)
    alpha = np.random.default_rng(9).uniform(-np.pi, np.pi, (T, L))
    qg = q + np.stack([alpha - sw.shift(alpha, 0, 1), alpha - sw.shift(alpha, 1, 1)], axis=-1)
    phig = np.exp(1j * alpha)[..., None] * phi
    U, Ug = sw.links(q), sw.links(qg)
    assert abs(sw.gauge_action(lat, U) - sw.gauge_action(lat, Ug)) < 1e-11
    assert abs(sw.fermion_action(lat, U, phi, solver) - sw.fermion_action(lat, Ug, phig, solver)) < 1e-9
    assert np.abs(sw.force(lat, U, phi, solver) - sw.force(lat, Ug, phig, solver)).max() < 1e-9
    C = sw.force_gradient(lat, U, phi, solver)
    Cg = sw.force_gradient(lat, Ug, phig, solver)
    assert np.abs(C - Cg).max() < 1e-8 * np.abs(C).max()


# ---------------------------------------------------- force-gradient term --

def test_c_gg_is_gradient_of_gauge_force_norm():
    # C_GG = d/dq |F_G|^2 (Eq. force_gradient restricted to S_G)
    lat, q, _ = setup(5, 4)
    C = sw.c_gg(lat, sw.links(q))
    g, _ = _fd_grad(lambda qq: np.sum(sw.gauge_force(lat, sw.links(qq)) ** 2), q)
    assert np.abs(C - g).max() < 1e-7 * np.abs(C).max()


def test_c_fg_is_twice_gauge_hessian_times_v():
    lat, q, _ = setup(4, 5)
    v = field(I.link_field(4, 5, 3), 4, 5)
    eps = 1e-5
    hv = (sw.gauge_force(lat, sw.links(q + eps * v)) - sw.gauge_force(lat, sw.links(q - eps * v))) / (2 * eps)
    assert np.abs(sw.c_fg(lat, sw.links(q), v) - 2 * hv).max() < 1e-7 * np.abs(hv).max()


def test_c_fermion_is_twice_fermion_hessian_times_v():
    # Eq. CFF / Z12 with f -> v:  4 Re[...] = 2 (Hess S_F) v
    lat, q, phi = setup(4, 4)
    solver = sw.Solver(tol=1e-14)
    v = field(I.link_field(4, 4, 4), 4, 4)
    U = sw.links(q)
    chi, xi = sw.chi_xi(lat, U, phi, solver)
    eps = 1e-5
    hv = (sw.fermion_force(lat, sw.links(q + eps * v), phi, solver)
          - sw.fermion_force(lat, sw.links(q - eps * v), phi, solver)) / (2 * eps)
    Cv = sw.c_fermion(lat, U, chi, xi, v, solver)
    assert np.abs(Cv - 2 * hv).max() < 1e-6 * np.abs(hv).max()


def test_full_force_gradient_is_gradient_of_force_norm():
    # Eq. force_gradient: C = 2 sum_m dS/dq_m d2S/dq_m dq_n = d/dq_n |F|^2
    lat, q, phi = setup(4, 4)
    solver = sw.Solver(tol=1e-14)
    C = sw.force_gradient(lat, sw.links(q), phi, solver)
    g, _ = _fd_grad(lambda qq: np.sum(sw.force(lat, sw.links(qq), phi, solver) ** 2), q)
    assert np.abs(C - g).max() < 1e-6 * np.abs(C).max()
    Cff = sw.force_gradient(lat, sw.links(q), phi, solver, "fermion")
    g, _ = _fd_grad(lambda qq: np.sum(sw.fermion_force(lat, sw.links(qq), phi, solver) ** 2), q)
    assert np.abs(Cff - g).max() < 1e-6 * np.abs(Cff).max()


def test_shifted_force_matches_force_gradient_to_fourth_order():
    # F(q - h^2/24 F) = F - (h^2/48) C + O(h^4)
    lat, q, phi = setup(4, 4)
    solver = sw.Solver(tol=1e-14)
    U = sw.links(q)
    F, C = sw.force_and_gradient(lat, U, phi, solver, "full")
    errs = []
    for h in (0.2, 0.1):
        Fs = sw.shifted_force(lat, q, phi, solver, h, "full")
        errs.append(np.abs(Fs - (F - h * h / 48 * C)).max())
    assert 3.5 < math.log2(errs[0] / errs[1]) < 4.5


# ---------------------------------------------------------------- schemes --

ALL = [("leapfrog", 1), ("five_stage", 1), ("five_stage_fg", 1), ("nested_leapfrog", 3),
       ("nested_five_stage", 3), ("nested_fg", 2), ("adapted_nested_fg", 2), ("eleven_stage", 1)]


def _state(lat, q, phi, tol=1e-14, seed=2):
    p = field(I.momenta(lat.L, lat.T, seed), lat.L, lat.T)
    return ig.State(lat, q.copy(), p, phi, sw.Solver(tol=tol))


@pytest.mark.parametrize("scheme,M", ALL)
@pytest.mark.parametrize("fg", ["exact", "shifted"])
def test_reversibility(scheme, M, fg):
    if fg == "shifted" and "fg" not in scheme:
        pytest.skip("no force-gradient kick")
    lat, q, phi = setup(4, 4, beta=2.0, kappa=0.2)
    st = _state(lat, q, phi)
    p0 = st.p.copy()
    ig.md_trajectory(st, scheme, 0.6, 3, M=M, fg=fg)
    st.p = -st.p
    ig.md_trajectory(st, scheme, 0.6, 3, M=M, fg=fg)
    assert np.abs(st.q - q).max() < 1e-10
    assert np.abs(st.p + p0).max() < 1e-10


def _golden_inversions():
    out = {}
    for line in open(os.path.join(GOLDEN, "inversions_per_step.txt")):
        if line.strip() and not line.startswith("#"):
            name, k = line.split()[:2]
            out[name] = int(k)
    return out


@pytest.mark.parametrize("key", sorted(_golden_inversions()))
def test_inversions_per_step_match_paper(key):
    scheme, _, fg = key.partition(":")
    lat, q, phi = setup(4, 4, beta=2.0, kappa=0.2)
    st = _state(lat, q, phi, tol=1e-8)
    ig.SCHEMES[scheme](st, 0.1, M=2, fg=fg or "exact")
    assert st.solver.inversions == _golden_inversions()[key]


def _dH_slope(scheme, M, fg="exact", ns=(4, 8, 16), tau=0.5):
    lat, q, phi = setup(4, 4, beta=2.0, kappa=0.2)
    errs = []
    for n in ns:
        st = _state(lat, q, phi)
        H0 = sw.hamiltonian(lat, st.q, st.p, phi, st.solver)
        ig.md_trajectory(st, scheme, tau, n, M=M(n) if callable(M) else M, fg=fg)
        errs.append(abs(sw.hamiltonian(lat, st.q, st.p, phi, st.solver) - H0))
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("scheme,M,fg,order", [
    ("leapfrog", 1, "exact", 2), ("five_stage", 1, "exact", 2),
    ("nested_leapfrog", 3, "exact", 2), ("nested_five_stage", 3, "exact", 2),
    ("five_stage_fg", 1, "exact", 4), ("five_stage_fg", 1, "shifted", 4),
    ("nested_fg", 2, "exact", 4), ("nested_fg", 2, "shifted", 4),
    # the adapted scheme is fourth order once the inner leapfrog error
    # O((h/M)^2) is negligible against O(h^4): M grows like 1/h^2 here
    ("adapted_nested_fg", lambda n: 2 * n * n, "exact", 4),
    ("adapted_nested_fg", lambda n: 2 * n * n, "shifted", 4),
    ("adapted_nested_fg", 1, "exact", 2),
    ("eleven_stage", 1, "exact", 4),
])
def test_delta_H_order(scheme, M, fg, order):
    s = _dH_slope(scheme, M, fg, ns=(5, 10) if callable(M) else (4, 8, 16))
    assert abs(s[-1] - order) < 0.6, s


def test_fg_sign_matters():
    """The opposite sign of the C term (as printed in Eq. 5stage_fg when C is
    read as grad |F|^2) loses fourth order: this pins the sign reading."""
    lat, q, phi = setup(4, 4, beta=2.0, kappa=0.2)

    def run(n, sgn):
        st = _state(lat, q, phi)
        H0 = sw.hamiltonian(lat, st.q, st.p, phi, st.solver)
        h = 0.5 / n
        for _ in range(n):
            ig.kick(st, h / 6, "full")
            ig.drift(st, h / 2)
            F, C = sw.force_and_gradient(lat, sw.links(st.q), phi, st.solver, "full")
            st.p = st.p - 2 * h / 3 * F + sgn * h ** 3 / 72 * C
            ig.drift(st, h / 2)
            ig.kick(st, h / 6, "full")
        return abs(sw.hamiltonian(lat, st.q, st.p, phi, st.solver) - H0)

    good = math.log2(run(8, +1) / run(16, +1))
    bad = math.log2(run(8, -1) / run(16, -1))
    assert good > 3.5 and bad < 2.6


def test_metropolis_decision():
    lat, q, _ = setup(4, 4, beta=2.0, kappa=0.2)
    p = field(I.momenta(4, 4, 3), 4, 4)
    eta = field(I.noise(4, 4, 4), 4, 4)
    r = ig.hmc_trajectory(lat, q, p, eta, 0.999999, "leapfrog", 1.0, 2, solver=sw.Solver(1e-12))
    assert r.accepted == (r.dH <= 0 or 0.999999 < math.exp(-r.dH))
    assert np.array_equal(r.q, r.q_md) == r.accepted
    r0 = ig.hmc_trajectory(lat, q, p, eta, 0.0, "leapfrog", 1.0, 2, solver=sw.Solver(1e-12))
    assert r0.accepted


def test_sf_start_from_noise_matches_the_solve():
    """H at the start with S_F = eta^dag eta (exact for phi = D^dag eta)
    against S_F = phi^dag (D^dag D)^{-1} phi by CG: the same trajectory, H0
    and Delta H equal to the solver's tolerance, the same decision."""
    lat, q, _ = setup(4, 6, beta=2.0, kappa=0.22)
    p = field(I.momenta(4, 6, 5), 4, 6)
    eta = field(I.noise(4, 6, 6), 4, 6)
    a = ig.hmc_trajectory(lat, q, p, eta, 0.5, "leapfrog", 1.0, 4, solver=sw.Solver(1e-14))
    b = ig.hmc_trajectory(lat, q, p, eta, 0.5, "leapfrog", 1.0, 4, solver=sw.Solver(1e-14),
                          sf_start="noise")
    assert abs(a.H0 - b.H0) < 1e-10 * abs(a.H0)
    assert abs(a.dH - b.dH) < 1e-10 * abs(a.H0)
    assert np.array_equal(a.q_md, b.q_md) and a.accepted == b.accepted
    # the identity it rests on, on a random field: phi^dag (D^dag D)^-1 phi = |eta|^2
    U = sw.links(q)
    phi = sw.apply_D(lat, U, eta, dagger=True)
    assert abs(sw.fermion_action(lat, U, phi, sw.Solver(1e-14)) - np.vdot(eta, eta).real) < 1e-10


def test_creutz_equality_on_markov_chain():
    """<exp(-Delta H)> = 1 in equilibrium (a consequence of reversibility and
    area preservation, Sec. 2.2), checked on an oracle HMC chain."""
    L, T = 4, 4
    lat = sw.Lattice(L, T, beta=1.0, m0=sw.kappa_to_m0(0.2))
    q = field(I.hot_links(L, T, 21), L, T)
    us = I.uniforms(400, 22)
    vals = []
    solver = sw.Solver(tol=1e-10)
    for k in range(400):
        p = field(I.momenta(L, T, 1000 + k), L, T)
        eta = field(I.noise(L, T, 5000 + k), L, T)
        r = ig.hmc_trajectory(lat, q, p, eta, us[k], "leapfrog", 1.0, 3, solver=solver)
        q = r.q
        if k >= 50:
            vals.append(math.exp(-r.dH))
    vals = np.array(vals)
    err = vals.std() / math.sqrt(len(vals))
    assert abs(vals.mean() - 1.0) < 3 * err + 1e-3, (vals.mean(), err)


# ------------------------------------------- 11-stage weights, BCH check --

def _free_log(seq, deg=5):
    """log of a product of exponentials exp(c X) (X = 'a' or 'b') in the free
    associative algebra truncated at degree `deg`: {word: coefficient}."""
    def mul(x, y):
        z = {}
        for w1, c1 in x.items():
            for w2, c2 in y.items():
                if len(w1) + len(w2) <= deg:
                    z[w1 + w2] = z.get(w1 + w2, 0.0) + c1 * c2
        return z
    prod = {"": 1.0}
    for letter, c in seq:
        prod = mul(prod, {letter * k: c ** k / math.factorial(k) for k in range(deg + 1)})
    z = {w: c for w, c in prod.items() if w}
    out, power = {}, {"": 1.0}
    for k in range(1, deg + 1):
        power = mul(power, z)
        for w, c in power.items():
            out[w] = out.get(w, 0.0) + (-1) ** (k + 1) * c / k
    return out


def _eleven_stage_seq(sigma, eta, lam, theta):
    """Eq. 11_stage as a word of exponentials: b = the force flow, a = drift."""
    mb, ma = (1 - 2 * (lam + sigma)) / 2, 1 - 2 * (theta + eta)
    return [("b", sigma), ("a", eta), ("b", lam), ("a", theta), ("b", mb), ("a", ma),
            ("b", mb), ("a", theta), ("b", lam), ("a", eta), ("b", sigma)]


def test_eleven_stage_weights_are_fourth_order():
    """log Delta_11 = h (A + B) + O(h^5): the degree-1 part is a + b, degrees 2
    and 4 vanish by symmetry, and the weights of Eq. (71) of Omelyan, Mryglod
    and Folk (used by the paper for Eq. 11_stage) cancel both degree-3
    commutators [a,[a,b]] = aab - 2 aba + baa and [b,[b,a]]: the coefficients
    of the words aab and bba.  Moving one weight by 1e-6 breaks it."""
    w = ig.OMELYAN_11
    lg = _free_log(_eleven_stage_seq(w["sigma"], w["eta"], w["lam"], w["theta"]))
    assert abs(lg["a"] - 1) < 1e-15 and abs(lg["b"] - 1) < 1e-15
    for word, c in lg.items():
        if len(word) in (2, 3, 4):
            assert abs(c) < 1e-14, (word, c)
    assert max(abs(c) for word, c in lg.items() if len(word) == 5) > 1e-5  # not sixth order
    bad = _free_log(_eleven_stage_seq(w["sigma"] + 1e-6, w["eta"], w["lam"], w["theta"]))
    assert max(abs(bad["aab"]), abs(bad["bba"])) > 1e-8
