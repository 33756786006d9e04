"""Schwinger-model lattice operators, actions, forces and force-gradient terms.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): a plain FP64 numpy
restatement of Sec. 3 of "Adapted nested force-gradient integrators: the
Schwinger model case" (arXiv:1512.03812).  Shares no code with the CUDA path.

Conventions (where the paper is silent, the reading taken is stated here)
-------------------------------------------------------------------------
* A lattice is L (space, x, paper direction mu=1) by T (time, t, paper
  mu=2).  Every field is a numpy array of shape (T, L, ...): site
  n = (x, t) sits at [t, x], so the C-order flattening is n = x + L*t.
  Direction index mu = 0 is x, mu = 1 is t.
* Links U_mu(n) = exp(i q_mu(n)) (Sec. 3, after Eq. gauge_action); the
  angles q and the momenta p have shape (T, L, 2).  Gauge links are
  periodic in both directions.
* Spinors have shape (T, L, 2) complex.  Fermions are periodic in x and
  antiperiodic in t: a fermion field read across the t = T-1 -> 0 boundary
  picks up the factor ``bc`` (default -1).  ``psi_shift`` is the only place
  this sign enters.
* The force is F = dS/dq (Eq. force); kicks are p <- p - eps F.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
# Pauli matrices sigma_1, sigma_2 of the Wilson-Dirac operator (Sec. 3).
SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
)
SIGMA3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)

# field arrays are indexed [t, x, ...]: direction mu runs along this axis
_AXIS = (1, 0)


@dataclass
class Lattice:
    """An L x T lattice with couplings beta (Eq. gauge_action) and m0 (the
    Wilson-Dirac operator); ``bc`` is the fermion time-boundary factor."""

    L: int
    T: int
    beta: float
    m0: float
    bc: float = -1.0

    @property
    def V(self) -> int:
        return self.L * self.T


def kappa_to_m0(kappa: float) -> float:
    """Hopping parameter to bare mass: kappa = 1 / (2 (2 + m0)) (the paper
    writes D with m0, Sec. 3; the configurations give kappa)."""
    return 1.0 / (2.0 * kappa) - 2.0


# ---------------------------------------------------------------- geometry --

def shift(a: np.ndarray, mu: int, d: int) -> np.ndarray:
    """a(n + d mu_hat) for a periodic (gauge) field."""
    return np.roll(a, -d, axis=_AXIS[mu])


def psi_shift(psi: np.ndarray, mu: int, d: int, bc: float) -> np.ndarray:
    """psi(n + d mu_hat) for a fermion field, d = +1 or -1: periodic in x,
    and in t a value brought across the t = T-1 <-> 0 boundary is
    multiplied by ``bc`` (the paper does not state the fermion boundary
    conditions; antiperiodic in t is the reading taken)."""
    out = np.roll(psi, -d, axis=_AXIS[mu]).copy()
    if mu == 1 and bc != 1.0:
        if d == +1:
            out[-1] *= bc  # row T-1 now holds row 0
        else:
            out[0] *= bc  # row 0 now holds row T-1
    return out


def links(q: np.ndarray) -> np.ndarray:
    """U_mu(n) = exp(i q_mu(n)) (Sec. 3, after Eq. gauge_action)."""
    return np.exp(1j * q)


def _pm(mat: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 2x2 spin matrix at every site."""
    return psi @ mat.T


# ------------------------------------------------------- Wilson-Dirac D ----

def apply_D(lat: Lattice, U: np.ndarray, psi: np.ndarray, dagger: bool = False) -> np.ndarray:
    """Wilson-Dirac operator of Sec. 3,

        (D psi)(n) = (2 + m0) psi(n)
                     - 1/2 sum_mu [ (1 - sigma_mu) U_mu(n) psi(n + mu)
                                   + (1 + sigma_mu) U_mu^dag(n - mu) psi(n - mu) ].

    With ``dagger`` the adjoint D^dag_{n,m} = conj(D_{m,n}): the two hops
    keep their links and swap their spin projectors (sigma_mu is
    hermitian)."""
    out = (2.0 + lat.m0) * psi
    for mu in (0, 1):
        p_fwd = I2 - SIGMA[mu]
        p_bwd = I2 + SIGMA[mu]
        if dagger:
            p_fwd, p_bwd = p_bwd, p_fwd
        fwd = U[..., mu, None] * psi_shift(psi, mu, +1, lat.bc)
        bwd = psi_shift(np.conj(U[..., mu])[..., None] * psi, mu, -1, lat.bc)
        out = out - 0.5 * (_pm(p_fwd, fwd) + _pm(p_bwd, bwd))
    return out


def apply_DdagD(lat: Lattice, U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """D^dag D psi, the normal operator of Eq. fer_action."""
    return apply_D(lat, U, apply_D(lat, U, psi), dagger=True)


def dense_D(lat: Lattice, U: np.ndarray) -> np.ndarray:
    """The matrix D_{n,m} of Sec. 3 built entry by entry from its Kronecker
    deltas (site-major, spin fastest: row 2n+s).  For tiny lattices only."""
    L, T = lat.L, lat.T
    D = np.zeros((2 * lat.V, 2 * lat.V), dtype=np.complex128)
    for t in range(T):
        for x in range(L):
            n = x + L * t
            D[2 * n:2 * n + 2, 2 * n:2 * n + 2] += (2.0 + lat.m0) * I2
            for mu in (0, 1):
                # delta_{n, m - mu}: column m = n + mu
                xp, tp = (x + 1) % L if mu == 0 else x, (t + 1) % T if mu == 1 else t
                sgn = lat.bc if (mu == 1 and t == T - 1) else 1.0
                m = xp + L * tp
                D[2 * n:2 * n + 2, 2 * m:2 * m + 2] += -0.5 * (I2 - SIGMA[mu]) * U[t, x, mu] * sgn
                # delta_{n, m + mu}: column m = n - mu, link U_mu(n - mu)^dag
                xm, tm = (x - 1) % L if mu == 0 else x, (t - 1) % T if mu == 1 else t
                sgn = lat.bc if (mu == 1 and t == 0) else 1.0
                m = xm + L * tm
                D[2 * n:2 * n + 2, 2 * m:2 * m + 2] += (
                    -0.5 * (I2 + SIGMA[mu]) * np.conj(U[tm, xm, mu]) * sgn)
    return D


# ------------------------------------------------------------ inversion ----

class Solver:
    """Textbook conjugate gradient on D^dag D x = b from x = 0.

    The paper does not name its solver (Sec. 3, end); CG on the normal
    equations is the reading used here.  It stops when the recursive
    residual satisfies |r| <= tol |b| and raises if ``maxit`` is reached.

    ``inversions`` counts inversions of D in the paper's units (Sec. 3,
    end): a solve of D^dag D for (chi, xi) is D^dag^{-1} followed by D^{-1},
    i.e. two; ``Dinv`` and ``Ddaginv`` count one each."""

    def __init__(self, tol: float = 1e-12, maxit: int = 100000):
        self.tol = tol
        self.maxit = maxit
        self.inversions = 0
        self.inversions_by_m0 = {}  # the same count split by the operator's bare mass
        self.cg_calls = 0
        self.cg_iterations = 0

    def _count(self, lat, k):
        self.inversions += k
        self.inversions_by_m0[lat.m0] = self.inversions_by_m0.get(lat.m0, 0) + k

    def cg(self, lat: Lattice, U: np.ndarray, b: np.ndarray) -> np.ndarray:
        self.cg_calls += 1
        x = np.zeros_like(b)
        r = b.copy()
        bb = np.vdot(b, b).real
        if bb == 0.0:
            return x
        p = r.copy()
        rr = bb
        for k in range(1, self.maxit + 1):
            Ap = apply_DdagD(lat, U, p)
            alpha = rr / np.vdot(p, Ap).real
            x = x + alpha * p
            r = r - alpha * Ap
            rr_new = np.vdot(r, r).real
            if np.sqrt(rr_new / bb) <= self.tol:
                self.cg_iterations += k
                return x
            p = r + (rr_new / rr) * p
            rr = rr_new
        raise RuntimeError(f"CG did not converge in {self.maxit} iterations")

    def DdagD_inv(self, lat, U, b):
        """(D^dag D)^{-1} b: counted as D^dag^{-1} then D^{-1}."""
        self._count(lat, 2)
        return self.cg(lat, U, b)

    def Dinv(self, lat, U, y):
        """D^{-1} y = (D^dag D)^{-1} D^dag y."""
        self._count(lat, 1)
        return self.cg(lat, U, apply_D(lat, U, y, dagger=True))

    def Ddaginv(self, lat, U, y):
        """D^dag^{-1} y = D (D^dag D)^{-1} y."""
        self._count(lat, 1)
        return apply_D(lat, U, self.cg(lat, U, y))


# ------------------------------------------------------------ gauge part ---

def link_at(U: np.ndarray, mu: int, dx: int, dt: int) -> np.ndarray:
    """U_mu(n + dx x_hat + dt t_hat) (periodic)."""
    return np.roll(np.roll(U[..., mu], -dx, axis=1), -dt, axis=0)


def plaquette(U: np.ndarray) -> np.ndarray:
    """P(n) = U_1(n) U_2(n+1) U_1^dag(n+2) U_2^dag(n) (Sec. 3)."""
    return (link_at(U, 0, 0, 0) * link_at(U, 1, 1, 0)
            * np.conj(link_at(U, 0, 0, 1)) * np.conj(link_at(U, 1, 0, 0)))


def gauge_action(lat: Lattice, U: np.ndarray) -> float:
    """S_G = beta sum_n (1 - Re P(n)) (Eq. gauge_action)."""
    return float(lat.beta * np.sum(1.0 - plaquette(U).real))


def oriented_plaquettes(U: np.ndarray, mu: int) -> list:
    """The plaquettes P_1 ... P_8 (n, mu) of the C_GG formula (Sec. 3.1),
    nu != mu, each written exactly as printed.  Index 0 is P_1."""
    nu = 1 - mu

    def u(d, a, b):
        # U_d(n + a mu_hat + b nu_hat)
        off = [0, 0]
        off[mu] += a
        off[nu] += b
        return link_at(U, d, off[0], off[1])

    c = np.conj
    return [
        u(mu, 0, 0) * u(nu, 1, 0) * c(u(mu, 0, 1)) * c(u(nu, 0, 0)),      # P1
        u(mu, 0, -1) * u(nu, 1, -1) * c(u(mu, 0, 0)) * c(u(nu, 0, -1)),   # P2
        u(mu, 1, 0) * u(nu, 2, 0) * c(u(mu, 1, 1)) * c(u(nu, 1, 0)),      # P3
        u(mu, 0, 1) * u(nu, 1, 1) * c(u(mu, 0, 2)) * c(u(nu, 0, 1)),      # P4
        u(mu, -1, 0) * u(nu, 0, 0) * c(u(mu, -1, 1)) * c(u(nu, -1, 0)),   # P5
        u(mu, -1, -1) * u(nu, 0, -1) * c(u(mu, -1, 0)) * c(u(nu, -1, -1)),  # P6
        u(mu, 0, -2) * u(nu, 1, -2) * c(u(mu, 0, -1)) * c(u(nu, 0, -2)),  # P7
        u(mu, 1, -1) * u(nu, 2, -1) * c(u(mu, 1, 0)) * c(u(nu, 1, -1)),   # P8
    ]


def gauge_force(lat: Lattice, U: np.ndarray) -> np.ndarray:
    """beta g(n, mu) = dS_G/dq_mu(n) = beta Im(P(n) - P(n - nu)) (Eq.
    force_gauge), read with the mu-oriented plaquettes P_1(n, mu) and
    P_2(n, mu) of Sec. 3.1 in place of P(n) and P(n - nu)."""
    F = np.empty(U.shape, dtype=np.float64)
    for mu in (0, 1):
        P = oriented_plaquettes(U, mu)
        F[..., mu] = lat.beta * np.imag(P[0] - P[1])
    return F


def c_gg(lat: Lattice, U: np.ndarray) -> np.ndarray:
    """C_GG(n, mu) (Eq. force_grad_de, closed form of Sec. 3.1):
    2 beta^2 [ Im(4P1 - P2 - P3 - P4 - P5) Re P1
               - Im(4P2 - P1 - P6 - P7 - P8) Re P2 ]."""
    C = np.empty(U.shape, dtype=np.float64)
    for mu in (0, 1):
        P = oriented_plaquettes(U, mu)
        C[..., mu] = 2.0 * lat.beta ** 2 * (
            np.imag(4 * P[0] - P[1] - P[2] - P[3] - P[4]) * P[0].real
            - np.imag(4 * P[1] - P[0] - P[5] - P[6] - P[7]) * P[1].real)
    return C


def c_fg(lat: Lattice, U: np.ndarray, v: np.ndarray) -> np.ndarray:
    """C_FG(n, mu) (closed form of Sec. 3.1) with the fermion force f
    replaced by an arbitrary link field v:

      2 beta [ (v(n,mu) + v(n+mu,nu) - v(n+nu,mu) - v(n,nu)) Re P1
             + (v(n,mu) - v(n+mu-nu,nu) - v(n-nu,mu) + v(n-nu,nu)) Re P2 ].

    With v = f it is C_FG; it equals 2 (Hess S_G) v for any v."""
    C = np.empty(U.shape, dtype=np.float64)
    for mu in (0, 1):
        nu = 1 - mu
        P = oriented_plaquettes(U, mu)

        def vv(d, a, b):
            off = [0, 0]
            off[mu] += a
            off[nu] += b
            return np.roll(np.roll(v[..., d], -off[0], axis=1), -off[1], axis=0)

        C[..., mu] = 2.0 * lat.beta * (
            (vv(mu, 0, 0) + vv(nu, 1, 0) - vv(mu, 0, 1) - vv(nu, 0, 0)) * P[0].real
            + (vv(mu, 0, 0) - vv(nu, 1, -1) - vv(mu, 0, -1) + vv(nu, 0, -1)) * P[1].real)
    return C


# ---------------------------------------------------------- fermion part ---

def chi_xi(lat: Lattice, U: np.ndarray, phi: np.ndarray, solver: Solver):
    """chi = D^dag^{-1} phi and xi = D^{-1} D^dag^{-1} phi (Eq.
    chi_xi_vectors), computed as xi = (D^dag D)^{-1} phi, chi = D xi."""
    xi = solver.DdagD_inv(lat, U, phi)
    chi = apply_D(lat, U, xi)
    return chi, xi


def fermion_action(lat: Lattice, U: np.ndarray, phi: np.ndarray, solver: Solver) -> float:
    """S_F = phi^dag (D^dag D)^{-1} phi (Eq. fer_action; the paper's
    pseudofermion field is called phi here)."""
    xi = solver.DdagD_inv(lat, U, phi)
    return float(np.vdot(phi, xi).real)


def fermion_force_from(lat: Lattice, U: np.ndarray, chi: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """f(n, mu) = -Im[ chi^dag(n) (1 - sigma_mu) U_mu(n) xi(n + mu)
                     - chi^dag(n + mu) (1 + sigma_mu) U_mu^dag(n) xi(n) ]
    (Eq. force_fermion)."""
    f = np.empty(U.shape, dtype=np.float64)
    for mu in (0, 1):
        xi_f = psi_shift(xi, mu, +1, lat.bc)
        chi_f = psi_shift(chi, mu, +1, lat.bc)
        a = U[..., mu] * np.sum(np.conj(chi) * _pm(I2 - SIGMA[mu], xi_f), axis=-1)
        b = np.conj(U[..., mu]) * np.sum(np.conj(chi_f) * _pm(I2 + SIGMA[mu], xi), axis=-1)
        f[..., mu] = -np.imag(a - b)
    return f


def fermion_force(lat: Lattice, U: np.ndarray, phi: np.ndarray, solver: Solver) -> np.ndarray:
    """f = dS_F/dq (Eq. force_fermion with Eq. chi_xi_vectors)."""
    chi, xi = chi_xi(lat, U, phi, solver)
    return fermion_force_from(lat, U, chi, xi)


def _w_sources(lat, U, chi, xi, v):
    """sum_{m,nu} w_{1,m,nu} v(m,nu) and sum_{m,nu} w_{2,m,nu} v(m,nu), with
    w_1 = (dD^dag/dq_nu(m)) chi and w_2 = (dD/dq_nu(m)) xi as printed in
    Sec. 3.1: each w has one term at site m and one at site m + nu."""
    s1 = np.zeros_like(chi)
    s2 = np.zeros_like(xi)
    for nu in (0, 1):
        Un = U[..., nu, None]
        vn = v[..., nu, None]
        # w_1: delta_{n,m+nu} (i/2)(1-sigma) U^dag chi(m) - delta_{n,m} (i/2)(1+sigma) U chi(m+nu)
        s1 = s1 + psi_shift(0.5j * vn * np.conj(Un) * _pm(I2 - SIGMA[nu], chi), nu, -1, lat.bc)
        s1 = s1 - 0.5j * vn * Un * _pm(I2 + SIGMA[nu], psi_shift(chi, nu, +1, lat.bc))
        # w_2: -delta_{n,m} (i/2)(1-sigma) U xi(m+nu) + delta_{n,m+nu} (i/2)(1+sigma) U^dag xi(m)
        s2 = s2 - 0.5j * vn * Un * _pm(I2 - SIGMA[nu], psi_shift(xi, nu, +1, lat.bc))
        s2 = s2 + psi_shift(0.5j * vn * np.conj(Un) * _pm(I2 + SIGMA[nu], xi), nu, -1, lat.bc)
    return s1, s2


def z_vectors(lat, U, chi, xi, v, solver):
    """Z_1 = D^dag^{-1} sum w_1 v,  Z_2 = D^{-1}(sum w_2 v + Z_1) (Eq. Z12
    with f replaced by v)."""
    s1, s2 = _w_sources(lat, U, chi, xi, v)
    Z1 = solver.Ddaginv(lat, U, s1)
    Z2 = solver.Dinv(lat, U, s2 + Z1)
    return Z1, Z2


def c_fermion(lat: Lattice, U: np.ndarray, chi: np.ndarray, xi: np.ndarray,
              v: np.ndarray, solver: Solver) -> np.ndarray:
    """C(n, mu) = 4 Re[ Z_1^dag w_{2,n,mu} + w_{1,n,mu}^dag Z_2
                        - chi^dag d^2D/dq_mu(n)^2 xi . v(n, mu) ]
    (Eq. CFF with Eq. Z12).  v = f gives C_FF; v = beta g gives C_GF."""
    Z1, Z2 = z_vectors(lat, U, chi, xi, v, solver)
    C = np.empty(U.shape, dtype=np.float64)
    for mu in (0, 1):
        Um = U[..., mu, None]
        xi_f = psi_shift(xi, mu, +1, lat.bc)
        chi_f = psi_shift(chi, mu, +1, lat.bc)
        Z1_f = psi_shift(Z1, mu, +1, lat.bc)
        Z2_f = psi_shift(Z2, mu, +1, lat.bc)
        # w_{2,n,mu}: -(i/2)(1-s) U xi(n+mu) at n ; (i/2)(1+s) U^dag xi(n) at n+mu
        w2_n = -0.5j * Um * _pm(I2 - SIGMA[mu], xi_f)
        w2_np = 0.5j * np.conj(Um) * _pm(I2 + SIGMA[mu], xi)
        # w_{1,n,mu}: -(i/2)(1+s) U chi(n+mu) at n ; (i/2)(1-s) U^dag chi(n) at n+mu
        w1_n = -0.5j * Um * _pm(I2 + SIGMA[mu], chi_f)
        w1_np = 0.5j * np.conj(Um) * _pm(I2 - SIGMA[mu], chi)
        z1w2 = np.sum(np.conj(Z1) * w2_n + np.conj(Z1_f) * w2_np, axis=-1)
        w1z2 = np.sum(np.conj(w1_n) * Z2 + np.conj(w1_np) * Z2_f, axis=-1)
        # d^2 D / dq_mu(n)^2 = +1/2 (1-s) U at (n, n+mu) and +1/2 (1+s) U^dag at (n+mu, n)
        d2 = (0.5 * np.sum(np.conj(chi) * Um * _pm(I2 - SIGMA[mu], xi_f), axis=-1)
              + 0.5 * np.sum(np.conj(chi_f) * np.conj(Um) * _pm(I2 + SIGMA[mu], xi), axis=-1))
        C[..., mu] = 4.0 * np.real(z1w2 + w1z2 - d2 * v[..., mu])
    return C


def force(lat: Lattice, U: np.ndarray, phi: np.ndarray, solver: Solver, part: str = "full") -> np.ndarray:
    """F = dS_G/dq + dS_F/dq (Eq. force); ``part`` selects 'gauge',
    'fermion' or 'full'."""
    if part == "gauge":
        return gauge_force(lat, U)
    if part == "fermion":
        return fermion_force(lat, U, phi, solver)
    return gauge_force(lat, U) + fermion_force(lat, U, phi, solver)


def force_and_gradient(lat: Lattice, U: np.ndarray, phi: np.ndarray, solver: Solver,
                       part: str = "full"):
    """The force F (Eq. force) and the force-gradient term C (Eq.
    force_gradient) as the sum of the parts of Eq. force_grad_de:
    'gauge' -> C_GG, 'fermion' -> C_FF, 'full' -> C_GG + C_FG + C_GF + C_FF.
    chi and xi are computed once and shared by f and the C parts."""
    if part == "gauge":
        return gauge_force(lat, U), c_gg(lat, U)
    chi, xi = chi_xi(lat, U, phi, solver)
    f = fermion_force_from(lat, U, chi, xi)
    if part == "fermion":
        return f, c_fermion(lat, U, chi, xi, f, solver)
    bg = gauge_force(lat, U)
    C = (c_gg(lat, U) + c_fg(lat, U, f) + c_fermion(lat, U, chi, xi, bg, solver)
         + c_fermion(lat, U, chi, xi, f, solver))
    return bg + f, C


def force_gradient(lat: Lattice, U: np.ndarray, phi: np.ndarray, solver: Solver,
                   part: str = "full") -> np.ndarray:
    """C = grad |F|^2 alone (Eq. force_gradient; see ``force_and_gradient``)."""
    return force_and_gradient(lat, U, phi, solver, part)[1]


def shifted_force(lat: Lattice, q: np.ndarray, phi: np.ndarray, solver: Solver,
                  h: float, part: str = "full") -> np.ndarray:
    """Force at the shifted field q - (h^2/24) F(q): its Taylor expansion
    is F - (h^2/48) C + O(h^4), the force-gradient kick of Eq. 5stage_fg
    with C approximated as proposed by Yin and Mawhinney (Sec. 2)."""
    F0 = force(lat, links(q), phi, solver, part)
    return force(lat, links(q - (h * h / 24.0) * F0), phi, solver, part)


# ------------------------------------- determinant split over two masses ---
#
# The paper's outlook (Conclusions) partitions the action into more than two
# parts by factorising the fermion determinant, so that the most expensive
# part needs the force-gradient information and the cheaper, faster parts
# only leapfrog steps.  The factorisation used is the mass split of
# Hasenbusch (Phys. Lett. B 519 (2001) 177): with D_h the Wilson-Dirac
# operator at the heavier bare mass m0 + dm,
#   det(D^dag D) = det(D_h^dag D_h) * det(W^dag W),  W = D D_h^{-1},
# each factor represented by a pseudofermion:
#   S_h = phi_h^dag (D_h^dag D_h)^{-1} phi_h      (heavy part)
#   S_r = phi_r^dag (W^dag W)^{-1} phi_r = psi^dag (D^dag D)^{-1} psi,
#         psi = D_h^dag phi_r                        (ratio part, the light one).

def heavy_lattice(lat: Lattice, dm: float) -> Lattice:
    """The same lattice and couplings with the bare mass m0 + dm (D_h)."""
    return Lattice(lat.L, lat.T, lat.beta, lat.m0 + dm, lat.bc)


def ratio_vectors(lat: Lattice, lat_h: Lattice, U: np.ndarray, phi_r: np.ndarray,
                  solver: Solver):
    """psi = D_h^dag phi_r, X = (D^dag D)^{-1} psi and a = D X - phi_r."""
    psi = apply_D(lat_h, U, phi_r, dagger=True)
    X = solver.DdagD_inv(lat, U, psi)
    a = apply_D(lat, U, X) - phi_r
    return psi, X, a


def ratio_action(lat: Lattice, lat_h: Lattice, U: np.ndarray, phi_r: np.ndarray,
                 solver: Solver) -> float:
    """S_r = phi_r^dag D_h (D^dag D)^{-1} D_h^dag phi_r."""
    psi = apply_D(lat_h, U, phi_r, dagger=True)
    X = solver.DdagD_inv(lat, U, psi)
    return float(np.vdot(psi, X).real)


def ratio_force(lat: Lattice, lat_h: Lattice, U: np.ndarray, phi_r: np.ndarray,
                solver: Solver) -> np.ndarray:
    """dS_r/dq.  The hopping terms of D and D_h are the same, so with
    dD = dD/dq_mu(n):  dS_r = 2 Re[phi_r^dag dD X] - 2 Re[(D X)^dag dD X]
    = -2 Re[a^dag dD X]: the bilinear of Eq. force_fermion with chi -> a,
    xi -> X."""
    _, X, a = ratio_vectors(lat, lat_h, U, phi_r, solver)
    return fermion_force_from(lat, U, a, X)


def ratio_force_and_gradient(lat: Lattice, lat_h: Lattice, U: np.ndarray, phi_r: np.ndarray,
                             solver: Solver):
    """F_r and C_r = grad |F_r|^2 = 2 (Hess S_r) F_r.  Along a direction v,
    dX = -(D^dag D)^{-1}(s_1 + D^dag s_2) and da = dD X + D dX with
    s_1 = (dD_v)^dag a, s_2 = (dD_v) X: the vectors Z_1, Z_2 of Eq. Z12 with
    (chi, xi) -> (a, X), so C_r is Eq. CFF with the same substitution."""
    _, X, a = ratio_vectors(lat, lat_h, U, phi_r, solver)
    F = fermion_force_from(lat, U, a, X)
    return F, c_fermion(lat, U, a, X, F, solver)


def heatbath_split(lat: Lattice, lat_h: Lattice, U: np.ndarray, eta_r: np.ndarray,
                   eta_h: np.ndarray, solver: Solver):
    """The two pseudofermions from Gaussian noise: phi_h = D_h^dag eta_h and
    phi_r = W^dag eta_r = D_h^dag^{-1} D^dag eta_r, so that S_h = eta_h^dag
    eta_h and S_r = eta_r^dag eta_r at the start."""
    phi_h = apply_D(lat_h, U, eta_h, dagger=True)
    phi_r = solver.Ddaginv(lat_h, U, apply_D(lat, U, eta_r, dagger=True))
    return phi_r, phi_h


def kinetic(p: np.ndarray) -> float:
    """1/2 sum p^2 (Eq. schwinger)."""
    return float(0.5 * np.sum(p * p))


def hamiltonian(lat: Lattice, q: np.ndarray, p: np.ndarray, phi: np.ndarray, solver: Solver) -> float:
    """H = 1/2 sum p^2 + S_G + S_F (Eq. schwinger)."""
    U = links(q)
    return kinetic(p) + gauge_action(lat, U) + fermion_action(lat, U, phi, solver)


def hamiltonian_split(lat: Lattice, lat_h: Lattice, q: np.ndarray, p: np.ndarray,
                      phi_r: np.ndarray, phi_h: np.ndarray, solver: Solver) -> float:
    """H = 1/2 sum p^2 + S_G + S_h + S_r with the determinant split over two
    masses."""
    U = links(q)
    return (kinetic(p) + gauge_action(lat, U) + fermion_action(lat_h, U, phi_h, solver)
            + ratio_action(lat, lat_h, U, phi_r, solver))
