"""MD schedules and the HMC trajectory (Sec. 2 of arXiv:1512.03812).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Every schedule is
written as the literal composition printed in the paper, with no merging of
consecutive kicks, so that the inversion counter reproduces the paper's
"D^{-1} per step" (Sec. 3, end).

Primitives (Sec. 2.1, the discrete updates e^{hA} and e^{hB}):
  drift  e^{eps A}: U -> exp(i eps P) U, i.e. q <- q + eps p
  kick   e^{eps B}: P -> P - eps F; for U(1) the momenta are real and the
         factor i of the Lie-algebra notation is dropped: p <- p - eps F
  fg     e^{(2/3) h B + h^3/72 C}: p <- p - (2h/3) F + (h^3/72) C, with
         C = grad |F|^2 of Eq. force_gradient.  This is the sign that gives
         fourth order (the paper prints both signs, Eq. 5stage_fg versus
         Eq. 5stage_multi_fg).  ``fg='shifted'`` replaces F and C by the
         force at the shifted field q - (h^2/24) F(q).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import schwinger as sw


@dataclass
class State:
    """The phase-space point (q, p) of one chain with its pseudofermion phi
    (fixed during a trajectory, Sec. 2.1).  With the fermion determinant
    split over two masses (the three-level schemes below), phi is the ratio
    pseudofermion phi_r, phi_h the heavy one and lat_h the lattice at the
    heavy mass."""
    lat: sw.Lattice
    q: np.ndarray
    p: np.ndarray
    phi: np.ndarray
    solver: sw.Solver
    lat_h: sw.Lattice | None = None
    phi_h: np.ndarray | None = None


def part_force(st: State, U: np.ndarray, part: str) -> np.ndarray:
    """The force of one part of the action: 'gauge', 'fermion' (one
    pseudofermion), 'full' (their sum), 'heavy' (S_h) or 'ratio' (S_r)."""
    if part == "heavy":
        return sw.fermion_force(st.lat_h, U, st.phi_h, st.solver)
    if part == "ratio":
        return sw.ratio_force(st.lat, st.lat_h, U, st.phi, st.solver)
    return sw.force(st.lat, U, st.phi, st.solver, part)


def drift(st: State, eps: float) -> None:
    """The link update e^{eps A}: q <- q + eps p (Sec. 2.1, U <- e^{i eps P} U
    for U(1) link angles; the momentum update printed there as P - i h F is
    read for the U(1) algebra element P = i p with p real, which gives the
    real kick p <- p - h F with F = dS/dq of Eq. force)."""
    st.q = st.q + eps * st.p


def kick(st: State, eps: float, part: str) -> None:
    """The momentum update e^{eps B}: p <- p - eps F(q) of one part of the
    action (Sec. 2.1; F = dS/dq, Eq. force)."""
    st.p = st.p - eps * part_force(st, sw.links(st.q), part)


def fg_kick(st: State, h: float, part: str, fg: str) -> None:
    """The force-gradient kick e^{(2/3) h B + (1/72) h^3 C} for step h, the
    middle kick of Eq. 5stage_fg; fg = "shifted"
    takes the force at the shifted field instead (Sec. 2, after Eq.
    5stage_fg).  The sign of the C term: Eq. 5stage_fg prints it negative,
    Eq. 5stage_multi_fg and Eq. ad_5stage_multi_fg positive; with C = grad |F|^2
    of Eq. force_gradient and the kick p <- p - eps F of Sec. 2.1 the
    composition is of fourth order only with the positive sign used here
    (Sec. 2.1, the force-gradient step of Eq. 5stage_fg)."""
    if fg == "exact":
        if part == "ratio":
            F, C = sw.ratio_force_and_gradient(st.lat, st.lat_h, sw.links(st.q), st.phi,
                                               st.solver)
        else:
            F, C = sw.force_and_gradient(st.lat, sw.links(st.q), st.phi, st.solver, part)
        st.p = st.p - (2.0 * h / 3.0) * F + (h ** 3 / 72.0) * C
    elif fg == "shifted":
        if part == "ratio":
            F0 = part_force(st, sw.links(st.q), part)
            Fs = part_force(st, sw.links(st.q - (h * h / 24.0) * F0), part)
        else:
            Fs = sw.shifted_force(st.lat, st.q, st.phi, st.solver, h, part)
        st.p = st.p - (2.0 * h / 3.0) * Fs
    else:
        raise ValueError(fg)


# ----------------------------------------------------------- basic schemes --

def leapfrog(st: State, h: float, **_) -> None:
    """Delta(h) = e^{hB/2} e^{hA} e^{hB/2} (Eq. leap)."""
    kick(st, h / 2, "full")
    drift(st, h)
    kick(st, h / 2, "full")


def five_stage(st: State, h: float, lam: float = 1.0 / 6.0, **_) -> None:
    """Delta_5(h) = e^{lam h B} e^{h A/2} e^{(1-2 lam) h B} e^{h A/2} e^{lam h B}
    (Eq. 5stage prints lam = 1/6)."""
    kick(st, lam * h, "full")
    drift(st, h / 2)
    kick(st, (1 - 2 * lam) * h, "full")
    drift(st, h / 2)
    kick(st, lam * h, "full")


def five_stage_fg(st: State, h: float, fg: str = "exact", **_) -> None:
    """Delta_5C(h) (Eq. 5stage_fg) with the full force gradient C, or its
    shifted-force approximation (Sec. 2, after Eq. 5stage_fg)."""
    kick(st, h / 6, "full")
    drift(st, h / 2)
    fg_kick(st, h, "full", fg)
    drift(st, h / 2)
    kick(st, h / 6, "full")


# The four weights of the 11-stage decomposition (Eq. 11_stage), which the
# paper takes from Eq. (71) of Omelyan, Mryglod and Folk (2003): sigma and
# lambda weight the force, eta and theta the drift.  They satisfy the two
# fourth-order conditions of the symmetric composition (the coefficients of
# [A,[A,B]] and [B,[B,A]] in log Delta_11 vanish; tests/test_oracle.py checks
# this with a truncated Baker-Campbell-Hausdorff expansion).
OMELYAN_11 = {"sigma": 0.08398315262876693, "eta": 0.2539785108410595,
              "lam": 0.6822365335719091, "theta": -0.03230286765269967}


def eleven_stage(st: State, h: float, **_) -> None:
    """Delta_11(h) (Eq. 11_stage): force weights sigma, lambda,
    (1 - 2 (lambda + sigma)) / 2 (twice), lambda, sigma; drift weights eta,
    theta, 1 - 2 (theta + eta), theta, eta, interleaved as printed."""
    w = OMELYAN_11
    sg, et, lm, th = w["sigma"], w["eta"], w["lam"], w["theta"]
    mid_b = (1 - 2 * (lm + sg)) / 2
    mid_a = 1 - 2 * (th + et)
    kick(st, sg * h, "full")
    drift(st, et * h)
    kick(st, lm * h, "full")
    drift(st, th * h)
    kick(st, mid_b * h, "full")
    drift(st, mid_a * h)
    kick(st, mid_b * h, "full")
    drift(st, th * h)
    kick(st, lm * h, "full")
    drift(st, et * h)
    kick(st, sg * h, "full")


# ---------------------------------------------------------- nested schemes --

def inner_leapfrog(st: State, h: float, M: int) -> None:
    """Delta_1(h)_M = (e^{h B1/2M} e^{h A/M} e^{h B1/2M})^M (Sec. 2, after
    Eq. leap_multi); B1 is the gauge action."""
    for _ in range(M):
        kick(st, h / (2 * M), "gauge")
        drift(st, h / M)
        kick(st, h / (2 * M), "gauge")


def inner_fg(st: State, h: float, M: int, fg: str) -> None:
    """Delta_2(h)_M: M five-stage force-gradient steps of size h/M on the
    gauge system, C_g = C_GG (Sec. 2, after Eq. 5stage_multi_fg)."""
    hm = h / M
    for _ in range(M):
        kick(st, hm / 6, "gauge")
        drift(st, hm / 2)
        fg_kick(st, hm, "gauge", fg)
        drift(st, hm / 2)
        kick(st, hm / 6, "gauge")


def nested_leapfrog(st: State, h: float, M: int = 1, **_) -> None:
    """hat Delta(h) = e^{h B2/2} Delta_1(h)_M e^{h B2/2} (Eq. leap_multi)."""
    kick(st, h / 2, "fermion")
    inner_leapfrog(st, h, M)
    kick(st, h / 2, "fermion")


def nested_five_stage(st: State, h: float, M: int = 1, lam: float = 1.0 / 6.0, **_) -> None:
    """hat Delta_5(h) (Eq. 5stage_multi), outer weights lam, 1-2 lam, lam."""
    kick(st, lam * h, "fermion")
    inner_leapfrog(st, h / 2, M)
    kick(st, (1 - 2 * lam) * h, "fermion")
    inner_leapfrog(st, h / 2, M)
    kick(st, lam * h, "fermion")


def nested_fg(st: State, h: float, M: int = 1, fg: str = "exact", **_) -> None:
    """hat Delta_5C(h) (Eq. 5stage_multi_fg): C_f = C_FF outside, the
    force-gradient inner scheme Delta_2 inside."""
    kick(st, h / 6, "fermion")
    inner_fg(st, h / 2, M, fg)
    fg_kick(st, h, "fermion", fg)
    inner_fg(st, h / 2, M, fg)
    kick(st, h / 6, "fermion")


def adapted_nested_fg(st: State, h: float, M: int = 1, fg: str = "exact", **_) -> None:
    """tilde Delta_5C(h) (Eq. ad_5stage_multi_fg): C_f = C_FF outside,
    plain leapfrog Delta_1 inside."""
    kick(st, h / 6, "fermion")
    inner_leapfrog(st, h / 2, M)
    fg_kick(st, h, "fermion", fg)
    inner_leapfrog(st, h / 2, M)
    kick(st, h / 6, "fermion")


# ------------------------------------------------------ three time scales --
#
# The paper's outlook (Conclusions): with the fermion determinant factorised,
# the action has more than two parts, and the adapted scheme keeps the
# force-gradient term only for the most expensive one, with leapfrog steps
# for the faster, cheaper parts.  Here H = A + B1 + B2 + B3 with B1 = S_G
# (fastest), B2 = S_h (the heavy pseudofermion) and B3 = S_r (the ratio
# part, the slowest and most expensive): the scheme of a level holds the
# level below in place of its drifts, as Eq. leap_multi and Eq.
# ad_5stage_multi_fg hold the gauge system.

def middle_leapfrog(st: State, h: float, M2: int, M: int) -> None:
    """Delta_2(h) = (e^{h B2/2M2} Delta_1(h/M2)_M e^{h B2/2M2})^{M2}: M2
    leapfrog steps on the heavy part, each with M gauge leapfrog steps
    inside."""
    for _ in range(M2):
        kick(st, h / (2 * M2), "heavy")
        inner_leapfrog(st, h / M2, M)
        kick(st, h / (2 * M2), "heavy")


def nested3_leapfrog(st: State, h: float, M: int = 1, M2: int = 1, **_) -> None:
    """e^{h B3/2} Delta_2(h) e^{h B3/2}: Eq. leap_multi on three levels."""
    kick(st, h / 2, "ratio")
    middle_leapfrog(st, h, M2, M)
    kick(st, h / 2, "ratio")


def adapted_nested3_fg(st: State, h: float, M: int = 1, M2: int = 1, fg: str = "exact",
                       **_) -> None:
    """Eq. ad_5stage_multi_fg with the ratio part outside and C_3 =
    {B3, {A, B3}} (the force gradient of S_r alone), the leapfrog levels
    Delta_2(h/2) of the heavy part and the gauge action inside."""
    kick(st, h / 6, "ratio")
    middle_leapfrog(st, h / 2, M2, M)
    fg_kick(st, h, "ratio", fg)
    middle_leapfrog(st, h / 2, M2, M)
    kick(st, h / 6, "ratio")


THREE_LEVEL = ("nested3_leapfrog", "adapted_nested3_fg")

SCHEMES = {
    "leapfrog": leapfrog,
    "five_stage": five_stage,
    "five_stage_fg": five_stage_fg,
    "nested_leapfrog": nested_leapfrog,
    "nested_five_stage": nested_five_stage,
    "nested_fg": nested_fg,
    "adapted_nested_fg": adapted_nested_fg,
    "eleven_stage": eleven_stage,
    "nested3_leapfrog": nested3_leapfrog,
    "adapted_nested3_fg": adapted_nested3_fg,
}

# Omelyan's second-order minimum-norm weight (Omelyan, Mryglod and Folk 2002),
# used for the "2MN" variant of the five-stage schemes.
LAMBDA_2MN = 0.1931833275037836


def md_trajectory(st: State, scheme: str, tau: float, n: int, M: int = 1,
                  lam: float = 1.0 / 6.0, fg: str = "exact", M2: int = 1) -> None:
    """n steps of size h = tau / n of one scheme of Sec. 2 (Eqs. leap,
    5stage, 5stage_fg, 11_stage, leap_multi, 5stage_multi, 5stage_multi_fg,
    ad_5stage_multi_fg) or of the three-level schemes (M2 heavy steps per
    middle block)."""
    h = tau / n
    step = SCHEMES[scheme]
    for _ in range(n):
        step(st, h, M=M, lam=lam, fg=fg, M2=M2)


@dataclass
class TrajectoryResult:
    q: np.ndarray          # links after the Metropolis step
    q_md: np.ndarray       # links at the end of the MD trajectory
    p_md: np.ndarray
    dH: float
    H0: float
    H1: float
    accepted: bool


def hmc_trajectory(lat: sw.Lattice, q0: np.ndarray, p0: np.ndarray, eta: np.ndarray,
                   u: float, scheme: str, tau: float, n: int, M: int = 1,
                   lam: float = 1.0 / 6.0, fg: str = "exact",
                   solver: sw.Solver | None = None, sf_start: str = "solve",
                   dm: float = 0.0, M2: int = 1) -> TrajectoryResult:
    """One HMC update (Sec. 2.1): pseudofermion heatbath phi = D^dag eta at
    the starting links, MD trajectory of length tau, Metropolis accept
    with probability min(1, e^{-Delta H}) decided as u < exp(-Delta H) for
    a supplied uniform u in [0, 1).  sf_start = "noise" takes S_F at the
    start as eta^dag eta, which phi^dag (D^dag D)^{-1} phi equals exactly
    for phi = D^dag eta, instead of solving for it.

    The three-level schemes use the determinant split over the masses m0
    and m0 + dm: eta is then the pair (eta_r, eta_h) stacked on a leading
    axis, the heatbath gives phi_r, phi_h (heatbath_split) and H holds
    S_h + S_r."""
    solver = solver or sw.Solver()
    if scheme in THREE_LEVEL:
        return _hmc_split(lat, q0, p0, eta, u, scheme, tau, n, M, lam, fg, solver, sf_start,
                          dm, M2)
    phi = sw.apply_D(lat, sw.links(q0), eta, dagger=True)
    if sf_start == "noise":
        U0 = sw.links(q0)
        H0 = sw.kinetic(p0) + sw.gauge_action(lat, U0) + float(np.vdot(eta, eta).real)
    else:
        H0 = sw.hamiltonian(lat, q0, p0, phi, solver)
    st = State(lat, q0.copy(), p0.copy(), phi, solver)
    md_trajectory(st, scheme, tau, n, M, lam, fg)
    H1 = sw.hamiltonian(lat, st.q, st.p, phi, solver)
    dH = H1 - H0
    accepted = bool(math.isfinite(dH) and (dH <= 0.0 or u < math.exp(-dH)))
    return TrajectoryResult(st.q if accepted else q0.copy(), st.q, st.p, dH, H0, H1, accepted)


def _hmc_split(lat, q0, p0, eta, u, scheme, tau, n, M, lam, fg, solver, sf_start, dm, M2):
    """hmc_trajectory with the determinant split over two masses."""
    lat_h = sw.heavy_lattice(lat, dm)
    U0 = sw.links(q0)
    eta_r, eta_h = eta[0], eta[1]
    phi_r, phi_h = sw.heatbath_split(lat, lat_h, U0, eta_r, eta_h, solver)
    if sf_start == "noise":
        H0 = (sw.kinetic(p0) + sw.gauge_action(lat, U0) + float(np.vdot(eta_r, eta_r).real)
              + float(np.vdot(eta_h, eta_h).real))
    else:
        H0 = sw.hamiltonian_split(lat, lat_h, q0, p0, phi_r, phi_h, solver)
    st = State(lat, q0.copy(), p0.copy(), phi_r, solver, lat_h, phi_h)
    md_trajectory(st, scheme, tau, n, M, lam, fg, M2)
    H1 = sw.hamiltonian_split(lat, lat_h, st.q, st.p, phi_r, phi_h, solver)
    dH = H1 - H0
    accepted = bool(math.isfinite(dH) and (dH <= 0.0 or u < math.exp(-dH)))
    return TrajectoryResult(st.q if accepted else q0.copy(), st.q, st.p, dH, H0, H1, accepted)
