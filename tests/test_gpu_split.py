"""The fermion determinant split over two masses (heavy part S_h, ratio part
S_r) and the three-level schemes on the GPU, through the C ABI, against the
oracle on ragged batches of seeded inputs: the forces of both parts, the
exact force-gradient term and the shifted force of the ratio part, the MD
trajectory of both three-level schemes, the HMC update (Delta H, decisions)
in both CG layouts, the inversion counts per step, and the trajectory
captured as a CUDA graph against the eager one.  Tolerances as in
test_gpu_parity: 1e-12 relative on FP64 forces and Delta H (CG tolerance
1e-14)."""
import numpy as np
import pytest

from oracle import integrators as ig
from oracle import schwinger as sw
from tests.gpu_util import Batch, rel_err

pytestmark = pytest.mark.gpu

DIMS = [(8, 8), (3, 5), (2, 2), (16, 8), (17, 9)]
DM = 0.3
TOL64 = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    P.build()
    return t


def split_batch(dims=DIMS, seed=0):
    n = len(dims)
    b = Batch(dims, np.resize([2.0, 1.0, 4.0, 2.0, 1.5], n), np.resize([0.24, 0.2, 0.22, 0.25, 0.21], n),
              seed=seed)
    b.lat.set_heavy(DM)
    b.olat_h = [sw.heavy_lattice(ol, DM) for ol in b.olat]
    return b


def cg(tol=1e-14, prec="f64", algo="auto"):
    import paper_1512_03812_gb300 as P
    return P.CG(tol=tol, maxit=50000, prec=prec, algo=algo, delta=0.01)


def test_heavy_and_ratio_forces(torch):
    b = split_batch()
    q, phi_r, phi_h = b.q(), b.spinor(7), b.spinor(8)
    qd = b.dev(q)
    Fh = b.lat.force(qd, b.dev(phi_h), "heavy", cg())
    Fr = b.lat.force(qd, b.dev(phi_r), "ratio", cg())
    for c in range(len(b.dims)):
        U = sw.links(b.chain(q, c))
        s = sw.Solver(1e-14)
        assert rel_err(b.chain(Fh, c), sw.fermion_force(b.olat_h[c], U, b.chain(phi_h, c), s)) < TOL64
        assert rel_err(b.chain(Fr, c), sw.ratio_force(b.olat[c], b.olat_h[c], U,
                                                       b.chain(phi_r, c), s)) < TOL64


def test_ratio_force_gradient_and_shifted_force(torch):
    b = split_batch(seed=1)
    q, phi_r = b.q(), b.spinor(9)
    qd = b.dev(q)
    F = torch.empty_like(qd)
    C = b.lat.force_gradient(qd, b.dev(phi_r), "ratio", cg(), F=F)
    Fs = b.lat.fg_shifted_force(qd, b.dev(phi_r), 0.2, "ratio", cg())
    for c in range(len(b.dims)):
        U = sw.links(b.chain(q, c))
        s = sw.Solver(1e-14)
        Fo, Co = sw.ratio_force_and_gradient(b.olat[c], b.olat_h[c], U, b.chain(phi_r, c), s)
        assert rel_err(b.chain(F, c), Fo) < TOL64
        assert rel_err(b.chain(C, c), Co) < 1e-11
        qs = b.chain(q, c) - (0.2 * 0.2 / 24.0) * Fo
        Fso = sw.ratio_force(b.olat[c], b.olat_h[c], sw.links(qs), b.chain(phi_r, c), s)
        assert rel_err(b.chain(Fs, c), Fso) < TOL64


def test_heavy_part_has_no_force_gradient_and_parts_need_the_split(torch):
    import paper_1512_03812_gb300 as P
    b = split_batch(dims=[(4, 4)])
    qd = b.dev(b.q())
    with pytest.raises(P.SchwingerError):
        b.lat.force_gradient(qd, b.dev(b.spinor(1)), "heavy", cg())
    plain = Batch([(4, 4)], 2.0, 0.24)
    with pytest.raises(P.SchwingerError):
        plain.lat.force(b.dev(plain.q()), b.dev(plain.spinor(1)), "ratio", cg())


SCHEMES3 = [("nested3_leapfrog", "exact"), ("adapted_nested3_fg", "exact"),
            ("adapted_nested3_fg", "shifted")]


@pytest.mark.parametrize("scheme,fg", SCHEMES3)
@pytest.mark.parametrize("merge", [True, False])
def test_three_level_md_trajectory(torch, scheme, fg, merge):
    import paper_1512_03812_gb300 as P
    b = split_batch(seed=2)
    q, p, phi_r, phi_h = b.q(), b.p(), b.spinor(10), b.spinor(11)
    qd, pd = b.dev(q), b.dev(p)
    phi = torch.cat([b.dev(phi_r), b.dev(phi_h)])
    md = P.MD(scheme=scheme, tau=0.6, n=3, M=2, M2=2, fg=fg, merge_kicks=merge, cg=cg())
    b.lat.md_trajectory(qd, pd, phi, md)
    for c in range(len(b.dims)):
        st = ig.State(b.olat[c], b.chain(q, c).copy(), b.chain(p, c).copy(), b.chain(phi_r, c),
                      sw.Solver(1e-14), b.olat_h[c], b.chain(phi_h, c))
        ig.md_trajectory(st, scheme, 0.6, 3, M=2, fg=fg, M2=2)
        assert rel_err(b.chain(qd, c), st.q) < TOL64
        assert rel_err(b.chain(pd, c), st.p) < 1e-11


@pytest.mark.parametrize("scheme,fg", SCHEMES3)
@pytest.mark.parametrize("algo", ["grid", "chain"])
def test_three_level_hmc_parity(torch, scheme, fg, algo):
    import paper_1512_03812_gb300 as P
    b = split_batch(seed=3)
    q, p = b.q(), b.p()
    eta_r, eta_h = b.eta(12), b.eta(13)
    eta = torch.cat([b.dev(eta_r), b.dev(eta_h)])
    us = np.linspace(0.05, 0.95, len(b.dims))
    md = P.MD(scheme=scheme, tau=0.8, n=4, M=2, M2=2, fg=fg, cg=cg(algo=algo))
    q_md = torch.empty_like(b.dev(q))
    dH, H0, acc = b.lat.hmc_trajectory(b.dev(q), b.dev(p), eta, us, md, q_md=q_md)
    for c in range(len(b.dims)):
        r = ig.hmc_trajectory(b.olat[c], b.chain(q, c), b.chain(p, c),
                              np.stack([b.chain(eta_r, c), b.chain(eta_h, c)]), us[c], scheme,
                              0.8, 4, M=2, fg=fg, solver=sw.Solver(1e-14), dm=DM, M2=2)
        assert abs(dH[c] - r.dH) <= 1e-12 * max(1.0, abs(r.H0)), (c, dH[c], r.dH)
        assert abs(H0[c] - r.H0) <= 1e-12 * abs(r.H0)
        assert bool(acc[c]) == r.accepted
        assert rel_err(b.chain(q_md, c), r.q_md) < TOL64


def test_three_level_hmc_mixed_precision(torch):
    """The mixed CG (FP32 iterations, FP64 reliable updates to 1e-12) in every
    solve of the split action: Delta H within 1e-8 of the oracle's FP64 and
    the same decisions."""
    import paper_1512_03812_gb300 as P
    b = split_batch(dims=[(16, 16), (32, 32), (8, 8)], seed=4)
    q, p = b.q(), b.p()
    eta_r, eta_h = b.eta(14), b.eta(15)
    eta = torch.cat([b.dev(eta_r), b.dev(eta_h)])
    us = np.array([0.2, 0.5, 0.8])
    md = P.MD(scheme="adapted_nested3_fg", tau=0.5, n=2, M=2, M2=2,
              cg=cg(tol=1e-12, prec="mixed"), tol_action=1e-12)
    dH, _, acc = b.lat.hmc_trajectory(b.dev(q), b.dev(p), eta, us, md)
    for c in range(len(b.dims)):
        r = ig.hmc_trajectory(b.olat[c], b.chain(q, c), b.chain(p, c),
                              np.stack([b.chain(eta_r, c), b.chain(eta_h, c)]), us[c],
                              "adapted_nested3_fg", 0.5, 2, M=2, solver=sw.Solver(1e-14),
                              dm=DM, M2=2)
        assert abs(dH[c] - r.dH) < 1e-8, (c, dH[c], r.dH)
        assert bool(acc[c]) == r.accepted


@pytest.mark.parametrize("scheme,fg", SCHEMES3)
def test_three_level_inversions_per_step(torch, scheme, fg):
    """Every kick evaluated (no merging): the oracle's count of inversions
    (light and heavy) per step."""
    import paper_1512_03812_gb300 as P
    b = split_batch(dims=[(4, 4)], seed=5)
    q, p = b.q(), b.p()
    phi = torch.cat([b.dev(b.spinor(1)), b.dev(b.spinor(2))])
    for M2 in (1, 3):
        md = P.MD(scheme=scheme, tau=1.0, n=1, M=2, M2=M2, fg=fg, merge_kicks=False,
                  cg=cg(1e-8))
        b.lat.md_step(b.dev(q), b.dev(p), phi, md, 0.1)
        st = ig.State(b.olat[0], b.chain(q, 0).copy(), b.chain(p, 0).copy(),
                      b.chain(b.spinor(1), 0), sw.Solver(1e-8), b.olat_h[0],
                      b.chain(b.spinor(2), 0))
        ig.SCHEMES[scheme](st, 0.1, M=2, M2=M2, fg=fg)
        assert b.lat.stats.inversions == st.solver.inversions, (M2, b.lat.stats.as_dict())


def test_three_level_graph_equals_eager_twice(torch):
    import paper_1512_03812_gb300 as P
    b = split_batch(dims=[(16, 16), (32, 32), (16, 16)], seed=6)
    md = P.MD(scheme="adapted_nested3_fg", tau=0.5, n=2, M=2, M2=2,
              cg=cg(tol=1e-10, prec="mixed"), tol_action=1e-12)
    q0 = b.q()
    ps = [b.p(20 + k) for k in range(2)]
    es = [torch.cat([b.dev(b.eta(30 + k)), b.dev(b.eta(40 + k))]) for k in range(2)]
    us = [np.array([0.3, 0.6, 0.9]), np.array([0.8, 0.1, 0.5])]
    qe = b.dev(q0)
    eager = [b.lat.hmc_trajectory(qe, b.dev(ps[k]), es[k], us[k], md, check=False)
             for k in range(2)]
    qg = b.dev(q0)
    p0 = torch.empty_like(b.dev(ps[0]))
    eta = torch.empty_like(es[0])
    g = b.lat.hmc_graph(qg, p0, eta, md)
    for k in range(2):
        p0.copy_(b.dev(ps[k]))
        eta.copy_(es[k])
        dH, H0, acc = g.run(us[k])
        assert np.array_equal(dH, eager[k][0]), (dH, eager[k][0])
        assert np.array_equal(acc, eager[k][2])
    torch.cuda.synchronize()
    assert torch.equal(qg, qe)
