"""Parity at the full sizes of the large-lattice and batched-chain
workloads: the 2048 x 2048 lattice (beta 8, kappa 0.255) for D, D^dag and the
fused D^dag D against the oracle over every site, the mixed-precision CG by
its FP64 true residual (a property that holds at any size), and a batch of
256 chains with sides from {16, 32, 48, 64, 128} (beta in {1, 2, 4}, kappa in
[0.20, 0.26]) against the oracle on sampled chains."""
import numpy as np
import pytest

from oracle import schwinger as sw
from paper_1512_03812_gb300 import inputs as I
from tests.gpu_util import Batch, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    P.build()
    return t


@pytest.fixture(scope="module")
def big(torch):
    import paper_1512_03812_gb300 as P
    L = T = 2048
    m0 = sw.kappa_to_m0(0.255)
    lat = P.Lattice(L, T, 8.0, m0)
    q = I.hot_links(L, T, 71)
    psi = I.spinor(L, T, 72)
    qd = torch.tensor(q, device="cuda")
    U64, U32 = lat.links(qd)
    olat = sw.Lattice(L, T, 8.0, m0)
    return P, lat, olat, q, psi, U64, U32


def test_2048_dslash_and_fused_ddagd_every_site(torch, big):
    P, lat, olat, q, psi, U64, U32 = big
    L = T = 2048
    pd = torch.tensor(psi, device="cuda")
    U = sw.links(q.reshape(T, L, 2))
    ref_d = sw.apply_D(olat, U, psi.reshape(T, L, 2))
    out = lat.apply_D(U64, pd).cpu().numpy().reshape(T, L, 2)
    assert rel_err(out, ref_d) < 1e-14
    ref = sw.apply_D(olat, U, ref_d, dagger=True)
    del ref_d
    out = lat.apply_DdagD(U64, pd).cpu().numpy().reshape(T, L, 2)
    assert rel_err(out, ref) < 1e-14
    out32 = lat.apply_DdagD(U32, pd.to(torch.complex64)).cpu().numpy().reshape(T, L, 2)
    assert rel_err(out32, ref) < 4e-6


@pytest.mark.parametrize("L,T", [(512, 512), (130, 2048)])
def test_single_chain_large_fp32_paths(torch, L, T):
    """2^18 sites or more in one chain: 512 x 512 takes the warp-streaming
    D^dag D (60-column strips) in both sm_apply_DdagD and the tiled CG;
    130 x 2048 is too narrow for 64-column windows (3 strips would read 192
    columns) and takes the 64 x 16 tiles instead, TMA-staged in the interior
    (x0 = 64) and cp.async-staged at the boundary."""
    import paper_1512_03812_gb300 as P
    m0 = sw.kappa_to_m0(0.24)
    lat = P.Lattice(L, T, 2.0, m0)
    q = I.hot_links(L, T, 91)
    psi = I.spinor(L, T, 92)
    U64, U32 = lat.links(torch.tensor(q, device="cuda"))
    pd = torch.tensor(psi, device="cuda")
    out = lat.apply_DdagD(U32, pd.to(torch.complex64)).cpu().numpy().reshape(T, L, 2)
    olat = sw.Lattice(L, T, 2.0, m0)
    ref = sw.apply_DdagD(olat, sw.links(q.reshape(T, L, 2)), psi.reshape(T, L, 2))
    assert rel_err(out, ref) < 4e-6
    x, iters, relres = lat.cg_solve(U64, U32, pd, P.CG(tol=1e-10, prec="mixed", delta=0.01))
    assert relres[0] <= 1e-10
    r = pd - lat.apply_DdagD(U64, x)
    assert float(torch.linalg.vector_norm(r)) <= 1.0000001e-10 * float(torch.linalg.vector_norm(pd))
    assert lat.check() == 0


def test_2048_mixed_cg_true_residual(torch, big):
    P, lat, olat, q, psi, U64, U32 = big
    b = torch.tensor(psi, device="cuda")
    x, iters, relres = lat.cg_solve(U64, U32, b, P.CG(tol=1e-10, prec="mixed", delta=0.01,
                                                       maxit=20000))
    assert relres[0] <= 1e-10
    r = b - lat.apply_DdagD(U64, x)
    assert float(torch.linalg.vector_norm(r)) <= 1.0000001e-10 * float(torch.linalg.vector_norm(b))
    assert lat.check() == 0


def test_256_ragged_chains_sampled(torch):
    import paper_1512_03812_gb300 as P
    n = 256
    sides = I.chain_sides(n, 81)
    betas, kappas = I.chain_couplings(n, 82)
    b = Batch([(int(s), int(s)) for s in sides], betas, kappas, seed=83)
    q, psi = b.q(), b.spinor()
    U64, U32 = b.lat.links(b.dev(q))
    out = b.lat.apply_DdagD(U32, b.dev(psi, torch.complex64))
    x, iters, relres = b.lat.cg_solve(U64, U32, b.dev(psi), P.CG(tol=1e-10, prec="mixed",
                                                                  delta=0.01))
    assert (relres <= 1e-10).all()
    rng = np.random.default_rng(84)
    for c in rng.choice(n, size=6, replace=False):
        ol = b.olat[c]
        U = sw.links(b.chain(q, c))
        ref = sw.apply_DdagD(ol, U, b.chain(psi, c))
        assert rel_err(b.chain(out, c), ref) < 4e-6
        r = b.chain(psi, c) - sw.apply_DdagD(ol, U, b.chain(x, c))
        assert np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(b.chain(psi, c))


def test_stream_ragged_batch_every_site(torch):
    """A ragged batch on the streaming form: a strip of 1 column at the right
    edge (301 = 5 x 60 + 1), one of 16 (256), whole strips (240), and a chain
    of 37 rows, fewer than a strip's window, whose rows wrap inside it."""
    import paper_1512_03812_gb300 as P
    shapes = [(301, 500), (256, 700), (240, 37)]
    betas, kappas = [2.0, 4.0, 1.0], [0.24, 0.25, 0.22]
    b = Batch(shapes, betas, kappas, seed=95)
    assert b.lat.N >= 1 << 18
    q, psi = b.q(), b.spinor()
    U64, U32 = b.lat.links(b.dev(q))
    out = b.lat.apply_DdagD(U32, b.dev(psi, torch.complex64))
    x, iters, relres = b.lat.cg_solve(U64, U32, b.dev(psi), P.CG(tol=1e-10, prec="mixed",
                                                                  delta=0.01))
    assert (relres <= 1e-10).all()
    for c in range(len(shapes)):
        ol = b.olat[c]
        U = sw.links(b.chain(q, c))
        ref = sw.apply_DdagD(ol, U, b.chain(psi, c))
        assert rel_err(b.chain(out, c), ref) < 4e-6
        r = b.chain(psi, c) - sw.apply_DdagD(ol, U, b.chain(x, c))
        assert np.linalg.norm(r) <= 1.0000001e-10 * np.linalg.norm(b.chain(psi, c))
    assert b.lat.check() == 0


def test_bench_workload_sampled_chains(torch):
    """The bench's launch configuration: 304 chains of 64 x 64 (beta 2,
    kappa 0.26), the autotuned chain-resident kernel, one trajectory of
    adapted nested FG (n 8, M 2, tau 1) with the mixed CG at 1e-10 (1e-12
    for H) and reliable-update factor 1e-3.  Two sampled chains, one from
    each wave of 152, against the oracle's FP64 trajectory at 1e-12: Delta H
    to the solver tolerance, and the same decision wherever u is not within
    1e-4 of exp(-Delta H)."""
    import paper_1512_03812_gb300 as P
    from oracle import integrators as ig
    B, L = 304, 64
    m0 = sw.kappa_to_m0(0.26)
    lat = P.Lattice([L] * B, [L] * B, 2.0, m0)
    # disordered but not hot: 0.3 x the seeded hot angles (CG converges in a
    # few hundred iterations, as on the bench's thermalised chains)
    q = np.concatenate([0.3 * I.hot_links(L, L, 400 + c) for c in range(B)])
    p = np.concatenate([I.momenta(L, L, 700 + c) for c in range(B)])
    eta = np.concatenate([I.noise(L, L, 900 + c) for c in range(B)])
    u = I.uniforms(B, 33)
    qd = torch.tensor(q, device="cuda")
    U64, U32 = lat.links(qd)
    cg = P.CG(tol=1e-10, maxit=20000, prec="mixed", delta=1e-3)
    lat.autotune_cg(U64, U32, torch.tensor(eta, device="cuda"), cg)
    md = P.MD(scheme="adapted_nested_fg", tau=1.0, n=8, M=2, fg="exact", cg=cg, tol_action=1e-12)
    dH, H0, acc = lat.hmc_trajectory(qd, torch.tensor(p, device="cuda"),
                                     torch.tensor(eta, device="cuda"), u, md)
    V = L * L
    ol = sw.Lattice(L, L, 2.0, m0)
    for c in (7, 230):
        sl = slice(c * V, (c + 1) * V)
        r = ig.hmc_trajectory(ol, q[sl].reshape(L, L, 2), p[sl].reshape(L, L, 2),
                              eta[sl].reshape(L, L, 2), u[c], "adapted_nested_fg", 1.0, 8, M=2,
                              solver=sw.Solver(1e-12))
        assert abs(dH[c] - r.dH) < 1e-6 * max(1.0, abs(r.dH)), (c, dH[c], r.dH)
        if abs(u[c] - np.exp(-r.dH)) > 1e-4:
            assert bool(acc[c]) == r.accepted


def test_hybrid_batch_fused_iteration(torch):
    """A batch mixing chains the chain-resident kernels hold (60 x 60) with
    one that only the grid-wide form can take (600 x 500): the small chains
    are solved on a side stream while the large one takes the fused
    streaming iteration (every chain is wide enough for the strips); all
    reach the FP64 true residual, also through a second solve on the same
    workspace."""
    import paper_1512_03812_gb300 as P
    shapes = [(60, 60), (600, 500), (60, 60)]
    b = Batch(shapes, [2.0, 2.0, 1.5], [0.24, 0.25, 0.23], seed=97)
    assert b.lat.N >= 1 << 18
    q, psi = b.q(), b.spinor()
    U64, U32 = b.lat.links(b.dev(q))
    for k in range(2):
        rhs = b.dev(psi if k == 0 else b.spinor(salt=9))
        x, iters, relres = b.lat.cg_solve(U64, U32, rhs, P.CG(tol=1e-10, prec="mixed",
                                                               delta=1e-3))
        assert (relres <= 1e-10).all(), relres
        r = rhs - b.lat.apply_DdagD(U64, x)
        for c in range(len(shapes)):
            assert np.linalg.norm(b.chain(r, c)) <= 1.0000001e-10 * np.linalg.norm(b.chain(rhs, c))
    assert b.lat.check() == 0


def test_tma_wait_give_up_is_reported_and_recovers(torch):
    """The bounded wait of a block for its TMA box copies, made to run out on
    purpose (limit 0: every interior tile of the 130 x 2048 lattice gives up
    at once; the copies themselves still land and the second, fully bounded
    wait lets them before the block leaves).  The lattice reports
    SM_ERR_TIMEOUT, the context stays usable, and with the default limit
    restored the same call matches the oracle."""
    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding as B
    L, T = 130, 2048
    m0 = sw.kappa_to_m0(0.24)
    lat = P.Lattice(L, T, 2.0, m0)
    with pytest.raises(B.SchwingerError):
        lat.set_wait_limit(-2)
    with pytest.raises(B.SchwingerError):
        lat.set_wait_limit(1 << 23)
    q = I.hot_links(L, T, 93)
    psi = I.spinor(L, T, 94)
    U64, U32 = lat.links(torch.tensor(q, device="cuda"))
    p32 = torch.tensor(psi, device="cuda").to(torch.complex64)
    assert lat.check() == 0
    lat.set_wait_limit(0)
    lat.apply_DdagD(U32, p32)
    with pytest.raises(B.SchwingerError) as e:
        lat.check()
    assert e.value.code == B.SM_ERR_TIMEOUT
    assert lat.check() == 0  # the word was cleared by the read
    lat.set_wait_limit(-1)
    out = lat.apply_DdagD(U32, p32).cpu().numpy().reshape(T, L, 2)
    assert lat.check() == 0
    olat = sw.Lattice(L, T, 2.0, m0)
    ref = sw.apply_DdagD(olat, sw.links(q.reshape(T, L, 2)), psi.reshape(T, L, 2))
    assert rel_err(out, ref) < 4e-6


def test_stencil_strip_height_autotuner(torch):
    """sm_autotune_ddagd on a 512 x 512 lattice (the streaming form): it times
    its candidate heights, keeps one of them, and sm_apply_DdagD with the
    chosen height still matches the oracle; a lattice too small for the
    streaming form reports height 0 and times nothing."""
    import paper_1512_03812_gb300 as P
    L = T = 512
    m0 = sw.kappa_to_m0(0.24)
    lat = P.Lattice(L, T, 2.0, m0)
    q = I.hot_links(L, T, 95)
    psi = I.spinor(L, T, 96)
    U64, U32 = lat.links(torch.tensor(q, device="cuda"))
    p32 = torch.tensor(psi, device="cuda").to(torch.complex64)
    h, cand = lat.autotune_ddagd(U32, p32)
    hs = [c[0] for c in cand]
    assert h in hs and len(hs) >= 2 and hs == sorted(hs) and all(t > 0 for _, t in cand)
    assert min(cand, key=lambda c: c[1])[0] == h
    out = lat.apply_DdagD(U32, p32).cpu().numpy().reshape(T, L, 2)
    olat = sw.Lattice(L, T, 2.0, m0)
    ref = sw.apply_DdagD(olat, sw.links(q.reshape(T, L, 2)), psi.reshape(T, L, 2))
    assert rel_err(out, ref) < 4e-6
    small = P.Lattice(16, 16, 2.0, m0)
    U64s, U32s = small.links(torch.zeros((256, 2), dtype=torch.float64, device="cuda"))
    assert small.autotune_ddagd(U32s, torch.ones((256, 2), dtype=torch.complex64,
                                                 device="cuda")) == (0, [])
