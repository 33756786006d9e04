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
