"""One HMC trajectory captured as a CUDA graph (sm_hmc_graph_*) reproduces the
eager sm_hmc_trajectory bitwise, over two runs in a row with refilled
momenta and noise, on a batch whose solves are all chain-resident."""
import numpy as np
import pytest

from tests.gpu_util import Batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    P.build()
    return t


@pytest.mark.parametrize("dims", [[(64, 64), (16, 8), (8, 8)],
                                  # a 128 x 128 chain takes the 4-block cluster kernel,
                                  # the others the one-block kernels on a side stream
                                  [(128, 128), (32, 32), (16, 16)]])
def test_graph_equals_eager_twice(torch, dims):
    import paper_1512_03812_gb300 as P
    b = Batch(dims, [2.0, 1.5, 2.5], [0.24, 0.22, 0.23], seed=12)
    md = P.MD(scheme="adapted_nested_fg", tau=0.5, n=2, M=2,
              cg=P.CG(tol=1e-10, prec="mixed", delta=0.01), tol_action=1e-12)
    q0 = b.q()
    ps = [b.p(20 + k) for k in range(2)]
    es = [b.eta(30 + k) for k in range(2)]
    us = [np.array([0.3, 0.6, 0.9]), np.array([0.8, 0.1, 0.5])]
    # eager
    qe = b.dev(q0)
    eager = []
    for k in range(2):
        eager.append(b.lat.hmc_trajectory(qe, b.dev(ps[k]), b.dev(es[k]), us[k], md, check=False))
    # graph
    qg = b.dev(q0)
    p0 = torch.empty_like(b.dev(ps[0]))
    eta = torch.empty_like(b.dev(es[0]))
    g = b.lat.hmc_graph(qg, p0, eta, md)
    for k in range(2):
        p0.copy_(b.dev(ps[k]))
        eta.copy_(b.dev(es[k]))
        dH, H0, acc = g.run(us[k])
        assert np.array_equal(dH, eager[k][0]), (dH, eager[k][0])
        assert np.array_equal(acc, eager[k][2])
    torch.cuda.synchronize()
    assert torch.equal(qg, qe)


def test_graph_needs_chain_resident_solves(torch):
    import paper_1512_03812_gb300 as P
    b = Batch([(8, 8)], 2.0, 0.24, seed=13)
    q = b.dev(b.q())
    md = P.MD(scheme="leapfrog", tau=0.2, n=2, cg=P.CG(tol=1e-10, prec="mixed", algo="grid"))
    with pytest.raises(P.SchwingerError):
        b.lat.hmc_graph(q, b.dev(b.p()), b.dev(b.eta()), md)


@pytest.mark.parametrize("variant", [6, 8])
def test_graph_equals_eager_longest_first(torch, variant):
    """160 chains of 64 x 64 on a column-pair kernel pinned (variant 6, or 8
    with the iterate in tensor memory): its launches take the chains in the
    order of their previous solve's iteration counts, which changes between
    solves; the results do not depend on it (graph and eager bitwise equal,
    and a chain's solution equal to that of the same chain solved alone)."""
    import paper_1512_03812_gb300 as P
    n = 160
    b = Batch([(64, 64)] * n, 2.0, 0.24, seed=14)
    b.lat.set_cg_variant(variant)
    md = P.MD(scheme="adapted_nested_fg", tau=0.25, n=1, M=2,
              cg=P.CG(tol=1e-10, prec="mixed", delta=0.01), tol_action=1e-12)
    q0 = b.q()
    ps = [b.p(40 + k) for k in range(2)]
    es = [b.eta(50 + k) for k in range(2)]
    rng = np.random.default_rng(3)
    us = [rng.random(n) for _ in range(2)]
    qe = b.dev(q0)
    eager = [b.lat.hmc_trajectory(qe, b.dev(ps[k]), b.dev(es[k]), us[k], md, check=False)
             for k in range(2)]
    qg = b.dev(q0)
    p0 = torch.empty_like(b.dev(ps[0]))
    eta = torch.empty_like(b.dev(es[0]))
    g = b.lat.hmc_graph(qg, p0, eta, md)
    for k in range(2):
        p0.copy_(b.dev(ps[k]))
        eta.copy_(b.dev(es[k]))
        dH, H0, acc = g.run(us[k])
        assert np.array_equal(dH, eager[k][0])
        assert np.array_equal(acc, eager[k][2])
    torch.cuda.synchronize()
    assert torch.equal(qg, qe)
    # chain c's result is the same when it is solved alone
    one = Batch([(64, 64)], 2.0, 0.24, seed=14)
    one.lat.set_cg_variant(variant)
    U64, U32 = b.lat.links(b.dev(q0))
    phi = b.dev(b.spinor())
    x, _, _ = b.lat.cg_solve(U64, U32, phi, P.CG(tol=1e-10, prec="mixed", delta=0.01))
    c = 137
    sl = slice(b.off[c], b.off[c + 1])
    U64c, U32c = one.lat.links(b.dev(q0)[sl].contiguous())
    xc, _, _ = one.lat.cg_solve(U64c, U32c, phi[sl].contiguous(),
                                P.CG(tol=1e-10, prec="mixed", delta=0.01))
    assert torch.equal(x[sl], xc)
