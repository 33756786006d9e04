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
