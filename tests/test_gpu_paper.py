"""The paper's own configuration (Sec. 5): a 32 x 32 lattice, beta = 1.0,
m0 = -0.231367, trajectory length tau = 2, the adapted nested force-gradient
scheme at the step size Table 1 gives it (h = 0.056, n = 36 outer steps) with
the micro step h/10 (M = 5 inner leapfrog steps per half step).  One HMC
trajectory of the CUDA path (FP64 CG, tolerance 1e-14) against the oracle on
a seeded start (the paper's thermalised configuration is not available):
Delta H, H at the start, the links at the end of the MD and the decision."""
import numpy as np
import pytest

from oracle import integrators as ig
from oracle import schwinger as sw
from tests.gpu_util import Batch, rel_err

pytestmark = pytest.mark.gpu

L = T = 32
BETA, M0, TAU, N, M = 1.0, -0.231367, 2.0, 36, 5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    P.build()
    return t


@pytest.mark.parametrize("fg", ["exact", "shifted"])
def test_paper_configuration_trajectory_matches_oracle(torch, fg):
    import paper_1512_03812_gb300 as P
    kappa = 1.0 / (2.0 * (M0 + 2.0))
    b = Batch([(L, T)], BETA, kappa, seed=1512)
    q, p, eta = b.q(), b.p(), b.eta()
    u = 0.5
    qd = b.dev(q)
    q_md = torch.empty_like(qd)
    md = P.MD(scheme="adapted_nested_fg", tau=TAU, n=N, M=M, fg=fg,
              cg=P.CG(tol=1e-14, maxit=50000, prec="f64"))
    dH, H0, acc = b.lat.hmc_trajectory(qd, b.dev(p), b.dev(eta), u, md, q_md=q_md)
    r = ig.hmc_trajectory(b.olat[0], b.chain(q, 0), b.chain(p, 0), b.chain(eta, 0), u,
                          "adapted_nested_fg", TAU, N, M=M, fg=fg, solver=sw.Solver(1e-14))
    scale = max(1.0, abs(r.H0))
    err_dH = abs(dH[0] - r.dH) / scale
    err_q = rel_err(b.chain(q_md, 0), r.q_md)
    print(f"paper config {fg}: dH gpu {dH[0]:.15e} oracle {r.dH:.15e} (rel to H {err_dH:.2e}), "
          f"q_md rel {err_q:.2e}")
    assert abs(H0[0] - r.H0) <= 1e-12 * abs(r.H0)
    assert err_dH <= 1e-12, (dH[0], r.dH)
    assert bool(acc[0]) == r.accepted
    assert err_q < 1e-10
