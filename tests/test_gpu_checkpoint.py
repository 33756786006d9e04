"""Resume from a checkpoint reproduces the following trajectories bit for
bit: the link angles and the caller's generator state are the whole state of
a batch between trajectories."""
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


def test_resume_reproduces_the_next_trajectories(torch, tmp_path):
    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import checkpoint as ck
    b = Batch([(8, 8), (16, 8)], [2.0, 1.5], [0.24, 0.22], seed=31)
    md = P.MD(scheme="adapted_nested_fg", tau=0.5, n=2, M=2,
              cg=P.CG(tol=1e-10, prec="mixed", delta=0.01))
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    N = b.lat.N

    def draw():
        p = torch.randn((N, 2), generator=g, device="cuda", dtype=torch.float64)
        e = torch.randn((N, 2, 2), generator=g, device="cuda", dtype=torch.float64)
        e = torch.view_as_complex(e * 0.5 ** 0.5).contiguous()
        u = torch.rand(b.lat.nchains, generator=g, device="cuda", dtype=torch.float64)
        return p, e, u.cpu().numpy()

    q = b.dev(b.q())
    for _ in range(2):
        b.lat.hmc_trajectory(q, *draw(), md)
    path = tmp_path / "batch.ckpt"
    ck.save(path, b.lat, q, 2, rng_state=g.get_state(), params={"tau": md.tau, "n": md.n})
    ref = []
    for _ in range(2):
        dH, _, acc = b.lat.hmc_trajectory(q, *draw(), md)
        ref.append((dH.copy(), acc.copy()))
    c = ck.load(path)
    assert c["trajectory"] == 2 and ck.matches(c, b.lat)
    q2 = torch.tensor(c["q"], device="cuda")
    g.set_state(c["rng_state"])
    for k in range(2):
        dH, _, acc = b.lat.hmc_trajectory(q2, *draw(), md)
        assert np.array_equal(dH, ref[k][0]) and np.array_equal(acc, ref[k][1])
    assert torch.equal(q2, q)
