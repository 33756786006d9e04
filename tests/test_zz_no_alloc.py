"""The entry point that allocates nothing (sm_apply_DdagD_noalloc), for
callers that cannot call cudaMalloc and so can create neither a workspace nor
a lattice object: its output must match the workspace-based sm_apply_DdagD,
within the tolerances the parity tests use, on two calls in a row.  This file
is collected last; it also passes on its own in a fresh process."""
import pytest

from oracle import schwinger as sw
from paper_1512_03812_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    P.build()
    return t


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("L,T", [(64, 64), (17, 9)])
def test_noalloc_matches_workspace_entry_point_twice(torch, L, T):
    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding
    m0 = sw.kappa_to_m0(0.25)
    lat = P.Lattice(L, T, 2.0, m0)
    q = torch.tensor(I.hot_links(L, T, 41), device="cuda")
    U64, U32 = lat.links(q)
    for call, seed in enumerate((42, 43)):  # two calls in a row, different inputs
        psi = torch.tensor(I.spinor(L, T, seed), device="cuda")
        ref64 = lat.apply_DdagD(U64, psi)
        ref32 = lat.apply_DdagD(U32, psi.to(torch.complex64))
        out64 = binding.apply_DdagD_noalloc(L, T, m0, U64, psi)
        out32 = binding.apply_DdagD_noalloc(L, T, m0, U32, psi.to(torch.complex64))
        torch.cuda.synchronize()
        assert _rel(out64, ref64) < 1e-14, call
        assert _rel(out32.to(torch.complex128), ref32.to(torch.complex128)) < 4e-6, call


def test_noalloc_rejects_lattices_beyond_its_scratch(torch):
    from paper_1512_03812_gb300 import binding
    L = T = 1024  # 1048576 sites > 262144 (FP64) and > 524288 (FP32)
    for dt in (torch.complex128, torch.complex64):
        U = torch.zeros((L * T, 2), dtype=dt, device="cuda")
        psi = torch.zeros((L * T, 2), dtype=dt, device="cuda")
        with pytest.raises(binding.SchwingerError, match="exceed"):
            binding.apply_DdagD_noalloc(L, T, 0.0, U, psi)
