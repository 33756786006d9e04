"""The bounds-checked debug build (-DSM_DEBUG): every entry point on the
smallest lattices (2 x 2, 3 x 5, 4 x 6 in one ragged batch) against the
oracle, with every site index of a field access and the neighbour and halo
indices of the small-lattice kernels checked; none may be out of range.  The
debug library runs in a process of its own (SM_LIBRARY=debug), so that this
process keeps the normal one, whose record is empty by construction."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def debug_run():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03812_gb300 import _build
    _build.build()
    _build.build(debug=True)
    env = dict(os.environ, SM_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_checks.py")],
                       capture_output=True, text=True, env=env, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])


def test_debug_build_sees_no_out_of_range_index(debug_run):
    rec = debug_run["debug"]
    assert rec["where"] != -2, "the checks were not compiled in"
    assert rec["violations"] == 0, rec
    assert debug_run["lattice_check"] == 0


def test_debug_build_matches_the_oracle(debug_run):
    err = debug_run["errors"]
    for k, e in err.items():
        if k.endswith("_same_decisions"):
            assert e == 1.0, k
        elif "_f32" in k:
            assert e < 4e-6, (k, e)
        elif k.startswith("cg_mixed"):
            assert e < 1e-10, (k, e)
        elif k.startswith("hmc_") and "_mixed" in k:
            assert e < 1e-8, (k, e)
        elif k.startswith("cg_"):
            assert e < 1e-11, (k, e)
        else:
            assert e < 1e-11, (k, e)


def test_normal_build_reports_no_checks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03812_gb300 import binding as B
    assert B.debug_read()["where"] == -2
