"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/schwinger.h declares.  No compute calls (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s\*]+(sm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_build_and_load():
    import paper_1512_03812_gb300 as P
    P.build()
    lib = P.load()
    assert lib.sm_version() == 1


def test_every_declared_symbol_is_exported_and_bound():
    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding
    lib = P.load()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(binding.exported_symbols())


def test_error_path_without_gpu_work():
    import ctypes
    import paper_1512_03812_gb300 as P
    lib = P.load()
    h = ctypes.c_void_p()
    rc = lib.sm_lattice_create(0, None, None, None, None, ctypes.byref(h))
    assert rc == 1 and b"nchains" in lib.sm_last_error()
    assert lib.sm_lattice_destroy(None) == 0


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets that a
    C compiler gives the header's structs (compiled with gcc, no GPU)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1512_03812_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sm_cg_params": B.CgParams, "sm_md_params": B.MdParams, "sm_stats": B.Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "schwinger.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            name, key, val = line.split()
            c[(name, key)] = int(val)
    for cname, py in structs.items():
        assert c[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert c[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_binding_constants_match_the_header():
    """The binding's scheme, precision, part, force-gradient and status codes
    and the number of chain-CG variants are the header's #defines."""
    from paper_1512_03812_gb300 import binding as B
    src = open(os.path.join(ROOT, "include", "schwinger.h")).read()
    d = {k: int(v) for k, v in re.findall(r"^#define (SM_\w+) (-?\d+)", src, flags=re.M)}
    names = {"leapfrog": "SM_LEAPFROG", "five_stage": "SM_FIVE_STAGE",
             "five_stage_fg": "SM_FIVE_STAGE_FG", "nested_leapfrog": "SM_NESTED_LEAPFROG",
             "nested_five_stage": "SM_NESTED_FIVE_STAGE", "nested_fg": "SM_NESTED_FG",
             "adapted_nested_fg": "SM_ADAPTED_NESTED_FG", "eleven_stage": "SM_ELEVEN_STAGE",
             "nested3_leapfrog": "SM_NESTED3_LEAPFROG",
             "adapted_nested3_fg": "SM_ADAPTED_NESTED3_FG"}
    assert set(B.SCHEMES) == set(names)
    for k, v in B.SCHEMES.items():
        assert v == d[names[k]], k
    for k in ("SM_OK", "SM_ERR_ARG", "SM_ERR_CUDA", "SM_ERR_NOT_CONVERGED", "SM_ERR_TIMEOUT",
              "SM_ERR_NAN", "SM_F64", "SM_F32", "SM_MIXED"):
        assert getattr(B, k) == d[k], k
    assert (B.PART_GAUGE, B.PART_FERMION, B.PART_FULL, B.PART_HEAVY, B.PART_RATIO) == (
        d["SM_PART_GAUGE"], d["SM_PART_FERMION"], d["SM_PART_FULL"], d["SM_PART_HEAVY"],
        d["SM_PART_RATIO"])
    assert (B.FG_EXACT, B.FG_SHIFTED) == (d["SM_FG_EXACT"], d["SM_FG_SHIFTED"])
    assert B.CG_VARIANTS == d["SM_CG_VARIANTS"]
    assert B.DDAGD_HEIGHTS == d["SM_DDAGD_HEIGHTS"]


def test_noalloc_binding_refuses_mismatched_tensors_before_launching():
    """The no-alloc entry point sees only pointers and L, T: the binding checks
    shapes, dtypes, contiguity and the device first (CPU tensors here, so a
    launch could not even start)."""
    import torch
    from paper_1512_03812_gb300 import binding
    L, T = 6, 4
    V = L * T
    good = torch.zeros((V, 2), dtype=torch.complex128)
    cases = [
        (good, torch.zeros((V + 1, 2), dtype=torch.complex128), None, "psi must have shape"),
        (torch.zeros((V, 2), dtype=torch.complex64), good, None, "U must have psi's dtype"),
        (torch.zeros((V - 2, 2), dtype=torch.complex128), good, None, "U must have shape"),
        (good, good, torch.zeros((V, 2), dtype=torch.complex64), "out must have psi's dtype"),
        (good, torch.zeros((2, V), dtype=torch.complex128).t(), None, "psi must be contiguous"),
        (good, torch.zeros((V, 2), dtype=torch.float64), None, "psi must be complex"),
        (good, good, None, "must be on the current CUDA device"),
    ]
    for U, psi, out, msg in cases:
        with pytest.raises(ValueError, match=msg):
            binding.apply_DdagD_noalloc(L, T, 0.1, U, psi, out)
