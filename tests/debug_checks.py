"""Run in a process that loads the bounds-checked debug library
(SM_LIBRARY=debug): every entry point on a ragged batch of the smallest
lattices (2 x 2, 3 x 5, 4 x 6) against the oracle, then the debug build's
record of out-of-range indices.  Prints one JSON line: the largest relative
error of each comparison and the record.  Used by tests/test_gpu_debug.py."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import integrators as ig  # noqa: E402
from oracle import schwinger as sw  # noqa: E402
from tests.gpu_util import Batch, rel_err  # noqa: E402

DIMS = [(2, 2), (3, 5), (4, 6)]


def main():
    import torch

    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding as B
    assert B.library_path().endswith("_debug.so"), B.library_path()
    b = Batch(DIMS, [2.0, 1.0, 3.0], [0.24, 0.2, 0.22], seed=3)
    err = {}

    def worst(name, gpu, ref_fn):
        err[name] = max(rel_err(b.chain(gpu, c), ref_fn(c)) for c in range(len(DIMS)))

    q, psi, p, eta, v = b.q(), b.spinor(), b.p(), b.eta(), b.v()
    qd = b.dev(q)
    U64, U32 = b.lat.links(qd)
    Uo = [sw.links(b.chain(q, c)) for c in range(len(DIMS))]
    pd = b.dev(psi)
    for dag in (False, True):
        worst(f"D{int(dag)}_f64", b.lat.apply_D(U64, pd, dagger=dag),
              lambda c: sw.apply_D(b.olat[c], Uo[c], b.chain(psi, c), dagger=dag))
        worst(f"D{int(dag)}_f32", b.lat.apply_D(U32, pd.to(torch.complex64), dagger=dag),
              lambda c: sw.apply_D(b.olat[c], Uo[c], b.chain(psi, c), dagger=dag))
    worst("DdagD_f64", b.lat.apply_DdagD(U64, pd),
          lambda c: sw.apply_DdagD(b.olat[c], Uo[c], b.chain(psi, c)))
    worst("DdagD_f32", b.lat.apply_DdagD(U32, pd.to(torch.complex64)),
          lambda c: sw.apply_DdagD(b.olat[c], Uo[c], b.chain(psi, c)))
    c1 = 1
    L1, T1 = DIMS[c1]
    one = P.Lattice(L1, T1, 1.0, b.m0[c1])
    U1, _ = one.links(b.dev(b.chain(q, c1).reshape(-1, 2)))
    out = B.apply_DdagD_noalloc(L1, T1, b.m0[c1], U1, b.dev(b.chain(psi, c1).reshape(-1, 2)))
    err["DdagD_noalloc"] = rel_err(out.cpu().numpy().reshape(T1, L1, 2),
                                   sw.apply_DdagD(b.olat[c1], Uo[c1], b.chain(psi, c1)))
    for prec, algo in (("f64", "grid"), ("f64", "chain"), ("mixed", "grid"), ("mixed", "chain")):
        x, _, _ = b.lat.cg_solve(U64, U32, pd, P.CG(tol=1e-13, prec=prec, algo=algo, delta=0.1))
        worst(f"cg_{prec}_{algo}", x,
              lambda c: sw.Solver(1e-14).cg(b.olat[c], Uo[c], b.chain(psi, c)))
    cg = P.CG(tol=1e-14, prec="f64")
    worst("gauge_force", b.lat.gauge_force(qd), lambda c: sw.gauge_force(b.olat[c], Uo[c]))
    phi = b.dev(np.concatenate([sw.apply_D(b.olat[c], Uo[c], b.chain(eta, c), dagger=True)
                                .reshape(-1, 2) for c in range(len(DIMS))]))
    ph = phi.cpu().numpy()
    worst("force_full", b.lat.force(qd, phi, "full", cg),
          lambda c: sw.force(b.olat[c], Uo[c], b.chain(ph, c), sw.Solver(1e-14), "full"))
    worst("force_gradient_full", b.lat.force_gradient(qd, phi, "full", cg),
          lambda c: sw.force_and_gradient(b.olat[c], Uo[c], b.chain(ph, c), sw.Solver(1e-14),
                                          "full")[1])
    vd = b.dev(v)
    worst("hvp_full", b.lat.hvp(qd, phi, vd, "full", cg),
          lambda c: 0.5 * (sw.c_fg(b.olat[c], Uo[c], b.chain(v, c)) +
                           sw.c_fermion(b.olat[c], Uo[c], *sw.chi_xi(b.olat[c], Uo[c],
                                                                     b.chain(ph, c),
                                                                     sw.Solver(1e-14)),
                                        b.chain(v, c), sw.Solver(1e-14))))
    worst("shifted_force_full", b.lat.fg_shifted_force(qd, phi, 0.1, "full", cg),
          lambda c: sw.shifted_force(b.olat[c], b.chain(q, c), b.chain(ph, c), sw.Solver(1e-14),
                                     0.1, "full"))
    us = np.array([0.2, 0.5, 0.8])
    for scheme, M in (("leapfrog", 1), ("five_stage_fg", 1), ("adapted_nested_fg", 2),
                      ("nested_fg", 2), ("eleven_stage", 1)):
        for algo in ("grid", "chain"):
            for prec in ("f64", "mixed"):
                md = P.MD(scheme=scheme, tau=1.0, n=3, M=M,
                          cg=P.CG(tol=1e-14 if prec == "f64" else 1e-12, prec=prec, algo=algo,
                                  delta=0.1))
                q_md = torch.empty_like(qd)
                dH, _, acc = b.lat.hmc_trajectory(b.dev(q), b.dev(p), b.dev(eta), us, md,
                                                  q_md=q_md)
                rs = [ig.hmc_trajectory(b.olat[c], b.chain(q, c), b.chain(p, c), b.chain(eta, c),
                                        us[c], scheme, 1.0, 3, M=M, solver=sw.Solver(1e-14))
                      for c in range(len(DIMS))]
                key = f"hmc_{scheme}_{algo}_{prec}"
                err[key] = max(abs(dH[c] - r.dH) / max(1.0, abs(r.H0)) for c, r in enumerate(rs))
                err[key + "_qmd"] = max(rel_err(b.chain(q_md, c), r.q_md) for c, r in enumerate(rs))
                err[key + "_same_decisions"] = float(all(bool(acc[c]) == r.accepted
                                                         for c, r in enumerate(rs)))
    torch.cuda.synchronize()
    rec = B.debug_read()
    print(json.dumps({"errors": err, "debug": rec, "lattice_check": b.lat.check()}), flush=True)


if __name__ == "__main__":
    main()
