"""FP64 CPU oracle for the two-flavour Wilson-fermion Schwinger-model HMC.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or
links this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
path: it is a plain, slow, obviously-correct numpy restatement of the paper
(arXiv:1512.03812), every function citing the section/equation it follows.

Modules
-------
schwinger    lattice operators, actions, forces and force-gradient terms
             (Sec. 3: Eq. gauge_action, fer_action, the Wilson-Dirac matrix,
             Eq. force, force_gauge, force_fermion, chi_xi_vectors,
             force_gradient, force_grad_de, CFF, Z12)
integrators  the MD schedules of Sec. 2 (Eq. leap, 5stage, 5stage_fg,
             leap_multi, 5stage_multi, 5stage_multi_fg,
             ad_5stage_multi_fg) and the HMC trajectory with its
             Metropolis step (Sec. 2.1)

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute force, finite differences, invariances,
the paper's inversion counts).  Functions without such a pin say
"parity unpinned" in their docstring; there are none at present.
"""
