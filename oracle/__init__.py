"""Plain, slow, FP64 CPU oracle for the Henry-problem MLMC hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm)
use it.  It shares no code with the CUDA path (no kernels, headers, helpers,
tables or constant generators); the only thing both sides see is the seeded
input generator module ``paper_2302_07804_gb300.inputs``, which holds none of
the method's arithmetic.

Contents, each function citing the passage of arXiv 2302.07804 it follows:

* ``philox``  - Philox4x32-10 counter-based generator (Salmon et al., SC'11,
  the published definition) and the exact map of its words to xi in (-1, 1);
  the paper draws xi_i iid uniform on [-1, 1] (Sec. 4, the recharge and
  porosity model).
* ``henry``   - the discrete cell-centred finite-volume form of Eqs.
  (e_cont_eq), (e_tran_eq), (e_Darcy_vel), (e_lin_density), (e_mol_diff) with
  the boundary conditions of Sec. 2.1, implicit Euler in time and Newton's
  method with a direct sparse solve (Sec. 2.3); QoIs.
* ``henry_vc`` - the paper's own vertex-centred finite volumes (two unknowns
  per grid vertex, Sec. 2.3 and Table tab:adaptiveTS_times), with the
  readings of its "consistent velocity" and partial upwinding stated in the
  module; the same equations, boundary conditions, time stepping and QoIs.
  Its CUDA counterpart so far is the assembly (``henry_vc_assemble``); the
  oracle fixes the target of the rest of that path.
* ``mg``      - the textbook definitions of the multigrid pieces the CUDA
  path uses (Galerkin coarse operator, red-black block Gauss-Seidel, V-cycle,
  right-preconditioned BiCGStab from the Templates book cited in Sec. 2.3).
* ``mg_vc``   - the same multigrid pieces for the vertex-centred scheme
  (vertex-nested grids, bilinear transfer, four-colour block Gauss-Seidel).
* ``mlmc``    - the telescoping estimator (Eqs. EgL, A, Def. Yell), its
  variance, and the sample allocation of Eq. (M_ell), with two-pass moments.

Parity status: every function is pinned by a ``-m "not gpu"`` test except
``henry.qoi`` values against the paper itself ("parity unpinned": the paper's
physics variant differs from the configuration solved here and its figures
carry no numbers).
"""
