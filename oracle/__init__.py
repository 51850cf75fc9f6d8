"""Plain FP64 CPU oracle of the FETI solvers compared in the paper
"Comparison of FETI-based domain decomposition methods for topology
optimization problems" (Medricky, Doskar, Pultarova, Zeman).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import it.  The CUDA library
never calls it and shares no code with it; the two meet only through the
seeded problem descriptions in ``workloads``.

Every routine is written for a reader checking it against the paper by eye:
dense per-subdomain matrices, explicit Boolean/signed constraint matrices,
and the steps of Algorithm 1 in the paper's order.  Nothing is blocked,
fused or reordered for speed.

Modules
-------
fem          SIMP interpolation (Eq. 1), Q4/H8 reference element stiffness.
mesh         Regular tile meshes: global <-> subdomain numbering.
assemble     Global system (Eq. 2) and local systems (Eq. 3), direct solve.
scaling      k-scaling (Eq. 15) and multiplicity scaling (Section 3.1).
tfeti        Total FETI (Section 2.1, Eqs. 4-7) and its projector.
fetidp       FETI-DP (Section 2.2, Eqs. 8-12) with corner primal DOFs, optionally
             with edge averages (a richer primal set, Section 5).
krylov       PCG, full orthogonalization, and Algorithm 1 (RR-S-FETI).
sensitivity  Compliance and the SIMP sensitivity.
sharded      Algorithm 1 for FETI-DP on CPU ranks of torch.distributed with the
             multi-GPU layout (subdomain blocks per rank, row-partitioned
             directions, halo exchanges and all-reduces); imported on demand.

Parity status of each function is stated in its docstring; functions without
an independent pin say "parity unpinned".
"""
from . import fem, mesh, assemble, scaling, tfeti, fetidp, krylov, sensitivity  # noqa: F401
from .solve import solve, build  # noqa: F401
