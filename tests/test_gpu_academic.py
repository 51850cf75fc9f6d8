"""GPU parity on the stand-ins for the academic problems of Section 4 (laminated
beam, laminated 3x3 grid with cross points, 4x4 grid of stiff inclusions): all
12 variants through the C ABI against the oracle -- the displacement against
the direct solution of Eq. (2), the iteration count against the oracle's own
run of the same variant (Algorithm 1 in a different summation order: within
10% or 2 iterations), and the k-scaling finding (less than half the PCG
iterations of multiplicity scaling on the laminated grid)."""
import numpy as np
import pytest

import workloads
from oracle.assemble import direct_solve
from oracle.solve import solve

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import rel, solve_u  # noqa: E402

TOL = 1e-6
PROBLEMS = {
    "beam": lambda: workloads.layered_beam(elems=7, layers=7),
    "grid": lambda: workloads.layered_grid(elems=8, layers=8),
    "inclusion": lambda: workloads.inclusion_grid(elems=8),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_twelve_variants_match_oracle(name):
    p = PROBLEMS[name]()
    ud = direct_solve(p)
    its = {}
    for method in ("tfeti", "fetidp"):
        for scaling in ("k", "mult"):
            for krylov in ("pcg", "fo", "rrs"):
                u, st, c, s = solve_u(p, method=method, scaling=scaling, krylov=krylov, tol=TOL, max_iter=400)
                s.close()
                _, _, info, _ = solve(p, method, scaling, krylov, tol=TOL, max_iter=400)
                key = (method, scaling, krylov)
                assert st.converged, key
                assert rel(u, ud) <= 1e-4, (key, rel(u, ud))
                assert abs(st.iterations - info.iterations) <= max(2, 0.1 * info.iterations), (
                    key, st.iterations, info.iterations)
                its[key] = st.iterations
    if name == "grid":
        for method in ("tfeti", "fetidp"):
            assert 2 * its[method, "k", "pcg"] < its[method, "mult", "pcg"], method
