"""The 3D workload at full size (8^3 subdomains of 8^3 H8 elements, 823,875
DOF), in the configuration bench.py times: properties that hold at any size,
checked with the oracle's independently assembled global stiffness K (Eq. 2):

* energy identity: a Galerkin solution satisfies u^T K u = f^T u; FETI
  solutions at relative dual residual 1e-6 meet it to ~1e-11 (oracle, 2^3 and
  3^3 tiles), a wrong block or map would not;
* equilibrium: ||(K u - f)_free|| / ||f|| small (oracle: 7e-6 at 2^3 tiles,
  3e-5 at 3^3 tiles);
* the compliance the library returns equals f^T u;
* the reduced-precision operators of the same full-size problem stay within
  their rounding of the FP64 operator on sampled directions.
"""
import numpy as np
import pytest

import workloads
from oracle.assemble import global_stiffness

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import rel, solve_u, torch_cuda  # noqa: E402


@pytest.fixture(scope="module")
def full3d():
    return workloads.config4(tiles=8, elems=8)


def test_full_size_3d_solution_properties(full3d):
    p = full3d
    u, st, comp, s = solve_u(p, tol=1e-6, max_iter=60)
    s.close()
    assert st.converged and st.iterations <= 40
    K = global_stiffness(p)
    fu = float(p.f @ u)
    assert comp == pytest.approx(fu, rel=1e-12)
    assert abs(float(u @ (K @ u)) / fu - 1.0) <= 1e-8
    free = ~np.asarray(p.dirichlet, bool)
    res = np.linalg.norm((K @ u - p.f)[free]) / np.linalg.norm(p.f)
    assert res <= 1e-3


@pytest.mark.parametrize("prec,bar", [("tf32x3", 2e-5), ("bf16x3", 2e-4)])
def test_full_size_3d_reduced_precision_apply(full3d, prec, bar):
    torch = torch_cuda()
    from gpu_helpers import make_solver
    p = full3d
    pr = {"tf32x3": fg.FETI_TF32X3, "bf16x3": fg.FETI_BF16X3}[prec]
    Ys = []
    for precision in (0, pr):
        s = make_solver(p, precision=precision)
        fg.feti_factorize(s.ctx)
        n = s.query(fg.FETI_Q_N_LAMBDA)
        X = torch.from_numpy(np.random.default_rng(7).standard_normal((16, n))).cuda()
        Y = torch.zeros_like(X)
        fg.feti_apply_dual(s.ctx, X, n, 16, Y, n)
        Ys.append(Y.cpu().numpy())
        s.close()
    d = rel(Ys[1], Ys[0])
    assert 0.0 < d <= bar
