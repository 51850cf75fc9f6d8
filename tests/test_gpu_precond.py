"""GPU parity of the preconditioner choices (Dirichlet S_s of Eq. 13, lumped
K_bb, super-lumped diag K_bb; Section 3) against the oracle: the block
preconditioner Z column by column, and PCG solves that reach the direct
solution of Eq. 2 with the oracle's iteration counts (+-2)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.assemble import direct_solve

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import lambda_perm, make_solver, rel, solve_u, torch_cuda  # noqa: E402

PC = {"dirichlet": 0, "lumped": 1, "superlumped": 2}


def moderate(tiles=4, elems=8):
    p = workloads.config2(tiles=tiles, elems=elems)
    p.rho = np.where(p.rho < 0.5, 0.3, 1.0)
    p.Emin = 1e-6
    return p


@pytest.mark.parametrize("method", ["fetidp", "tfeti"])
@pytest.mark.parametrize("pc", ["lumped", "superlumped"])
def test_precond_columns_match_oracle(method, pc):
    torch = torch_cuda()
    p = moderate() if method == "fetidp" else workloads.config1()
    op = oracle.build(p, method, "k", precond=pc)
    s = make_solver(p, method=method, precond=PC[pc])
    fg.feti_factorize(s.ctx)
    perm = lambda_perm(op, fg.feti_lambda_layout(s.ctx), method)
    n = perm.size
    ro = np.random.default_rng(11).standard_normal(n)
    Zo = op.precond_columns(ro)
    r = torch.from_numpy(ro[perm].copy()).cuda()
    Z = torch.zeros((p.n_subdomains, n), dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    fg.feti_apply_precond(s.ctx, r, Z, n, z)
    assert rel(Z.cpu().numpy().T, Zo[perm]) <= 1e-12
    assert rel(z.cpu().numpy(), Zo.sum(axis=1)[perm]) <= 1e-12


@pytest.mark.parametrize("method", ["tfeti", "fetidp"])
@pytest.mark.parametrize("pc", ["dirichlet", "lumped", "superlumped"])
def test_pcg_solves_match_oracle(method, pc):
    p = workloads.config1()
    ud = direct_solve(p)
    _, _, info, _ = oracle.solve(p, method, "k", "pcg", tol=1e-12, max_iter=2000, precond=pc)
    u, st, c, s = solve_u(p, method=method, krylov="pcg", tol=1e-12, max_iter=2000, precond=PC[pc])
    assert st.converged
    assert rel(u, ud) <= 1e-8
    assert abs(st.iterations - info.iterations) <= max(2, 0.1 * info.iterations), (st.iterations, info.iterations)


def test_lumped_rrs_and_reduced_precision():
    # the lumped blocks with the multi-direction solver and with the tensor-core operator
    p = moderate()
    ud = direct_solve(p)
    for kw in ({"krylov": "rrs"}, {"krylov": "rrs", "precision": fg.FETI_TF32X3}):
        u, st, c, s = solve_u(p, tol=1e-10, precond=PC["lumped"], max_iter=400, **kw)
        assert st.converged and rel(u, ud) <= 1e-8
