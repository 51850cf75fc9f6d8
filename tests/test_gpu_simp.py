"""GPU checks of the differentiation form: compliance through the C ABI behind
torch.autograd, its gradient against the oracle's sensitivity and central
finite differences, and a short optimality-criteria loop with warm starts."""
import numpy as np
import pytest

import workloads
from oracle.assemble import direct_solve
from oracle.sensitivity import compliance as oracle_compliance
from oracle.sensitivity import compliance_gradient

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")


def _problem():
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.3, 1.0, size=8 * 8)
    return workloads.tile_problem("fd", 2, (2, 2), (4, 4), rho, Emin=1e-6)


def test_autograd_gradient_matches_oracle_and_fd():
    import torch
    from paper_2111_11728_gb300 import simp
    p = _problem()
    cp = simp.ComplianceProblem(p, krylov=fg.FETI_RRS, tol=1e-12)
    rho = torch.tensor(p.rho, dtype=torch.float64, device="cuda", requires_grad=True)
    c = simp.compliance(rho, cp)
    c.backward()
    ud = direct_solve(p)
    assert float(c.detach()) == pytest.approx(oracle_compliance(p, ud), rel=1e-9)
    g_ref = compliance_gradient(p, ud)
    g = rho.grad.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    # central differences of the GPU compliance itself on 20 seeded elements
    rng = np.random.default_rng(5)
    for e in rng.choice(p.rho.size, 20, replace=False):
        h = 1e-4 * p.rho[e]
        vals = []
        for sgn in (1, -1):
            r2 = rho.detach().clone()
            r2[e] += sgn * h
            vals.append(float(simp.compliance(r2, cp)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + 1e-9 * np.abs(g).max()


def test_oc_loop_decreases_compliance_with_warm_start():
    import torch
    from paper_2111_11728_gb300 import simp
    p = workloads.config5(tiles=4, elems=8)
    cp = simp.ComplianceProblem(p, krylov=fg.FETI_PCG, tol=1e-8)
    rho0 = torch.tensor(p.rho, dtype=torch.float64, device="cuda")
    rho, hist = simp.optimize(cp, rho0, volfrac=0.4, iterations=6)
    cs = [h[0] for h in hist]
    assert cs[-1] < cs[0]
    assert abs(float(rho.mean()) - 0.4) <= 1e-3
    assert float(rho.min()) >= 1e-3 - 1e-12 and float(rho.max()) <= 1.0


def test_warm_start_shortens_the_solve():
    """The relative stopping test is measured from the method's own initial
    multiplier, so restarting from the solution needs no iteration and a
    nearby design needs fewer iterations than a cold start."""
    import torch
    from gpu_helpers import make_solver
    p = workloads.config5(tiles=4, elems=8)
    rng = np.random.default_rng(3)
    p.rho = rng.uniform(0.3, 1.0, size=p.rho.size)
    s = make_solver(p, krylov="pcg", tol=1e-8, dedup=False)
    fg.feti_factorize(s.ctx)
    n = s.query(fg.FETI_Q_N_LAMBDA)
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st_cold = fg.feti_solve_dual(s.ctx, lam)
    assert st_cold.converged and st_cold.iterations > 5
    _, st_again = fg.feti_solve_dual(s.ctx, lam)
    assert st_again.converged and st_again.iterations <= 1
    rho2 = torch.from_numpy(p.rho * (1.0 + 0.02 * rng.standard_normal(p.rho.size))).cuda()
    fg.feti_set_density(s.ctx, rho2, True)
    fg.feti_factorize(s.ctx)
    _, st_warm = fg.feti_solve_dual(s.ctx, lam)
    _, st_cold2 = fg.feti_solve_dual(s.ctx, None)
    assert st_warm.converged and st_cold2.converged
    assert st_warm.iterations < st_cold2.iterations
