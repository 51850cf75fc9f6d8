"""One-call driver of the oracle: build the dual problem, run the Krylov
solver, recover the global displacement (test infrastructure only)."""
from .fetidp import FETIDP
from .krylov import solve_dual
from .tfeti import TFETI


def build(problem, method="fetidp", scaling="k", precond="dirichlet", primal="corners", jump_ratio=10.0):
    if method == "tfeti":
        if primal != "corners":
            raise ValueError("primal sets are a FETI-DP choice")
        return TFETI(problem, scaling, precond=precond)
    if method == "fetidp":
        return FETIDP(problem, scaling, precond=precond, primal=primal, jump_ratio=jump_ratio)
    raise ValueError(method)


def solve(problem, method="fetidp", scaling="k", krylov="rrs", tol=1e-6, max_iter=500,
          rr_tol=1e-10, op=None, precond="dirichlet", primal="corners", jump_ratio=10.0):
    """Returns (u_global, lambda, info, op)."""
    op = op or build(problem, method, scaling, precond, primal, jump_ratio)
    lam, info = solve_dual(op, tol=tol, max_iter=max_iter, rr_tol=rr_tol, variant=krylov)
    return op.recover(lam), lam, info, op
