"""Compliance c(rho) = f^T u(rho) behind torch.autograd, and an optimality-
criteria SIMP loop (Section 1: state solves alternate with density updates).

The forward pass runs the library's whole pipeline through the C ABI
(feti_set_density, feti_factorize, feti_solve_dual with the previous
multiplier as warm start, feti_recover_displacements); the backward pass
calls the library's sensitivity kernel (feti_compliance_grad), which forms
the self-adjoint SIMP sensitivity -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e from
the recovered displacement: no adjoint solve is needed because the
compliance problem is self-adjoint.  This module only marshals tensors.
"""
import torch

from . import (FETI_ENOTCONV, FETI_FETIDP, FETI_OK, FETI_PCG, FETI_SCALING_K, FETI_Q_N_LAMBDA, Solver,
               feti_compliance_grad, feti_factorize, feti_recover_displacements, feti_set_density,
               feti_solve_dual, feti_query)


class ComplianceProblem:
    """Owns one library context for a fixed mesh; densities change per call."""

    def __init__(self, problem, method=FETI_FETIDP, scaling=FETI_SCALING_K, krylov=FETI_PCG, tol=1e-6,
                 max_iter=2000, warm_start=True, device="cuda"):
        self.problem = problem
        self.device = torch.device(device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.solver = Solver(method, scaling, krylov, tol=tol, max_iter=max_iter, dedup=False, stream=stream)
        rho = torch.as_tensor(problem.rho, dtype=torch.float64, device=self.device)
        self.f = torch.as_tensor(problem.f, dtype=torch.float64, device=self.device)
        self.solver.setup(problem, rho=rho, f=self.f, on_device=True)
        self.n_lambda = feti_query(self.solver.ctx, FETI_Q_N_LAMBDA)
        self.lam = torch.zeros(self.n_lambda, dtype=torch.float64, device=self.device) if warm_start else None
        self.u = torch.empty(problem.n_dofs, dtype=torch.float64, device=self.device)
        self.last_stats = None

    def solve(self, rho):
        rho = rho.detach().to(torch.float64).contiguous()
        feti_set_density(self.solver.ctx, rho, True)
        feti_factorize(self.solver.ctx)
        status, st = feti_solve_dual(self.solver.ctx, self.lam, allow_notconv=True)
        self.last_stats = st
        c = feti_recover_displacements(self.solver.ctx, self.u, True)
        return c, status in (FETI_OK, FETI_ENOTCONV)

    def grad(self):
        g = torch.empty(self.problem.n_elements, dtype=torch.float64, device=self.device)
        feti_compliance_grad(self.solver.ctx, g, True)
        return g


class _Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, cp):
        c, _ = cp.solve(rho)
        ctx.cp = cp
        return torch.tensor(c, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad_out):
        return grad_out * ctx.cp.grad(), None


def compliance(rho, cp):
    """c = f^T u(rho); differentiable in rho through the library's sensitivity kernel."""
    return _Compliance.apply(rho, cp)


def oc_update(rho, dc, volfrac, move=0.2, eta=0.5, rho_min=1e-3):
    """Optimality-criteria update with bisection on the volume multiplier
    (textbook SIMP update; the paper does not specify its optimizer)."""
    lo, hi = 0.0, 1e9
    dc = torch.clamp(dc, max=0.0)
    target = volfrac * rho.numel()
    new = rho
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        be = torch.pow(torch.clamp(-dc / mid, min=1e-30), eta)
        new = torch.clamp(rho * be, min=torch.clamp(rho - move, min=rho_min), max=torch.clamp(rho + move, max=1.0))
        if float(new.sum()) > target:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-12 * max(1.0, hi):
            break
    return new


def optimize(cp, rho0, volfrac, iterations=50, callback=None):
    """Run `iterations` OC steps; returns the final densities and the history
    of (compliance, Krylov iterations)."""
    rho = rho0.clone()
    hist = []
    for it in range(iterations):
        r = rho.clone().requires_grad_(True)
        c = compliance(r, cp)
        c.backward()
        hist.append((float(c), cp.last_stats.iterations))
        if callback:
            callback(it, rho, float(c), cp.last_stats)
        rho = oc_update(rho, r.grad, volfrac)
    return rho, hist
