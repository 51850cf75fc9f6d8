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
import os

import numpy as np
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


def save_checkpoint(path, iteration, rho, lam, history):
    """The whole state of the design loop after `iteration` completed steps:
    the densities, the multiplier that warm-starts the next state solve (or
    None) and the history of (compliance, Krylov iterations).  Written to a
    temporary file first and renamed, so an interrupted save leaves the
    previous checkpoint intact."""
    arrays = {"iteration": np.array(iteration), "rho": rho.detach().cpu().numpy(),
              "history": np.array(history, dtype=np.float64).reshape(-1, 2)}
    if lam is not None:
        arrays["lam"] = lam.detach().cpu().numpy()
    tmp = str(path) + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, str(path))


def load_checkpoint(path, device="cuda"):
    """(iteration, densities, multiplier or None, history) saved by save_checkpoint."""
    with np.load(str(path)) as z:
        lam = torch.as_tensor(z["lam"], device=device) if "lam" in z.files else None
        hist = [(float(c), int(k)) for c, k in z["history"]]
        return int(z["iteration"]), torch.as_tensor(z["rho"], device=device), lam, hist


def optimize(cp, rho0, volfrac, iterations=50, callback=None, checkpoint=None, start=0, history=None):
    """Run OC steps `start` .. `iterations` - 1; returns the final densities and
    the history of (compliance, Krylov iterations).  With `checkpoint` (a path)
    the state is saved after every step; resume with load_checkpoint and pass
    its iteration, history and multiplier (cp.lam) back."""
    rho = rho0.clone()
    hist = list(history or [])
    for it in range(start, iterations):
        r = rho.clone().requires_grad_(True)
        c = compliance(r, cp)
        c.backward()
        cval = float(c.detach())
        hist.append((cval, cp.last_stats.iterations))
        if callback:
            callback(it, rho, cval, cp.last_stats)
        rho = oc_update(rho, r.grad, volfrac)
        if checkpoint is not None:
            save_checkpoint(checkpoint, it + 1, rho, cp.lam, hist)
    return rho, hist


def _fd_check(problem, n_check, rel_h, tol, seed=7):
    """Central differences of the compliance on n_check seeded elements against
    the sensitivity kernel, at the problem's own densities.  Each evaluation
    uses a fresh context with module sharing on, so that perturbing one element
    refactorizes only the modules that changed."""
    import numpy as np

    def comp(rho_np):
        s = Solver(FETI_FETIDP, FETI_SCALING_K, FETI_PCG, tol=tol, max_iter=5000, dedup=True,
                   stream=torch.cuda.current_stream().cuda_stream)
        pr = problem
        old = pr.rho
        pr.rho = rho_np
        s.setup(pr, rho=torch.from_numpy(rho_np).cuda(), f=torch.from_numpy(pr.f).cuda(), on_device=True)
        pr.rho = old
        feti_factorize(s.ctx)
        feti_solve_dual(s.ctx, allow_notconv=True)
        u = torch.empty(pr.n_dofs, dtype=torch.float64, device="cuda")
        c = feti_recover_displacements(s.ctx, u, True)
        g = torch.empty(pr.n_elements, dtype=torch.float64, device="cuda")
        feti_compliance_grad(s.ctx, g, True)
        s.close()
        return c, g

    rho0 = np.ascontiguousarray(problem.rho, dtype=np.float64)
    c0, g0 = comp(rho0)
    g0 = g0.cpu().numpy()
    rng = np.random.default_rng(seed)
    worst = 0.0
    rows = []
    for e in rng.choice(rho0.size, n_check, replace=False):
        h = rel_h * rho0[e]
        vals = []
        for sgn in (1.0, -1.0):
            r = rho0.copy()
            r[e] += sgn * h
            vals.append(comp(r)[0])
        fd = (vals[0] - vals[1]) / (2.0 * h)
        err = abs(fd - g0[e]) / max(abs(g0[e]), 1e-300)
        worst = max(worst, err)
        rows.append({"element": int(e), "grad": float(g0[e]), "fd": float(fd), "rel_err": float(err)})
    gmax = max(abs(r["grad"]) for r in rows)
    abs_err = max(abs(r["fd"] - r["grad"]) for r in rows)
    big = [r["rel_err"] for r in rows if abs(r["grad"]) >= 1e-2 * gmax]
    return {"compliance": c0, "elements": rows, "max_rel_err": worst,
            "max_abs_err_over_max_grad": abs_err / gmax,
            "max_rel_err_where_grad_ge_1pct_of_max": max(big) if big else None,
            "rel_h": rel_h, "tol": tol}


def main(argv=None):
    """Optimality-criteria run on the MBB-type beam: gradient check by central
    differences, then `iterations` design steps with the multipliers
    warm-started between state solves.  One JSON line per step and a summary."""
    import argparse
    import json
    import os
    import sys
    import time

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--tiles", type=int, default=32)
    ap.add_argument("--elems", type=int, default=64)
    ap.add_argument("--volfrac", type=float, default=0.4)
    ap.add_argument("--iterations", type=int, default=50)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--fd", type=int, default=20)
    ap.add_argument("--fd-rel-h", type=float, default=1e-3)
    ap.add_argument("--fd-tol", type=float, default=1e-12)
    ap.add_argument("--checkpoint", default=None, help="save the loop's state (.npz) after every design step")
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
    a = ap.parse_args(argv)

    p = workloads.config5(tiles=a.tiles, elems=a.elems, volfrac=a.volfrac)
    print(json.dumps({"workload": p.name, "n_dofs": p.n_dofs, "n_elements": p.n_elements}), flush=True)
    if a.fd > 0:
        t0 = time.perf_counter()
        fd = _fd_check(p, a.fd, a.fd_rel_h, a.fd_tol)
        fd["seconds"] = time.perf_counter() - t0
        print(json.dumps({"fd_check": fd}), flush=True)
    cp = ComplianceProblem(p, krylov=FETI_PCG, tol=a.tol, warm_start=True)
    rho = torch.tensor(p.rho, dtype=torch.float64, device="cuda")
    start, history = 0, None
    if a.resume and a.checkpoint and os.path.exists(a.checkpoint):
        start, rho, lam, history = load_checkpoint(a.checkpoint)
        if lam is not None:
            cp.lam.copy_(lam)
    t_last = [time.perf_counter()]

    def cb(it, r, c, st):
        torch.cuda.synchronize()
        now = time.perf_counter()
        print(json.dumps({"it": it, "compliance": c, "pcg_iterations": st.iterations, "converged": bool(st.converged),
                          "seconds": now - t_last[0], "volume": float(r.mean())}), flush=True)
        t_last[0] = now

    t0 = time.perf_counter()
    rho, hist = optimize(cp, rho, a.volfrac, iterations=a.iterations, callback=cb, checkpoint=a.checkpoint,
                         start=start, history=history)
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    # the same final state solve without the warm start, for comparison
    cold = ComplianceProblem(p, krylov=FETI_PCG, tol=a.tol, warm_start=False)
    cold.solve(rho)
    warm_its = [h[1] for h in hist]
    print(json.dumps({"summary": {"iterations": a.iterations, "seconds": total, "compliance_first": hist[0][0],
                                  "compliance_last": hist[-1][0], "pcg_iterations_mean_warm": sum(warm_its) / len(warm_its),
                                  "pcg_iterations_last_warm": warm_its[-1],
                                  "pcg_iterations_last_design_cold": cold.last_stats.iterations,
                                  "volume": float(rho.mean())}}), flush=True)


if __name__ == "__main__":
    main()
