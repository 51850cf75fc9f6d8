"""Helpers shared by the GPU parity tests: drive the C ABI through the thin
binding and map the library's multiplier / DOF orderings onto the oracle's."""
import numpy as np

import paper_2111_11728_gb300 as fg

METHOD = {"tfeti": fg.FETI_TFETI, "fetidp": fg.FETI_FETIDP}
SCALING = {"k": fg.FETI_SCALING_K, "mult": fg.FETI_SCALING_MULT}
KRYLOV = {"pcg": fg.FETI_PCG, "fo": fg.FETI_FO, "rrs": fg.FETI_RRS}


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def make_solver(problem, method="fetidp", scaling="k", krylov="rrs", tol=1e-10, max_iter=500, dedup=True,
                on_device=True, rr_tol=1e-10, precision=0, inner_tol=None, precond=0):
    torch = torch_cuda()
    s = fg.Solver(METHOD[method], SCALING[scaling], KRYLOV[krylov], tol=tol, max_iter=max_iter, rr_tol=rr_tol,
                  dedup=dedup, stream=torch.cuda.current_stream().cuda_stream, precision=precision,
                  inner_tol=inner_tol, precond=precond)
    if on_device:
        rho = torch.from_numpy(problem.rho).cuda()
        f = torch.from_numpy(problem.f).cuda()
        s.setup(problem, rho=rho, f=f, on_device=True)
    else:
        s.setup(problem, on_device=False)
    return s


def solve_u(problem, **kw):
    """Full pipeline on the GPU; returns (u numpy, stats, compliance, solver)."""
    torch = torch_cuda()
    s = make_solver(problem, **kw)
    fg.feti_factorize(s.ctx)
    status, st = fg.feti_solve_dual(s.ctx, allow_notconv=True)
    u = torch.empty(problem.n_dofs, dtype=torch.float64, device="cuda")
    c = fg.feti_recover_displacements(s.ctx, u, True)
    return u.cpu().numpy(), st, c, s


def lambda_perm(op, layout, method):
    """perm[i] = oracle row of library multiplier i (signs checked)."""
    key_to_row = {}
    for l, ent in enumerate(op.cons.entries):
        key = []
        for (s, k, sg) in ent:
            ld = int(op.r_loc[s][k]) if method == "fetidp" else int(k)
            key.append((int(s), ld, int(sg)))
        key_to_row[tuple(key)] = l
    perm = np.empty(layout.shape[0], np.int64)
    for i, row in enumerate(layout):
        key = [(int(row[0]), int(row[1]), int(row[2]))]
        if row[3] >= 0:
            key.append((int(row[3]), int(row[4]), int(row[5])))
        perm[i] = key_to_row[tuple(key)]
    assert np.unique(perm).size == perm.size
    return perm


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
