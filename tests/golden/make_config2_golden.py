"""Writes config2_fetidp_k_rrs.json: the oracle's FETI-DP + k-scaling + RRS
solution of the full modular workload (16x16 subdomains of 32x32 Q4, contrast
1e9) at relative tolerance 1e-6, sampled at 256 seeded DOFs, plus the same DOFs
of a sparse direct solve of Eq. 2.  Calls only the oracle.

Run from the repository root:  python tests/golden/make_config2_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402
from oracle.assemble import direct_solve  # noqa: E402


def main():
    p = workloads.config2()
    u, lam, info, op = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-6)
    ud = direct_solve(p)
    rng = np.random.Generator(np.random.PCG64(2026))
    free = np.flatnonzero(p.dirichlet == 0)
    idx = np.sort(rng.choice(free, 256, replace=False))
    out = {
        "workload": "config2: 16x16 subdomains of 32x32 Q4, 4 binary modules, contrast 1e9",
        "method": "FETI-DP, k-scaling, rank-revealing S-FETI, rel. tol 1e-6, rr_tol 1e-10",
        "iterations": info.iterations, "ranks": info.ranks, "eps_history": info.eps_history,
        "f_applies": info.f_applies, "n_lambda": op.n_lam,
        "dof": idx.tolist(), "u_oracle": u[idx].tolist(), "u_direct": ud[idx].tolist(),
        "u_oracle_norm2": float(np.linalg.norm(u)), "u_direct_norm2": float(np.linalg.norm(ud)),
        "u_oracle_maxabs": float(np.abs(u).max()),
        "rel_err_oracle_vs_direct": float(np.linalg.norm(u - ud) / np.linalg.norm(ud)),
        "compliance_oracle": float(p.f @ u), "compliance_direct": float(p.f @ ud),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_fetidp_k_rrs.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
