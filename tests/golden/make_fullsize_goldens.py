"""Writes the full-size goldens of the dual operator, the preconditioner and the
3D solution.  Calls only the oracle (oracle/) and the seeded generators
(workloads); no value comes from the CUDA library.

  fullsize_config2.npz   16x16 tiles of 32x32 Q4, 4 binary modules (contrast 1e9):
                         sampled rows of F X for a 256-column block (Eq. 12), the
                         preconditioner columns Z and z = Z 1 of a residual at those
                         rows (Eq. 13), and the error-bound scales below
  fullsize_config4.npz   8^3 tiles of 8^3 H8, smoothed field (contrast 1e9):
                         sampled rows of F X for a 512-column block and the bound scales
  solve_config2.npz      the bench workload's own solve (FETI-DP + k + Algorithm 1,
                         tol 1e-6) at 4096 sampled DOFs and its compliance, and the same
                         for the solve with the moduli perturbed at the unit roundoff
  solve_config4_4x4x4.npz  4^3 tiles of 8^3 H8 (same field recipe): Algorithm 1
                         (FETI-DP, k-scaling) solution at tol 1e-10, the same solve
                         with the densities perturbed at the unit roundoff (below), the
                         sparse direct solution of Eq. 2, and the scaled condition number

Test blocks are workloads.multiplier_block of each multiplier's canonical
(subdomain, DOF) pair, so the GPU test rebuilds them from the library's own
multiplier layout; stored rows are multiplied by the oracle's sign on the
row's canonical first copy (the test does the same with the library's sign).

Tolerance scales (per sampled row i and column j; x_s = B_s^T X_j, the interface
vector of subdomain s; V = Kbar_cc^{-1} F_rc^T X the coarse correction):

  A_loc = sum over the copies (s, k) of row i of (|F_s| |x_s|)_k + (|F_rc,s| |V_s|)_k
          -- rounding of the local products: an implementation that rounds F_s,
          F_rc, x and V to a format of unit roundoff u_f and accumulates K terms in
          FP32 is off by at most (2 u_f + (K + 8) u_32) A_loc (first order).
  A_cc  = sum over (s, k) of (|F_rc,s| |Kbar^{-1}| c~)_k, c~ = sum_s B_c,s^T |F_rc,s|^T |x_s|
          -- an error (u_x + n u_32) |F_rc|^T |x| in the corner reduction reaches Y
          through the exact coarse solve, at most (u_x + n u_32) A_cc.
  Y_pert (and Z_pert) -- the conditioning of the FP64 operator itself.  F_s, F_rc
          and Kbar_cc come from inverses of the local stiffness; the normwise bound
          n u kappa_2 of a Cholesky-based inverse is vacuous here (the diagonally
          scaled local stiffness has kappa_2 ~ 1e12 at contrast 1e9, so n u kappa ~ 1).
          Instead the oracle is run a second time with every density multiplied by
          (1 + 2u xi_e / p), xi_e ~ U[-1, 1] seeded (each SIMP modulus moved by ~2u, u =
          2^-53): the change Y_pert - Y is a one-sample statistical estimate of how far
          an FP64 perturbation of the inputs moves the output (Kenney and Laub, "Small-
          sample statistical condition estimates for general matrix functions", SIAM
          J. Sci. Comput. 15, 1994).  The test scales it by the local problem size n_r
          (a factorization's backward error is ~n u rather than 2u).

Run from the repository root:
    python tests/golden/make_fullsize_goldens.py config2|config4|solve4|solve2
"""
import gc
import os
import sys
import time

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402
from oracle.assemble import direct_solve, global_stiffness  # noqa: E402
from oracle.fetidp import FETIDP  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
U64 = 2.0 ** -53
SEED_X, SEED_R, SEED_ROWS, SEED_PERT = 2111, 11728, 2026, 53
N_ROWS = 256


def log(*a):
    print(f"[{time.strftime('%H:%M:%S')}]", *a, flush=True)


def sample_rows(op, rng, n):
    """n multiplier rows: three quarters uniformly, one quarter among the rows of
    DOFs shared by three or more subdomains (the pair-wise redundant cross-point rows)."""
    multi = np.array([len(sh) >= 3 for sh in op.cons.sharing])
    n_multi = min(n // 4, int(multi.sum()))
    a = rng.choice(np.flatnonzero(multi), n_multi, replace=False) if n_multi else np.zeros(0, np.int64)
    rest = np.setdiff1d(np.arange(op.n_lam), a)
    b = rng.choice(rest, n - n_multi, replace=False)
    return np.sort(np.concatenate([a, b]).astype(np.int64))


def perturbed(problem, seed):
    """The problem with every density moved by a relative 2u xi_e / p (see above)."""
    import copy
    q = copy.copy(problem)
    xi = np.random.default_rng(seed).uniform(-1.0, 1.0, problem.rho.size)
    q.rho = problem.rho * (1.0 + 2.0 * U64 * xi / problem.p)
    return q


def operator_golden(problem, build, m, with_precond):
    """Rows of F X (and of the perturbed operator's F X), the rounding scales and,
    optionally, the preconditioner columns.  ``build(problem)`` returns the oracle's
    FETI-DP operator; the perturbed one is built and released first, so that only
    one full set of local blocks is held at a time."""
    op_pert = build(perturbed(problem, SEED_PERT))
    ent = op_pert.row_entries()
    keys, sign = workloads.multiplier_pairs(ent)
    rows = sample_rows(op_pert, np.random.default_rng(SEED_ROWS), N_ROWS)
    log("test block", op_pert.n_lam, "x", m)
    X = workloads.multiplier_block(keys, sign, m, seed=SEED_X)
    log("perturbed F X at", rows.size, "rows")
    Yp = op_pert.apply_F_rows(X, rows)
    if with_precond:
        r = workloads.multiplier_block(keys, sign, 1, seed=SEED_R)[:, 0]
        Zp = op_pert.precond_columns(r)
    del op_pert
    gc.collect()
    op = build(problem)
    assert np.array_equal(ent, op.row_entries())
    n_lam, ns = op.n_lam, op.n_sub
    log("F X at", rows.size, "rows")
    Y = op.apply_F_rows(X, rows)
    # corner reduction and coarse correction, per subdomain
    C = np.zeros((op.n_c, m))
    Ct = np.zeros((op.n_c, m))       # c~ = sum B_c^T |F_rc|^T |x_s|
    touched = set(int(s) for s in ent[rows][:, [0, 3]].ravel() if s >= 0)
    cache = {}
    for s in range(ns):
        M = op.mod(s)
        xs = op.Br[s][:, op.bset[s]].T @ X                         # [n_b, m]
        cg = op.c_glob[s]
        if cg.size:
            np.add.at(C, cg, M.Frc_b.T @ xs)
            np.add.at(Ct, cg, np.abs(M.Frc_b).T @ np.abs(xs))
        if s in touched:
            cache[s] = xs
    V = sla.cho_solve(op.Kbar_cho, C)
    cc = np.abs(sla.cho_solve(op.Kbar_cho, np.eye(op.n_c))) @ Ct
    R = rows.size
    A_loc = np.zeros((R, m))
    A_cc = np.zeros((R, m))
    for t in (0, 3):
        for ii, l in enumerate(rows):
            s = int(ent[l, t])
            if s < 0:
                continue
            M = op.mod(s)
            b = op.bset[s]
            kk = int(np.flatnonzero(op.r_loc[s][b] == ent[l, t + 1])[0])   # the copy's place in b
            cg = op.c_glob[s]
            A_loc[ii] += np.abs(M.Fb[kk]) @ np.abs(cache[s])
            if cg.size:
                fr = np.abs(M.Frc_b[kk])
                A_loc[ii] += fr @ np.abs(V[cg])
                A_cc[ii] += fr @ cc[cg]
    sha = np.frombuffer(__import__("hashlib").sha1(problem.rho.tobytes()).digest(), np.uint8)
    out = dict(keys=keys[rows], Y=sign[rows, None] * Y, Y_pert=sign[rows, None] * Yp,
               A_loc=A_loc.astype(np.float32), A_cc=A_cc.astype(np.float32), m=np.int64(m),
               n_lam=np.int64(n_lam), n_c=np.int64(op.n_c), seed_x=np.int64(SEED_X), rho_sha1=sha,
               n_r_max=np.int64(max(r.size for r in op.r_loc)), n_b_max=np.int64(max(b.size for b in op.bset)))
    if with_precond:
        log("preconditioner columns")
        Z = op.precond_columns(r)
        out.update(seed_r=np.int64(SEED_R), Z=sign[rows, None] * Z[rows], z=sign[rows] * Z.sum(axis=1)[rows],
                   Z_pert=sign[rows, None] * Zp[rows], z_pert=sign[rows] * Zp.sum(axis=1)[rows])
    return out


def config2():
    p = workloads.config2()
    log("oracle FETI-DP builds, config 2")
    out = operator_golden(p, lambda q: FETIDP(q, "k"), 256, with_precond=True)
    path = os.path.join(HERE, "fullsize_config2.npz")
    np.savez_compressed(path, **out)
    log(path)


def config4():
    p = workloads.config4()
    log("oracle FETI-DP operator builds, config 4 (operator only)")
    out = operator_golden(p, lambda q: FETIDP(q, "k", operator_only=True), 512, with_precond=False)
    path = os.path.join(HERE, "fullsize_config4.npz")
    np.savez_compressed(path, **out)
    log(path)


def solve4():
    """Algorithm 1 on the 4^3-tile version of the 3D recipe, and the scaled
    condition number kappa_2(D^-1/2 K D^-1/2) of its free-DOF stiffness (the
    factor that turns round-off into displacement error)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    p = workloads.config4(tiles=4)
    log("oracle solve, 4^3 tiles of 8^3")
    u, lam, info, op = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-10, max_iter=200)
    log("iterations", info.iterations, "converged", info.converged, "eps", info.eps_history[-1])
    ud = direct_solve(p)
    K = global_stiffness(p)
    free = np.flatnonzero(p.dirichlet == 0)
    Kff = K[free][:, free].tocsc()
    dinv = sp.diags(1.0 / np.sqrt(Kff.diagonal()))
    Kh = (dinv @ Kff @ dinv).tocsc()
    hi = spla.eigsh(Kh, k=1, which="LA", return_eigenvectors=False)[0]
    lo = spla.eigsh(Kh, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    log("scaled kappa", hi / lo)
    u_pert, _, info_p, _ = oracle.solve(perturbed(p, SEED_PERT), "fetidp", "k", "rrs", tol=1e-10, max_iter=200)
    log("perturbed solve", info_p.iterations, "iterations; moved by", np.linalg.norm(u_pert - u) / np.linalg.norm(u))
    out = dict(u_oracle=u, u_direct=ud, u_pert=u_pert, iterations=np.int64(info.iterations),
               converged=np.bool_(info.converged),
               eps=np.array(info.eps_history), ranks=np.array(info.ranks), kappa_scaled=np.float64(hi / lo),
               n_free=np.int64(free.size), tol=np.float64(1e-10),
               rho_sha1=np.frombuffer(__import__("hashlib").sha1(p.rho.tobytes()).digest(), np.uint8))
    path = os.path.join(HERE, "solve_config4_4x4x4.npz")
    np.savez_compressed(path, **out)
    log(path, "oracle vs direct", np.linalg.norm(u - ud) / np.linalg.norm(ud))


def solve2():
    """The bench workload's own solve (FETI-DP + k + Algorithm 1 at relative
    tolerance 1e-6): the oracle's displacements at 4096 seeded DOFs, its
    compliance and norms, and the same for the solve with the moduli perturbed
    at the unit roundoff (how far FP64 round-off moves this solve)."""
    p = workloads.config2()
    log("oracle solve, config 2")
    u, lam, info, op = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-6)
    log("iterations", info.iterations, "ranks", info.ranks)
    del op
    gc.collect()
    u_pert, _, info_p, _ = oracle.solve(perturbed(p, SEED_PERT), "fetidp", "k", "rrs", tol=1e-6)
    log("perturbed solve", info_p.iterations, "iterations; moved by", np.linalg.norm(u_pert - u) / np.linalg.norm(u))
    free = np.flatnonzero(p.dirichlet == 0)
    idx = np.sort(np.random.default_rng(SEED_ROWS).choice(free, 4096, replace=False))
    out = dict(dof=idx, u_oracle=u[idx], u_pert=u_pert[idx], u_norm=np.float64(np.linalg.norm(u)),
               pert_norm=np.float64(np.linalg.norm(u_pert - u)), pert_max=np.float64(np.abs(u_pert - u).max()),
               u_max=np.float64(np.abs(u).max()), compliance=np.float64(p.f @ u),
               compliance_pert=np.float64(p.f @ u_pert), iterations=np.int64(info.iterations),
               iterations_pert=np.int64(info_p.iterations), ranks=np.array(info.ranks), tol=np.float64(1e-6),
               n_r_max=np.int64(2 * 33 * 33 - 8),
               rho_sha1=np.frombuffer(__import__("hashlib").sha1(p.rho.tobytes()).digest(), np.uint8))
    path = os.path.join(HERE, "solve_config2.npz")
    np.savez_compressed(path, **out)
    log(path)


if __name__ == "__main__":
    {"config2": config2, "config4": config4, "solve4": solve4, "solve2": solve2}[sys.argv[1]]()
