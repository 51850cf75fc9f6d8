"""Subdomain-sharded Algorithm 1 for FETI-DP and TFETI on CPU ranks (oracle).

Test infrastructure only (see the package docstring): a check, on gloo ranks
of torch.distributed, that the multi-GPU layout of the method gives the
serial result.  Nothing on the GPU path imports it.

The layout (one rank per GPU):
* rank r owns a contiguous block of subdomains in lexicographic tile order
  (slabs along the slowest axis) and every multiplier row whose lowest
  subdomain it owns;
* direction blocks W, Q, the residual, lambda~ and the stored history are
  partitioned by rows; the Gram-type products Delta = Q^T W, gamma = W^T r,
  Psi_j = Q_j^T W and r^T z are partial sums over owned rows, summed across
  ranks (all-reduce of m x m or m x 1 blocks); the rank-revealing
  factorization of Delta runs redundantly on every rank (same input, same
  result) and the transforms and updates are row-local;
* the dual-operator apply (Eq. 12) needs, for an owned subdomain, the rows of
  W it touches that other ranks own (a halo), produces its local products, a
  partial coarse right-hand side sum_s F_rc,s^T X_b(s) (all-reduced, then the
  coarse solve is replicated) and contributions to rows owned elsewhere
  (returned to their owners); the preconditioner columns (Eq. 13) likewise;
* TFETI: the rows of G = -R^T B^T belong to their subdomain's rank; G X is a
  partial (rigid modes x m) block per rank, all-reduced, and the small solve
  with G G^T is replicated; G^T t is row-local.
Here each exchange is written as a sum-all-reduce of a full-length array in
which every rank fills only what it contributes (a row is contributed by its
owner, a column of Z by the owner of its subdomain); the bytes a real halo
exchange would move are counted separately.

Pin (tests/test_sharded_cpu.py): on 2 and 3 ranks the same iterations and
retained ranks as the serial Algorithm 1 of krylov.py and the same solution.
"""
import dataclasses

import numpy as np
import scipy.linalg as sla
import torch
import torch.distributed as dist

from .krylov import KrylovInfo, rank_revealing_cholesky


@dataclasses.dataclass
class ShardStats:
    halo_rows: int = 0           # multiplier rows this rank reads but does not own
    owned_rows: int = 0
    owned_subdomains: int = 0
    halo_bytes: int = 0          # point-to-point volume of the halo exchanges (both directions)
    allreduce_bytes: int = 0     # payload of the small all-reduces (coarse RHS, Gram-type blocks)


def _allreduce(a):
    """Sum over ranks into a new array (the argument is left untouched)."""
    t = torch.from_numpy(np.array(a, dtype=np.float64, copy=True))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def partition(op, world):
    """Owner rank of every subdomain (contiguous blocks) and of every multiplier row."""
    ns = op.n_sub
    sub_owner = np.array([s * world // ns for s in range(ns)])
    row_owner = np.array([sub_owner[min(s for (s, _, _) in ent)] for ent in op.cons.entries])
    return sub_owner, row_owner


def solve_dual_sharded(op, tol=1e-6, max_iter=500, rr_tol=1e-10):
    """Algorithm 1 (one direction per subdomain, full orthogonalization) on the
    current process group, for a FETIDP or TFETI operator object.  Returns
    (lambda on every rank, KrylovInfo, ShardStats)."""
    tfeti = hasattr(op, "G")
    rank, world = dist.get_rank(), dist.get_world_size()
    sub_owner, row_owner = partition(op, world)
    mine = np.flatnonzero(sub_owner == rank)
    own = row_owner == rank
    nl = op.n_lam
    Bsub = op.B if tfeti else op.Br                 # signed B^s (TFETI) or B_r^s (FETI-DP)
    touched = np.zeros(nl, bool)
    for s in mine:
        touched[np.unique(Bsub[s].tocoo().row)] = True
    stats = ShardStats(halo_rows=int(np.count_nonzero(touched & ~own)), owned_rows=int(own.sum()),
                       owned_subdomains=int(mine.size))

    def rows(x):                    # keep this rank's rows of a full-length block
        y = np.zeros_like(x)
        y[own] = x[own]
        return y

    def gather_full(x_part, m):     # halo: every rank assembles the rows it reads
        stats.halo_bytes += 2 * stats.halo_rows * m * 8
        return _allreduce(x_part)

    def apply_F(W_part):
        m = W_part.shape[1]
        X = gather_full(W_part, m)
        if tfeti:                   # F = sum_s B^s K^+_s B^sT (Eq. 7)
            Yp = np.zeros((nl, m))
            for s in mine:
                Yp += op.B[s] @ (op.Kp[s] @ (op.B[s].T @ X))
            stats.halo_bytes += 2 * stats.halo_rows * m * 8
            return rows(_allreduce(Yp))
        Vp = np.zeros((op.n_c, m))
        for s in mine:
            Bb = op.Br[s][:, op.bset[s]]
            np.add.at(Vp, op.c_glob[s], op.mod(s).Frc_b.T @ (Bb.T @ X))
        stats.allreduce_bytes += Vp.size * 8
        V = sla.cho_solve(op.Kbar_cho, _allreduce(Vp))
        Yp = np.zeros((nl, m))
        for s in mine:
            Bb = op.Br[s][:, op.bset[s]]
            M = op.mod(s)
            Yp += Bb @ (M.Fb @ (Bb.T @ X) + M.Frc_b @ V[op.c_glob[s]])
        stats.halo_bytes += 2 * stats.halo_rows * m * 8
        return rows(_allreduce(Yp))     # contributions to rows owned elsewhere go to their owners

    def precond_columns(r_part):
        r = gather_full(r_part[:, None], 1)[:, 0]
        Zp = np.zeros((nl, op.n_sub))
        for s in mine:
            Bt = (op.Bt if tfeti else op.Brt)[s][:, op.bset[s]]
            Zp[:, s] = Bt @ (op.precond_block(s) @ (Bt.T @ r))
        stats.halo_bytes += 2 * stats.halo_rows * mine.size * 8
        return rows(_allreduce(Zp))

    def project(X_part):            # P X = X - G^T (G G^T)^{-1} G X (TFETI; identity for FETI-DP)
        if not tfeti:
            return X_part
        m = X_part.shape[1]
        X = gather_full(X_part, m)
        nr = op.n_rbm
        GXp = np.zeros((op.G.shape[0], m))
        for s in mine:
            GXp[s * nr:(s + 1) * nr] = op.G[s * nr:(s + 1) * nr] @ X
        stats.allreduce_bytes += GXp.size * 8
        t = sla.cho_solve(op.GGt_cho, _allreduce(GXp))
        return X_part - rows(op.G.T @ t)

    def dot(a, b):
        stats.allreduce_bytes += 8
        return float(_allreduce(np.array([a[own] @ b[own]]))[0])

    def gram(A, B):                 # A^T B over all rows
        p = A[own].T @ B[own]
        stats.allreduce_bytes += p.size * 8
        return _allreduce(p)

    info = KrylovInfo()
    lam0 = op.lam0                  # FETI-DP: 0; TFETI: G^T (G G^T)^{-1} e (replicated set-up)
    r0 = rows(op.d)[:, None] - apply_F(rows(lam0)[:, None])      # d - F lambda_0 on the owned rows
    r = project(r0)[:, 0]
    Z = precond_columns(r)
    W = project(Z)
    lam_t = np.zeros(nl)
    hist = []
    eps = np.sqrt(max(dot(r, Z.sum(axis=1)), 0.0))
    eps0 = eps
    info.eps_history.append(eps)
    i = 0
    while eps > tol * eps0 and i < max_iter:
        Q = apply_F(W)
        info.f_applies += W.shape[1]
        Delta = gram(Q, W)
        Delta = 0.5 * (Delta + Delta.T)
        perm, k, Lt = rank_revealing_cholesky(Delta, rr_tol)
        info.ranks.append(k)
        if k == 0 or not np.all(np.isfinite(Lt)):
            info.breakdown = True
            break
        T = np.zeros((W.shape[1], k))
        T[perm[:k], :] = sla.solve_triangular(Lt, np.eye(k), lower=True).T
        W, Q = W @ T, Q @ T
        gamma = gram(W, r[:, None])[:, 0]
        lam_t = lam_t + W @ gamma
        r = r - project((Q @ gamma)[:, None])[:, 0]
        Z = precond_columns(r)
        hist.append((W, Q))
        Wn = project(Z)
        for Wj, Qj in hist:
            Wn = Wn - Wj @ gram(Qj, Wn)
        W = Wn
        i += 1
        eps = np.sqrt(max(dot(r, Z.sum(axis=1)), 0.0))
        info.eps_history.append(eps)
        if not np.isfinite(eps):
            info.breakdown = True
            break
    info.iterations = i
    info.converged = bool(eps <= tol * eps0)
    lam = lam0 + _allreduce(lam_t)
    return lam, info, stats
