"""Krylov solvers for the FETI dual problems (oracle).

Test infrastructure only (see the package docstring).

``solve_dual`` carries out Algorithm 1 (Rank-Revealing Simultaneous FETI,
Section 3.3) in the paper's order.  Starting from the projected residual of
lambda_0, each subdomain contributes its own preconditioned residual as a
search direction (the columns of Z, projected by P to give W).  One pass of
the loop: apply F to the whole block W to get Q; form the Gram matrix
Delta = Q^T W; factor it with a pivoted, rank-revealing Cholesky and keep
only the independent directions, mapping W and Q through the inverse of the
retained triangular factor so the kept block is F-orthonormal; step the
multiplier and the residual along the block with the coefficients W^T r;
precondition the new residual column by column; and F-orthogonalise the new
block against every stored block in turn (modified Gram-Schmidt, oldest
first).  The loop stops when sqrt(r^T Z 1) is small enough.

The three Krylov variants of the paper (Sections 3.2-3.3) are this loop with:
  "rrs": as printed (one direction per subdomain, full history);
  "fo":  the single direction w = W 1 = P Z 1 (Section 3.3) and the full
         history loop (full orthogonalization, Section 3.2);
  "pcg": the single direction and orthogonalization against the previous
         direction only, which is projected PCG with F-normalised directions.

Readings (the paper is silent on them):
* eps is relative: stop when sqrt(r_i^T Z_i 1) <= tol * sqrt(r_0^T Z_0 1).
* lambda~_0 = 0 and the returned multiplier is lambda_0 + lambda~.
* Rank-revealing Cholesky: diagonal pivoting on the remaining Schur
  complement, measured relative to each column's own Delta_jj (so that the
  test for linear dependence does not depend on the scale of a direction);
  the largest ratio is taken next, exact ties going to the lowest original
  column; stop when the best ratio is <= rr_tol.  Columns with
  Delta_jj <= (2^-52)^2 * max Delta are treated as zero and never taken.

Pins (tests/test_oracle_dual.py): the PCG variant equals a textbook projected
PCG; F-orthonormality of every kept block and F-orthogonality to every stored
block; the rank-revealing factorization against a brute-force subset search;
all twelve variants reach the direct solution; the qualitative finding that
plain TFETI stalls at high contrast while FETI-DP + k + Algorithm 1 converges.
"""
import dataclasses
from typing import List

import numpy as np
import scipy.linalg as sla

EPS2 = np.finfo(np.float64).eps ** 2


@dataclasses.dataclass
class KrylovInfo:
    iterations: int = 0
    converged: bool = False
    breakdown: bool = False
    eps_history: List[float] = dataclasses.field(default_factory=list)
    ranks: List[int] = dataclasses.field(default_factory=list)
    f_applies: int = 0        # columns of F applied


def rank_revealing_cholesky(Delta, rr_tol):
    """Rank-revealing pivoted Cholesky of the Gram matrix (Algorithm 1).

    Returns (perm, k, Lt) with Delta[perm][:, perm][:k, :k] = Lt Lt^T."""
    A = np.array(Delta, dtype=np.float64, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    d0 = np.diag(A).copy()
    dmax = d0.max() if n else 0.0
    alive = d0 > EPS2 * dmax if dmax > 0 else np.zeros(n, bool)
    L = np.zeros((n, n))
    k = 0
    for j in range(n):
        best, bt = -np.inf, -1
        for t in range(j, n):
            if not alive[perm[t]]:
                continue
            ratio = A[t, t] / d0[perm[t]]
            if ratio > best or (ratio == best and perm[t] < perm[bt]):
                best, bt = ratio, t
        if bt < 0 or not (best > rr_tol):
            break
        if bt != j:   # symmetric swap of positions j and bt
            A[[j, bt], :] = A[[bt, j], :]
            A[:, [j, bt]] = A[:, [bt, j]]
            L[[j, bt], :j] = L[[bt, j], :j]
            perm[[j, bt]] = perm[[bt, j]]
        piv = np.sqrt(A[j, j])
        L[j, j] = piv
        L[j + 1:, j] = A[j + 1:, j] / piv
        A[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], L[j + 1:, j])
        k = j + 1
    return perm, k, L[:k, :k]


def solve_dual(op, tol=1e-6, max_iter=500, rr_tol=1e-10, variant="rrs", lam0=None, callback=None):
    """Algorithm 1 on a FETI operator object ``op`` (TFETI or FETIDP).

    ``callback(stage, i, data)`` (tests only) sees the F-orthonormalised block
    right after the rank-revealing step (stage "orth", data = (W_i, Q_i)) and
    the new block after the full-orthogonalization loop (stage "conj",
    data = (W_{i+1}, history)).
    """
    lam0 = op.lam0 if lam0 is None else lam0
    info = KrylovInfo()

    def directions(r):
        Z = op.precond_columns(r)
        return Z if variant == "rrs" else Z.sum(axis=1, keepdims=True)

    r = op.project_T(op.d - op.apply_F(lam0[:, None])[:, 0])
    Z = directions(r)
    W = op.project(Z)
    lam_t = np.zeros_like(lam0)
    hist = []
    eps = np.sqrt(max(r @ Z.sum(axis=1), 0.0))
    eps0 = eps
    info.eps_history.append(eps)
    i = 0
    while eps > tol * eps0 and i < max_iter:
        Q = op.apply_F(W)
        info.f_applies += W.shape[1]
        Delta = Q.T @ W
        Delta = 0.5 * (Delta + Delta.T)
        perm, k, Lt = rank_revealing_cholesky(Delta, rr_tol)
        info.ranks.append(k)
        if k == 0 or not np.all(np.isfinite(Lt)):
            info.breakdown = True
            break
        T = np.zeros((W.shape[1], k))
        T[perm[:k], :] = sla.solve_triangular(Lt, np.eye(k), lower=True).T    # N^T [L~^{-T}; 0]
        W = W @ T
        Q = Q @ T
        if callback:
            callback("orth", i, (W, Q))
        gamma = W.T @ r
        lam_t = lam_t + W @ gamma
        r = r - op.project_T(Q @ gamma)
        Z = directions(r)
        hist.append((W, Q))
        Wn = op.project(Z)
        js = range(len(hist)) if variant in ("rrs", "fo") else [len(hist) - 1]
        for j in js:
            Wj, Qj = hist[j]
            Psi = Qj.T @ Wn
            Wn = Wn - Wj @ Psi
        W = Wn
        if callback:
            callback("conj", i, (W, hist))
        i += 1
        eps = np.sqrt(max(r @ Z.sum(axis=1), 0.0))
        info.eps_history.append(eps)
        if not np.isfinite(eps):
            info.breakdown = True
            break
    info.iterations = i
    info.converged = bool(eps <= tol * eps0)
    return lam0 + lam_t, info
