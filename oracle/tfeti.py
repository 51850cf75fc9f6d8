"""Total FETI (Section 2.1, Eqs. 4-7) with the Dirichlet preconditioner (oracle).

Test infrastructure only (see the package docstring).

Every subdomain keeps all of its DOFs and floats: Dirichlet conditions are
rows of B with the prescribed value in c (Eq. 4).  With K^+ the
Moore-Penrose pseudo-inverse of the block-diagonal K and R its null-space
basis (rigid-body modes, 3 per subdomain in 2D, 6 in 3D), the dual problem
is Eq. (7):

    [F  G^T] [lambda]   [d]      F = B K^+ B^T,   d = B K^+ f - c,
    [G  0  ] [alpha ] = [e],     G = -R^T B^T,    e = -R^T f,

solved by PCG projected with P = I - G^T (G G^T)^{-1} G (Section 3.3), from
lambda_0 = G^T (G G^T)^{-1} e.  The primal solution follows from the first
row of Eq. (6): u = K^+ (f - B^T lambda) + R alpha, with alpha from the
first row of Eq. (7): G^T alpha = d - F lambda.

Reading (a DOF that is both fixed and shared): each copy of a fixed DOF gets
its own Dirichlet row and no continuity row is added for it, so B has full
row rank apart from the pair-wise redundancy at cross points.

Pins (tests/test_oracle_dual.py): the dense saddle systems of Eqs. (6)-(7),
K^+ against an SVD pseudo-inverse, the rigid-body null space of floating
subdomains, the projector identities and G lambda_0 = e, the direct solution.
"""
import numpy as np
import scipy.linalg as sla

from .assemble import local_dirichlet, local_load, local_stiffness, mesh_of, gather_global, element_moduli
from .fem import element_stiffness, rigid_body_modes
from .scaling import Constraints, pairwise_rows, row_weights


def moore_penrose_psd(K, R):
    """Moore-Penrose pseudo-inverse of a symmetric PSD K whose null space is
    exactly span(R): with Rh an orthonormal basis of span(R),
    K^+ = (K + Rh Rh^T)^{-1} - Rh Rh^T (the two terms act on orthogonal
    complements).  The tests pin it against an SVD pseudo-inverse."""
    Rh, _ = np.linalg.qr(R)
    PR = Rh @ Rh.T
    Kp = np.linalg.inv(K + PR) - PR
    return 0.5 * (Kp + Kp.T)


def schur_complement(K, bset):
    """S = K_bb - K_bi K_ii^{-1} K_ib for the DOF subset ``bset`` (Eq. 13)."""
    n = K.shape[0]
    mask = np.zeros(n, bool)
    mask[bset] = True
    iset = np.flatnonzero(~mask)
    Kbb = K[np.ix_(bset, bset)]
    if iset.size == 0:
        return Kbb
    Kib = K[np.ix_(iset, bset)]
    Kii = K[np.ix_(iset, iset)]
    return Kbb - Kib.T @ sla.cho_solve(sla.cho_factor(Kii, lower=True), Kib)


class TFETI:
    def __init__(self, problem, scaling="k", precond="dirichlet"):
        if precond not in ("dirichlet", "lumped", "superlumped"):
            raise ValueError(precond)
        self.precond = precond
        self.problem = problem
        mesh = self.mesh = mesh_of(problem)
        dim = self.dim = problem.dim
        k0 = element_stiffness(dim, problem.nu)
        E = element_moduli(problem)
        ns = self.n_sub = mesh.n_sub
        self.n_loc = mesh.n_loc_dofs
        self.K = [local_stiffness(problem, mesh, s, k0, E) for s in range(ns)]
        self.f = [local_load(problem, mesh, s) for s in range(ns)]
        self.R = [rigid_body_modes(mesh.local_node_coords(s).astype(np.float64)) for s in range(ns)]
        self.Kp = [moore_penrose_psd(self.K[s], self.R[s]) for s in range(ns)]
        # --- constraints B u = c (Eq. 4) ---
        entries, sharing, cvals = [], [], []
        for gn in range(mesh.n_nodes):
            own = mesh.owners[gn]
            for d in range(dim):
                g = gn * dim + d
                copies = [(s, ln * dim + d) for (s, ln) in own]
                if problem.dirichlet[g]:
                    for (s, k) in copies:
                        entries.append([(s, k, 1.0)])
                        sharing.append([(s, k)])
                        cvals.append(0.0)
                elif len(copies) >= 2:
                    for row in pairwise_rows(copies):
                        entries.append(row)
                        sharing.append(copies)
                        cvals.append(0.0)
        self.cons = Constraints(entries, sharing, np.array(cvals))
        self.n_lam = self.cons.n_lam
        self.B = [self.cons.B_sub(s, self.n_loc) for s in range(ns)]
        diagK = [np.diag(Ks).copy() for Ks in self.K]
        self.weights = row_weights(self.cons, diagK, scaling)
        self.Bt = [self.cons.B_sub(s, self.n_loc, self.weights) for s in range(ns)]
        # --- Dirichlet preconditioner pieces (Eq. 13): b = DOFs touched by B ---
        self.bset = [np.unique(self.B[s].indices) for s in range(ns)]
        self.S = [schur_complement(self.K[s], self.bset[s]) for s in range(ns)]
        self.Kbb = [self.K[s][np.ix_(self.bset[s], self.bset[s])] for s in range(ns)]
        # --- G, e, d (Eq. 7) and the coarse matrix G G^T ---
        nr = self.R[0].shape[1]
        self.n_rbm = nr
        self.G = np.vstack([-(self.B[s] @ self.R[s]).T for s in range(ns)])    # [ns*nr, n_lam]
        self.e = np.concatenate([-(self.R[s].T @ self.f[s]) for s in range(ns)])
        self.GGt = self.G @ self.G.T
        self.GGt_cho = sla.cho_factor(self.GGt, lower=True)
        self.d = sum(self.B[s] @ (self.Kp[s] @ self.f[s]) for s in range(ns)) - self.cons.c
        self.lam0 = self.G.T @ sla.cho_solve(self.GGt_cho, self.e)

    # -- operators used by the Krylov solvers --------------------------------
    def apply_F(self, X):
        """F X = sum_s B^s K^+_s B^sT X for X [n_lam, m]."""
        X = np.atleast_2d(X.T).T
        return sum(self.B[s] @ (self.Kp[s] @ (self.B[s].T @ X)) for s in range(self.n_sub))

    def project(self, X):
        """P X with P = I - G^T (G G^T)^{-1} G."""
        return X - self.G.T @ sla.cho_solve(self.GGt_cho, self.G @ X)

    project_T = project   # P is symmetric

    def precond_block(self, s):
        """Dirichlet S^s (Eq. 13), lumped K_bb or super-lumped diag(K_bb)."""
        if self.precond == "dirichlet":
            return self.S[s]
        if self.precond == "lumped":
            return self.Kbb[s]
        return np.diag(np.diag(self.Kbb[s]))

    def precond_columns(self, r):
        """Z = [... , B~^s P^s B~^sT r, ...] one column per subdomain (the block preconditioner of Algorithm 1)."""
        Z = np.zeros((self.n_lam, self.n_sub))
        for s in range(self.n_sub):
            Bb = self.Bt[s][:, self.bset[s]]
            Z[:, s] = Bb @ (self.precond_block(s) @ (Bb.T @ r))
        return Z

    # -- dense forms for tiny problems (brute-force pins) -----------------------
    def dense(self):
        """Concatenated K (block diagonal), B, f, R, K^+ as dense arrays."""
        K = sla.block_diag(*self.K)
        B = np.hstack([Bs.toarray() for Bs in self.B])
        f = np.concatenate(self.f)
        R = sla.block_diag(*self.R)
        Kp = sla.block_diag(*self.Kp)
        return K, B, f, R, Kp

    # -- recovery -------------------------------------------------------------
    def recover_local(self, lam):
        """alpha from G^T alpha = d - F lambda, then u^s = K^+ (f^s - B^sT lambda) + R^s alpha_s."""
        alpha = sla.cho_solve(self.GGt_cho, self.G @ (self.d - self.apply_F(lam[:, None])[:, 0]))
        nr = self.n_rbm
        us = []
        for s in range(self.n_sub):
            us.append(self.Kp[s] @ (self.f[s] - self.B[s].T @ lam) + self.R[s] @ alpha[s * nr:(s + 1) * nr])
        return us, alpha

    def recover(self, lam):
        us, _ = self.recover_local(lam)
        return gather_global(self.mesh, self.dim, us, self.problem.dirichlet)
