"""FETI-DP (Section 2.2, Eqs. 8-12) with corner primal DOFs (oracle).

Test infrastructure only (see the package docstring).

Each subdomain's DOFs split into primal corner DOFs c and the remaining DOFs
r (Eq. 8); u_c^s = B_c^s u_c selects them from the global primal vector
(Eq. 9); continuity of the r-DOFs is B_r u_r = 0 (Eq. 10).  Eliminating u_r
from Eq. (11) gives Eq. (12):

    F_rr   = B_r K_rr^{-1} B_r^T          F_rc = B_r K_rr^{-1} K_rc
    Kbar_cc = K_cc - K_cr K_rr^{-1} K_rc  d_r  = B_r K_rr^{-1} f_r
    fbar_c  = f_c - K_cr K_rr^{-1} f_r

and condensing u_c (Section 2.2, last paragraph; u_c from the second row of
Eq. 12) the dual problem on lambda alone:

    (F_rr + F_rc Kbar_cc^{-1} F_rc^T) lambda = d_r - F_rc Kbar_cc^{-1} fbar_c.

Readings:
* Primal set: every non-fixed DOF at a vertex of the tile grid (the corner
  nodes of the regular partition, Section 2.2), including vertices on the
  outer boundary.
* Optional richer primal set (primal="edges"; the paper names richer and
  adaptive primal sets as future work, Section 5): in addition, one average
  per component over the interior nodes of every tile-grid edge shared by two
  or more subdomains (3D: the edges of the tiles; 2D: their sides) whose
  nodes are all free in that component.  It is introduced by a change of
  basis on each such edge with nodes e_1 .. e_n (ordered by the global
  coordinate along the edge): the new variables are the average ubar (stored
  in the slot of e_1) and the fluctuations v_j (j >= 2, in the slots of e_j),
  u_{e_1} = ubar - sum_j v_j,  u_{e_j} = ubar + v_j,  so u = T u^ with T
  identical on every sharer.  K^s and f^s are replaced by T^T K^s T and
  T^T f^s; ubar joins the primal DOFs (global, one per edge and component)
  and the fluctuations keep the pair-wise rows of B_r; the recovered u^ is
  mapped back by T.  The k-scaling weights use the diagonal of the
  untransformed K^s.
* Adaptive selection (primal="adaptive"; the paper names adaptive primal sets
  as future work, Section 5, without a rule): an edge of the "edges" reading
  gets its average in component d only where the stiffness jumps across it,
  i.e. where on some interior node of the edge the sharers' diagonal stiffness
  entries K^s_dd (the quantities k-scaling weighs) differ by a factor of at
  least ``jump_ratio`` (default 10).  Edges inside homogeneous material keep
  corners only; an edge where a stiff region meets a compliant one is averaged.
* The printed fbar_c carries the index "kk" on K^{-1}; it is read as K_rr.
* Fixed (Dirichlet) DOFs are eliminated from K^s; FETI-DP has no c-vector.
* K_rr^{-1} is only ever needed on the DOFs that B_r touches (the "b" DOFs)
  and on K_rc; the oracle forms those restrictions once per distinct
  subdomain matrix (identical modules share them, Section 1).

Pins: tests/test_oracle_dual.py (the blocks of Eq. 12 against the dense Eq. 11
and global inverses, module deduplication exact, the direct solution),
tests/test_oracle_precond.py (the three preconditioner blocks),
tests/test_oracle_edges.py (the edge-average reading: direct solution,
closed-form sizes, the primal value is the edge mean on every sharer; the
adaptive selection: its limits equal corners and all edges, direct solution,
fewer iterations than corners where the laminae meet the interfaces).
"""
import hashlib

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .assemble import local_dirichlet, local_load, local_stiffness, mesh_of, gather_global, element_moduli
from .fem import element_stiffness
from .scaling import Constraints, pairwise_rows, row_weights
from .tfeti import schur_complement


PRECONDS = ("dirichlet", "lumped", "superlumped")


class _Module:
    """Per-distinct-subdomain factorisation data (shared by identical modules).

    ``keep_factor=False`` keeps only the dense blocks the dual operator and the
    preconditioner use (F_s, F_rc restricted to b, the local Kbar_cc, S and
    K_bb) and releases K_rr, K_rc and the Cholesky factor: same blocks, less
    host memory (the right-hand sides and the recovery need the factor);
    K_bb is then kept only for the lumped preconditioners (keep_kbb)."""

    def __init__(self, Ks, r_loc, c_loc, b_in_r, keep_factor=True, keep_kbb=True):
        self.Krr = Ks[np.ix_(r_loc, r_loc)]
        self.Krc = Ks[np.ix_(r_loc, c_loc)]
        self.Kcc = Ks[np.ix_(c_loc, c_loc)]
        self.cho = sla.cho_factor(self.Krr, lower=True)
        nr = self.Krr.shape[0]
        Eb = np.zeros((nr, b_in_r.size))
        Eb[b_in_r, np.arange(b_in_r.size)] = 1.0
        KinvEb = sla.cho_solve(self.cho, Eb)
        self.KinvKrc = sla.cho_solve(self.cho, self.Krc)             # K_rr^{-1} K_rc   [nr, nc]
        self.Fb = KinvEb[b_in_r]                                       # [K_rr^{-1}]_bb  [nb, nb]
        self.Fb = 0.5 * (self.Fb + self.Fb.T)
        self.Frc_b = self.KinvKrc[b_in_r]                              # [K_rr^{-1} K_rc]_b
        self.Kbar = self.Kcc - self.Krc.T @ self.KinvKrc               # local Kbar_cc^s
        self.S = schur_complement(self.Krr, b_in_r)                    # Eq. (13) on r-DOFs
        self.Kbb = self.Krr[np.ix_(b_in_r, b_in_r)]                    # lumped: K_bb instead of S
        if not keep_factor:
            del self.Krr, self.Krc, self.Kcc, self.cho, self.KinvKrc
            if not keep_kbb:
                del self.Kbb


PRIMALS = ("corners", "edges", "adaptive")


def edge_stiffness_jump(mesh, dim, diagK, nodes, d):
    """The stiffness jump across an edge in component d: the largest, over the
    edge's interior nodes, ratio between the sharers' diagonal stiffness entries
    K^s_dd of that node (the quantities k-scaling weighs, Eq. 15)."""
    jump = 1.0
    for gn in nodes:
        vals = [diagK[s][ln * dim + d] for (s, ln) in mesh.owners[gn]]
        jump = max(jump, max(vals) / min(vals))
    return jump


def edge_averages(problem, mesh):
    """The averaged edges of the primal="edges" reading: a list of
    (nodes along the edge in increasing coordinate, component), one entry per
    edge and free component, for every tile-grid edge (nodes with exactly
    dim - 1 coordinates on tile-grid planes) shared by two or more subdomains."""
    dim = problem.dim
    coords = mesh.node_coords()
    edges = {}
    for gn in range(mesh.n_nodes):
        ijk = coords[gn]
        on = [ijk[a] % mesh.elems[a] == 0 for a in range(dim)]
        if sum(on) != dim - 1 or len(mesh.owners[gn]) < 2:
            continue
        run = on.index(False)
        start = list(ijk)
        start[run] -= ijk[run] % mesh.elems[run]
        edges.setdefault((run, tuple(start)), []).append((int(ijk[run]), gn))
    out = []
    for key in sorted(edges):
        nodes = [gn for _, gn in sorted(edges[key])]
        for d in range(dim):
            if not any(problem.dirichlet[gn * dim + d] for gn in nodes):
                out.append((nodes, d))
    return out


class FETIDP:
    def __init__(self, problem, scaling="k", dedup=True, precond="dirichlet", primal="corners",
                 operator_only=False, jump_ratio=10.0):
        """``operator_only``: build the blocks of the dual operator, the coarse
        matrix and the preconditioner only (no right-hand sides, no recovery),
        releasing each module's factor after use -- for operator-level checks at
        sizes where keeping every factor would not fit in host memory."""
        self.operator_only = operator_only
        if precond not in PRECONDS:
            raise ValueError(precond)
        if primal not in PRIMALS:
            raise ValueError(primal)
        self.precond = precond
        self.primal_set = primal
        self.problem = problem
        mesh = self.mesh = mesh_of(problem)
        dim = self.dim = problem.dim
        k0 = element_stiffness(dim, problem.nu)
        E = element_moduli(problem)
        ns = self.n_sub = mesh.n_sub
        # --- global primal numbering (Eq. 9) ---
        corner_nodes = [gn for gn in range(mesh.n_nodes) if mesh.is_tile_vertex(gn)]
        self.primal = {}
        for gn in corner_nodes:
            for d in range(dim):
                if not problem.dirichlet[gn * dim + d]:
                    self.primal[gn * dim + d] = len(self.primal)
        # the untransformed local stiffness (its diagonal gives the k-scaling weights
        # and the adaptive selection's stiffness jumps)
        Ks_raw = [local_stiffness(problem, mesh, s, k0, E) for s in range(ns)]
        self.diagK = [np.diag(K).copy() for K in Ks_raw]
        # edge averages: the primal unknown sits in the slot of the first edge node
        self.edges = edge_averages(problem, mesh) if primal in ("edges", "adaptive") else []
        if primal == "adaptive":
            self.edges = [(nodes, d) for nodes, d in self.edges
                          if edge_stiffness_jump(mesh, dim, self.diagK, nodes, d) >= jump_ratio]
        avg_dofs = set()
        for nodes, d in self.edges:
            self.primal[nodes[0] * dim + d] = len(self.primal)
            avg_dofs.add(nodes[0] * dim + d)
        self.n_c = len(self.primal)
        # --- per-subdomain split (Eq. 8) ---
        self.r_loc, self.c_loc, self.c_glob = [], [], []
        self.f_r, self.f_c = [], []
        self.mod_key = []
        self.modules = {}
        Ks_cache = {}
        self.T = []
        for s in range(ns):
            Ks = Ks_raw[s]
            Ks_raw[s] = None
            fs = local_load(problem, mesh, s)
            fixed = local_dirichlet(problem, mesh, s)
            g2 = mesh.local_to_global_nodes(s)
            is_corner = np.repeat(np.array([mesh.is_tile_vertex(g) for g in g2]), dim)
            gdofs = (g2[:, None] * dim + np.arange(dim)[None, :]).ravel()
            Ts = None
            if self.edges:
                loc_of = {int(g): ln for ln, g in enumerate(g2)}
                Ts = np.eye(mesh.n_loc_dofs)
                for nodes, d in self.edges:
                    if nodes[0] not in loc_of:
                        continue
                    l1 = loc_of[nodes[0]] * dim + d
                    for gn in nodes[1:]:
                        lj = loc_of[gn] * dim + d
                        Ts[l1, lj] = -1.0
                        Ts[lj, l1] = 1.0
                    is_corner[l1] = True                   # the average joins the primal set
                Ks = Ts.T @ Ks @ Ts
                fs = Ts.T @ fs
            self.T.append(Ts)
            r_loc = np.flatnonzero(~fixed & ~is_corner)
            c_loc = np.flatnonzero(~fixed & is_corner)
            self.r_loc.append(r_loc)
            self.c_loc.append(c_loc)
            self.c_glob.append(np.array([self.primal[g] for g in gdofs[c_loc]], dtype=np.int64))
            self.f_r.append(fs[r_loc])
            self.f_c.append(fs[c_loc])
            Ks_cache[s] = Ks
        # --- B_r rows (Eq. 10): pair-wise rows at shared non-corner, non-fixed DOFs ---
        pos_in_r = []
        for s in range(ns):
            p = -np.ones(mesh.n_loc_dofs, np.int64)
            p[self.r_loc[s]] = np.arange(self.r_loc[s].size)
            pos_in_r.append(p)
        entries, sharing = [], []
        for gn in range(mesh.n_nodes):
            own = mesh.owners[gn]
            if len(own) < 2 or mesh.is_tile_vertex(gn):
                continue
            for d in range(dim):
                if problem.dirichlet[gn * dim + d] or gn * dim + d in avg_dofs:
                    continue
                copies = [(s, ln * dim + d) for (s, ln) in own]
                for row in pairwise_rows(copies):
                    entries.append(row)
                    sharing.append(copies)
        cons_loc = Constraints(entries, sharing, np.zeros(len(entries)))
        w = row_weights(cons_loc, self.diagK, scaling)
        # re-express the rows on r-local indices
        entries_r = [[(s, int(pos_in_r[s][k]), sg) for (s, k, sg) in ent] for ent in entries]
        self.cons = Constraints(entries_r, sharing, np.zeros(len(entries)))
        self.weights = w
        self.n_lam = self.cons.n_lam
        self.Br = [self.cons.B_sub(s, self.r_loc[s].size) for s in range(ns)]
        self.Brt = [self.cons.B_sub(s, self.r_loc[s].size, w) for s in range(ns)]
        self.bset = [np.unique(self.Br[s].indices) for s in range(ns)]
        self.Bc = [sp.csr_matrix((np.ones(cg.size), (np.arange(cg.size), cg)), shape=(cg.size, self.n_c))
                   for cg in self.c_glob]
        # --- per-module factorisations ---
        for s in range(ns):
            Ks = Ks_cache.pop(s)
            h = hashlib.sha1()
            for a in (Ks, self.r_loc[s], self.c_loc[s], self.bset[s]):
                h.update(np.ascontiguousarray(a).tobytes())
            key = h.hexdigest() if dedup else s
            if key not in self.modules:
                self.modules[key] = _Module(Ks, self.r_loc[s], self.c_loc[s], self.bset[s],
                                            keep_factor=not operator_only,
                                            keep_kbb=not operator_only or precond != "dirichlet")
            self.mod_key.append(key)
        # --- coarse problem and right-hand sides (Eq. 12) ---
        Kbar = np.zeros((self.n_c, self.n_c))
        fbar = np.zeros(self.n_c)
        d_r = np.zeros(self.n_lam)
        for s in range(ns):
            M = self.mod(s)
            cg = self.c_glob[s]
            Kbar[np.ix_(cg, cg)] += M.Kbar
            if operator_only:
                continue
            y = sla.cho_solve(M.cho, self.f_r[s])                      # K_rr^{-1} f_r^s
            np.add.at(fbar, cg, self.f_c[s] - M.Krc.T @ y)
            d_r += self.Br[s] @ y
        self.Kbar = 0.5 * (Kbar + Kbar.T)
        self.Kbar_cho = sla.cho_factor(self.Kbar, lower=True)
        self.lam0 = np.zeros(self.n_lam)
        if operator_only:
            self.fbar = self.d_r = self.d = None
            return
        self.fbar = fbar
        self.d_r = d_r
        self.d = d_r - self.apply_Frc(sla.cho_solve(self.Kbar_cho, fbar)[:, None])[:, 0]

    def mod(self, s):
        return self.modules[self.mod_key[s]]

    # -- blocks of Eq. (12) ---------------------------------------------------
    def apply_Frr(self, X):
        Y = np.zeros((self.n_lam, X.shape[1]))
        for s in range(self.n_sub):
            b = self.bset[s]
            Bb = self.Br[s][:, b]
            Y += Bb @ (self.mod(s).Fb @ (Bb.T @ X))
        return Y

    def apply_FrcT(self, X):
        V = np.zeros((self.n_c, X.shape[1]))
        for s in range(self.n_sub):
            b = self.bset[s]
            Bb = self.Br[s][:, b]
            np.add.at(V, self.c_glob[s], self.mod(s).Frc_b.T @ (Bb.T @ X))
        return V

    def apply_Frc(self, V):
        Y = np.zeros((self.n_lam, V.shape[1]))
        for s in range(self.n_sub):
            b = self.bset[s]
            Bb = self.Br[s][:, b]
            Y += Bb @ (self.mod(s).Frc_b @ V[self.c_glob[s]])
        return Y

    # -- condensed operator used by the Krylov solvers --------------------------
    def apply_F(self, X):
        """(F_rr + F_rc Kbar_cc^{-1} F_rc^T) X for X [n_lam, m]."""
        X = np.atleast_2d(X.T).T
        V = sla.cho_solve(self.Kbar_cho, self.apply_FrcT(X))
        return self.apply_Frr(X) + self.apply_Frc(V)

    def apply_F_rows(self, X, rows):
        """Rows ``rows`` of apply_F(X): the same sums restricted to those
        multipliers.  Only the subdomains that own one of the rows contribute
        their local term; the coarse correction V = Kbar_cc^{-1} F_rc^T X still
        gathers every subdomain.  For operator checks at sizes where forming
        all of F X is too slow.  Pinned against apply_F (tests/test_oracle_dual.py)."""
        X = np.atleast_2d(X.T).T
        rows = np.asarray(rows, dtype=np.int64)
        V = sla.cho_solve(self.Kbar_cho, self.apply_FrcT(X))
        Y = np.zeros((rows.size, X.shape[1]))
        for s in range(self.n_sub):
            b = self.bset[s]
            Bb_R = self.Br[s][rows][:, b]
            if Bb_R.nnz == 0:
                continue
            M = self.mod(s)
            xb = self.Br[s][:, b].T @ X
            Y += Bb_R @ (M.Fb @ xb + M.Frc_b @ V[self.c_glob[s]])
        return Y

    def row_entries(self):
        """The multipliers as int64 [n_lam, 6] rows (s1, local dof1, sign1,
        s2, local dof2, sign2), local DOFs numbered in the subdomain (not in
        its r-set); s2 = -1 for a single-subdomain row."""
        out = -np.ones((self.n_lam, 6), np.int64)
        for l, ent in enumerate(self.cons.entries):
            for t, (s, k, sg) in enumerate(ent):
                out[l, 3 * t:3 * t + 3] = (s, int(self.r_loc[s][k]), int(sg))
        return out

    def project(self, X):
        return X            # FETI-DP needs no projector

    project_T = project

    def precond_block(self, s):
        """The local block of the preconditioner: the Dirichlet choice S^s of
        Eq. 13 (Schur complement onto the interface), the lumped choice K_bb
        (the interface block of the stiffness, no interior solve) or the
        super-lumped choice diag(K_bb) (Section 3)."""
        M = self.mod(s)
        if self.precond == "dirichlet":
            return M.S
        if self.precond == "lumped":
            return M.Kbb
        return np.diag(np.diag(M.Kbb))

    def precond_columns(self, r):
        """Z = [..., B~_r^s P^s B~_r^sT r, ...]: one column per subdomain (Eq. 13 on r-DOFs)."""
        Z = np.zeros((self.n_lam, self.n_sub))
        for s in range(self.n_sub):
            Bb = self.Brt[s][:, self.bset[s]]
            Z[:, s] = Bb @ (self.precond_block(s) @ (Bb.T @ r))
        return Z

    # -- recovery (second row of Eq. 12, then the second row of Eq. 11) ----------
    def recover_local(self, lam):
        uc = sla.cho_solve(self.Kbar_cho, self.fbar + self.apply_FrcT(lam[:, None])[:, 0])
        us = []
        for s in range(self.n_sub):
            M = self.mod(s)
            ucs = uc[self.c_glob[s]]
            ur = sla.cho_solve(M.cho, self.f_r[s] - M.Krc @ ucs - self.Br[s].T @ lam)
            u = np.zeros(self.mesh.n_loc_dofs)
            u[self.r_loc[s]] = ur
            u[self.c_loc[s]] = ucs
            if self.T[s] is not None:
                u = self.T[s] @ u                          # back to nodal values
            us.append(u)
        return us, uc

    def recover(self, lam):
        us, _ = self.recover_local(lam)
        return gather_global(self.mesh, self.dim, us, self.problem.dirichlet)
