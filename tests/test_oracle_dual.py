"""Pins of the oracle's TFETI / FETI-DP dual problems and Algorithm 1.

What pins what (none of these re-run the oracle's own formula):
* the assembled global system solved by a sparse direct solver (Eq. 2) pins
  u for every one of the 12 variants;
* the dense saddle-point systems Eq. (6) and Eq. (11), solved by least
  squares on tiny meshes, pin the constraint matrices and the recovery;
* the dense dual system Eq. (7) pins F, G, d, e including their signs;
* global block-diagonal inverses pin the per-subdomain restriction used for
  the Eq. (12) blocks;
* invariants stated by the paper: rigid-body null space (Section 2.1),
  G lambda = e and the projector (Section 3.3), B u = c / B_r u_r = 0
  (Eqs. 4, 10), admissibility Eq. (14), k-scaling = multiplicity for a
  homogeneous material (Section 3.1), F-orthonormality after the
  rank-revealing step and F-orthogonality to the history (Section 3.3);
* a textbook projected PCG written here from scratch pins the "pcg" variant;
* a brute-force subset search pins the rank-revealing pivot rule.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads
from oracle.assemble import direct_solve, global_stiffness
from oracle.fetidp import FETIDP
from oracle.krylov import rank_revealing_cholesky, solve_dual
from oracle.tfeti import TFETI, moore_penrose_psd


def tiny(tiles=(2, 2), elems=(2, 2), seed=3, lo=0.2, Emin=1e-6, bc="clamped_left"):
    rng = np.random.default_rng(seed)
    n = np.prod([t * e for t, e in zip(tiles, elems)])
    rho = rng.uniform(lo, 1.0, size=n)
    return workloads.tile_problem("tiny", len(tiles), tiles, elems, rho, Emin=Emin, bc=bc)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- direct solve
def test_direct_solve_residual():
    p = workloads.config1()
    u = direct_solve(p)
    K = global_stiffness(p)
    free = p.dirichlet == 0
    r = (K @ u - p.f)[free]
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(p.f)
    assert np.all(u[~free] == 0)


# ------------------------------------------------------------- 12 variants
@pytest.mark.parametrize("method", ["tfeti", "fetidp"])
@pytest.mark.parametrize("scaling", ["k", "mult"])
@pytest.mark.parametrize("krylov", ["pcg", "fo", "rrs"])
def test_twelve_variants_reach_direct_solution(method, scaling, krylov):
    p = workloads.config1()
    ud = direct_solve(p)
    u, lam, info, op = oracle.solve(p, method, scaling, krylov, tol=1e-12, max_iter=400)
    assert info.converged and not info.breakdown
    assert rel(u, ud) <= 1e-9


def test_three_dimensional_fetidp_rrs():
    p = tiny(tiles=(2, 2, 2), elems=(2, 2, 2), seed=5)
    ud = direct_solve(p)
    u, lam, info, op = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-12)
    assert info.converged and rel(u, ud) <= 1e-9
    u2, _, info2, _ = oracle.solve(p, "tfeti", "k", "rrs", tol=1e-12)
    assert info2.converged and rel(u2, ud) <= 1e-9


# --------------------------------------------------------- TFETI brute force
def test_tfeti_saddle_point_eq6_and_dual_eq7():
    p = tiny()
    op = TFETI(p, "k")
    K, B, f, R, Kp = op.dense()
    n, nl = K.shape[0], B.shape[0]
    A = np.block([[K, B.T], [B, np.zeros((nl, nl))]])
    sol = np.linalg.lstsq(A, np.concatenate([f, op.cons.c]), rcond=None)[0]
    u_eq6 = sol[:n]
    # Eq. (7) formed densely from its definitions
    F = B @ Kp @ B.T
    G = -R.T @ B.T
    d = B @ Kp @ f - op.cons.c
    e = -R.T @ f
    ng = G.shape[0]
    A7 = np.block([[F, G.T], [G, np.zeros((ng, ng))]])
    sol7 = np.linalg.lstsq(A7, np.concatenate([d, e]), rcond=None)[0]
    lam7, alpha7 = sol7[:nl], sol7[nl:]
    u_eq7 = Kp @ (f - B.T @ lam7) + R @ alpha7
    assert rel(u_eq7, u_eq6) <= 1e-8
    # the oracle's operators agree with the dense definitions
    assert rel(op.apply_F(np.eye(nl)), F) <= 1e-12
    assert rel(op.G, G) <= 1e-14 and rel(op.d, d) <= 1e-12 and rel(op.e, e) <= 1e-14
    # and its solve reproduces Eq. (6)
    lam, info = solve_dual(op, tol=1e-13)
    us, alpha = op.recover_local(lam)
    assert rel(np.concatenate(us), u_eq6) <= 1e-8
    assert np.allclose(G @ lam, e, atol=1e-10 * np.abs(e).max())           # G lambda = e
    assert np.allclose(B @ np.concatenate(us), op.cons.c, atol=1e-9)       # B u = c


def test_pseudo_inverse_matches_svd():
    p = tiny()
    op = TFETI(p, "k")
    for s in range(op.n_sub):
        Kp_svd = np.linalg.pinv(op.K[s], rcond=1e-12, hermitian=True)
        assert rel(op.Kp[s], Kp_svd) <= 1e-9
        assert rel(moore_penrose_psd(op.K[s], op.R[s]), Kp_svd) <= 1e-9


def test_rigid_body_null_space_of_floating_subdomains():
    p = tiny(tiles=(3, 2))
    op = TFETI(p, "k")
    for s in range(op.n_sub):
        assert np.abs(op.K[s] @ op.R[s]).max() <= 1e-12 * np.abs(op.K[s]).max()
        ev = np.linalg.eigvalsh(op.K[s])
        assert np.sum(ev < 1e-10 * ev.max()) == 3            # three RBMs in 2D (Section 2.1)


def test_projector_properties():
    op = TFETI(tiny(tiles=(3, 2)), "k")
    nl = op.n_lam
    P = op.project(np.eye(nl))
    assert np.allclose(P @ P, P, atol=1e-12)
    assert np.allclose(P, P.T, atol=1e-12)
    assert np.abs(op.G @ P).max() <= 1e-12 * np.abs(op.G).max()
    assert np.allclose(op.G @ op.lam0, op.e)


# ------------------------------------------------------- FETI-DP brute force
def test_fetidp_eq11_and_eq12_blocks():
    p = tiny(tiles=(3, 3), elems=(2, 2))      # load on a boundary edge node: d_r != 0
    op = FETIDP(p, "k", dedup=False)
    ns = op.n_sub
    Krr = sla.block_diag(*[op.mod(s).Krr for s in range(ns)])
    Br = np.hstack([op.Br[s].toarray() for s in range(ns)])
    Bc = [op.Bc[s].toarray() for s in range(ns)]
    Kcc = sum(Bc[s].T @ op.mod(s).Kcc @ Bc[s] for s in range(ns))
    Kcr = np.hstack([Bc[s].T @ op.mod(s).Krc.T for s in range(ns)])
    fr = np.concatenate(op.f_r)
    fc = sum(Bc[s].T @ op.f_c[s] for s in range(ns))
    nc, nr, nl = Kcc.shape[0], Krr.shape[0], Br.shape[0]
    A11 = np.block([[Kcc, Kcr, np.zeros((nc, nl))],
                    [Kcr.T, Krr, Br.T],
                    [np.zeros((nl, nc)), Br, np.zeros((nl, nl))]])
    sol = np.linalg.lstsq(A11, np.concatenate([fc, fr, np.zeros(nl)]), rcond=None)[0]
    uc, ur = sol[:nc], sol[nc:nc + nr]
    # global u from Eq. (11) equals the direct solve
    ud = direct_solve(p)
    us, off = [], 0
    for s in range(ns):
        u = np.zeros(op.mesh.n_loc_dofs)
        n_r = op.r_loc[s].size
        u[op.r_loc[s]] = ur[off:off + n_r]
        u[op.c_loc[s]] = uc[op.c_glob[s]]
        off += n_r
        us.append(u)
    from oracle.assemble import gather_global
    assert rel(gather_global(op.mesh, 2, us, p.dirichlet), ud) <= 1e-9
    # Eq. (12) blocks from global dense inverses
    Kinv = np.linalg.inv(Krr)
    Frr = Br @ Kinv @ Br.T
    Frc = Br @ Kinv @ Kcr.T
    Kbar = Kcc - Kcr @ Kinv @ Kcr.T
    dr = Br @ Kinv @ fr
    fbar = fc - Kcr @ Kinv @ fr
    assert rel(op.apply_Frr(np.eye(nl)), Frr) <= 1e-10
    assert rel(op.apply_Frc(np.eye(nc)), Frc) <= 1e-10
    assert rel(op.apply_FrcT(np.eye(nl)), Frc.T) <= 1e-10
    assert np.linalg.norm(dr) > 0
    assert rel(op.Kbar, Kbar) <= 1e-10 and rel(op.d_r, dr) <= 1e-10 and rel(op.fbar, fbar) <= 1e-10
    # the condensed system gives lambda; recovery matches Eq. (11)
    lam, info = solve_dual(op, tol=1e-13)
    us2, uc2 = op.recover_local(lam)
    assert rel(uc2, uc) <= 1e-8
    ur2 = np.concatenate([us2[s][op.r_loc[s]] for s in range(ns)])
    assert np.abs(Br @ ur2).max() <= 1e-9 * np.abs(ur2).max()            # B_r u_r = 0


def test_fetidp_row_restricted_apply_and_operator_only_build():
    """apply_F_rows against the dense condensed operator of Eq. (12) built from
    global inverses; the operator-only build gives the same operator and
    preconditioner bit for bit; row_entries reproduces B_r."""
    p = tiny(tiles=(3, 3), elems=(2, 2))
    op = FETIDP(p, "k", dedup=False)
    ns = op.n_sub
    Krr = sla.block_diag(*[op.mod(s).Krr for s in range(ns)])
    Br = np.hstack([op.Br[s].toarray() for s in range(ns)])
    Bc = [op.Bc[s].toarray() for s in range(ns)]
    Kcc = sum(Bc[s].T @ op.mod(s).Kcc @ Bc[s] for s in range(ns))
    Kcr = np.hstack([Bc[s].T @ op.mod(s).Krc.T for s in range(ns)])
    Kinv = np.linalg.inv(Krr)
    Frc = Br @ Kinv @ Kcr.T
    F = Br @ Kinv @ Br.T + Frc @ np.linalg.solve(Kcc - Kcr @ Kinv @ Kcr.T, Frc.T)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((op.n_lam, 5))
    rows = np.sort(rng.choice(op.n_lam, 7, replace=False))
    assert rel(op.apply_F_rows(X, rows), (F @ X)[rows]) <= 1e-10
    lean = FETIDP(p, "k", dedup=False, operator_only=True)
    assert lean.d is None and not hasattr(lean.mod(0), "cho")
    assert np.array_equal(lean.apply_F(X), op.apply_F(X))
    assert np.array_equal(lean.precond_columns(X[:, 0]), op.precond_columns(X[:, 0]))
    # row_entries: the signed jumps of local vectors (full local numbering) equal B_r u_r
    ent = op.row_entries()
    us = [rng.standard_normal(op.mesh.n_loc_dofs) for _ in range(ns)]
    jump = np.zeros(op.n_lam)
    for t in (0, 3):
        for l in range(op.n_lam):
            if ent[l, t] >= 0:
                jump[l] += ent[l, t + 2] * us[ent[l, t]][ent[l, t + 1]]
    ur = np.concatenate([us[s][op.r_loc[s]] for s in range(ns)])
    assert np.allclose(jump, Br @ ur, rtol=0, atol=1e-14)


def test_multiplier_block_is_independent_of_row_order_and_orientation():
    """Two numberings of the same multipliers (rows permuted, some rows with the
    copies listed the other way round and negated) get the same test block up to
    that permutation and sign, so B^T X is the same interface vector."""
    op = FETIDP(tiny(tiles=(3, 2), elems=(2, 2)), "k")
    ent = op.row_entries()
    rng = np.random.default_rng(1)
    perm = rng.permutation(op.n_lam)
    flip = rng.random(op.n_lam) < 0.5
    other = ent[perm].copy()
    f = flip[perm]
    other[f] = other[f][:, [3, 4, 5, 0, 1, 2]]
    other[f, 2] *= -1
    other[f, 5] *= -1
    Xa = workloads.multiplier_block(*workloads.multiplier_pairs(ent), 4, seed=9)
    Xb = workloads.multiplier_block(*workloads.multiplier_pairs(other), 4, seed=9)
    sgn = np.where(f, -1.0, 1.0)[:, None]
    assert np.array_equal(Xb, sgn * Xa[perm])
    assert np.all(np.abs(Xa) <= 1.0) and Xa.std() > 0.4


def test_fetidp_dedup_is_exact():
    p = workloads.config2(tiles=4, elems=4)
    a = FETIDP(p, "k", dedup=True)
    b = FETIDP(p, "k", dedup=False)
    assert len(a.modules) < len(b.modules)
    X = np.random.default_rng(0).standard_normal((a.n_lam, 3))
    assert np.array_equal(a.apply_F(X), b.apply_F(X))


# ---------------------------------------------------------------- scaling
@pytest.mark.parametrize("method", ["tfeti", "fetidp"])
@pytest.mark.parametrize("scaling", ["k", "mult"])
def test_scaling_admissibility_eq14(method, scaling):
    p = tiny(tiles=(3, 3), elems=(2, 2), lo=1e-3)
    op = TFETI(p, scaling) if method == "tfeti" else FETIDP(p, scaling, dedup=False)
    Bs = op.B if method == "tfeti" else op.Br
    Bts = op.Bt if method == "tfeti" else op.Brt
    M = sum((Bs[s] @ Bts[s].T).toarray() for s in range(op.n_sub))
    for j in range(op.n_sub):
        Bj = Bs[j].toarray()
        assert np.abs(M @ Bj - Bj).max() <= 1e-13


def test_k_scaling_equals_multiplicity_for_homogeneous_material():
    p = tiny(tiles=(3, 3), elems=(2, 2))
    p.rho[:] = 0.7
    for cls in (TFETI, FETIDP):
        a, b = cls(p, "k"), cls(p, "mult")
        for wa, wb in zip(a.weights, b.weights):
            assert np.allclose(wa, wb, rtol=1e-13)


def test_block_preconditioner_sums_to_classic_one():
    # Section 3.3: w = W 1 restores the classic preconditioned direction.
    op = FETIDP(tiny(tiles=(3, 2)), "k", dedup=False)
    r = np.random.default_rng(2).standard_normal(op.n_lam)
    Fbar_inv = sum((op.Brt[s][:, op.bset[s]] @ op.mod(s).S @ op.Brt[s][:, op.bset[s]].T)
                   for s in range(op.n_sub))
    assert rel(op.precond_columns(r).sum(axis=1), Fbar_inv @ r) <= 1e-13


# ---------------------------------------------------------------- Krylov
def _textbook_pcpg(op, n_it):
    """Projected PCG with the classic beta recurrence (written independently)."""
    lam = op.lam0.copy()
    r = op.project_T(op.d - op.apply_F(lam[:, None])[:, 0])
    z = op.precond_columns(r).sum(axis=1)
    y = op.project(z[:, None])[:, 0]
    pdir = y.copy()
    rz = r @ y
    out = []
    for _ in range(n_it):
        q = op.apply_F(pdir[:, None])[:, 0]
        a = rz / (pdir @ q)
        lam = lam + a * pdir
        r = r - a * op.project_T(q[:, None])[:, 0]
        z = op.precond_columns(r).sum(axis=1)
        y = op.project(z[:, None])[:, 0]
        rz_new = r @ y
        pdir = y + (rz_new / rz) * pdir
        rz = rz_new
        out.append(lam.copy())
    return out


@pytest.mark.parametrize("method", ["tfeti", "fetidp"])
def test_pcg_variant_equals_textbook_pcpg(method):
    p = workloads.config1()
    op = oracle.build(p, method, "k")
    ref = _textbook_pcpg(op, 6)
    for k in range(1, 7):
        lam, info = solve_dual(op, tol=0.0, max_iter=k, variant="pcg")
        assert rel(lam, ref[k - 1]) <= 1e-10


def test_rrs_orthogonality_invariants():
    p = workloads.config1()
    op = oracle.build(p, "fetidp", "k")
    worst = {"orth": 0.0, "conj": 0.0}

    def cb(stage, i, data):
        if stage == "orth":
            W, Q = data
            worst["orth"] = max(worst["orth"], np.abs(W.T @ op.apply_F(W) - np.eye(W.shape[1])).max())
        else:
            W, hist = data
            Wn = W / np.linalg.norm(W, axis=0, keepdims=True).clip(1e-300)
            for (Wj, Qj) in hist:
                worst["conj"] = max(worst["conj"], np.abs(Qj.T @ Wn).max() / max(1.0, np.abs(Qj).max()))
    lam, info = solve_dual(op, tol=1e-10, callback=cb, variant="rrs")
    assert info.converged
    assert worst["orth"] <= 1e-8
    assert worst["conj"] <= 1e-8


def _brute_force_rank_revealing(Delta, rr_tol):
    """Greedy selection by explicit Schur complements of the chosen subset."""
    n = Delta.shape[0]
    d0 = np.diag(Delta)
    chosen = []
    alive = [j for j in range(n) if d0[j] > np.finfo(float).eps ** 2 * d0.max()]
    while True:
        best, bj = -np.inf, -1
        for j in alive:
            if j in chosen:
                continue
            if chosen:
                A = Delta[np.ix_(chosen, chosen)]
                v = Delta[np.ix_(chosen, [j])]
                schur = Delta[j, j] - (v.T @ np.linalg.solve(A, v))[0, 0]
            else:
                schur = Delta[j, j]
            ratio = schur / d0[j]
            if ratio > best:
                best, bj = ratio, j
        if bj < 0 or not best > rr_tol:
            return chosen
        chosen.append(bj)


def test_rank_revealing_cholesky_against_brute_force():
    rng = np.random.default_rng(11)
    for trial in range(20):
        m, rank = 9, int(rng.integers(1, 9))
        A = rng.standard_normal((40, rank)) @ rng.standard_normal((rank, m))
        A[:, rng.integers(0, m)] *= 1e-6 ** rng.integers(0, 2)    # scale spread
        if trial % 4 == 0:
            A[:, 2] = 0.0                                             # an exactly zero direction
        Delta = A.T @ A
        perm, k, Lt = rank_revealing_cholesky(Delta, 1e-10)
        true_rank = np.linalg.matrix_rank(A)
        assert k == true_rank
        assert list(perm[:k]) == _brute_force_rank_revealing(Delta, 1e-10)
        sub = Delta[np.ix_(perm[:k], perm[:k])]
        assert rel(Lt @ Lt.T, sub) <= 1e-12


# ------------------------------------------------------------ qualitative
def test_qualitative_plain_tfeti_stalls_fetidp_rrs_k_converges():
    """Sections 4-6: plain (multiplicity-scaled) TFETI converges very slowly at
    severe contrast while FETI-DP with multiple directions and k-scaling
    converges quickly."""
    p = workloads.config2(tiles=4, elems=8)
    _, _, good, _ = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-6, max_iter=200)
    _, _, bad, _ = oracle.solve(p, "tfeti", "mult", "pcg", tol=1e-6, max_iter=200)
    assert good.converged and good.iterations <= 20
    assert (not bad.converged) or bad.iterations >= 5 * good.iterations
