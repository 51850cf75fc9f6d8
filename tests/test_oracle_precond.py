"""Pins of the oracle's preconditioner choices (the Dirichlet block S^s of
Eq. 13, the lumped block K_bb and the super-lumped diag(K_bb), Section 3):

* with no interior DOF the Schur complement is K_bb itself, so the Dirichlet and
  lumped blocks coincide exactly (left tile of a 2x1 mesh of single elements
  with the left edge clamped: every DOF is touched by B in TFETI);
* the super-lumped block of a single unit Q4 element in plane stress is its
  diagonal (1/2 - nu/6) / (1 - nu^2) E (closed form);
* S^s <= K_bb in the Loewner order (K_bb - S^s = K_bi K_ii^-1 K_ib is PSD);
* every choice leads PCG to the direct solution of Eq. 2;
* preconditioning quality orders the iteration counts Dirichlet < lumped <
  super-lumped (textbook behaviour).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.assemble import direct_solve
from oracle.fetidp import FETIDP
from oracle.tfeti import TFETI


def _two_elements():
    return workloads.tile_problem("2x1 single elements", 2, (2, 1), (1, 1), np.array([1.0, 0.7]), Emin=1e-6)


def test_no_interior_dofs_dirichlet_equals_lumped():
    p = _two_elements()
    d = TFETI(p, "k", precond="dirichlet")
    lu = TFETI(p, "k", precond="lumped")
    assert d.bset[0].size == 8                       # every DOF of the left tile is in B
    assert np.array_equal(d.precond_block(0), lu.precond_block(0))
    assert not np.allclose(d.precond_block(1), lu.precond_block(1))   # the right tile has interior DOFs


def test_superlumped_diagonal_closed_form():
    p = _two_elements()
    op = TFETI(p, "k", precond="superlumped")
    nu = p.nu
    E = p.Emin + 1.0 ** p.p * (p.E0 - p.Emin)
    expect = (0.5 - nu / 6.0) / (1.0 - nu * nu) * E
    blk = op.precond_block(0)
    assert np.allclose(np.diag(blk), expect, rtol=1e-14)
    assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0


@pytest.mark.parametrize("cls", [TFETI, FETIDP])
def test_schur_complement_below_lumped_block(cls):
    p = workloads.config1()
    d = cls(p, "k", precond="dirichlet")
    lu = cls(p, "k", precond="lumped")
    rng = np.random.default_rng(4)
    for s in range(d.n_sub):
        D = lu.precond_block(s) - d.precond_block(s)
        x = rng.standard_normal((D.shape[0], 20))
        q = np.einsum("ij,ij->j", x, D @ x)
        assert np.all(q >= -1e-12 * np.abs(np.einsum("ij,ij->j", x, lu.precond_block(s) @ x)))


@pytest.mark.parametrize("method", ["tfeti", "fetidp"])
def test_every_preconditioner_reaches_the_direct_solution_in_order(method):
    p = workloads.config1()
    ud = direct_solve(p)
    its = {}
    for pc in ("dirichlet", "lumped", "superlumped"):
        u, _, info, _ = oracle.solve(p, method, "k", "pcg", tol=1e-12, max_iter=2000, precond=pc)
        assert info.converged
        assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
        its[pc] = info.iterations
    assert its["dirichlet"] < its["lumped"] < its["superlumped"]
