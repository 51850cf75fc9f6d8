"""Pins of compliance and the SIMP sensitivity: central finite differences of
direct solves (Eq. 2) on 20 seeded elements, and c = f^T u = u^T K u > 0."""
import numpy as np

import oracle
import workloads
from oracle.assemble import direct_solve, global_stiffness
from oracle.sensitivity import compliance, compliance_gradient


def _problem():
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.3, 1.0, size=8 * 8)
    return workloads.tile_problem("fd", 2, (2, 2), (4, 4), rho, Emin=1e-6)


def test_compliance_is_strain_energy():
    p = _problem()
    u = direct_solve(p)
    K = global_stiffness(p)
    c = compliance(p, u)
    assert c > 0 and abs(c - u @ (K @ u)) <= 1e-12 * c


def test_gradient_central_differences():
    p = _problem()
    u = direct_solve(p)
    g = compliance_gradient(p, u)
    rng = np.random.default_rng(5)
    for e in rng.choice(p.rho.size, 20, replace=False):
        h = 1e-4 * p.rho[e]     # O(h^2) truncation ~1e-8; keeps direct-solve noise below 1e-6
        cs = []
        for sgn in (+1, -1):
            q = workloads.tile_problem("fd", 2, p.tiles, p.elems, p.rho.copy(), Emin=p.Emin)
            q.rho[e] += sgn * h
            cs.append(compliance(q, direct_solve(q)))
        fd = (cs[0] - cs[1]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + 1e-12 * np.abs(g).max()


def test_gradient_from_feti_solution():
    p = _problem()
    u, *_ = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-12)
    g_ref = compliance_gradient(p, direct_solve(p))
    assert np.linalg.norm(compliance_gradient(p, u) - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
