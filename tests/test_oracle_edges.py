"""Pins of the oracle's richer FETI-DP primal set (corners plus one average per
component over every tile-grid edge shared by two or more subdomains; the
paper names richer primal sets as future work, Section 5), introduced by a
change of basis on each edge (the reading stated in oracle/fetidp.py):

* the method still solves Eq. (2): every Krylov variant and both scalings
  reach the direct solution;
* closed-form sizes on a clamped 2x2x2 cube of tiles: 18 free vertices and 26
  averaged edges give 3 * (18 + 26) = 132 primal unknowns, and each averaged
  edge component removes its first node's pair-wise rows (168 rows in all,
  counted by brute force from the node owners);
* the change of basis is the average: on every subdomain the recovered nodal
  values along an averaged edge have the primal value as their mean, the same
  on every sharer;
* the richer coarse space pays off in 3D: fewer PCG and simultaneous-variant
  iterations than corners alone.
"""
import itertools

import numpy as np
import pytest

import workloads
from oracle.assemble import direct_solve
from oracle.fetidp import FETIDP, edge_averages
from oracle.mesh import TileMesh
from oracle.solve import solve


def _cube(tiles=2, elems=3):
    return workloads.config4(tiles=tiles, elems=elems)


@pytest.mark.parametrize("krylov", ["pcg", "fo", "rrs"])
@pytest.mark.parametrize("scaling", ["k", "mult"])
def test_edges_reach_the_direct_solution_3d(krylov, scaling):
    p = _cube()
    u, _, info, op = solve(p, "fetidp", scaling, krylov, tol=1e-10, max_iter=500, primal="edges")
    assert info.converged
    ud = direct_solve(p)
    assert np.linalg.norm(u - ud) <= 1e-6 * np.linalg.norm(ud)


def test_edges_reach_the_direct_solution_2d():
    p = workloads.layered_grid(elems=8, layers=8)
    u, _, info, _ = solve(p, "fetidp", "k", "pcg", tol=1e-10, max_iter=500, primal="edges")
    assert info.converged
    ud = direct_solve(p)
    assert np.linalg.norm(u - ud) <= 1e-6 * np.linalg.norm(ud)


def test_closed_form_sizes_on_the_clamped_cube():
    p = _cube()
    corners = FETIDP(p, "k")
    edges = FETIDP(p, "k", primal="edges")
    assert corners.n_c == 3 * 18
    # averaged edges: per axis, the tile-grid segments not on an edge of the
    # domain (one owner) and not inside the clamped face x = 0
    mesh = TileMesh(3, p.tiles, p.elems)
    n_edges = 0
    for run in range(3):
        others = [a for a in range(3) if a != run]
        for seg in range(2):
            for i, j in itertools.product(range(3), repeat=2):
                on_domain_edge = i in (0, 2) and j in (0, 2)
                clamped = (others[0] == 0 and i == 0) or (others[1] == 0 and j == 0)
                if not on_domain_edge and not clamped:
                    n_edges += 1
    assert n_edges == 26
    assert len(edge_averages(p, mesh)) == 3 * n_edges
    assert edges.n_c == 3 * (18 + n_edges)
    removed = sum(len(mesh.owners[nodes[0]]) * (len(mesh.owners[nodes[0]]) - 1) // 2
                  for nodes, _ in edge_averages(p, mesh))
    assert removed == 168
    assert edges.n_lam == corners.n_lam - removed


def test_primal_value_is_the_edge_average_on_every_sharer():
    p = _cube(tiles=2, elems=4)
    op = FETIDP(p, "k", primal="edges")
    _, lam, info, _ = solve(p, "fetidp", "k", "rrs", tol=1e-10, op=op)
    us, uc = op.recover_local(lam)
    mesh = op.mesh
    dim = 3
    for nodes, d in op.edges:
        ubar = uc[op.primal[nodes[0] * dim + d]]
        for s, _ in mesh.owners[nodes[0]]:
            g2 = list(mesh.local_to_global_nodes(s))
            vals = [us[s][g2.index(gn) * dim + d] for gn in nodes]
            assert np.mean(vals) == pytest.approx(ubar, rel=1e-10, abs=1e-14 * max(1.0, abs(ubar)))


@pytest.mark.parametrize("krylov", ["pcg", "rrs"])
def test_edge_averages_reduce_iterations_in_3d(krylov):
    p = _cube(tiles=3, elems=3)
    _, _, ic, _ = solve(p, "fetidp", "k", krylov, tol=1e-8, primal="corners")
    _, _, ie, _ = solve(p, "fetidp", "k", krylov, tol=1e-8, primal="edges")
    assert ie.iterations < ic.iterations
