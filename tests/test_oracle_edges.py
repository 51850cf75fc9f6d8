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
  iterations than corners alone;
* the adaptive selection (averages only across stiffness jumps): its limits are
  the two fixed sets bit for bit; on the laminated grid it averages exactly the
  horizontal tile sides (where a stiff lamina meets a compliant one), on the grid
  of inclusions nothing; it reaches the direct solution in 2D and 3D with fewer
  PCG iterations than corners alone.
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


# ---- adaptive selection (primal="adaptive") ------------------------------------------
def test_adaptive_selection_limits_are_corners_and_all_edges():
    """A jump ratio of 1 selects every shared edge, an infinite one none: the
    operators then equal those of the two fixed primal sets bit for bit."""
    p = workloads.layered_grid(elems=6, layers=6)
    X = np.random.default_rng(3).standard_normal
    all_edges = FETIDP(p, "k", primal="edges")
    none = FETIDP(p, "k", primal="corners")
    a1 = FETIDP(p, "k", primal="adaptive", jump_ratio=1.0)
    ainf = FETIDP(p, "k", primal="adaptive", jump_ratio=np.inf)
    assert a1.edges == all_edges.edges and not ainf.edges
    for got, want in ((a1, all_edges), (ainf, none)):
        assert got.n_c == want.n_c and got.n_lam == want.n_lam
        Y = X((want.n_lam, 3))
        assert np.array_equal(got.apply_F(Y), want.apply_F(Y))


def test_adaptive_selection_follows_the_stiffness_jumps():
    """On the laminated grid the horizontal interfaces join a stiff lamina to a
    compliant one and the vertical ones join equal laminae: exactly the
    horizontal tile sides are averaged.  On the grid of inclusions every
    interface is homogeneous: nothing is.  The selection still solves Eq. (2)
    and needs fewer PCG iterations than corners alone."""
    p = workloads.layered_grid(elems=8, layers=8)
    op = FETIDP(p, "k", primal="adaptive")
    mesh = op.mesh
    coords = mesh.node_coords()
    assert op.edges
    for nodes, d in op.edges:
        ys = {int(coords[g][1]) for g in nodes}
        assert len(ys) == 1 and next(iter(ys)) % p.elems[1] == 0        # runs along x: a horizontal side
    horizontal = [e for e in edge_averages(p, mesh) if len({int(coords[g][1]) for g in e[0]}) == 1]
    assert sorted(op.edges) == sorted(horizontal)
    ud = direct_solve(p)
    u, _, info, _ = solve(p, "fetidp", "k", "pcg", tol=1e-10, max_iter=500, primal="adaptive")
    _, _, info_c, _ = solve(p, "fetidp", "k", "pcg", tol=1e-10, max_iter=500, primal="corners")
    assert info.converged and np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    assert info.iterations < info_c.iterations
    q = workloads.inclusion_grid(elems=8)
    assert not FETIDP(q, "k", primal="adaptive").edges


def test_adaptive_selection_reaches_the_direct_solution_3d():
    p = _cube()
    u, _, info, op = solve(p, "fetidp", "k", "rrs", tol=1e-10, max_iter=500, primal="adaptive")
    assert 0 < len(op.edges) < len(edge_averages(p, op.mesh))
    assert info.converged
    ud = direct_solve(p)
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
