"""Pins of the tile mesh and the tearing counts.

Section 4.2 prints one structural number: 96 modules of 30x30 bilinear
elements give 184,512 DOFs in total, which is the torn (subdomain-wise)
count 96 * 31^2 * 2.
"""
import numpy as np

import workloads
from oracle.mesh import TileMesh


def test_paper_torn_dof_count_section_4_2():
    for layout in [(12, 8), (16, 6), (8, 12), (24, 4)]:
        m = TileMesh(2, layout, (30, 30))
        assert m.n_sub == 96
        assert m.n_sub * m.n_loc_dofs == 184512


def test_global_numbering_lexicographic():
    m = TileMesh(2, (3, 2), (2, 3))
    assert m.nnod == (7, 7)
    assert m.node_index([6, 0]) == 6 and m.node_index([0, 1]) == 7
    # every local node maps to a distinct global node inside one subdomain,
    # and the union covers the grid
    seen = set()
    for s in range(m.n_sub):
        g = m.local_to_global_nodes(s)
        assert len(set(g)) == g.size == m.n_loc_nodes
        seen.update(g.tolist())
    assert seen == set(range(m.n_nodes))
    # elements partition exactly
    allel = np.concatenate([m.local_elements(s) for s in range(m.n_sub)])
    assert np.array_equal(np.sort(allel), np.arange(m.n_elements))


def test_owner_multiplicity():
    m = TileMesh(2, (3, 3), (2, 2))
    mult = np.array([len(o) for o in m.owners])
    assert mult.max() == 4 and np.sum(mult == 4) == 4        # the 4 interior cross points
    m3 = TileMesh(3, (2, 2, 2), (2, 2, 2))
    mult3 = np.array([len(o) for o in m3.owners])
    assert mult3.max() == 8 and np.sum(mult3 == 8) == 1


def test_workload_shapes():
    p = workloads.config1()
    assert p.n_dofs == 578 and p.rho.size == 256
    assert p.dirichlet.sum() == 34 and p.f.sum() == -1.0
    p2 = workloads.config2(tiles=4, elems=8)
    assert set(np.unique(p2.rho)) <= {1e-3, 1.0}
    p4 = workloads.config4(tiles=2, elems=2)
    assert p4.dim == 3 and p4.rho.min() >= 1e-3 and p4.rho.max() <= 1.0
    # same seed, same bits
    assert np.array_equal(workloads.config2(tiles=4, elems=8).rho, p2.rho)
