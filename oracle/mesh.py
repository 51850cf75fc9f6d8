"""Regular tile meshes: global and subdomain-local numbering (oracle).

Test infrastructure only (see the package docstring).

Section 2: the domain is split into N_s disjoint subdomains; Section 1 and
Section 4.2: in modular problems every module (tile) is one subdomain, so
the partition is fixed and regular.  Subdomain s is the tile with
lexicographic index s (x fastest).  Inside a subdomain, nodes and elements
are numbered lexicographically as well, and local DOF = dim * node + d.

Pins (tests/test_oracle_mesh.py): the torn DOF count Section 4.2 prints
(96 modules of 31 x 31 interior-edge nodes: 184,512), lexicographic global
numbering, owner multiplicities, workload shapes.
"""
import itertools
from functools import cached_property

import numpy as np

from .fem import Q4_NODES, H8_NODES


class TileMesh:
    def __init__(self, dim, tiles, elems):
        self.dim = int(dim)
        self.tiles = tuple(int(t) for t in tiles)
        self.elems = tuple(int(e) for e in elems)
        assert len(self.tiles) == self.dim and len(self.elems) == self.dim
        self.nel = tuple(t * e for t, e in zip(self.tiles, self.elems))
        self.nnod = tuple(n + 1 for n in self.nel)
        self.n_nodes = int(np.prod(self.nnod))
        self.n_elements = int(np.prod(self.nel))
        self.n_dofs = self.n_nodes * self.dim
        self.n_sub = int(np.prod(self.tiles))
        self.loc_nnod = tuple(e + 1 for e in self.elems)
        self.n_loc_nodes = int(np.prod(self.loc_nnod))
        self.n_loc_dofs = self.n_loc_nodes * self.dim
        self.n_loc_elems = int(np.prod(self.elems))

    # -- global grid -------------------------------------------------------------
    def node_index(self, ijk):
        idx, stride = 0, 1
        for a in range(self.dim):
            idx += ijk[a] * stride
            stride *= self.nnod[a]
        return idx

    def node_coords(self):
        """[n_nodes, dim] integer coordinates of the global nodes."""
        grids = np.meshgrid(*[np.arange(n) for n in self.nnod], indexing="ij")
        return np.stack([g.ravel(order="F") for g in grids], axis=1)

    def element_nodes_global(self):
        """[n_elements, 2^dim] global node ids per element (oracle node order)."""
        ref = Q4_NODES if self.dim == 2 else H8_NODES
        grids = np.meshgrid(*[np.arange(n) for n in self.nel], indexing="ij")
        base = np.stack([g.ravel(order="F") for g in grids], axis=1)
        out = np.empty((self.n_elements, ref.shape[0]), np.int64)
        for a, off in enumerate(ref):
            c = base + off
            out[:, a] = self.node_index([c[:, d] for d in range(self.dim)])
        return out

    # -- subdomains --------------------------------------------------------------
    def tile_of(self, s):
        return np.unravel_index(s, self.tiles, order="F")

    def local_to_global_nodes(self, s):
        """Global node id of every local node of subdomain s (local lexicographic order)."""
        t = self.tile_of(s)
        grids = np.meshgrid(*[np.arange(n) for n in self.loc_nnod], indexing="ij")
        loc = np.stack([g.ravel(order="F") for g in grids], axis=1)
        glob = loc + np.array([t[a] * self.elems[a] for a in range(self.dim)])
        return self.node_index([glob[:, d] for d in range(self.dim)])

    def local_elements(self, s):
        """Global element id of every local element of subdomain s (local lexicographic order)."""
        t = self.tile_of(s)
        grids = np.meshgrid(*[np.arange(n) for n in self.elems], indexing="ij")
        loc = np.stack([g.ravel(order="F") for g in grids], axis=1)
        glob = loc + np.array([t[a] * self.elems[a] for a in range(self.dim)])
        idx, stride = 0, 1
        for a in range(self.dim):
            idx = idx + glob[:, a] * stride
            stride *= self.nel[a]
        return idx

    @cached_property
    def local_element_nodes(self):
        """[n_loc_elems, 2^dim] local node ids per local element (same for every subdomain)."""
        ref = Q4_NODES if self.dim == 2 else H8_NODES
        grids = np.meshgrid(*[np.arange(n) for n in self.elems], indexing="ij")
        base = np.stack([g.ravel(order="F") for g in grids], axis=1)
        out = np.empty((self.n_loc_elems, ref.shape[0]), np.int64)
        for a, off in enumerate(ref):
            c = base + off
            idx, stride = 0, 1
            for d in range(self.dim):
                idx = idx + c[:, d] * stride
                stride *= self.loc_nnod[d]
            out[:, a] = idx
        return out

    @cached_property
    def owners(self):
        """For every global node, the sorted list of (subdomain, local node) copies."""
        own = [[] for _ in range(self.n_nodes)]
        for s in range(self.n_sub):
            for ln, gn in enumerate(self.local_to_global_nodes(s)):
                own[gn].append((s, ln))
        return own

    def is_tile_vertex(self, gn):
        """True if global node gn is a vertex of the tile grid (a subdomain corner)."""
        ijk = np.unravel_index(gn, self.nnod, order="F")
        return all(ijk[a] % self.elems[a] == 0 for a in range(self.dim))

    def local_node_coords(self, s):
        return self.node_coords()[self.local_to_global_nodes(s)]


def dof_list(nodes, dim):
    """DOF ids (node-major) of a node list."""
    nodes = np.asarray(nodes, dtype=np.int64)
    return (nodes[:, None] * dim + np.arange(dim)[None, :]).ravel()


def all_pairs(items):
    return list(itertools.combinations(items, 2))
