"""Global system (Eq. 2), local subdomain systems (Eq. 3), direct solve (oracle).

Test infrastructure only (see the package docstring).

The assembled global problem K^Omega u^Omega = f^Omega (Eq. 2) is the plain
definition of what every FETI variant must reproduce; ``direct_solve`` solves
it with a sparse direct factorisation after eliminating the Dirichlet DOFs.
``local_stiffness`` builds K^s of Eq. (3) for one subdomain as a dense
matrix, including all of its DOFs (Dirichlet ones too; TFETI keeps them).

Pins: tests/test_oracle_dual.py (the direct solve's residual of Eq. 2; every
FETI variant reaches it), tests/test_oracle_sensitivity.py (compliance equal
to the strain energy).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import element_stiffness, simp_modulus
from .mesh import TileMesh


def mesh_of(problem):
    return TileMesh(problem.dim, problem.tiles, problem.elems)


def element_moduli(problem):
    """Eq. (1) per element."""
    return simp_modulus(problem.rho, problem.E0, problem.Emin, problem.p)


def global_stiffness(problem, mesh=None):
    """K^Omega of Eq. (2) as a scipy CSR matrix [n_dofs, n_dofs]."""
    mesh = mesh or mesh_of(problem)
    dim = problem.dim
    k0 = element_stiffness(dim, problem.nu)
    E = element_moduli(problem)
    en = mesh.element_nodes_global()
    edofs = (en[:, :, None] * dim + np.arange(dim)[None, None, :]).reshape(en.shape[0], -1)
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).ravel()
    cols = np.tile(edofs, (1, nd)).ravel()
    vals = (E[:, None, None] * k0[None, :, :]).reshape(en.shape[0], -1).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(mesh.n_dofs, mesh.n_dofs)).tocsr()
    K.sum_duplicates()
    return K


def direct_solve(problem, mesh=None):
    """Solve Eq. (2) with Dirichlet DOFs fixed to zero; returns u [n_dofs]."""
    K = global_stiffness(problem, mesh)
    free = np.flatnonzero(problem.dirichlet == 0)
    u = np.zeros(K.shape[0])
    Kff = K[free][:, free].tocsc()
    u[free] = spla.spsolve(Kff, problem.f[free])
    return u


def local_stiffness(problem, mesh, s, k0=None, E=None):
    """Dense K^s (Eq. 3) of subdomain s over all its local DOFs."""
    dim = problem.dim
    k0 = element_stiffness(dim, problem.nu) if k0 is None else k0
    E = element_moduli(problem) if E is None else E
    Es = E[mesh.local_elements(s)]
    conn = mesh.local_element_nodes
    n = mesh.n_loc_dofs
    Ks = np.zeros((n, n))
    for e in range(conn.shape[0]):
        dofs = (conn[e][:, None] * dim + np.arange(dim)[None, :]).ravel()
        Ks[np.ix_(dofs, dofs)] += Es[e] * k0
    return Ks


def local_load(problem, mesh, s):
    """f^s of Eq. (3): the global nodal load of a node shared by several
    subdomains is given to its lowest-index owner (any split sums to the same
    global load; this one is deterministic)."""
    dim = problem.dim
    g2 = mesh.local_to_global_nodes(s)
    fs = np.zeros(mesh.n_loc_dofs)
    for ln, gn in enumerate(g2):
        if mesh.owners[gn][0][0] == s:
            fs[ln * dim:(ln + 1) * dim] = problem.f[gn * dim:(gn + 1) * dim]
    return fs


def local_dirichlet(problem, mesh, s):
    """Boolean mask over the local DOFs of subdomain s that are fixed."""
    dim = problem.dim
    g2 = mesh.local_to_global_nodes(s)
    gd = (g2[:, None] * dim + np.arange(dim)[None, :]).ravel()
    return problem.dirichlet[gd].astype(bool)


def gather_global(mesh, dim, u_loc_list, dirichlet):
    """Global nodal field from subdomain copies: the mean of all copies of a node
    (copies agree up to the solver tolerance); fixed DOFs are set to zero."""
    u = np.zeros(mesh.n_dofs)
    cnt = np.zeros(mesh.n_nodes)
    for s, us in enumerate(u_loc_list):
        g2 = mesh.local_to_global_nodes(s)
        for d in range(dim):
            np.add.at(u, g2 * dim + d, us[d::dim])
        np.add.at(cnt, g2, 1.0)
    u /= np.repeat(cnt, dim)
    u[dirichlet.astype(bool)] = 0.0
    return u
