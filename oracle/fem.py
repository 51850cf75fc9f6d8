"""SIMP interpolation and reference element stiffness matrices (oracle).

Test infrastructure only (see the package docstring).

* Eq. (1): E(x) = E_min + rho(x)^p (E_0 - E_min); with an isotropic material
  and a fixed Poisson ratio the element stiffness is E_e * k0(nu).
* Section 4.2: bilinear quadrilateral elements, 2 DOF per node, plane
  stress, unit thickness; trilinear hexahedra (3 DOF per node) for the 3D
  workloads.  Elements are unit squares / cubes.

k0 is integrated with the 2-point (per axis) Gauss rule, which is exact for
the bilinear / trilinear element on an undistorted square / cube; the tests
(tests/test_oracle_fem.py) pin it against exact symbolic integration, the
patch test and the rigid-body null space, and Eq. (1) against its closed form.

Element node order (local to the oracle):
  Q4: (0,0) (1,0) (1,1) (0,1)
  H8: (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1)
DOF order inside an element: node-major, [ux, uy(, uz)] per node.
"""
import itertools

import numpy as np

Q4_NODES = np.array([(0, 0), (1, 0), (1, 1), (0, 1)], dtype=np.int64)
H8_NODES = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                     (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)], dtype=np.int64)


def simp_modulus(rho, E0, Emin, p):
    """Eq. (1): Young's modulus of each element from its relative density."""
    rho = np.asarray(rho, dtype=np.float64)
    return Emin + rho ** p * (E0 - Emin)


def elasticity_matrix(dim, nu):
    """Isotropic constitutive matrix for E = 1 (plane stress in 2D), Voigt order
    [xx, yy, xy] in 2D and [xx, yy, zz, yz, xz, xy] in 3D (engineering shear)."""
    if dim == 2:
        return np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, 0.5 * (1.0 - nu)]]) / (1.0 - nu * nu)
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def _shape_gradients(nodes, xi):
    """Gradients dN_a/dx at point xi of the multilinear unit element."""
    dim = nodes.shape[1]
    grads = np.zeros((nodes.shape[0], dim))
    for a, na in enumerate(nodes):
        fac = [xi[d] if na[d] == 1 else 1.0 - xi[d] for d in range(dim)]
        dfac = [1.0 if na[d] == 1 else -1.0 for d in range(dim)]
        for d in range(dim):
            g = dfac[d]
            for e in range(dim):
                if e != d:
                    g *= fac[e]
            grads[a, d] = g
    return grads


def strain_matrix(nodes, xi):
    """Strain-displacement matrix B (Voigt rows) of the unit element at xi."""
    dim = nodes.shape[1]
    G = _shape_gradients(nodes, xi)
    n = nodes.shape[0]
    if dim == 2:
        B = np.zeros((3, 2 * n))
        B[0, 0::2] = G[:, 0]
        B[1, 1::2] = G[:, 1]
        B[2, 0::2] = G[:, 1]
        B[2, 1::2] = G[:, 0]
        return B
    B = np.zeros((6, 3 * n))
    B[0, 0::3] = G[:, 0]
    B[1, 1::3] = G[:, 1]
    B[2, 2::3] = G[:, 2]
    B[3, 1::3] = G[:, 2]
    B[3, 2::3] = G[:, 1]
    B[4, 0::3] = G[:, 2]
    B[4, 2::3] = G[:, 0]
    B[5, 0::3] = G[:, 1]
    B[5, 1::3] = G[:, 0]
    return B


def element_stiffness(dim, nu):
    """k0 = integral over the unit element of B^T D B (E = 1), 2-point Gauss per axis."""
    nodes = Q4_NODES if dim == 2 else H8_NODES
    D = elasticity_matrix(dim, nu)
    g = 0.5 / np.sqrt(3.0)
    pts = [0.5 - g, 0.5 + g]
    w = 0.5
    k0 = np.zeros((dim * nodes.shape[0],) * 2)
    for xi in itertools.product(pts, repeat=dim):
        B = strain_matrix(nodes, np.array(xi))
        k0 += (w ** dim) * B.T @ D @ B
    return 0.5 * (k0 + k0.T)


def rigid_body_modes(coords):
    """Rigid-body displacement fields at nodes with coordinates ``coords``
    [n, dim]: 3 in 2D (2 translations, 1 rotation), 6 in 3D.  Returned as
    [n*dim, n_rbm] in node-major DOF order."""
    coords = np.asarray(coords, dtype=np.float64)
    n, dim = coords.shape
    if dim == 2:
        R = np.zeros((2 * n, 3))
        R[0::2, 0] = 1.0
        R[1::2, 1] = 1.0
        R[0::2, 2] = -coords[:, 1]
        R[1::2, 2] = coords[:, 0]
        return R
    R = np.zeros((3 * n, 6))
    for d in range(3):
        R[d::3, d] = 1.0
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    R[1::3, 3] = -z; R[2::3, 3] = y      # rotation about x
    R[0::3, 4] = z;  R[2::3, 4] = -x     # rotation about y
    R[0::3, 5] = -y; R[1::3, 5] = x      # rotation about z
    return R
