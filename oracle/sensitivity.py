"""Compliance and its SIMP sensitivity (oracle).

Test infrastructure only (see the package docstring).

Section 1: SIMP alternates state solves with density updates driven by the
sensitivities of the objective.  For compliance c(rho) = f^T u(rho) with
K(rho) u = f and K = sum_e E_e(rho_e) k0 (Eq. 1), the problem is
self-adjoint, so dc/drho_e = -u^T (dK/drho_e) u
                           = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e.
Pinned in the tests by central finite differences of direct solves.
"""
import numpy as np

from .assemble import mesh_of
from .fem import element_stiffness


def compliance(problem, u):
    return float(problem.f @ u)


def compliance_gradient(problem, u):
    mesh = mesh_of(problem)
    dim = problem.dim
    k0 = element_stiffness(dim, problem.nu)
    en = mesh.element_nodes_global()
    ue = u[(en[:, :, None] * dim + np.arange(dim)[None, None, :]).reshape(en.shape[0], -1)]
    energy = np.einsum("ei,ij,ej->e", ue, k0, ue)
    return -problem.p * problem.rho ** (problem.p - 1.0) * (problem.E0 - problem.Emin) * energy
