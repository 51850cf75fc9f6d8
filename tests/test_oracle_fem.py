"""Pins of the oracle's finite-element layer (Eq. 1; Section 4.2 elements).

k0 is checked against (a) the Hessian of the exact strain energy of the
interpolated displacement field, integrated symbolically, (b) the patch test
(a uniform strain field stores exactly eps^T D eps per unit volume), and (c)
its null space (3 rigid modes in 2D, 6 in 3D).  None of these reuse the
oracle's strain-displacement matrix or quadrature.
"""
import numpy as np
import pytest

from oracle import fem


def test_simp_modulus_closed_form():
    # Eq. (1): E(0) = Emin, E(1) = E0, E(1/2) = Emin + (E0 - Emin) / 2^p.
    E = fem.simp_modulus(np.array([0.0, 1.0, 0.5]), 2.0, 1e-3, 3.0)
    assert E[0] == pytest.approx(1e-3, rel=1e-15)
    assert E[1] == pytest.approx(2.0, rel=1e-15)
    assert E[2] == pytest.approx(1e-3 + (2.0 - 1e-3) / 8.0, rel=1e-15)


def _symbolic_k0(dim, nu):
    sympy = pytest.importorskip("sympy")
    xs = sympy.symbols("x0:%d" % dim)
    nodes = fem.Q4_NODES if dim == 2 else fem.H8_NODES
    q = sympy.symbols("q0:%d" % (dim * len(nodes)))
    disp = []
    for d in range(dim):
        expr = 0
        for a, na in enumerate(nodes):
            N = 1
            for ax in range(dim):
                N *= xs[ax] if na[ax] == 1 else (1 - xs[ax])
            expr += N * q[dim * a + d]
        disp.append(expr)
    nu_s = sympy.Rational(str(nu))
    if dim == 2:
        exx, eyy = sympy.diff(disp[0], xs[0]), sympy.diff(disp[1], xs[1])
        gxy = sympy.diff(disp[0], xs[1]) + sympy.diff(disp[1], xs[0])
        # plane-stress energy density for E = 1
        w = (exx ** 2 + eyy ** 2 + 2 * nu_s * exx * eyy) / (2 * (1 - nu_s ** 2)) + gxy ** 2 / (4 * (1 + nu_s))
    else:
        lam = nu_s / ((1 + nu_s) * (1 - 2 * nu_s))
        mu = 1 / (2 * (1 + nu_s))
        grad = [[sympy.diff(disp[i], xs[j]) for j in range(3)] for i in range(3)]
        eps = [[(grad[i][j] + grad[j][i]) / 2 for j in range(3)] for i in range(3)]
        tr = eps[0][0] + eps[1][1] + eps[2][2]
        w = lam / 2 * tr ** 2 + mu * sum(eps[i][j] ** 2 for i in range(3) for j in range(3))
    w = sympy.expand(w)
    for x in xs:
        w = sympy.integrate(w, (x, 0, 1))
    H = sympy.hessian(w, q)
    return np.array(H.evalf(), dtype=np.float64)


@pytest.mark.parametrize("dim", [2, 3])
def test_k0_equals_exact_energy_hessian(dim):
    k0 = fem.element_stiffness(dim, 0.3)
    ref = _symbolic_k0(dim, 0.3)
    assert np.abs(k0 - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_k0_patch_test(dim):
    nu = 0.3
    k0 = fem.element_stiffness(dim, nu)
    nodes = fem.Q4_NODES if dim == 2 else fem.H8_NODES
    rng = np.random.default_rng(7)
    for _ in range(5):
        G = rng.standard_normal((dim, dim))       # u(x) = G x
        u = (nodes.astype(float) @ G.T).ravel()
        eps = 0.5 * (G + G.T)
        if dim == 2:
            # plane stress energy density, E = 1
            w = (eps[0, 0] ** 2 + eps[1, 1] ** 2 + 2 * nu * eps[0, 0] * eps[1, 1]) / (1 - nu ** 2) \
                + 2 * eps[0, 1] ** 2 / (1 + nu)
        else:
            lam = nu / ((1 + nu) * (1 - 2 * nu))
            mu = 1 / (2 * (1 + nu))
            w = lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)
        assert u @ k0 @ u == pytest.approx(w, rel=1e-13)


@pytest.mark.parametrize("dim,n_rbm", [(2, 3), (3, 6)])
def test_k0_null_space_is_rigid_motion(dim, n_rbm):
    k0 = fem.element_stiffness(dim, 0.3)
    nodes = fem.Q4_NODES if dim == 2 else fem.H8_NODES
    R = fem.rigid_body_modes(nodes)
    assert np.abs(k0 @ R).max() < 1e-14
    ev = np.linalg.eigvalsh(k0)
    assert np.sum(ev < 1e-12) == n_rbm
    assert ev.min() > -1e-14
    assert np.allclose(k0, k0.T)


def test_rigid_body_modes_are_rigid():
    # a rigid motion has zero symmetric gradient: check on random points
    rng = np.random.default_rng(1)
    for dim in (2, 3):
        pts = rng.standard_normal((10, dim))
        R = fem.rigid_body_modes(pts)
        for q in range(R.shape[1]):
            U = R[:, q].reshape(-1, dim)
            # fit U = A x + b exactly and check A antisymmetric
            X = np.hstack([pts, np.ones((10, 1))])
            coef, *_ = np.linalg.lstsq(X, U, rcond=None)
            A = coef[:dim].T
            assert np.allclose(A + A.T, 0, atol=1e-12)
            assert np.allclose(X @ coef, U, atol=1e-12)
