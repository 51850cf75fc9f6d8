"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: both sides compute in FP64 with different summation orders and
different (equally valid) factorisation routes, so at moderate stiffness
contrast block-level quantities agree to ~1e-11 relative and solves at
tol 1e-12 reach the direct solution of Eq. (2) to <= 1e-8 relative
displacement error (the bar for the FP64 path).  At the 1e9 contrast of the
modular workload no FP64 route reaches 1e-8 (the oracle itself stops at
~2e-6 against the direct solve, set by the conditioning), so there the GPU
must be as accurate as the oracle: error <= 3x the oracle's, or 1e-8.  The
full-size workloads are compared in tests/test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.assemble import direct_solve
from oracle.sensitivity import compliance_gradient

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import lambda_perm, make_solver, rel, solve_u, torch_cuda  # noqa: E402


def moderate_modules(tiles=4, elems=8):
    """The modular workload's layout with densities {0.3, 1} and Emin = 1e-6 (contrast ~40)."""
    p = workloads.config2(tiles=tiles, elems=elems)
    p.rho = np.where(p.rho < 0.5, 0.3, 1.0)
    p.Emin = 1e-6
    return p


@pytest.fixture(scope="module")
def small_dp():
    p = moderate_modules()
    op = oracle.build(p, "fetidp", "k")
    return p, op


def test_local_blocks_match_oracle(small_dp):
    p, op = small_dp
    s = make_solver(p)
    fg.feti_factorize(s.ctx)
    for sub in range(p.n_subdomains):
        blk = fg.feti_local_blocks(s.ctx, sub)
        M = op.mod(sub)
        r_loc = op.r_loc[sub]
        o_b = r_loc[op.bset[sub]]                       # oracle b DOFs (local ids)
        pos = {int(d): k for k, d in enumerate(o_b)}
        perm = np.array([pos[int(d)] for d in blk["bdofs"]])
        assert sorted(blk["cdofs"].tolist()) == sorted(op.c_loc[sub].tolist())
        cpos = {int(d): k for k, d in enumerate(op.c_loc[sub])}
        cperm = np.array([cpos[int(d)] for d in blk["cdofs"]])
        assert rel(blk["F"], M.Fb[np.ix_(perm, perm)]) <= 1e-11
        assert rel(blk["S"], M.S[np.ix_(perm, perm)]) <= 1e-11
        assert rel(blk["Frc"], M.Frc_b[np.ix_(perm, cperm)]) <= 1e-11


@pytest.mark.parametrize("m", [1, 7, 16])
def test_apply_dual_matches_oracle(small_dp, m):
    torch = torch_cuda()
    p, op = small_dp
    s = make_solver(p)
    fg.feti_factorize(s.ctx)
    perm = lambda_perm(op, fg.feti_lambda_layout(s.ctx), "fetidp")
    n = perm.size
    Xo = np.random.default_rng(m).standard_normal((n, m))
    Yo = op.apply_F(Xo)
    X = torch.from_numpy(np.ascontiguousarray(Xo[perm].T)).cuda()     # column-major n x m
    Y = torch.zeros_like(X)
    fg.feti_apply_dual(s.ctx, X, n, m, Y, n)
    assert rel(Y.cpu().numpy().T, Yo[perm]) <= 1e-12


def test_precond_matches_oracle(small_dp):
    torch = torch_cuda()
    p, op = small_dp
    s = make_solver(p)
    fg.feti_factorize(s.ctx)
    perm = lambda_perm(op, fg.feti_lambda_layout(s.ctx), "fetidp")
    n = perm.size
    ro = np.random.default_rng(3).standard_normal(n)
    Zo = op.precond_columns(ro)
    r = torch.from_numpy(ro[perm].copy()).cuda()
    Z = torch.zeros((p.n_subdomains, n), dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    fg.feti_apply_precond(s.ctx, r, Z, n, z)
    assert rel(Z.cpu().numpy().T, Zo[perm]) <= 1e-12
    assert rel(z.cpu().numpy(), Zo.sum(axis=1)[perm]) <= 1e-12


@pytest.mark.parametrize("method", ["tfeti", "fetidp"])
@pytest.mark.parametrize("scaling", ["k", "mult"])
@pytest.mark.parametrize("krylov", ["pcg", "fo", "rrs"])
def test_twelve_variants_config1(method, scaling, krylov):
    p = workloads.config1()
    ud = direct_solve(p)
    u, st, c, _ = solve_u(p, method=method, scaling=scaling, krylov=krylov, tol=1e-12, max_iter=400)
    assert st.converged
    assert rel(u, ud) <= 1e-8
    _, _, info, _ = oracle.solve(p, method, scaling, krylov, tol=1e-12, max_iter=400)
    assert abs(st.iterations - info.iterations) <= max(2, 0.1 * info.iterations)
    assert c == pytest.approx(p.f @ ud, rel=1e-8)


def test_fetidp_rrs_moderate_contrast_matches_oracle(small_dp):
    p, op = small_dp
    ud = direct_solve(p)
    u, st, c, _ = solve_u(p, tol=1e-12)
    uo, _, info, _ = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-12, op=op)
    assert st.converged
    assert rel(u, uo) <= 1e-8 and rel(u, ud) <= 1e-8
    assert abs(st.iterations - info.iterations) <= max(2, 0.1 * info.iterations)


@pytest.mark.parametrize("tiles,elems", [(4, 8), (5, 12)])
def test_fetidp_rrs_contrast_1e9_as_accurate_as_oracle(tiles, elems):
    p = workloads.config2(tiles=tiles, elems=elems)
    ud = direct_solve(p)
    u, st, c, _ = solve_u(p, tol=1e-10)
    uo, _, info, _ = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-10)
    assert st.converged
    e_gpu, e_orc = rel(u, ud), rel(uo, ud)
    # at contrast 1e9 the iteration count depends on round-off; accuracy is what is unique
    assert e_gpu <= max(1e-8, 3.0 * e_orc), (e_gpu, e_orc, st.iterations, info.iterations)


def test_ragged_tiles_and_host_inputs():
    # non-square tiles and elements, densities and loads from host memory
    rng = np.random.default_rng(9)
    rho = rng.uniform(0.05, 1.0, size=(3 * 5) * (2 * 3))
    p = workloads.tile_problem("ragged", 2, (3, 2), (5, 3), rho, Emin=1e-6)
    ud = direct_solve(p)
    for method in ("fetidp", "tfeti"):
        u, st, _, _ = solve_u(p, method=method, tol=1e-12, on_device=False)
        assert st.converged and rel(u, ud) <= 1e-8


def test_three_dimensional_small():
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.2, 1.0, size=4 * 4 * 4)
    p = workloads.tile_problem("3d", 3, (2, 2, 2), (2, 2, 2), rho, Emin=1e-6)
    ud = direct_solve(p)
    for method in ("fetidp", "tfeti"):
        u, st, _, _ = solve_u(p, method=method, tol=1e-12)
        assert st.converged and rel(u, ud) <= 1e-8


def test_compliance_gradient_matches_oracle():
    torch = torch_cuda()
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.3, 1.0, size=8 * 8)
    p = workloads.tile_problem("fd", 2, (2, 2), (4, 4), rho, Emin=1e-6)
    u, st, c, s = solve_u(p, tol=1e-12)
    g = torch.empty(p.n_elements, dtype=torch.float64, device="cuda")
    fg.feti_compliance_grad(s.ctx, g, True)
    g_ref = compliance_gradient(p, direct_solve(p))
    assert rel(g.cpu().numpy(), g_ref) <= 1e-8


def test_module_dedup_is_exact():
    p = workloads.config2(tiles=4, elems=8)
    a = solve_u(p, dedup=True, tol=1e-10)
    b = solve_u(p, dedup=False, tol=1e-10)
    assert a[3].query(fg.FETI_Q_N_MODULES) < b[3].query(fg.FETI_Q_N_MODULES)
    assert np.array_equal(a[0], b[0])


def test_deterministic_repeat():
    p = workloads.config2(tiles=4, elems=8)
    u1 = solve_u(p, tol=1e-8)[0]
    u2 = solve_u(p, tol=1e-8)[0]
    assert np.array_equal(u1, u2)


def test_call_order_and_bad_arguments():
    torch = torch_cuda()
    p = workloads.config1()
    s = make_solver(p)
    with pytest.raises(fg.FetiError) as e:
        fg.feti_solve_dual(s.ctx)
    assert e.value.status == fg.FETI_ESTATE
    fg.feti_factorize(s.ctx)
    with pytest.raises(fg.FetiError) as e:
        fg.feti_recover_displacements(s.ctx, None, True)
    assert e.value.status == fg.FETI_ESTATE
    n = s.query(fg.FETI_Q_N_LAMBDA)
    X = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(fg.FetiError) as e:
        fg.feti_apply_dual(s.ctx, X, n - 1, 1, X, n)
    assert e.value.status == fg.FETI_EINVAL


def test_singular_stiffness_reports_breakdown():
    # zero density with Emin = 0: K_ii is singular; the library must report it, not fault
    p = workloads.config2(tiles=2, elems=4)
    p.rho[:] = 0.0
    s = make_solver(p)
    with pytest.raises(fg.FetiError) as e:
        fg.feti_factorize(s.ctx)
    assert e.value.status == fg.FETI_EBREAKDOWN


def test_fetidp_rrs_8x8_modules_accuracy():
    """A larger case of the modular workload at tol 1e-6.  At contrast 1e9 the
    iteration count of this case depends on round-off (the same oracle needs
    59 iterations on an x86 host and 14 on an Arm host; the GPU ~48), so only
    the accuracy against the direct solve is compared: no worse than 3x the
    oracle's."""
    p = workloads.config2(tiles=8, elems=32)
    ud = direct_solve(p)
    u, st, _, _ = solve_u(p, tol=1e-6)
    uo, _, info, _ = oracle.solve(p, "fetidp", "k", "rrs", tol=1e-6)
    assert st.converged and info.converged
    e_gpu, e_orc = rel(u, ud), rel(uo, ud)
    assert e_gpu <= max(1e-8, 3.0 * e_orc), (e_gpu, e_orc, st.iterations, info.iterations)
