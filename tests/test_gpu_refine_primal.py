"""The FP64 primal residual r = f - K u (element by element, Eq. 2 with the
moduli of Eq. 1) and the precision form refined on it (FETI_REFINE_PRIMAL).

* feti_primal_residual against the oracle's assembled K (2D and 3D, batch of
  uneven problems too): element by element, within the FP64 rounding of the
  element sums.
* At moderate stiffness contrast the primal refinement with split-precision
  blocks reaches the mixed-path bar (<= 1e-6 relative displacement error
  against a direct solve of Eq. 2) and its reported residual ratio is the one
  feti_primal_residual gives for the recovered u.
"""
import numpy as np
import pytest

import workloads
from oracle.assemble import direct_solve, global_stiffness

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import make_solver, rel, torch_cuda  # noqa: E402


def moderate(dim=2, tiles=3, elems=6, seed=7):
    if dim == 2:
        p = workloads.config2(tiles=tiles, elems=elems)
    else:
        p = workloads.config4(tiles=tiles, elems=elems)
    rng = np.random.default_rng(seed)
    p.rho = np.where(rng.random(p.rho.size) < 0.3, 0.3, 1.0)
    p.Emin = 1e-9
    return p


def oracle_residual(p, u):
    K = global_stiffness(p)
    r = p.f - K @ u
    r[np.asarray(p.dirichlet, bool)] = 0.0
    bound = np.abs(K) @ np.abs(u) + np.abs(p.f)
    return r, bound


@pytest.mark.parametrize("dim", [2, 3])
def test_primal_residual_matches_oracle(dim):
    torch = torch_cuda()
    p = moderate(dim=dim, tiles=3, elems=5 if dim == 3 else 7)
    s = make_solver(p)
    fg.feti_factorize(s.ctx)
    u = np.random.default_rng(3).standard_normal(p.n_dofs)
    u_d = torch.from_numpy(u).cuda()
    r_d = torch.empty_like(u_d)
    ratio = fg.feti_primal_residual(s.ctx, u_d, r_d)
    r = r_d.cpu().numpy()
    r_o, bound = oracle_residual(p, u)
    # each entry sums at most 8 (2D: 4) element rows of 24 (8) products
    assert np.all(np.abs(r - r_o) <= 64 * np.finfo(float).eps * bound)
    free = ~np.asarray(p.dirichlet, bool)
    assert ratio == pytest.approx(np.linalg.norm(r_o) / np.linalg.norm(p.f[free]), rel=1e-12)
    # u = 0: the free part of f
    r0 = torch.empty_like(u_d)
    assert fg.feti_primal_residual(s.ctx, None, r0) == pytest.approx(1.0, rel=1e-15)
    f_free = np.where(free, p.f, 0.0)
    assert np.array_equal(r0.cpu().numpy(), f_free)
    s.close()


def test_primal_residual_of_a_batch():
    torch = torch_cuda()
    probs = workloads.config3(n_problems=3, tile_range=(2, 3), elem_range=(4, 6), seed=9)
    o = fg.feti_options_default()
    ctx = fg.feti_create(o, torch.cuda.current_stream().cuda_stream)
    keep, structs = [], []
    for p in probs:
        rho = torch.from_numpy(p.rho).cuda()
        f = torch.from_numpy(p.f).cuda()
        d = np.ascontiguousarray(p.dirichlet, np.uint8)
        keep += [rho, f, d]
        structs.append(fg.make_problem(p.dim, p.tiles, p.elems, p.E0, p.Emin, p.nu, p.p, rho, d, f, True))
    fg.feti_setup_batch(ctx, structs)
    fg.feti_factorize(ctx)
    n = sum(p.n_dofs for p in probs)
    u = np.random.default_rng(5).standard_normal(n)
    u_d = torch.from_numpy(u).cuda()
    r_d = torch.empty_like(u_d)
    fg.feti_primal_residual(ctx, u_d, r_d)
    r = r_d.cpu().numpy()
    off = 0
    for p in probs:
        r_o, bound = oracle_residual(p, u[off:off + p.n_dofs])
        assert np.all(np.abs(r[off:off + p.n_dofs] - r_o) <= 64 * np.finfo(float).eps * bound)
        off += p.n_dofs
    fg.feti_destroy(ctx)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_primal_refinement_reaches_mixed_bar(precision):
    torch = torch_cuda()
    prec = {"bf16x3": fg.FETI_BF16X3, "tf32x3": fg.FETI_TF32X3}[precision]
    p = moderate(dim=2, tiles=4, elems=8)
    s = fg.Solver(fg.FETI_FETIDP, fg.FETI_SCALING_K, fg.FETI_RRS, tol=1e-10, max_iter=500,
                  stream=torch.cuda.current_stream().cuda_stream, precision=prec,
                  refine=fg.FETI_REFINE_PRIMAL, max_refine=12)
    s.setup(p, rho=torch.from_numpy(p.rho).cuda(), f=torch.from_numpy(p.f).cuda(), on_device=True)
    fg.feti_factorize(s.ctx)
    status, st = fg.feti_solve_dual(s.ctx, allow_notconv=True)
    u = torch.empty(p.n_dofs, dtype=torch.float64, device="cuda")
    fg.feti_recover_displacements(s.ctx, u, True)
    ud = direct_solve(p)
    assert st.refinements >= 1
    assert rel(u.cpu().numpy(), ud) <= 1e-6, (st.refinements, st.eps)
    # the reported ratio is the primal residual of the accumulated solution;
    # the recovered u (from the summed multipliers) has the same one up to rounding
    ratio = fg.feti_primal_residual(s.ctx, u)
    assert ratio <= max(10 * st.eps, 1e-9)
    s.close()
