"""The precision form: local dual blocks F_s / S_s as diagonally scaled TF32
products on the tensor cores (tcgen05, FP32 accumulation) inside FP64
iterative refinement on the dual residual.

* The tensor-core operator against the FP64 operator: normwise relative
  difference of F X within the TF32 rounding of the scaled blocks (<= 3e-3).
* The three-pass split-TF32 operator (hi*hi + hi*lo + lo*hi) is FP32-class:
  within 2e-5 of the FP64 operator and at least 20x closer than one pass.
* BF16 (kind::f16 with BF16 inputs): one pass within the BF16 rounding of the
  scaled blocks (<= 1e-2), the split product within 2e-4 and at least 20x
  closer than one pass; the refined split-BF16 solve reaches the FP64 bar.
* At moderate stiffness contrast the refined solution reaches the FP64 bar
  (<= 1e-8 relative displacement error against a direct solve of Eq. 2).
"""
import numpy as np
import pytest

import workloads
from oracle.assemble import direct_solve

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import make_solver, rel, solve_u, torch_cuda  # noqa: E402


def moderate(tiles=4, elems=8, lo=0.1):
    p = workloads.config2(tiles=tiles, elems=elems)
    p.rho = np.where(p.rho < 0.5, lo, 1.0)
    p.Emin = 1e-9
    return p


@pytest.mark.parametrize("m", [1, 16, 64, 300])
def test_tensor_core_operator_close_to_fp64(m):
    torch = torch_cuda()
    p = moderate(tiles=5, elems=12)
    s64 = make_solver(p)
    s32 = make_solver(p, precision=fg.FETI_TF32)
    fg.feti_factorize(s64.ctx)
    fg.feti_factorize(s32.ctx)
    n = s64.query(fg.FETI_Q_N_LAMBDA)
    X = torch.from_numpy(np.random.default_rng(m).standard_normal((m, n))).cuda()
    Y64 = torch.zeros_like(X)
    Y32 = torch.zeros_like(X)
    fg.feti_apply_dual(s64.ctx, X, n, m, Y64, n)
    fg.feti_apply_dual(s32.ctx, X, n, m, Y32, n)
    a, b = Y32.cpu().numpy(), Y64.cpu().numpy()
    assert rel(a, b) <= 3e-3
    assert rel(a, b) > 0.0          # the tensor-core path really ran in reduced precision


@pytest.mark.parametrize("m", [1, 37, 256])
def test_split_tf32_operator_is_fp32_class(m):
    torch = torch_cuda()
    p = moderate(tiles=5, elems=12)
    s64 = make_solver(p)
    s1 = make_solver(p, precision=fg.FETI_TF32)
    s3 = make_solver(p, precision=fg.FETI_TF32X3)
    for s in (s64, s1, s3):
        fg.feti_factorize(s.ctx)
    n = s64.query(fg.FETI_Q_N_LAMBDA)
    X = torch.from_numpy(np.random.default_rng(100 + m).standard_normal((m, n))).cuda()
    Ys = []
    for s in (s64, s1, s3):
        Y = torch.zeros_like(X)
        fg.feti_apply_dual(s.ctx, X, n, m, Y, n)
        Ys.append(Y.cpu().numpy())
    d1, d3 = rel(Ys[1], Ys[0]), rel(Ys[2], Ys[0])
    assert 0.0 < d3 <= 2e-5
    assert d3 * 20 <= d1


def test_refined_split_tf32_solve_needs_few_refinements():
    # with inner solves to 1e-5 (near the split product's accuracy) two or
    # three FP64 refinement steps reach 1e-10; one TF32 pass cannot do that
    p = moderate()
    ud = direct_solve(p)
    u, st, c, _ = solve_u(p, tol=1e-10, precision=fg.FETI_TF32X3, inner_tol=1e-5)
    assert st.converged and 1 <= st.refinements <= 3
    assert rel(u, ud) <= 1e-8
    _, st1, _, _ = solve_u(p, tol=1e-10, precision=fg.FETI_TF32, inner_tol=1e-5, max_iter=300)
    assert st1.refinements > st.refinements or not st1.converged


@pytest.mark.parametrize("method", ["fetidp", "tfeti"])
def test_refined_tf32_solve_reaches_fp64_accuracy(method):
    p = moderate() if method == "fetidp" else workloads.config1()
    ud = direct_solve(p)
    u, st, c, _ = solve_u(p, method=method, tol=1e-10, precision=fg.FETI_TF32)
    assert st.converged and st.refinements >= 1
    assert rel(u, ud) <= 1e-8
    u64, st64, _, _ = solve_u(p, method=method, tol=1e-10)
    assert rel(u, u64) <= 1e-8


@pytest.mark.parametrize("m", [1, 40, 300])
def test_bf16_operators(m):
    torch = torch_cuda()
    p = moderate(tiles=5, elems=12)
    solvers = [make_solver(p), make_solver(p, precision=fg.FETI_BF16), make_solver(p, precision=fg.FETI_BF16X3)]
    for s in solvers:
        fg.feti_factorize(s.ctx)
    n = solvers[0].query(fg.FETI_Q_N_LAMBDA)
    X = torch.from_numpy(np.random.default_rng(200 + m).standard_normal((m, n))).cuda()
    Ys = []
    for s in solvers:
        Y = torch.zeros_like(X)
        fg.feti_apply_dual(s.ctx, X, n, m, Y, n)
        Ys.append(Y.cpu().numpy())
    d1, d3 = rel(Ys[1], Ys[0]), rel(Ys[2], Ys[0])
    assert 0.0 < d1 <= 1e-2
    assert 0.0 < d3 <= 2e-4
    assert d3 * 20 <= d1


@pytest.mark.parametrize("method", ["fetidp", "tfeti"])
def test_refined_split_bf16_solve_reaches_fp64_accuracy(method):
    p = moderate() if method == "fetidp" else workloads.config1()
    ud = direct_solve(p)
    u, st, c, _ = solve_u(p, method=method, tol=1e-10, precision=fg.FETI_BF16X3, max_iter=600)
    assert st.converged and st.refinements >= 1
    assert rel(u, ud) <= 1e-8
