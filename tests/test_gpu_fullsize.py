"""Full-size GPU parity: the dual operator (Eq. 12), the preconditioner (Eq. 13)
and the 3D solution against goldens the oracle wrote
(tests/golden/make_fullsize_goldens.py), element by element, in the launch
configurations bench.py times.

* 2D modular workload (16x16 subdomains of 32x32 Q4, contrast 1e9): F X for a
  256-column block at 256 sampled multipliers, FP64 and every reduced-precision
  form; the preconditioner columns Z and z = Z 1 of a residual.
* 3D workload (8^3 subdomains of 8^3 H8, contrast 1e9): F X for a 512-column
  block at 256 sampled multipliers, FP64 and every reduced-precision form.
* 3D solution (4^3 subdomains of 8^3 H8, the same field recipe): Algorithm 1 in
  FP64 and the refined split-BF16 / split-TF32 forms on every DOF, to the bars
  1e-8 (FP64) and 1e-6 (refined forms).

The test blocks are workloads.multiplier_block of each multiplier's
(subdomain, DOF) pair, rebuilt here from the library's own multiplier layout.

Tolerances (per element; derivations in the golden script's docstring):
* conditioning of the FP64 operator: the oracle's own output moves by
  delta = |Y_pert - Y| when every SIMP modulus is perturbed by ~2u (u = 2^-53);
  two FP64 implementations whose backward errors are n u (n = the local
  problem size n_r) may differ by up to n_r / 2 times that change.  The scale is
  the largest change in the element's column (one statistical sample, Kenney
  and Laub 1994), so the element bar is (n_r / 2) max_i delta_ij.
* rounding of the products: (2 u_f + (K + 8) u_32) A_loc for operands rounded to
  a format of unit roundoff u_f and FP32 accumulation over K terms, plus
  (2 u_f + (n_b + n_c + 8) u_32) A_cc (n_c <= 64) for the corner reduction (the
  same rounded operands on the tensor cores) and the FP32 coarse correction;
  u_f = 2^-11 (TF32), 2^-8 (BF16), 3 t^2 for the three-pass
  split of a format with unit roundoff t (its representation error t^2 and the
  dropped lo*lo term).
"""
import json
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import make_solver, rel, solve_u, torch_cuda  # noqa: E402

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U64, U32 = 2.0 ** -53, 2.0 ** -24
FORMATS = {  # precision -> (name, unit roundoff of the operands as multiplied)
    fg.FETI_TF32: ("tf32", 2.0 ** -11),
    fg.FETI_TF32X3: ("tf32x3", 3.0 * 2.0 ** -22),
    fg.FETI_BF16: ("bf16", 2.0 ** -8),
    fg.FETI_BF16X3: ("bf16x3", 3.0 * 2.0 ** -16),
}
REPORT = os.environ.get("FETI_PARITY_REPORT")


def report(name, **kv):
    """Measured error / tolerance ratios, appended to $FETI_PARITY_REPORT when set."""
    if REPORT:
        with open(REPORT, "a") as fh:
            fh.write(json.dumps({"test": name, **kv}) + "\n")


def load(name):
    path = os.path.join(GOLD, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    return dict(np.load(path))


def rho_hash_ok(problem, gold):
    import hashlib
    return hashlib.sha1(problem.rho.tobytes()).digest() == gold["rho_sha1"].tobytes()


def rows_of(layout, keys):
    """Library rows of the canonical keys, and the library's sign on every row."""
    kall, sign = workloads.multiplier_pairs(layout)
    index = {tuple(k): i for i, k in enumerate(map(tuple, kall.tolist()))}
    idx = np.array([index[tuple(k)] for k in keys.tolist()], np.int64)
    return idx, kall, sign


def apply_rows(solver, gold, m):
    """The library's F X at the golden's rows (sign-normalised), X rebuilt from its layout."""
    torch = torch_cuda()
    layout = fg.feti_lambda_layout(solver.ctx)
    idx, kall, sign = rows_of(layout, gold["keys"])
    n = kall.shape[0]
    assert n == int(gold["n_lam"])
    Xh = workloads.multiplier_block(kall, sign, m, seed=int(gold["seed_x"]))
    X = torch.from_numpy(np.ascontiguousarray(Xh.T)).cuda()           # column-major n x m
    del Xh
    Y = torch.zeros_like(X)
    fg.feti_apply_dual(solver.ctx, X, n, m, Y, n)
    torch.cuda.synchronize()
    Yr = Y[:, torch.from_numpy(idx).cuda()].T.cpu().numpy() * sign[idx, None]
    del X, Y
    return Yr


def fp64_scale(gold, key="Y"):
    """(n_r / 2) times the column-wise largest change of the oracle's output under a
    2u perturbation of the moduli."""
    d = np.abs(gold[key + "_pert"] - gold[key])
    return 0.5 * float(gold["n_r_max"]) * d.max(axis=0, keepdims=True)


def check_apply(name, Y, gold, precision):
    Yo = gold["Y"]
    A_loc = gold["A_loc"].astype(np.float64)
    A_cc = gold["A_cc"].astype(np.float64)
    K = int(gold["n_b_max"]) + 96
    if precision == fg.FETI_FP64:
        tol = fp64_scale(gold) + (K + 4) * U64 * A_loc
    else:
        uf = FORMATS[precision][1]
        tol = (fp64_scale(gold) + (2 * uf + (K + 8) * U32) * A_loc
               + (2 * uf + (int(gold["n_b_max"]) + 72) * U32) * A_cc)
    err = np.abs(Y - Yo)
    ratio = err / tol
    report(name, precision=precision, max_ratio=float(ratio.max()), median_ratio=float(np.median(ratio)),
           rel_err=rel(Y, Yo), max_err_over_colmax=float((err.max(0) / np.abs(Yo).max(0)).max()),
           pert_over_colmax=float((np.abs(gold["Y_pert"] - Yo).max(0) / np.abs(Yo).max(0)).max()))
    assert np.all(np.isfinite(Y))
    assert np.all(err <= tol), (name, float(ratio.max()), rel(Y, Yo))


# ------------------------------------------------------------------ 2D workload
@pytest.fixture(scope="module")
def gold2():
    g = load("fullsize_config2.npz")
    p = workloads.config2()
    assert rho_hash_ok(p, g)
    return p, g


@pytest.mark.parametrize("precision", [fg.FETI_FP64, fg.FETI_TF32, fg.FETI_TF32X3, fg.FETI_BF16, fg.FETI_BF16X3])
def test_config2_apply_matches_oracle(gold2, precision):
    p, g = gold2
    s = make_solver(p, tol=1e-6, precision=precision)
    fg.feti_factorize(s.ctx)
    Y = apply_rows(s, g, int(g["m"]))
    s.close()
    check_apply(f"config2_apply_{precision}", Y, g, precision)


def test_config2_precond_matches_oracle(gold2):
    torch = torch_cuda()
    p, g = gold2
    s = make_solver(p, tol=1e-6)
    fg.feti_factorize(s.ctx)
    layout = fg.feti_lambda_layout(s.ctx)
    idx, kall, sign = rows_of(layout, g["keys"])
    n = kall.shape[0]
    ns = p.n_subdomains
    r = torch.from_numpy(workloads.multiplier_block(kall, sign, 1, seed=int(g["seed_r"]))[:, 0].copy()).cuda()
    Z = torch.zeros((ns, n), dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    fg.feti_apply_precond(s.ctx, r, Z, n, z)
    s.close()
    Zr = Z.cpu().numpy()[:, idx].T * sign[idx, None]
    zr = z.cpu().numpy()[idx] * sign[idx]
    # conditioning scale from the perturbed oracle, per column; the products' rounding
    # (n_b + 4) u |S| |y| is below it by orders of magnitude at this size
    n_r = float(g["n_r_max"])
    tolZ = 0.5 * n_r * np.abs(g["Z_pert"] - g["Z"]).max(axis=0, keepdims=True) \
        + (int(g["n_b_max"]) + 4) * U64 * np.abs(g["Z"]).max(axis=0, keepdims=True)
    tolz = 0.5 * n_r * np.abs(g["z_pert"] - g["z"]).max() + (int(g["n_b_max"]) + 4) * U64 * np.abs(g["z"]).max()
    errZ = np.abs(Zr - g["Z"])
    report("config2_precond", max_ratio_Z=float(np.max(np.divide(errZ, tolZ, out=np.zeros_like(errZ), where=tolZ > 0))),
           max_ratio_z=float((np.abs(zr - g["z"]) / tolz).max()), rel_Z=rel(Zr, g["Z"]), rel_z=rel(zr, g["z"]))
    # block structure: column s is zero outside subdomain s's multipliers
    assert np.array_equal(Zr == 0, g["Z"] == 0)
    assert np.all(np.abs(Zr - g["Z"]) <= tolZ)
    assert np.all(np.abs(zr - g["z"]) <= tolz)


# ------------------------------------------------------------------ 3D workload
@pytest.fixture(scope="module")
def gold4():
    g = load("fullsize_config4.npz")
    p = workloads.config4()
    assert rho_hash_ok(p, g)
    return p, g


@pytest.mark.parametrize("precision", [fg.FETI_FP64, fg.FETI_TF32, fg.FETI_TF32X3, fg.FETI_BF16, fg.FETI_BF16X3])
def test_config4_apply_matches_oracle(gold4, precision):
    p, g = gold4
    s = make_solver(p, tol=1e-6, precision=precision)
    fg.feti_factorize(s.ctx)
    Y = apply_rows(s, g, int(g["m"]))
    s.close()
    check_apply(f"config4_apply_{precision}", Y, g, precision)


# ------------------------------------------------------------------ 3D solution
@pytest.fixture(scope="module")
def gold4s():
    g = load("solve_config4_4x4x4.npz")
    p = workloads.config4(tiles=4)
    assert rho_hash_ok(p, g)
    return p, g


@pytest.mark.parametrize("precision", [fg.FETI_FP64, fg.FETI_TF32X3, fg.FETI_BF16X3])
def test_config4_4x4x4_solution_matches_oracle(gold4s, precision):
    """Every DOF of the solution against the oracle's at the same tolerance (1e-10),
    to the stated bars: relative displacement error <= 1e-8 for the FP64 path and
    <= 1e-6 for the refined reduced-precision forms.  This field is well conditioned
    after diagonal scaling (kappa_2(D^-1/2 K D^-1/2) ~ 2e4, stored in the golden:
    kappa u ~ 1e-12), and the oracle's solution moves by only ~1e-14 when the moduli
    are perturbed by 2u, so both bars hold with margin for any backward-stable route;
    elementwise, no DOF may differ by more than the bar times the largest displacement."""
    p, g = gold4s
    u, st, c, s = solve_u(p, tol=float(g["tol"]), max_iter=200, precision=precision)
    s.close()
    uo = g["u_oracle"]
    bar = 1e-8 if precision == fg.FETI_FP64 else 1e-6
    assert float(g["kappa_scaled"]) * U64 < 1e-3 * bar
    report(f"config4_4x4x4_solution_{precision}", iterations=st.iterations, oracle_iterations=int(g["iterations"]),
           refinements=st.refinements, rel_err=rel(u, uo), rel_pert=rel(g["u_pert"], uo),
           rel_direct=rel(u, g["u_direct"]), oracle_rel_direct=rel(uo, g["u_direct"]))
    assert st.converged
    assert rel(u, uo) <= bar
    assert np.abs(u - uo).max() <= bar * np.abs(uo).max()
    assert c == pytest.approx(float(p.f @ uo), rel=bar)
    if precision == fg.FETI_FP64:     # Algorithm 1 on both sides: iteration counts within 10% or 2
        assert abs(st.iterations - int(g["iterations"])) <= max(2, 0.1 * int(g["iterations"]))


# ------------------------------------------------------------------ 2D bench solve
def test_config2_bench_solve_matches_oracle():
    """The bench workload's own solve (FETI-DP + k + Algorithm 1, tol 1e-6, the
    launch configuration bench.py times) against the oracle's at 4,096 sampled
    DOFs and in the compliance.  At contrast 1e9 the solve amplifies round-off:
    the oracle's own solution moves by ||u_pert - u|| when the SIMP moduli are
    perturbed by 2u; both solutions carry the round-off of n_r-sized local
    solves, so the bar is (n_r / 2) times that change (elementwise: times its
    largest entry; the compliance: times the change of the compliance)."""
    g = load("solve_config2.npz")
    p = workloads.config2()
    assert rho_hash_ok(p, g)
    u, st, c, s = solve_u(p, tol=float(g["tol"]))
    s.close()
    idx = g["dof"]
    scale = 0.5 * float(g["n_r_max"])
    d_el = np.abs(u[idx] - g["u_oracle"]).max()
    report("config2_bench_solve", iterations=st.iterations, oracle_iterations=int(g["iterations"]),
           rel_sampled=rel(u[idx], g["u_oracle"]), pert_rel=float(g["pert_norm"] / g["u_norm"]),
           ratio_elem=float(d_el / (scale * g["pert_max"])),
           ratio_compliance=float(abs(c - g["compliance"]) / (scale * abs(g["compliance_pert"] - g["compliance"]))))
    assert st.converged
    assert abs(st.iterations - int(g["iterations"])) <= max(2, 0.1 * int(g["iterations"]))
    assert d_el <= scale * float(g["pert_max"])
    assert abs(c - float(g["compliance"])) <= scale * abs(float(g["compliance_pert"]) - float(g["compliance"]))
