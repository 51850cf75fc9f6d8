"""The failure path of the tensor-core pipeline's bounded waits (FETI_ETIMEOUT),
driven without any fault: the test hook feti_test_skip_copy makes the first
tile of the next TF32 product stop before one of its copies, so the MMA lane's
wait for it runs out (1 s limit).  The call must report FETI_ETIMEOUT within a
few seconds, and the same context must then give the same operator as before,
bit for bit, and still solve."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import make_solver, torch_cuda  # noqa: E402


def test_bounded_wait_times_out_and_context_recovers():
    torch = torch_cuda()
    p = workloads.config2(tiles=3, elems=8)
    p.rho = np.where(p.rho < 0.5, 0.1, 1.0)
    s = make_solver(p, tol=1e-8, precision=fg.FETI_TF32)
    fg.feti_factorize(s.ctx)
    n = s.query(fg.FETI_Q_N_LAMBDA)
    X = torch.from_numpy(np.random.default_rng(5).standard_normal((16, n))).cuda()
    Y0 = torch.zeros_like(X)
    fg.feti_apply_dual(s.ctx, X, n, 16, Y0, n)
    Y1 = torch.zeros_like(X)
    fg.feti_test_skip_copy(s.ctx, 1)
    t0 = time.perf_counter()
    with pytest.raises(fg.FetiError) as e:
        fg.feti_apply_dual(s.ctx, X, n, 16, Y1, n)
    elapsed = time.perf_counter() - t0
    assert e.value.status == fg.FETI_ETIMEOUT
    assert "timed out" in fg.feti_last_error(s.ctx)
    assert elapsed < 20.0
    # the hook acted once; the context is usable and gives the same operator
    Y2 = torch.zeros_like(X)
    fg.feti_apply_dual(s.ctx, X, n, 16, Y2, n)
    assert torch.equal(Y2, Y0)
    status, st = fg.feti_solve_dual(s.ctx)
    assert st.converged
    s.close()
