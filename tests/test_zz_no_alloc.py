"""The allocation-free preconditioner entry point against the allocating one.

feti_apply_precond_noalloc is for callers that cannot let the library call
cudaMalloc while they run; it keeps its work vectors in a static device array
instead of context memory.  Through the C ABI it must give the same Z and z as
feti_apply_precond (same kernels, same order, so equality is expected; the
check uses the parity tolerance 1e-12), on two calls in a row (the array keeps
the previous call's contents), and reject problems too large for the array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_precond_matches_allocating_entry_point_twice():
    import torch
    assert torch.cuda.is_available()
    p = workloads.config2(tiles=4, elems=8)
    s = fg.Solver(fg.FETI_FETIDP, fg.FETI_SCALING_K, fg.FETI_RRS,
                  stream=torch.cuda.current_stream().cuda_stream)
    s.setup(p)
    fg.feti_factorize(s.ctx)
    n = s.query(fg.FETI_Q_N_LAMBDA)
    ns = s.query(fg.FETI_Q_N_SUBDOMAINS)
    rng = np.random.default_rng(17)
    for call in range(2):
        r = torch.from_numpy(rng.standard_normal(n)).cuda()
        Z_ref = torch.full((ns, n), 7.0, dtype=torch.float64, device="cuda")
        z_ref = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
        fg.feti_apply_precond(s.ctx, r, Z_ref, n, z_ref)
        Z = torch.full((ns, n), -3.0, dtype=torch.float64, device="cuda")
        z = torch.full((n,), -3.0, dtype=torch.float64, device="cuda")
        fg.feti_apply_precond_noalloc(s.ctx, r, Z, n, z)
        assert _rel(Z.cpu().numpy(), Z_ref.cpu().numpy()) <= 1e-12, call
        assert _rel(z.cpu().numpy(), z_ref.cpu().numpy()) <= 1e-12, call
    s.close()


def test_noalloc_precond_rejects_oversized_interface():
    import torch
    # 32 x 32 tiles of 48 x 48 elements: 1984 interfaces x 47 nodes x 2 DOF x 2 copies = 372,992 > 262,144
    p = workloads.config2(tiles=32, elems=48)
    s = fg.Solver(fg.FETI_FETIDP, fg.FETI_SCALING_K, fg.FETI_PCG, stream=torch.cuda.current_stream().cuda_stream)
    s.setup(p)
    assert s.query(fg.FETI_Q_N_B_TOTAL) > 262144
    fg.feti_factorize(s.ctx)
    n = s.query(fg.FETI_Q_N_LAMBDA)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(fg.FetiError) as e:
        fg.feti_apply_precond_noalloc(s.ctx, r, None, n, z)
    assert e.value.status == fg.FETI_EINVAL
    s.close()
