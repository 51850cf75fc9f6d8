"""The allocation-free preconditioner entry point against the allocating one.

feti_apply_precond_noalloc is for callers that cannot let the library call
cudaMalloc while they run; it keeps its work vectors in a static device array
instead of context memory.  Through the C ABI it must give the same Z and z as
feti_apply_precond (same kernels, same order, so equality is expected; the
check uses the parity tolerance 1e-12), on two calls in a row (the array keeps
the previous call's contents), without moving the device's free memory, and
reject problems too large for the array.
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
        torch.cuda.synchronize()
        # the call allocates nothing: neither the context's device memory nor the
        # device's free memory moves (checked from the second call on; the first
        # call on a device may load the library's module)
        bytes0 = s.query(fg.FETI_Q_DEVICE_BYTES)
        free0 = torch.cuda.mem_get_info()[0]
        fg.feti_apply_precond_noalloc(s.ctx, r, Z, n, z)
        if call > 0:
            assert s.query(fg.FETI_Q_DEVICE_BYTES) == bytes0
            assert torch.cuda.mem_get_info()[0] == free0
        assert _rel(Z.cpu().numpy(), Z_ref.cpu().numpy()) <= 1e-12, call
        assert _rel(z.cpu().numpy(), z_ref.cpu().numpy()) <= 1e-12, call
    s.close()


def test_noalloc_precond_rejects_oversized_interface():
    import torch
    # 64 x 64 tiles of 12 x 12 elements: 8064 interfaces x 11 nodes x 2 DOF x 2 copies = 354,816 > 262,144;
    # the size is rejected right after set-up, before any factorization
    p = workloads.config2(tiles=64, elems=12)
    s = fg.Solver(fg.FETI_FETIDP, fg.FETI_SCALING_K, fg.FETI_PCG, stream=torch.cuda.current_stream().cuda_stream)
    s.setup(p)
    assert s.query(fg.FETI_Q_N_B_TOTAL) > 262144
    n = s.query(fg.FETI_Q_N_LAMBDA)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(fg.FetiError) as e:
        fg.feti_apply_precond_noalloc(s.ctx, r, None, n, z)
    assert e.value.status == fg.FETI_EINVAL
    s.close()
