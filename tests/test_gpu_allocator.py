"""The boundary's ownership rule: a context's internal device memory comes from
the caller's allocator when one is installed (feti_set_allocator), here
PyTorch's caching allocator.  The solve then makes no device allocation of its
own: every byte the library holds during set-up, factorization and the solve
(including the Krylov history blocks allocated while iterating) is accounted for
by the allocator, and all of it is returned at destroy; the results equal those
of a context on the default (stream-ordered) allocation bit for bit."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

fg = pytest.importorskip("paper_2111_11728_gb300")
from gpu_helpers import torch_cuda  # noqa: E402


def _solve(p, allocator):
    torch = torch_cuda()
    s = fg.Solver(fg.FETI_FETIDP, fg.FETI_SCALING_K, fg.FETI_RRS, tol=1e-10,
                  stream=torch.cuda.current_stream().cuda_stream, allocator=allocator)
    s.setup(p, rho=torch.from_numpy(p.rho).cuda(), f=torch.from_numpy(p.f).cuda(), on_device=True)
    fg.feti_factorize(s.ctx)
    return s


def test_torch_allocator_serves_all_internal_memory():
    torch = torch_cuda()
    p = workloads.config2(tiles=4, elems=8)
    # the driver loads a kernel's code on its first launch (lazy module loading),
    # in device memory of its own: launch every kernel of the pipeline once, in a
    # throwaway context, before measuring
    w = _solve(p, None)
    fg.feti_solve_dual(w.ctx)
    fg.feti_recover_displacements(w.ctx, torch.empty(p.n_dofs, dtype=torch.float64, device="cuda"), True)
    w.close()
    torch.cuda.synchronize()
    alloc = fg.TorchAllocator()
    s = _solve(p, alloc)
    assert alloc.n_alloc > 0 and alloc.bytes_held == s.query(fg.FETI_Q_DEVICE_BYTES)
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    outside0 = total - free0 - torch.cuda.memory_reserved()       # device memory torch does not manage
    n0 = alloc.n_alloc
    status, st = fg.feti_solve_dual(s.ctx)
    u = torch.empty(p.n_dofs, dtype=torch.float64, device="cuda")
    fg.feti_recover_displacements(s.ctx, u, True)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    outside1 = total - free1 - torch.cuda.memory_reserved()
    assert alloc.n_alloc > n0                       # the history blocks came from the allocator
    assert outside1 == outside0                     # and nothing from anywhere else
    assert alloc.bytes_held == s.query(fg.FETI_Q_DEVICE_BYTES)
    s.close()
    assert alloc.bytes_held == 0 and alloc.n_free == alloc.n_alloc
    # the same solve on the default allocation
    s2 = _solve(p, None)
    fg.feti_solve_dual(s2.ctx)
    u2 = torch.empty(p.n_dofs, dtype=torch.float64, device="cuda")
    fg.feti_recover_displacements(s2.ctx, u2, True)
    s2.close()
    assert st.converged and np.array_equal(u.cpu().numpy(), u2.cpu().numpy())


def test_allocator_only_before_setup():
    torch = torch_cuda()
    p = workloads.config2(tiles=2, elems=4)
    s = _solve(p, None)
    with pytest.raises(fg.FetiError) as e:
        fg.feti_set_allocator(s.ctx, fg.TorchAllocator())
    assert e.value.status == fg.FETI_ESTATE
    s.close()
