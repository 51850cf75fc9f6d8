"""The multi-GPU layout of FETI-DP / TFETI + Algorithm 1, checked on gloo ranks of
torch.distributed (CPU): subdomains in contiguous blocks per rank, multiplier
rows owned by the rank of their lowest subdomain, halo exchanges around the
dual-operator apply and the preconditioner, all-reduces of the coarse
right-hand side (FETI-DP) or of G X (TFETI) and of the Gram-type blocks.  On
2 and 3 ranks the sharded
solve takes the serial oracle's iterations and reaches its solution."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import workloads
    p = workloads.config2(tiles=4, elems=6)
    p.rho = np.where(p.rho < 0.5, 0.3, 1.0)      # moderate contrast: solutions comparable to ~1e-10
    p.Emin = 1e-6
    return p


def _worker(rank, world, port, method, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.solve import build
    from oracle.sharded import solve_dual_sharded
    op = build(_problem(), method, "k")
    lam, info, st = solve_dual_sharded(op, tol=1e-10)
    out[rank] = (op.recover(lam), info.iterations, info.ranks, st.halo_rows, st.owned_rows, st.owned_subdomains,
                 st.halo_bytes, st.allreduce_bytes)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("method,world", [("fetidp", 2), ("fetidp", 3), ("tfeti", 2)])
def test_sharded_algorithm1_matches_serial(method, world):
    sys.path.insert(0, ROOT)
    from oracle.solve import solve
    with mp.get_context("spawn").Manager() as mgr:          # no fork of this (threaded) process
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), method, out), nprocs=world, join=True)
        out = dict(out)
    u_ser, _, info, op = solve(_problem(), method, "k", "rrs", tol=1e-10)
    for r in range(world):
        u, its, ranks, halo, owned, nsub, hb, ab = out[r]
        assert its == info.iterations and ranks == info.ranks
        assert np.linalg.norm(u - u_ser) <= 1e-9 * np.linalg.norm(u_ser)
        assert halo < op.n_lam and nsub > 0 and ab > 0
    # rows belong to the rank of their lowest subdomain: the first rank reads no
    # foreign row, every later one reads the rows it shares with lower ranks
    assert out[0][3] == 0 and all(out[r][3] > 0 and out[r][6] > 0 for r in range(1, world))
    assert sum(out[r][4] for r in range(world)) == op.n_lam          # every row owned once
    assert sum(out[r][5] for r in range(world)) == op.n_sub
