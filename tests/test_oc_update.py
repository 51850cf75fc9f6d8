"""CPU pins of the optimality-criteria update of the differentiation form's
design loop (paper_2111_11728_gb300/simp.py; the paper does not fix its
optimizer, the textbook OC update with bisection on the volume multiplier is
used): bounds and move limits hold, the volume constraint is met, and at equal
density a larger sensitivity never gets a smaller update."""
import torch

from paper_2111_11728_gb300.simp import oc_update


def _case(seed, n=4000):
    g = torch.Generator().manual_seed(seed)
    rho = 0.05 + 0.9 * torch.rand(n, dtype=torch.float64, generator=g)
    dc = -torch.rand(n, dtype=torch.float64, generator=g) * 10.0 ** (4 * torch.rand(n, dtype=torch.float64, generator=g))
    return rho, dc


def test_bounds_move_limits_and_volume():
    for seed in range(5):
        rho, dc = _case(seed)
        vf = float(rho.mean()) * 0.97                      # a reachable target close to the current volume
        new = oc_update(rho, dc, vf, move=0.2, eta=0.5, rho_min=1e-3)
        assert float(new.min()) >= 1e-3 and float(new.max()) <= 1.0
        assert float((new - rho).abs().max()) <= 0.2 + 1e-15
        assert abs(float(new.sum()) - vf * rho.numel()) <= 1e-6 * vf * rho.numel()


def test_update_is_monotone_in_the_sensitivity():
    rho = torch.full((200,), 0.4, dtype=torch.float64)
    dc = -torch.logspace(-3, 3, 200, dtype=torch.float64)
    new = oc_update(rho, dc, 0.4, move=0.2, eta=0.5, rho_min=1e-3)
    assert bool(torch.all(new[1:] >= new[:-1]))
    assert float(new[0]) < 0.4 < float(new[-1])            # weak elements shrink, strong ones grow
