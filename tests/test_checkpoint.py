"""Checkpoint / resume of the differentiation form's design loop on the CPU
(paper_2111_11728_gb300/simp.py): the densities and the warm-start multiplier
are the loop's whole state.  With a stand-in state solver (an analytic
compliance and a multiplier updated from it) an interrupted run resumed from
its checkpoint ends bit-identical to an uninterrupted one."""
import numpy as np
import torch

from paper_2111_11728_gb300 import simp


class _Stats:
    iterations = 3


class _FakeProblem:
    """c(rho) = sum_e w_e / rho_e (convex, decreasing in rho, like a compliance);
    the 'multiplier' is a running quantity that the next solve reads back."""

    def __init__(self, n=64, seed=0):
        self.w = torch.as_tensor(np.random.default_rng(seed).uniform(0.5, 2.0, n))
        self.lam = torch.zeros(n, dtype=torch.float64)
        self.last_stats = _Stats()
        self._rho = None

    def solve(self, rho):
        self._rho = rho.detach()
        self.lam = 0.5 * self.lam + self._rho          # depends on the previous multiplier
        return float((self.w / self._rho).sum() + 1e-3 * self.lam.sum()), True

    def grad(self):
        return -self.w / self._rho ** 2


def test_resume_is_bit_identical(tmp_path):
    rho0 = torch.full((64,), 0.4, dtype=torch.float64)
    ref, hist_ref = simp.optimize(_FakeProblem(), rho0, 0.4, iterations=8)
    ck = tmp_path / "state.npz"
    cp = _FakeProblem()
    simp.optimize(cp, rho0, 0.4, iterations=5, checkpoint=ck)       # interrupted after 5 steps
    it, rho, lam, hist = simp.load_checkpoint(ck, device="cpu")
    assert it == 5 and len(hist) == 5
    cp2 = _FakeProblem()
    cp2.lam = lam
    out, hist_out = simp.optimize(cp2, rho, 0.4, iterations=8, start=it, history=hist)
    assert torch.equal(out, ref)
    assert hist_out == hist_ref
