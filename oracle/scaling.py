"""Signed constraint matrices B^s and their scaled versions B~^s (oracle).

Test infrastructure only (see the package docstring).

Constraint rows (Eq. 4 for TFETI, Eq. 10 for FETI-DP) are kept as explicit
lists of (subdomain, local DOF, sign).  A DOF shared by more than two
subdomains gets one row per pair of copies (Section 3.1 keeps the pair-wise
rows although they are redundant at cross points), each row being
u^a - u^b = 0 with a < b.  A fixed DOF in TFETI gets one row per copy,
u^s = 0 (the Dirichlet part of c in Eq. 4).

Scaling (Section 3.1): B~^s = W^s B^s with W^s diagonal over the rows.
* k-scaling, Eq. (15): on a row joining s and r, W^s = K^r_dd / (sum of
  K^q_dd over every subdomain q that shares the DOF), where K^q_dd is the
  diagonal stiffness entry of that DOF in subdomain q; for two sharers this
  is K^r / (K^s + K^r).
* multiplicity scaling: W^s = 1 / (number of sharers).
A single-subdomain (Dirichlet) row has weight 1.  Both choices satisfy the
admissibility condition Eq. (14); the tests pin that identity.

Pins: tests/test_oracle_dual.py (Eq. 14 for both scalings and methods; k equal
to multiplicity for homogeneous material), tests/test_oracle_academic.py
(equal weights on homogeneous interfaces, unequal across laminae), and the
library's own tearing against these rows (tests/test_host_tearing.py).
"""
import dataclasses
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Constraints:
    entries: List[List[Tuple[int, int, float]]]   # per row: (s, local dof, sign)
    sharing: List[List[Tuple[int, int]]]          # per row: every (s, local dof) copy of the DOF
    c: np.ndarray                                 # right-hand side of B u = c

    @property
    def n_lam(self):
        return len(self.entries)

    def entries_of(self, s):
        """(row, position in the row, local dof, sign) of every entry of subdomain
        s, in row order (indexed once for all subdomains)."""
        if not hasattr(self, "_by_sub"):
            self._by_sub = {}
            for l, ent in enumerate(self.entries):
                for t, (q, k, sg) in enumerate(ent):
                    self._by_sub.setdefault(q, []).append((l, t, k, sg))
        return self._by_sub.get(s, [])

    def B_sub(self, s, n_loc, weights=None):
        """B^s (or B~^s when ``weights`` is given) as CSR [n_lam, n_loc]."""
        rows, cols, vals = [], [], []
        for l, t, k, sg in self.entries_of(s):
            rows.append(l)
            cols.append(k)
            vals.append(sg * (1.0 if weights is None else weights[l][t]))
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_lam, n_loc))


def pairwise_rows(copies):
    """Rows u^a - u^b = 0 for every pair a < b of the (s, dof) copies."""
    out = []
    for i in range(len(copies)):
        for j in range(i + 1, len(copies)):
            (a, ka), (b, kb) = copies[i], copies[j]
            out.append([(a, ka, 1.0), (b, kb, -1.0)])
    return out


def row_weights(cons: Constraints, diagK, kind="k"):
    """Per-row, per-entry weights W^s (aligned with ``cons.entries``).

    ``diagK[s]`` is the diagonal of K^s over its local DOFs (used by k-scaling).
    """
    out = []
    for ent, share in zip(cons.entries, cons.sharing):
        if len(ent) == 1:
            out.append([1.0])
            continue
        if kind == "k":
            denom = sum(diagK[q][k] for (q, k) in share)
            (a, ka, _), (b, kb, _) = ent
            out.append([diagK[b][kb] / denom, diagK[a][ka] / denom])
        elif kind in ("mult", "multiplicity"):
            w = 1.0 / len(share)
            out.append([w, w])
        else:
            raise ValueError(kind)
    return out
