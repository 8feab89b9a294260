"""CPU FP64 reference (oracle) of the hyperbox LP special case of Gurung & Ray,
"Simultaneous Solving of Batched Linear Programs on a GPU" (arXiv
1802.08557), Section 4.4, Eq. 7.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use
it; the CUDA library never imports it.

For a box B = [lo_1, hi_1] x ... x [lo_n, hi_n] and a direction l, Eq. 7
gives  max_{x in B} l.x = sum_i l_i h_i  with h_i = lo_i where l_i < 0 and
h_i = hi_i otherwise (the paper's a_i, b_i are lo_i, hi_i here), and h is a
maximiser.  This module evaluates exactly that definition: h by the sign test,
then the sum of the products l_i * h_i in ascending i, each product rounded
and then added (FP64, no fused multiply-add).
"""
from __future__ import annotations

import numpy as np


def hyperbox_solve(L, lo, hi):
    """Eq. 7 for every row of ``L`` (num_lps x dim).

    ``lo`` and ``hi`` are either one box (shape (dim,)) shared by all rows or
    one box per row (shape (num_lps, dim)).  Returns (obj, x): obj[k] =
    max over the box of L[k] . x, and x[k] the maximiser h of Eq. 7."""
    L = np.asarray(L, dtype=np.float64)
    if L.ndim != 2:
        raise ValueError("L must be num_lps x dim")
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), L.shape)
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), L.shape)
    h = np.where(L < 0.0, lo, hi)
    obj = np.zeros(L.shape[0])
    for i in range(L.shape[1]):
        obj = obj + L[:, i] * h[:, i]
    return obj, np.ascontiguousarray(h)
