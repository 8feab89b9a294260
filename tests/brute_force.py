"""Brute-force LP solver for tiny LPs, independent of the simplex oracle.

max c^T x  s.t.  A x <= b, x >= 0  (Eq. 1-3 of Gurung & Ray, arXiv 1802.08557).

The feasible set P = {x : G x <= h} with G = [A; -I], h = [b; 0] is pointed
(it lies in the orthant), so
  * P is empty  <=> no n-subset of the m+n constraints, taken tight, gives a
    feasible point (a vertex);
  * the LP is unbounded <=> P is non-empty and some d >= 0 with A d <= 0 has
    c^T d > 0; such a d can be normalised to 1^T d = 1, and the maximum of c^T d
    over the polytope {d >= 0, A d <= 0, 1^T d = 1} is attained at one of its
    vertices, found by taking n-1 of the m+n inequalities tight;
  * otherwise the optimum is the best vertex.
Exponential in n; meant for n <= 4, m <= 6.
"""
from __future__ import annotations

import itertools

import numpy as np


def _vertices(G, h, eq=None, tol=1e-9):
    """All points where `k` rows of G x <= h are tight (k = dim - #eq), plus
    the equality rows, that satisfy every inequality within tol."""
    nrow, dim = G.shape
    neq = 0 if eq is None else eq[0].shape[0]
    k = dim - neq
    pts = []
    for S in itertools.combinations(range(nrow), k):
        M = G[list(S)]
        r = h[list(S)]
        if neq:
            M = np.vstack([M, eq[0]])
            r = np.concatenate([r, eq[1]])
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        try:
            x = np.linalg.solve(M, r)
        except np.linalg.LinAlgError:
            continue
        scale = max(1.0, np.abs(h).max(initial=0.0), np.abs(x).max(initial=0.0))
        if np.all(G @ x <= h + tol * scale):
            pts.append(x)
    return pts


def brute_force(A, b, c, tol=1e-9):
    """Return (status, value): status 0 optimal, 1 infeasible, 2 unbounded."""
    A = np.asarray(A, float)
    b = np.asarray(b, float)
    c = np.asarray(c, float)
    m, n = A.shape
    G = np.vstack([A, -np.eye(n)])
    h = np.concatenate([b, np.zeros(n)])
    verts = _vertices(G, h, tol=tol)
    if not verts:
        return 1, None
    # recession cone  {d >= 0, A d <= 0}  cut by 1^T d = 1
    Gd = np.vstack([A, -np.eye(n)])
    hd = np.zeros(m + n)
    rays = _vertices(Gd, hd, eq=(np.ones((1, n)), np.ones(1)), tol=tol)
    if rays and max(float(c @ d) for d in rays) > 1e-9:
        return 2, None
    return 0, max(float(c @ x) for x in verts)
