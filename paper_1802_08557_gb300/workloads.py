"""Seeded synthetic LP batches shaped like the workloads of Gurung & Ray,
"Simultaneous Solving of Batched Linear Programs on a GPU" (arXiv 1802.08557):
small dense random LPs (Section 5) and support-function LPs of a fixed
polytope (Section 2, Table 1).

This module only draws random numbers and lays them out; it holds none of the
simplex arithmetic.  It feeds both the CUDA solver and the CPU oracle.

Every LP is drawn from its own counter-based generator, numpy's Philox-4x64
keyed by (workload seed, LP index), so any LP of a batch can be regenerated
alone.  Shared data of a family (the polytope, the shared matrix) uses LP
index 2**63 - 1.

Batch layout (the solver's C-ABI layout): per-LP sizes ``m``, ``n`` (int32)
and element offsets ``a_off``, ``b_off``, ``c_off`` (int64) into flat float64
arrays ``A`` (row-major m x n blocks), ``b`` and ``c``.  Offsets may repeat
(shared matrix families).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SHARED_INDEX = (1 << 63) - 1

# Workload seeds: 0x180208557 xor workload id.
_BASE_SEED = 0x180208557


def workload_seed(wid: int) -> int:
    return _BASE_SEED ^ int(wid)


def lp_generator(seed: int, index: int) -> np.random.Generator:
    """The generator of LP ``index`` of a workload (Philox-4x64, 128-bit key)."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(index) & (2**64 - 1)]))


@dataclass
class LPBatch:
    """A batch of LPs  max c^T x  s.t.  A x <= b,  x >= 0  in offset layout."""
    name: str
    m: np.ndarray        # int32 [N]
    n: np.ndarray        # int32 [N]
    a_off: np.ndarray    # int64 [N]
    b_off: np.ndarray    # int64 [N]
    c_off: np.ndarray    # int64 [N]
    A: np.ndarray        # float64, flat
    b: np.ndarray        # float64, flat
    c: np.ndarray        # float64, flat
    kind: np.ndarray = field(default=None)  # int8 [N]: construction tag (see KIND_*)

    @property
    def num_lps(self) -> int:
        return int(self.m.shape[0])

    def lp(self, k: int):
        m, n = int(self.m[k]), int(self.n[k])
        a0, b0, c0 = int(self.a_off[k]), int(self.b_off[k]), int(self.c_off[k])
        return (self.A[a0:a0 + m * n].reshape(m, n), self.b[b0:b0 + m], self.c[c0:c0 + n])

    def subset(self, idx) -> "LPBatch":
        """A new packed batch holding the LPs ``idx`` (copies the data)."""
        idx = np.asarray(idx, dtype=np.int64)
        lps = [self.lp(int(k)) for k in idx]
        kind = None if self.kind is None else self.kind[idx].copy()
        return pack(self.name + "[subset]", lps, kind=kind)

    def x_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n.astype(np.int64))[:-1]]).astype(np.int64)

    def y_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.m.astype(np.int64))[:-1]]).astype(np.int64)


KIND_FEASIBLE_START = 0   # b >= 0: the slack basis is feasible
KIND_PHASE1 = 1           # some b_i < 0 drawn at random
KIND_INFEASIBLE = 2       # made infeasible by construction
KIND_UNBOUNDED = 3        # made unbounded by construction


def pack(name: str, lps, kind=None) -> LPBatch:
    """Pack a list of (A, b, c) into one offset-layout batch."""
    N = len(lps)
    m = np.array([np.shape(L[0])[0] for L in lps], dtype=np.int32)
    n = np.array([np.shape(L[0])[1] for L in lps], dtype=np.int32)
    mn = m.astype(np.int64) * n.astype(np.int64)
    a_off = np.concatenate([[0], np.cumsum(mn)[:-1]]).astype(np.int64) if N else np.zeros(0, np.int64)
    b_off = np.concatenate([[0], np.cumsum(m.astype(np.int64))[:-1]]).astype(np.int64) if N else np.zeros(0, np.int64)
    c_off = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]]).astype(np.int64) if N else np.zeros(0, np.int64)
    A = np.concatenate([np.ascontiguousarray(L[0], np.float64).ravel() for L in lps]) if N else np.zeros(0)
    b = np.concatenate([np.ascontiguousarray(L[1], np.float64) for L in lps]) if N else np.zeros(0)
    c = np.concatenate([np.ascontiguousarray(L[2], np.float64) for L in lps]) if N else np.zeros(0)
    kind = np.zeros(N, np.int8) if kind is None else np.asarray(kind, np.int8)
    return LPBatch(name, m, n, a_off, b_off, c_off, A, b, c, kind)


# ---------------------------------------------------------------------------
# Uniform-size dense random LPs (the paper's Section 5 random LPs)
# ---------------------------------------------------------------------------

def positive_dense(num_lps: int, m: int, n: int, a_rng=(1.0, 10.0), b_rng=(10.0, 100.0),
                   c_rng=(1.0, 10.0), wid: int = 1, start: int = 0) -> LPBatch:
    """Dense LPs with positive A, b, c: the slack basis is feasible and every
    LP is bounded (Section 5 draws A, b, c from positive ranges).  Default
    ranges: 5x5 batch with A~U[1,10], b~U[10,100], c~U[1,10]."""
    seed = workload_seed(wid)
    A = np.empty((num_lps, m, n))
    b = np.empty((num_lps, m))
    c = np.empty((num_lps, n))
    for k in range(num_lps):
        g = lp_generator(seed, start + k)
        A[k] = g.uniform(*a_rng, size=(m, n))
        b[k] = g.uniform(*b_rng, size=m)
        c[k] = g.uniform(*c_rng, size=n)
    return _uniform_batch(f"positive_dense_{m}x{n}", A, b, c, np.zeros(num_lps, np.int8))


def mixed_sign_dense(num_lps: int, m: int = 50, n: int = 50, wid: int = 2, start: int = 0,
                     p_phase1: float = 0.20, p_infeasible: float = 0.025,
                     p_unbounded: float = 0.025) -> LPBatch:
    """Dense LPs with A~U[-1,1], c~U[-1,1].  A fraction ``p_phase1`` draws
    b~U[-5,10] (the slack basis is then usually infeasible: phase I); the rest
    draw b~U[1,10].  Of the latter, ``p_infeasible`` are made infeasible (row
    k := -row j, b_k := -(b_j + U[0.5,1]) with b_j~U[1,4]) and ``p_unbounded``
    unbounded (one column j with A[:,j]~U[-1,0] and c_j~U[0.5,1]).
    Other LPs are whatever they are (random-sign A may be unbounded too)."""
    seed = workload_seed(wid)
    A = np.empty((num_lps, m, n))
    b = np.empty((num_lps, m))
    c = np.empty((num_lps, n))
    kind = np.zeros(num_lps, np.int8)
    for k in range(num_lps):
        g = lp_generator(seed, start + k)
        u = g.uniform()
        Ak = g.uniform(-1.0, 1.0, size=(m, n))
        ck = g.uniform(-1.0, 1.0, size=n)
        if u < p_phase1:
            bk = g.uniform(-5.0, 10.0, size=m)
            kind[k] = KIND_PHASE1 if (bk < 0).any() else KIND_FEASIBLE_START
        else:
            bk = g.uniform(1.0, 10.0, size=m)
            if u < p_phase1 + p_infeasible and m >= 2:
                j = int(g.integers(m))
                kk = (j + 1 + int(g.integers(m - 1))) % m
                bk[j] = g.uniform(1.0, 4.0)
                Ak[kk] = -Ak[j]
                bk[kk] = -(bk[j] + g.uniform(0.5, 1.0))
                kind[k] = KIND_INFEASIBLE
            elif u < p_phase1 + p_infeasible + p_unbounded:
                j = int(g.integers(n))
                Ak[:, j] = g.uniform(-1.0, 0.0, size=m)
                ck[j] = g.uniform(0.5, 1.0)
                kind[k] = KIND_UNBOUNDED
        A[k], b[k], c[k] = Ak, bk, ck
    return _uniform_batch(f"mixed_sign_dense_{m}x{n}", A, b, c, kind)


def _uniform_batch(name, A, b, c, kind) -> LPBatch:
    N, m, n = A.shape
    return LPBatch(
        name=name,
        m=np.full(N, m, np.int32), n=np.full(N, n, np.int32),
        a_off=np.arange(N, dtype=np.int64) * (m * n),
        b_off=np.arange(N, dtype=np.int64) * m,
        c_off=np.arange(N, dtype=np.int64) * n,
        A=A.reshape(-1), b=b.reshape(-1), c=c.reshape(-1), kind=kind)


# ---------------------------------------------------------------------------
# Support-function LPs of one polytope (Section 2, Table 1)
# ---------------------------------------------------------------------------

def support_function(num_dirs: int, dim: int = 10, halfspaces: int = 40, wid: int = 3,
                     start: int = 0) -> LPBatch:
    """Support function of one polytope P = {z : a_i.z <= b_i} in R^dim, with
    unit normals a_i (normalised Gaussians) and b_i~U[1,2], sampled in
    ``num_dirs`` directions l (uniform on the unit sphere).  z is free, so it is
    split z = x+ - x- : constraint matrix [A, -A] (halfspaces x 2*dim) and
    objective [l, -l].  The origin is interior, so no phase I.  A and b are
    shared by every LP (repeated offsets)."""
    seed = workload_seed(wid)
    g = lp_generator(seed, SHARED_INDEX)
    a = g.standard_normal((halfspaces, dim))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    bb = g.uniform(1.0, 2.0, size=halfspaces)
    Afull = np.concatenate([a, -a], axis=1)
    C = np.empty((num_dirs, 2 * dim))
    for k in range(num_dirs):
        gk = lp_generator(seed, start + k)
        l = gk.standard_normal(dim)
        l /= np.linalg.norm(l)
        C[k, :dim] = l
        C[k, dim:] = -l
    N = num_dirs
    return LPBatch(
        name=f"support_function_{halfspaces}x{dim}",
        m=np.full(N, halfspaces, np.int32), n=np.full(N, 2 * dim, np.int32),
        a_off=np.zeros(N, np.int64), b_off=np.zeros(N, np.int64),
        c_off=np.arange(N, dtype=np.int64) * (2 * dim),
        A=Afull.reshape(-1).copy(), b=bb.copy(), c=C.reshape(-1), kind=np.zeros(N, np.int8))


def hyperbox_directions(num_dirs: int, dim: int = 28, wid: int = 6, start: int = 0):
    """Support function of one hyperbox (Section 4.4, Eq. 7) sampled in
    ``num_dirs`` directions uniform on the unit sphere of R^dim (normalised
    Gaussians), the shape of the paper's state-space exploration LPs (Section
    6: a 28-variable helicopter model, a 5-dimensional system).  Box: lo~U[-2,0],
    hi = lo + U[0.5,3].  Returns (L [num_dirs x dim], lo [dim], hi [dim]).
    Directions are drawn in blocks of 4096 from generators keyed by the index
    of the block's first direction, so a block is reproducible alone."""
    seed = workload_seed(wid)
    g = lp_generator(seed, SHARED_INDEX)
    lo = g.uniform(-2.0, 0.0, dim)
    hi = lo + g.uniform(0.5, 3.0, dim)
    L = np.empty((num_dirs, dim))
    blk = 4096
    for b0 in range(0, num_dirs, blk):
        gb = lp_generator(seed, start + b0)
        n = min(blk, num_dirs - b0)
        v = gb.standard_normal((n, dim))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        L[b0:b0 + n] = v
    return L, lo, hi


# ---------------------------------------------------------------------------
# Uneven batch (sizes log-uniform)
# ---------------------------------------------------------------------------

def uneven_dense(num_lps: int, lo: int = 10, hi: int = 500, wid: int = 4, start: int = 0,
                 max_elems: int | None = None) -> LPBatch:
    """LPs with m, n drawn independently as floor(exp(U[ln lo, ln hi])), dense
    A~U[0,1], b~U[1,100], c~U[0,1] (all feasible at the slack basis and
    bounded).  ``max_elems`` (optional) caps m*n by redrawing."""
    seed = workload_seed(wid)
    lps = []
    for k in range(num_lps):
        g = lp_generator(seed, start + k)
        while True:
            m = int(math.floor(math.exp(g.uniform(math.log(lo), math.log(hi)))))
            n = int(math.floor(math.exp(g.uniform(math.log(lo), math.log(hi)))))
            if max_elems is None or m * n <= max_elems:
                break
        lps.append((g.uniform(0.0, 1.0, size=(m, n)), g.uniform(1.0, 100.0, size=m),
                    g.uniform(0.0, 1.0, size=n)))
    return pack(f"uneven_dense_{lo}_{hi}", lps)


# ---------------------------------------------------------------------------
# Parametric family with a shared matrix
# ---------------------------------------------------------------------------

def shared_matrix_family(num_lps: int, m: int = 200, n: int = 100, wid: int = 5,
                         start: int = 0) -> LPBatch:
    """Shared A (m x n, U[0,1]) and b0~U[1,100]; per LP b = b0*(1 + 0.1*N(0,1))
    (negative entries possible: phase I) and c~U[0,1]."""
    seed = workload_seed(wid)
    g = lp_generator(seed, SHARED_INDEX)
    A = g.uniform(0.0, 1.0, size=(m, n))
    b0 = g.uniform(1.0, 100.0, size=m)
    B = np.empty((num_lps, m))
    C = np.empty((num_lps, n))
    kind = np.zeros(num_lps, np.int8)
    for k in range(num_lps):
        gk = lp_generator(seed, start + k)
        B[k] = b0 * (1.0 + 0.1 * gk.standard_normal(m))
        C[k] = gk.uniform(0.0, 1.0, size=n)
        kind[k] = KIND_PHASE1 if (B[k] < 0).any() else KIND_FEASIBLE_START
    N = num_lps
    return LPBatch(
        name=f"shared_matrix_{m}x{n}",
        m=np.full(N, m, np.int32), n=np.full(N, n, np.int32),
        a_off=np.zeros(N, np.int64), b_off=np.arange(N, dtype=np.int64) * m,
        c_off=np.arange(N, dtype=np.int64) * n,
        A=A.reshape(-1).copy(), b=B.reshape(-1), c=C.reshape(-1), kind=kind)


def shared_matrix_family_blocks(num_lps: int, m: int = 200, n: int = 100, wid: int = 5,
                                start: int = 0) -> LPBatch:
    """The same family as shared_matrix_family (same A and b0), drawn in blocks
    of 4096 LPs per generator for large training sets.  The block generators
    are keyed apart from the per-LP ones, so these LPs are not copies of
    shared_matrix_family's."""
    seed = workload_seed(wid)
    g = lp_generator(seed, SHARED_INDEX)
    A = g.uniform(0.0, 1.0, size=(m, n))
    b0 = g.uniform(1.0, 100.0, size=m)
    B = np.empty((num_lps, m))
    C = np.empty((num_lps, n))
    blk = 4096
    for k0 in range(0, num_lps, blk):
        gb = lp_generator(seed ^ 0xB10C_0000_0000, start + k0)
        cnt = min(blk, num_lps - k0)
        B[k0:k0 + cnt] = b0 * (1.0 + 0.1 * gb.standard_normal((cnt, m)))
        C[k0:k0 + cnt] = gb.uniform(0.0, 1.0, size=(cnt, n))
    kind = np.where((B < 0).any(axis=1), KIND_PHASE1, KIND_FEASIBLE_START).astype(np.int8)
    N = num_lps
    return LPBatch(
        name=f"shared_matrix_{m}x{n}_blocks",
        m=np.full(N, m, np.int32), n=np.full(N, n, np.int32),
        a_off=np.zeros(N, np.int64), b_off=np.arange(N, dtype=np.int64) * m,
        c_off=np.arange(N, dtype=np.int64) * n,
        A=A.reshape(-1).copy(), b=B.reshape(-1), c=C.reshape(-1), kind=kind)


# ---------------------------------------------------------------------------
# Named workloads (sizes of the five benchmark configurations)
# ---------------------------------------------------------------------------

WORKLOADS = {
    "dense5x5_1k": lambda num=1000, start=0: positive_dense(num, 5, 5, start=start),
    "dense50x50_phase1_100k": lambda num=100_000, start=0: mixed_sign_dense(num, 50, 50, start=start),
    "support40x10_100k": lambda num=100_000, start=0: support_function(num, start=start),
    "uneven10to500_20k": lambda num=20_000, start=0: uneven_dense(num, start=start),
    "shared200x100_100k": lambda num=100_000, start=0: shared_matrix_family(num, start=start),
}
