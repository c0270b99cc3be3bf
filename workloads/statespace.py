"""Seeded synthetic concurrent-system models for state-space exploration.

The paper's model-checking workloads (Section 3.2: a model is a finite set of
finite-state processes in parallel composition, explored by BFS from the
vector of initial local states) come from models that are not available
here.  This module draws stand-in models of the same kind.  It produces the
model *tables* only; what a state's successors are is computed separately by
the oracle and by the CUDA path, each from the definition below.

Model format (shared by both sides as a document, not as code)
--------------------------------------------------------------
* ``C`` components (processes), C <= CMAX.  Component c has ``L[c]`` local
  states, 2 <= L[c] <= LMAX, stored in b[c] = ceil(log2 L[c]) bits.
* A state vector packs the local states LSB-first: component c occupies bits
  [o_c, o_c + b_c) with o_c = b_0 + ... + b_{c-1}.  The initial state is all
  zero.  A model with sum(b) <= 31 uses 32-bit keys, otherwise 64-bit keys
  (sum(b) <= 63).
* Component c in local state u has ``deg[c,u]`` (<= DMAX) outgoing
  transitions j with target ``tgt[c,u,j]`` and label ``lab[c,u,j]``.
  Label 0 is a local action; label p+1 ties the transition to sync pair p.
* ``pairs[p] = (c1, c2)``, c1 != c2.
* Successors of a state s (interleaving with binary synchronisation):
  - for every component c and every transition j of c at u = s_c with label
    0: s with s_c replaced by tgt[c,u,j];
  - for every pair p = (c1, c2), every transition j1 of c1 at s_c1 with label
    p+1 and every transition j2 of c2 at s_c2 with label p+1: s with s_c1 and
    s_c2 replaced by their targets.
  Labelled transitions never fire alone.

Generator (``random_model``): each component c gets a main cycle
0 -> 1 -> ... -> R_c-1 -> 0 through its first R_c local states plus extra
random transitions inside that window, so exactly R_c local states are
reachable when nothing synchronises; states R_c..L_c-1 exist in the tables
but are never reached.  Each transition of a component that belongs to a
pair is labelled with that pair with probability ``p_sync``.  With
p_sync = 0 the reachable set is the product of the windows, which the tests
use as a closed form.
"""
from dataclasses import dataclass, field

import numpy as np

LMAX = 32   # local states per component (table rows)
DMAX = 4    # transitions per local state (table columns)
CMAX = 16   # components
PMAX = 8    # sync pairs


@dataclass
class Model:
    C: int
    L: np.ndarray          # (C,) local-state counts
    bits: np.ndarray       # (CMAX,) uint8, bits per component (0 past C)
    deg: np.ndarray        # (CMAX, LMAX) uint8
    tgt: np.ndarray        # (CMAX, LMAX, DMAX) uint8
    lab: np.ndarray        # (CMAX, LMAX, DMAX) uint8
    pairs: np.ndarray      # (P, 2) uint8
    meta: dict = field(default_factory=dict)

    @property
    def P(self):
        return int(self.pairs.shape[0])

    @property
    def total_bits(self):
        return int(self.bits[:self.C].sum())

    @property
    def key_width(self):
        b = self.total_bits
        return 32 if b <= 31 else (64 if b <= 63 else 128)

    def pair_arrays(self):
        c1 = np.zeros(PMAX, dtype=np.uint8)
        c2 = np.zeros(PMAX, dtype=np.uint8)
        c1[:self.P] = self.pairs[:, 0]
        c2[:self.P] = self.pairs[:, 1]
        return c1, c2


def _bits_for(n):
    return max(1, int(np.ceil(np.log2(n))))


def random_model(seed, C, L, R, p_sync=0.0, P=0, deg_lo=1, deg_hi=3):
    """Draw a model; ``L`` and ``R`` are ints or per-component sequences.

    R[c] (2 <= R[c] <= L[c]) is the window of local states reachable when no
    transition is synchronised.  Draw order: per component, per local state:
    degree, then per transition a target; then the pairs; then the labels.
    """
    if not 1 <= C <= CMAX:
        raise ValueError("1 <= C <= CMAX")
    L = np.broadcast_to(np.asarray(L, dtype=np.int64), (C,)).copy()
    R = np.broadcast_to(np.asarray(R, dtype=np.int64), (C,)).copy()
    if (L < 2).any() or (L > LMAX).any() or (R < 1).any() or (R > L).any():
        raise ValueError("need 2 <= L <= LMAX and 1 <= R <= L")
    if not 0 <= P <= PMAX or (P > 0 and C < 2):
        raise ValueError("0 <= P <= PMAX, and pairs need two components")
    if deg_hi > DMAX or deg_lo < 1 or deg_lo > deg_hi:
        raise ValueError("1 <= deg_lo <= deg_hi <= DMAX")
    rng = np.random.Generator(np.random.PCG64(seed))
    bits = np.zeros(CMAX, dtype=np.uint8)
    deg = np.zeros((CMAX, LMAX), dtype=np.uint8)
    tgt = np.zeros((CMAX, LMAX, DMAX), dtype=np.uint8)
    lab = np.zeros((CMAX, LMAX, DMAX), dtype=np.uint8)
    for c in range(C):
        bits[c] = _bits_for(L[c])
        for u in range(L[c]):
            d = int(rng.integers(deg_lo, deg_hi + 1))
            deg[c, u] = d
            for j in range(d):
                if u < R[c]:
                    v = (u + 1) % R[c] if j == 0 else int(rng.integers(0, R[c]))
                else:
                    v = int(rng.integers(0, L[c]))
                tgt[c, u, j] = v
    pairs = np.zeros((P, 2), dtype=np.uint8)
    for p in range(P):
        c1 = int(rng.integers(0, C))
        c2 = int(rng.integers(0, C - 1))
        c2 = c2 + 1 if c2 >= c1 else c2
        pairs[p] = (c1, c2)
    if P and p_sync > 0.0:
        for c in range(C):
            mine = [p for p in range(P) if c in (pairs[p, 0], pairs[p, 1])]
            for u in range(L[c]):
                for j in range(deg[c, u]):
                    r = rng.random()
                    if mine and r < p_sync:
                        lab[c, u, j] = mine[0] + 1
    if bits.sum() > 127:
        raise ValueError("state vector exceeds 127 bits")
    return Model(C=C, L=L, bits=bits, deg=deg, tgt=tgt, lab=lab, pairs=pairs,
                 meta=dict(seed=seed, R=R.tolist(), p_sync=p_sync, P=P))


def config3_model(seed=3, p_sync=0.25):
    """12 components x 32 local states (5 bits each, 60-bit vectors), 4 sync
    pairs, out-degree 1-3.  Windows of 4-5 reachable local states set the
    reachable state count near 10^8."""
    R = [5] * 8 + [4] * 4
    return random_model(seed, C=12, L=32, R=R, p_sync=p_sync, P=4)


def batched_models(count, seed):
    """Uneven explorations: 6-10 components of 8-32 local states each.

    The window sizes are drawn so that the unsynchronised product size is
    log-uniform in [2^10, 2^20]; sync pairs then shrink it.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        C = int(rng.integers(6, 11))
        L = rng.integers(8, 33, size=C)
        target = 2.0 ** rng.uniform(10, 20)
        per = target ** (1.0 / C)
        R = np.clip(np.round(per * np.exp(rng.normal(0, 0.15, size=C))), 2, L).astype(np.int64)
        out.append(random_model(int(rng.integers(0, 2**31)), C=C, L=L, R=R,
                                p_sync=0.15, P=int(rng.integers(1, 5))))
    return out
