"""Container for one LR superblock problem (data only, no arithmetic of the method).

A superblock Hamiltonian in the LR form of Sec. 4.1 is H_SB = sum_a c_a A_a (x) B_a
(Eq. 9), where A_a acts on the enlarged left block L = l+1 and B_a on the enlarged
right block R = r+1.  With the U(1) symmetries of Sec. 3 every operator is stored as a
list of dense blocks A_{q_i -> q_j} (Sec. 4.1, the paragraph around Eq. 11), and the
state vector X is the concatenation of the dense segments X_{ik} over the valid sector
pairs (i, k) whose quantum numbers add up to the target Q.

Layout conventions (shared by every consumer of this container):

* sector pair p = (i, k) holds a row-major segment of shape [dL[i], dR[k]], i.e.
  element psi(a, b) sits at x[offset[p] + a * dR[k] + b];
* segments follow the order of ``pairs``;
* a block operator maps input sector i to output sector j with a dense row-major
  matrix of shape [d_j, d_i];
* a term (coef, a, b) contributes coef * (A_a (x) B_b); an index of -1 names the
  identity on that side.

The container only records the problem.  Nothing in this module applies an operator.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np

IDENTITY = -1


@dataclass
class BlockOp:
    """A block-sparse operator: {(i_in, j_out): dense [d_j, d_i] float64 array}."""

    blocks: Dict[Tuple[int, int], np.ndarray] = field(default_factory=dict)
    name: str = ""


@dataclass
class Superblock:
    qL: List[Tuple[int, ...]]          # quantum numbers of the enlarged-left sectors
    dL: np.ndarray                     # their dimensions (int64)
    qR: List[Tuple[int, ...]]
    dR: np.ndarray
    Q: Tuple[int, ...]                 # target quantum number of the superblock
    pairs: List[Tuple[int, int]]       # valid (i, k) pairs in storage order
    opsL: List[BlockOp]
    opsR: List[BlockOp]
    terms: List[Tuple[float, int, int]]  # (coef, a_op or IDENTITY, b_op or IDENTITY)
    meta: dict = field(default_factory=dict)

    # ---- bookkeeping helpers (index arithmetic only) ----
    def offsets(self) -> np.ndarray:
        sizes = np.array([int(self.dL[i]) * int(self.dR[k]) for i, k in self.pairs],
                         dtype=np.int64)
        off = np.zeros(len(sizes) + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        return off

    @property
    def n(self) -> int:
        return int(self.offsets()[-1])

    def pair_index(self) -> Dict[Tuple[int, int], int]:
        return {p: idx for idx, p in enumerate(self.pairs)}

    def segment(self, x: np.ndarray, p: int) -> np.ndarray:
        """View of segment p of a flat vector as a [dL[i], dR[k]] matrix."""
        off = self.offsets()
        i, k = self.pairs[p]
        return x[off[p]:off[p + 1]].reshape(int(self.dL[i]), int(self.dR[k]))

    def validate(self) -> None:
        """Structural checks: shapes of all blocks and pairs; raises ValueError."""
        nL, nR = len(self.dL), len(self.dR)
        if len(self.qL) != nL or len(self.qR) != nR:
            raise ValueError("sector tables disagree in length")
        seen = set()
        for i, k in self.pairs:
            if not (0 <= i < nL and 0 <= k < nR):
                raise ValueError(f"pair ({i},{k}) out of range")
            if (i, k) in seen:
                raise ValueError(f"pair ({i},{k}) repeated")
            seen.add((i, k))
            qs = tuple(a + b for a, b in zip(self.qL[i], self.qR[k]))
            if qs != tuple(self.Q):
                raise ValueError(f"pair ({i},{k}) has quantum number {qs} != {self.Q}")
        for side, ops, d in (("L", self.opsL, self.dL), ("R", self.opsR, self.dR)):
            for op in ops:
                for (i, j), blk in op.blocks.items():
                    if blk.shape != (int(d[j]), int(d[i])):
                        raise ValueError(f"{side} op {op.name} block {(i, j)} has shape "
                                         f"{blk.shape}, expected {(int(d[j]), int(d[i]))}")
        for coef, a, b in self.terms:
            if a != IDENTITY and not (0 <= a < len(self.opsL)):
                raise ValueError("term names a missing left operator")
            if b != IDENTITY and not (0 <= b < len(self.opsR)):
                raise ValueError("term names a missing right operator")


def pairs_for_target(qL, qR, Q) -> List[Tuple[int, int]]:
    """All (i, k) with qL[i] + qR[k] == Q, ordered by i then k."""
    out = []
    for i, a in enumerate(qL):
        for k, b in enumerate(qR):
            if tuple(x + y for x, y in zip(a, b)) == tuple(Q):
                out.append((i, k))
    return out


def save_npz(sb: Superblock, path: str) -> None:
    """Serialise a superblock into one .npz file (used as a checkpoint of a problem)."""
    arrs = {
        "qL": np.array(sb.qL, dtype=np.int64).reshape(len(sb.qL), -1),
        "qR": np.array(sb.qR, dtype=np.int64).reshape(len(sb.qR), -1),
        "dL": np.asarray(sb.dL, dtype=np.int64), "dR": np.asarray(sb.dR, dtype=np.int64),
        "Q": np.array(sb.Q, dtype=np.int64),
        "pairs": np.array(sb.pairs, dtype=np.int64).reshape(-1, 2),
        "terms_coef": np.array([t[0] for t in sb.terms], dtype=np.float64),
        "terms_ab": np.array([[t[1], t[2]] for t in sb.terms], dtype=np.int64).reshape(-1, 2),
    }
    for side, ops in (("L", sb.opsL), ("R", sb.opsR)):
        arrs[f"n_ops{side}"] = np.array(len(ops))
        for o, op in enumerate(ops):
            keys = sorted(op.blocks)
            arrs[f"op{side}{o}_keys"] = np.array(keys, dtype=np.int64).reshape(-1, 2)
            for bi, key in enumerate(keys):
                arrs[f"op{side}{o}_b{bi}"] = op.blocks[key]
    np.savez(path, **arrs)


def load_npz(path: str) -> Superblock:
    z = np.load(path)
    ops = {}
    for side in ("L", "R"):
        lst = []
        for o in range(int(z[f"n_ops{side}"])):
            keys = [tuple(int(v) for v in r) for r in z[f"op{side}{o}_keys"]]
            lst.append(BlockOp({key: np.array(z[f"op{side}{o}_b{bi}"])
                                for bi, key in enumerate(keys)}))
        ops[side] = lst
    return Superblock(
        qL=[tuple(int(v) for v in r) for r in z["qL"]], dL=np.array(z["dL"]),
        qR=[tuple(int(v) for v in r) for r in z["qR"]], dR=np.array(z["dR"]),
        Q=tuple(int(v) for v in z["Q"]),
        pairs=[(int(a), int(b)) for a, b in z["pairs"]],
        opsL=ops["L"], opsR=ops["R"],
        terms=[(float(c), int(a), int(b)) for c, (a, b) in zip(z["terms_coef"], z["terms_ab"])],
    )


@dataclass
class SuperblockL11r:
    """One superblock problem in the l-1-1-r form of Sec. 4.2: H_SB = sum_a c_a A_a (x)
    a_a (x) b_a (x) B_a (Eq. 12), with A_a on the block l, a_a and b_a on the two middle
    sites and B_a on the block r.

    Layout conventions:

    * the site states are their own sectors (each has one quantum number ``qs[s]``), so
      a site operator is a dense q x q matrix ``sops[o]`` with element [s_out, s_in];
    * a segment (i, s1, s2, k) -- block-l sector i, site states s1 and s2, block-r
      sector k -- is a row-major [dl[i], dr[k]] matrix; segments follow ``segs`` and
      hold every combination whose quantum numbers add up to Q;
    * a term (coef, a, s1, s2, b) contributes coef * (A_a (x) sops[s1] (x) sops[s2] (x)
      B_b); an index of -1 names the identity of that subsystem.

    The container only records the problem; nothing here applies an operator."""

    ql: List[Tuple[int, ...]]
    dl: np.ndarray
    qs: List[Tuple[int, ...]]
    qr: List[Tuple[int, ...]]
    dr: np.ndarray
    Q: Tuple[int, ...]
    segs: List[Tuple[int, int, int, int]]
    opsl: List[BlockOp]
    sops: List[np.ndarray]
    opsr: List[BlockOp]
    terms: List[Tuple[float, int, int, int, int]]
    meta: dict = field(default_factory=dict)

    def offsets(self) -> np.ndarray:
        sizes = np.array([int(self.dl[i]) * int(self.dr[k]) for i, _, _, k in self.segs],
                         dtype=np.int64)
        off = np.zeros(len(sizes) + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        return off

    @property
    def n(self) -> int:
        return int(self.offsets()[-1])

    @property
    def q(self) -> int:
        return len(self.qs)

    def seg_index(self) -> Dict[Tuple[int, int, int, int], int]:
        return {s: idx for idx, s in enumerate(self.segs)}


def segs_for_target(ql, qs, qr, Q) -> List[Tuple[int, int, int, int]]:
    """All (i, s1, s2, k) whose quantum numbers add up to Q, ordered by i, s1, s2, k."""
    out = []
    for i, a in enumerate(ql):
        for s1, b in enumerate(qs):
            for s2, c in enumerate(qs):
                for k, d in enumerate(qr):
                    if tuple(w + x + y + z for w, x, y, z in zip(a, b, c, d)) == tuple(Q):
                        out.append((i, s1, s2, k))
    return out
