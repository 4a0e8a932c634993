"""Seeded synthetic superblock problems shaped like the paper's Heisenberg / Hubbard runs.

This module is an input generator.  It builds the enlarged-block operators of an
infinite-lattice warm-up (Algorithm 1 with the LR strategy of Sec. 4.1) for the
Heisenberg chain (Eq. 1) or the spin-1/2 Hubbard chain (Eq. 4), keeping every operator
in the sector-blocked form of Sec. 4.1, and returns the final mid-chain superblock as a
:class:`dmrg_inputs.superblock.Superblock`.  It never applies H_SB to a vector, never
runs an eigensolver on the superblock and shares no code with the oracle.

Truncation recipe (a stand-in for the density-matrix step, which needs the ground state
and therefore the method itself):

* how many states each sector keeps comes from a Gaussian profile over the block's
  quantum numbers, centred on the block's mean filling, whose variance grows with
  ln(m).  The variance laws were fitted to the kept-state histograms of a real
  infinite-lattice DMRG at m = 32..256 (Heisenberg: var(2 S^z) = 1.2 ln m - 0.6;
  Hubbard, in charge / spin coordinates N_up + N_down and N_up - N_down:
  var_c = 0.1 ln m + 0.7, var_s = 0.4 ln m + 0.8); counts are found by water-filling so
  that exactly min(m, dim) states are kept;
* which states a sector keeps: the lowest eigenvectors of that sector's block of the
  enlarged-block Hamiltonian (an energy truncation), each signed so its
  largest-magnitude entry is positive;
* with m >= the full block dimension nothing is truncated and the superblock is the
  exact one, so its lowest eigenvalue equals exact diagonalisation of the chain.

Fermion signs follow the mode order of Eqs. 5-6 (sites left to right, down before up):
a hop from the last site of the left block to the first site of the right block is
(c^dag P) (x) c with P the parity of the whole left block; inside a block the string of
the edge operator is carried by the block (left side) or is absent (right side).
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

from .superblock import (IDENTITY, BlockOp, Superblock, SuperblockL11r, pairs_for_target,
                         segs_for_target)

Blocks = Dict[Tuple[int, int], np.ndarray]


# ------------------------------------------------------------------ sites
def _heis_site():
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])          # S+ in basis (up, down), Eq. 3
    sz = np.diag([0.5, -0.5])
    return [(1,), (-1,)], {"H": np.zeros((2, 2)), "Sp": sp, "Sz": sz}


def _hub_site(U):
    c = np.array([[0.0, 1.0], [0.0, 0.0]])           # Eq. 8 (annihilator)
    phi = np.diag([1.0, -1.0])                         # Eq. 7
    eye = np.eye(2)
    c_dn = np.kron(c, eye)                             # mode order down, up (Eq. 6)
    c_up = np.kron(phi, c)
    H = U * np.diag(np.diag(c_dn.T @ c_dn) * np.diag(c_up.T @ c_up))
    return ([(0, 0), (1, 0), (0, 1), (1, 1)],          # (N_up, N_down) of index 2 n_dn + n_up
            {"H": H, "cdag_up": c_up.T.copy(), "cdag_dn": c_dn.T.copy(),
             "P": np.diag([1.0, -1.0, -1.0, 1.0])})


def _add(q1, q2):
    return tuple(a + b for a, b in zip(q1, q2))


# ------------------------------------------------------------------ block-sparse block
class SBlock:
    """Sector-blocked basis (quantum numbers q, dims d) plus named block operators."""

    def __init__(self, q: List[tuple], d: List[int], ops: Dict[str, Blocks]):
        self.q, self.d, self.ops = list(q), list(d), ops

    @property
    def dim(self):
        return int(sum(self.d))

    def parity(self) -> List[float]:
        return [(-1.0) ** (sum(qq) % 2) for qq in self.q]


def _site_block(labels, ops):
    # one sector per site state (quantum numbers of the site states are distinct)
    q = list(labels)
    blocks = {}
    for name, M in ops.items():
        bl = {}
        for i in range(len(q)):
            for j in range(len(q)):
                if M[j, i] != 0.0:
                    bl[(i, j)] = np.array([[M[j, i]]])
        blocks[name] = bl
    return SBlock(q, [1] * len(q), blocks)


class _Layout:
    """Enlarged sectors of block (x) site: each sector lists (sigma, a) in sigma order."""

    def __init__(self, blk: SBlock, slabels):
        combos = {}
        for s, qs in enumerate(slabels):
            for a, qa in enumerate(blk.q):
                combos.setdefault(_add(qa, qs), []).append((s, a))
        self.q = sorted(combos)
        self.index = {qq: n for n, qq in enumerate(self.q)}
        self.pos = {}
        self.d = []
        for n, qq in enumerate(self.q):
            off = 0
            for s, a in combos[qq]:
                self.pos[(s, a)] = (n, off)
                off += blk.d[a]
            self.d.append(off)


def _embed(layout: _Layout, blk: SBlock, bops: Blocks, sop: np.ndarray) -> Blocks:
    """Blocks of (block operator) (x) (site operator) on the enlarged sectors.
    ``bops`` None means the block identity, ``sop`` None the site identity."""
    ns = len({s for s, _ in layout.pos})
    site_elems = ([(s, s, 1.0) for s in range(ns)] if sop is None else
                  [(s, t, sop[t, s]) for s in range(ns) for t in range(ns) if sop[t, s] != 0.0])
    blk_elems = ({(a, a): None for a in range(len(blk.d))} if bops is None else bops)
    out: Blocks = {}
    for (a, b), B in blk_elems.items():
        for s, t, v in site_elems:
            if (s, a) not in layout.pos or (t, b) not in layout.pos:
                continue
            ni, ci = layout.pos[(s, a)]
            nj, rj = layout.pos[(t, b)]
            key = (ni, nj)
            if key not in out:
                out[key] = np.zeros((layout.d[nj], layout.d[ni]))
            if B is None:
                out[key][rj:rj + blk.d[a], ci:ci + blk.d[a]] += v * np.eye(blk.d[a])
            else:
                out[key][rj:rj + blk.d[b], ci:ci + blk.d[a]] += v * B
    return out


def _bsum(*terms) -> Blocks:
    out: Blocks = {}
    for coef, bl in terms:
        for key, M in bl.items():
            if key in out:
                out[key] = out[key] + coef * M
            else:
                out[key] = coef * M
    return out


def _bmul(X: Blocks, Y: Blocks) -> Blocks:
    """Product X @ Y of two block operators (blocks keyed (in, out))."""
    out: Blocks = {}
    for (a, b), Yb in Y.items():
        for (c, d), Xb in X.items():
            if c == b:
                key = (a, d)
                out[key] = out.get(key, 0.0) + Xb @ Yb
    return out


def _btrans(X: Blocks) -> Blocks:
    return {(j, i): M.T.copy() for (i, j), M in X.items()}


def _bdiag_sign(signs: List[float], d: List[int]) -> Blocks:
    return {(i, i): s * np.eye(d[i]) for i, s in enumerate(signs)}


# ------------------------------------------------------------------ enlargement
def enlarge(blk: SBlock, model: str, side: str, J=1.0, delta=1.0, t=1.0, U=4.0) -> SBlock:
    """One site added to the centre side of a block: left block -> l (x) s,
    right block -> s (x) r (Sec. 4.1)."""
    if model == "heisenberg":
        slabels, sops = _heis_site()
    else:
        slabels, sops = _hub_site(U)
    lay = _Layout(blk, slabels)
    E = lambda bops, sop: _embed(lay, blk, bops, sop)
    if model == "heisenberg":
        sp, sz = sops["Sp"], sops["Sz"]
        H = _bsum((1.0, E(blk.ops["H"], None)),
                  (0.5 * J, E(blk.ops["Sp"], sp.T)), (0.5 * J, E(_btrans(blk.ops["Sp"]), sp)),
                  (J * delta, E(blk.ops["Sz"], sz)))
        ops = {"H": H, "Sp": E(None, sp), "Sz": E(None, sz)}
    else:
        H_parts = [(1.0, E(blk.ops["H"], None)), (1.0, E(None, sops["H"]))]
        ops = {}
        Pb = _bdiag_sign(blk.parity(), blk.d)
        for sig in ("up", "dn"):
            cd_s = sops["cdag_" + sig]
            cd_e = blk.ops["cdag_" + sig]
            if side == "L":
                hop = E(_bmul(cd_e, Pb), cd_s.T)           # (c^dag_e P_l) (x) c_s
                ops["cdag_" + sig] = E(Pb, cd_s)           # P_l (x) c^dag_s
            else:
                hop = E(_btrans(cd_e), cd_s @ sops["P"])   # (c^dag_s P_s) (x) c_e
                ops["cdag_" + sig] = E(None, cd_s)         # c^dag_s (x) 1
            H_parts += [(-t, hop), (-t, _btrans(hop))]
        ops["H"] = _bsum(*H_parts)
    # drop exact-zero blocks so the sparsity pattern is the symmetry's
    for name in ops:
        ops[name] = {k: v for k, v in ops[name].items() if np.any(v != 0.0)}
    return SBlock(lay.q, lay.d, ops)


# ------------------------------------------------------------------ truncation
def _profile_weights(q: List[tuple], model: str, nsites: int, m: int, filling: float):
    lm = math.log(max(m, 2))
    if model == "heisenberg":
        var = max(1.0, 1.2 * lm - 0.6)
        return [math.exp(-(qq[0] ** 2) / (2 * var)) for qq in q]
    var_c = 0.1 * lm + 0.7
    var_s = 0.4 * lm + 0.8
    centre = filling * nsites
    w = []
    for nu, nd in q:
        c = nu + nd - centre
        s = nu - nd
        w.append(math.exp(-(c * c) / (2 * var_c) - (s * s) / (2 * var_s)))
    return w


def allocate(d: List[int], w: List[float], m: int) -> List[int]:
    """Kept states per sector: min(d, round(scale * w)) with the scale found so that the
    total is exactly min(m, sum d); remainders go to the heaviest sectors with room."""
    total = min(m, int(sum(d)))
    if total == sum(d):
        return list(d)
    lo, hi = 0.0, 1.0
    cnt = lambda s: sum(min(di, int(math.floor(s * wi + 0.5))) for di, wi in zip(d, w))
    while cnt(hi) < total:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if cnt(mid) < total:
            lo = mid
        else:
            hi = mid
    keep = [min(di, int(math.floor(lo * wi + 0.5))) for di, wi in zip(d, w)]
    order = sorted(range(len(d)), key=lambda i: (-w[i], i))
    short = total - sum(keep)
    while short > 0:
        for i in order:
            if short == 0:
                break
            if keep[i] < d[i]:
                keep[i] += 1
                short -= 1
    return keep


def truncate(blk: SBlock, keep: List[int]) -> SBlock:
    P = {}
    for i, (di, ki) in enumerate(zip(blk.d, keep)):
        if ki == 0:
            continue
        if ki == di:
            P[i] = None
            continue
        Hq = blk.ops["H"].get((i, i), np.zeros((di, di)))
        w, v = np.linalg.eigh(0.5 * (Hq + Hq.T))
        v = v[:, :ki].copy()
        for c in range(ki):
            if v[np.argmax(np.abs(v[:, c])), c] < 0:
                v[:, c] = -v[:, c]
        P[i] = v
    remap = {old: new for new, old in enumerate(sorted(P))}
    ops = {}
    for name, bl in blk.ops.items():
        nb = {}
        for (i, j), M in bl.items():
            if i not in P or j not in P:
                continue
            R = M if P[i] is None else M @ P[i]
            R = R if P[j] is None else P[j].T @ R
            nb[(remap[i], remap[j])] = R
        ops[name] = nb
    return SBlock([blk.q[i] for i in sorted(P)], [keep[i] for i in sorted(P)], ops)


# ------------------------------------------------------------------ superblock
def _to_blockop(bl: Blocks, name: str) -> BlockOp:
    return BlockOp({k: np.ascontiguousarray(v) for k, v in bl.items()}, name=name)


def target(model: str, N: int, filling: float = 1.0):
    if model == "heisenberg":
        return (0,)
    n = int(round(filling * N / 2))
    return (n, n)


def superblock_from_blocks(Lb: SBlock, Rb: SBlock, model: str, Q, J=1.0, delta=1.0, t=1.0) -> Superblock:
    opsL, opsR, terms = [], [], []

    def aL(bl, name):
        opsL.append(_to_blockop(bl, name))
        return len(opsL) - 1

    def aR(bl, name):
        opsR.append(_to_blockop(bl, name))
        return len(opsR) - 1

    terms.append((1.0, aL(Lb.ops["H"], "H_L"), IDENTITY))
    terms.append((1.0, IDENTITY, aR(Rb.ops["H"], "H_R")))
    if model == "heisenberg":
        spL, smL = aL(Lb.ops["Sp"], "Sp"), aL(_btrans(Lb.ops["Sp"]), "Sm")
        szL = aL(Lb.ops["Sz"], "Sz")
        spR, smR = aR(Rb.ops["Sp"], "Sp"), aR(_btrans(Rb.ops["Sp"]), "Sm")
        szR = aR(Rb.ops["Sz"], "Sz")
        terms += [(0.5 * J, spL, smR), (0.5 * J, smL, spR), (J * delta, szL, szR)]
    else:
        PL = _bdiag_sign(Lb.parity(), Lb.d)
        for sig in ("up", "dn"):
            cdP = _bmul(Lb.ops["cdag_" + sig], PL)
            a1, a2 = aL(cdP, "cdagP_" + sig), aL(_btrans(cdP), "Pc_" + sig)
            b1 = aR(_btrans(Rb.ops["cdag_" + sig]), "c_" + sig)
            b2 = aR(Rb.ops["cdag_" + sig], "cdag_" + sig)
            terms += [(-t, a1, b1), (-t, a2, b2)]
    pairs = pairs_for_target(Lb.q, Rb.q, Q)
    sb = Superblock(qL=list(Lb.q), dL=np.array(Lb.d, dtype=np.int64),
                    qR=list(Rb.q), dR=np.array(Rb.d, dtype=np.int64),
                    Q=tuple(Q), pairs=pairs, opsL=opsL, opsR=opsR, terms=terms)
    return sb


def _warmup_blocks(model: str, L: int, m: int, J, delta, t, U, filling):
    """The blocks l and r of L/2 - 1 sites each that the last step of the warm-up
    enlarges (Algorithm 1 with the LR strategy, truncated by the recipe above)."""
    if L < 4 or L % 2:
        raise ValueError("L must be even and >= 4")
    if model == "heisenberg":
        labels, sops = _heis_site()
        sops = {"H": sops["H"], "Sp": sops["Sp"], "Sz": sops["Sz"]}
    elif model == "hubbard":
        labels, sops = _hub_site(U)
        sops = {"H": sops["H"], "cdag_up": sops["cdag_up"], "cdag_dn": sops["cdag_dn"]}
    else:
        raise ValueError(model)
    left = _site_block(labels, sops)
    right = _site_block(labels, sops)
    kw = dict(J=J, delta=delta, t=t, U=U)
    nsites = 1
    while 2 * (nsites + 1) < L:
        Lb = enlarge(left, model, "L", **kw)
        Rb = enlarge(right, model, "R", **kw)
        nsites += 1
        keepL = allocate(Lb.d, _profile_weights(Lb.q, model, nsites, m, filling), m)
        keepR = allocate(Rb.d, _profile_weights(Rb.q, model, nsites, m, filling), m)
        left, right = truncate(Lb, keepL), truncate(Rb, keepR)
    return left, right


def warmup_superblock(model: str, L: int, m: int, J=1.0, delta=1.0, t=1.0, U=4.0,
                      filling=1.0) -> Superblock:
    """Mid-chain LR superblock of an L-site chain (L even, L >= 4): blocks of
    l = r = L/2 - 1 sites, enlarged to L/2 sites each, target sector of Sec. 3."""
    left, right = _warmup_blocks(model, L, m, J, delta, t, U, filling)
    kw = dict(J=J, delta=delta, t=t, U=U)
    Lb = enlarge(left, model, "L", **kw)
    Rb = enlarge(right, model, "R", **kw)
    sb = superblock_from_blocks(Lb, Rb, model, target(model, L, filling), J=J, delta=delta, t=t)
    sb.meta = {"model": model, "L": L, "m": m, "J": J, "delta": delta, "t": t, "U": U,
               "filling": filling}
    return sb


def superblock_l11r_from_blocks(lb: SBlock, rb: SBlock, model: str, Q, J=1.0, delta=1.0,
                                t=1.0, U=4.0) -> SuperblockL11r:
    """The same superblock Hamiltonian in the l-1-1-r form (Sec. 4.2, Eq. 12): the terms of
    H_SB = H_l + bond(l, s1) + H_s1 + bond(s1, s2) + H_s2 + bond(s2, r) + H_r, each a
    product of one factor per subsystem.  The bonds are those that the LR form builds into
    its enlarged blocks (l, s1) and (s2, r) and across them; for fermions the hop out of a
    subsystem X carries the parity P_X of all of X (c^dag_X P_X (x) c_Y and its transpose),
    with the modes ordered l, s1, s2, r and, inside a site, down before up (Eqs. 5-6)."""
    opsl, sops, opsr, terms = [], [], [], []

    def al(bl, name):
        opsl.append(_to_blockop(bl, name))
        return len(opsl) - 1

    def ar(bl, name):
        opsr.append(_to_blockop(bl, name))
        return len(opsr) - 1

    def as_(M):
        sops.append(np.ascontiguousarray(M, dtype=np.float64))
        return len(sops) - 1

    I = IDENTITY
    if model == "heisenberg":
        qs, s = _heis_site()
        sp, sm, sz = as_(s["Sp"]), as_(s["Sp"].T), as_(s["Sz"])
        terms += [(1.0, al(lb.ops["H"], "H_l"), I, I, I), (1.0, I, I, I, ar(rb.ops["H"], "H_r"))]
        spl, sml, szl = al(lb.ops["Sp"], "Sp"), al(_btrans(lb.ops["Sp"]), "Sm"), al(lb.ops["Sz"], "Sz")
        spr, smr, szr = ar(rb.ops["Sp"], "Sp"), ar(_btrans(rb.ops["Sp"]), "Sm"), ar(rb.ops["Sz"], "Sz")
        for a1, a2, a3, a4 in ((spl, sm, I, I), (sml, sp, I, I), (I, sp, sm, I),
                               (I, sm, sp, I), (I, I, sp, smr), (I, I, sm, spr)):
            terms.append((0.5 * J, a1, a2, a3, a4))
        terms += [(J * delta, szl, sz, I, I), (J * delta, I, sz, sz, I), (J * delta, I, I, sz, szr)]
    elif model == "hubbard":
        qs, s = _hub_site(U)
        P = s["P"]
        terms += [(1.0, al(lb.ops["H"], "H_l"), I, I, I), (1.0, I, as_(s["H"]), I, I),
                  (1.0, I, I, as_(s["H"]), I), (1.0, I, I, I, ar(rb.ops["H"], "H_r"))]
        Pl = _bdiag_sign(lb.parity(), lb.d)
        for sig in ("up", "dn"):
            cd = s["cdag_" + sig]
            cdP = _bmul(lb.ops["cdag_" + sig], Pl)              # c^dag_l P_l
            lcdP, lPc = al(cdP, "cdagP_" + sig), al(_btrans(cdP), "Pc_" + sig)
            rc, rcd = ar(_btrans(rb.ops["cdag_" + sig]), "c_" + sig), ar(rb.ops["cdag_" + sig], "cdag_" + sig)
            c_s, cd_s = as_(cd.T), as_(cd)
            cdP_s, Pc_s = as_(cd @ P), as_((cd @ P).T)
            terms += [(-t, lcdP, c_s, I, I), (-t, lPc, cd_s, I, I),      # bond (l, s1)
                      (-t, I, cdP_s, c_s, I), (-t, I, Pc_s, cd_s, I),    # bond (s1, s2)
                      (-t, I, I, cdP_s, rc), (-t, I, I, Pc_s, rcd)]      # bond (s2, r)
    else:
        raise ValueError(model)
    segs = segs_for_target(lb.q, qs, rb.q, Q)
    return SuperblockL11r(ql=list(lb.q), dl=np.array(lb.d, dtype=np.int64), qs=list(qs),
                          qr=list(rb.q), dr=np.array(rb.d, dtype=np.int64), Q=tuple(Q),
                          segs=segs, opsl=opsl, sops=sops, opsr=opsr, terms=terms)


def warmup_superblock_l11r(model: str, L: int, m: int, J=1.0, delta=1.0, t=1.0, U=4.0,
                           filling=1.0) -> SuperblockL11r:
    """The mid-chain superblock of ``warmup_superblock`` with the same arguments, in the
    l-1-1-r form: the same blocks l and r (L/2 - 1 sites each) and the two middle sites
    kept apart instead of enlarging the blocks (Sec. 4.2)."""
    left, right = _warmup_blocks(model, L, m, J, delta, t, U, filling)
    sb = superblock_l11r_from_blocks(left, right, model, target(model, L, filling), J=J,
                                     delta=delta, t=t, U=U)
    sb.meta = {"model": model, "L": L, "m": m, "J": J, "delta": delta, "t": t, "U": U,
               "filling": filling}
    return sb


def start_vector(n: int, seed: int = 0) -> np.ndarray:
    """Seeded uniform(-1, 1) start vector of length n (NumPy PCG64), normalised."""
    x = np.random.default_rng(seed).uniform(-1.0, 1.0, n)
    return x / np.linalg.norm(x)


# named workloads (sizes of the paper-shaped configurations)
WORKLOADS = {
    "heis_L16_m64": dict(model="heisenberg", L=16, m=64),
    "heis_L100_m1024": dict(model="heisenberg", L=100, m=1024),
    "hub_L64_m2048": dict(model="hubbard", L=64, m=2048, U=4.0, t=1.0),
    "hub_L100_m4096_quarter": dict(model="hubbard", L=100, m=4096, U=8.0, t=1.0, filling=0.5),
}


def workload(name: str) -> Superblock:
    return warmup_superblock(**WORKLOADS[name])


def workload_l11r(name: str) -> SuperblockL11r:
    """The named workload's superblock in the l-1-1-r form (same Hamiltonian)."""
    return warmup_superblock_l11r(**WORKLOADS[name])


def batched_workload(count: int = 64, ms=(256, 512, 1024, 2048), L: int = 100, seed: int = 1234,
                     model: str = "heisenberg"):
    """Independent superblocks of uneven size: m_i drawn uniformly from ``ms`` (NumPy
    PCG64, ``seed``).  Problems that draw the same m share the (deterministic) operator
    blocks; each problem has its own start vector (seed i).  Returns (superblocks, m list,
    start vectors)."""
    rng = np.random.default_rng(seed)
    draws = [int(m) for m in rng.choice(np.asarray(ms), size=count)]
    cache = {}
    sbs, x0s = [], []
    for i, m in enumerate(draws):
        if m not in cache:
            cache[m] = warmup_superblock(model, L, m)
        sbs.append(cache[m])
        x0s.append(start_vector(cache[m].n, seed=i))
    return sbs, draws, x0s
