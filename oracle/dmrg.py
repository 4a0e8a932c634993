"""Infinite-lattice DMRG with the LR strategy (oracle; test infrastructure).

Algorithm 1 (Sec. 4): starting from the four-site superblock (one-site blocks), every
iteration enlarges the left block l and the right block r by one site each (L = l+1,
R = r+1, Sec. 4.1), forms the superblock H_SB = sum_a A_a (x) B_a (Eq. 9), finds its
lowest eigenstate with the Davidson method (Algorithm 3), builds the density matrix of
each enlarged block from that state, diagonalises it and keeps the m states of largest
weight.

Blocks are kept here as dense matrices on the block space plus one quantum-number label
per basis state; the superblock handed to the projection is the sector-blocked form of
Sec. 4.1.  Readings where the paper is silent:

* the right block is grown on its own (a site is added on its left), not mirrored;
* fermion signs: with modes ordered left to right and, inside a site, down before up
  (Eqs. 5, 6), a hop between the last site of L and the first site of R is
  (c^dagger_{s_L} P_L) (x) c_{s_R} with P_L = (-1)^{N_L}; inside the right block the new
  first site carries no string and the hop into the old block carries the site parity;
* truncation keeps exactly min(m, dim) states: density-matrix eigenvalues sorted in
  descending order, ties broken by (sector order, in-sector order); each kept vector is
  signed so that its largest-magnitude entry is positive;
* the target sector of a chain of N sites is S^z = 0 (Heisenberg, N even) or
  N_up = N_down = round(filling * N / 2) (Hubbard, filling = particles per site).
"""
from __future__ import annotations

import numpy as np

from dmrg_inputs.superblock import IDENTITY, BlockOp, Superblock, pairs_for_target

from . import sites
from .davidson import davidson
from .projection import diagonal, project_blocks


class Block:
    """Dense operators of a block on its (possibly truncated) basis, with labels."""

    def __init__(self, labels, ops):
        self.labels = [tuple(q) for q in labels]
        self.ops = ops            # name -> dense matrix

    @property
    def dim(self):
        return len(self.labels)


# ---------------- single sites ----------------

def heisenberg_site():
    # basis (up, down): 2 S^z = +1, -1 (Eq. 3)
    return Block([(1,), (-1,)], {"H": np.zeros((2, 2)), "Sp": sites.S_PLUS.copy(),
                                 "Sz": sites.S_Z.copy()})


def _hubbard_site_ops(U):
    # site = mode(down) (x) mode(up); index = 2 n_down + n_up (Eq. 6 order)
    c_dn = np.kron(sites.C_ANN, sites.EYE2)
    c_up = np.kron(sites.PHI, sites.C_ANN)
    n_dn = c_dn.T @ c_dn
    n_up = c_up.T @ c_up
    parity = np.kron(sites.PHI, sites.PHI)
    H = U * (n_dn @ n_up)          # (U/2) sum_{s != s'} n_s n_s' for F = 1/2 (Eq. 4)
    labels = [(0, 0), (1, 0), (0, 1), (1, 1)]   # (N_up, N_down)
    return labels, {"H": H, "cdag_up": c_up.T.copy(), "cdag_dn": c_dn.T.copy(),
                    "P": parity}


def hubbard_site(U):
    labels, ops = _hubbard_site_ops(U)
    return Block(labels, {"H": ops["H"], "cdag_up": ops["cdag_up"],
                          "cdag_dn": ops["cdag_dn"]})


def _parity(block):
    return np.diag([(-1.0) ** (sum(q)) for q in block.labels])


# ---------------- enlargement (Sec. 4.1: L = l + 1, R = r + 1) ----------------

def enlarge_left_heis(blk, J, delta):
    s = heisenberg_site()
    Il, Is = np.eye(blk.dim), np.eye(2)
    Sp_e, Sz_e = blk.ops["Sp"], blk.ops["Sz"]
    H = (np.kron(blk.ops["H"], Is) + np.kron(Il, s.ops["H"])
         + 0.5 * J * (np.kron(Sp_e, s.ops["Sp"].T) + np.kron(Sp_e.T, s.ops["Sp"]))
         + J * delta * np.kron(Sz_e, s.ops["Sz"]))
    labels = [tuple(a + b for a, b in zip(qa, qs)) for qa in blk.labels for qs in s.labels]
    return Block(labels, {"H": H, "Sp": np.kron(Il, s.ops["Sp"]), "Sz": np.kron(Il, s.ops["Sz"])})


def enlarge_right_heis(blk, J, delta):
    s = heisenberg_site()
    Ir, Is = np.eye(blk.dim), np.eye(2)
    Sp_e, Sz_e = blk.ops["Sp"], blk.ops["Sz"]
    H = (np.kron(s.ops["H"], Ir) + np.kron(Is, blk.ops["H"])
         + 0.5 * J * (np.kron(s.ops["Sp"], Sp_e.T) + np.kron(s.ops["Sp"].T, Sp_e))
         + J * delta * np.kron(s.ops["Sz"], Sz_e))
    labels = [tuple(a + b for a, b in zip(qs, qb)) for qs in s.labels for qb in blk.labels]
    return Block(labels, {"H": H, "Sp": np.kron(s.ops["Sp"], Ir), "Sz": np.kron(s.ops["Sz"], Ir)})


def enlarge_left_hub(blk, t, U):
    slabels, sops = _hubbard_site_ops(U)
    Il, Is = np.eye(blk.dim), np.eye(4)
    Pl = _parity(blk)
    H = np.kron(blk.ops["H"], Is) + np.kron(Il, sops["H"])
    new = {}
    for sig in ("up", "dn"):
        cd_e = blk.ops["cdag_" + sig]
        c_s = sops["cdag_" + sig].T
        hop = np.kron(cd_e @ Pl, c_s)          # c^dag_edge c_site with the string P_l
        H = H - t * (hop + hop.T)
        new["cdag_" + sig] = np.kron(Pl, sops["cdag_" + sig])
    labels = [tuple(a + b for a, b in zip(qa, qs)) for qa in blk.labels for qs in slabels]
    new["H"] = H
    return Block(labels, new)


def enlarge_right_hub(blk, t, U):
    slabels, sops = _hubbard_site_ops(U)
    Ir, Is = np.eye(blk.dim), np.eye(4)
    H = np.kron(sops["H"], Ir) + np.kron(Is, blk.ops["H"])
    new = {}
    for sig in ("up", "dn"):
        cd_s = sops["cdag_" + sig]
        c_e = blk.ops["cdag_" + sig].T
        hop = np.kron(cd_s @ sops["P"], c_e)   # c^dag_site c_edge with the site parity
        H = H - t * (hop + hop.T)
        new["cdag_" + sig] = np.kron(cd_s, Ir)
    labels = [tuple(a + b for a, b in zip(qs, qb)) for qs in slabels for qb in blk.labels]
    new["H"] = H
    return Block(labels, new)


# ---------------- superblock in sector-blocked form ----------------

def _sectorise(block):
    qs = sorted(set(block.labels))
    members = [np.array([s for s, q in enumerate(block.labels) if q == qq], dtype=np.int64)
               for qq in qs]
    return qs, members


def _block_op(dense, members, name):
    bo = BlockOp(name=name)
    for i, mi in enumerate(members):
        for j, mj in enumerate(members):
            blk = dense[np.ix_(mj, mi)]
            if np.any(blk != 0.0):
                bo.blocks[(i, j)] = blk.copy()
    return bo


def build_superblock(Lb, Rb, Q, model, J=1.0, delta=1.0, t=1.0):
    qL, memL = _sectorise(Lb)
    qR, memR = _sectorise(Rb)
    pairs = pairs_for_target(qL, qR, Q)
    opsL, opsR, terms = [], [], []

    def addL(M, name):
        opsL.append(_block_op(M, memL, name))
        return len(opsL) - 1

    def addR(M, name):
        opsR.append(_block_op(M, memR, name))
        return len(opsR) - 1

    hL, hR = addL(Lb.ops["H"], "H_L"), addR(Rb.ops["H"], "H_R")
    terms += [(1.0, hL, IDENTITY), (1.0, IDENTITY, hR)]
    if model == "heisenberg":
        spL, smL, szL = addL(Lb.ops["Sp"], "Sp"), addL(Lb.ops["Sp"].T, "Sm"), addL(Lb.ops["Sz"], "Sz")
        spR, smR, szR = addR(Rb.ops["Sp"], "Sp"), addR(Rb.ops["Sp"].T, "Sm"), addR(Rb.ops["Sz"], "Sz")
        terms += [(0.5 * J, spL, smR), (0.5 * J, smL, spR), (J * delta, szL, szR)]
    else:
        PL = _parity(Lb)
        for sig in ("up", "dn"):
            cd = Lb.ops["cdag_" + sig]
            a1 = addL(cd @ PL, "cdagP_" + sig)       # c^dag_{s_L} P_L
            a2 = addL(PL @ cd.T, "Pc_" + sig)        # its transpose
            b1 = addR(Rb.ops["cdag_" + sig].T, "c_" + sig)
            b2 = addR(Rb.ops["cdag_" + sig], "cdag_" + sig)
            terms += [(-t, a1, b1), (-t, a2, b2)]
    sb = Superblock(qL=qL, dL=np.array([len(m) for m in memL], dtype=np.int64),
                    qR=qR, dR=np.array([len(m) for m in memR], dtype=np.int64),
                    Q=tuple(Q), pairs=pairs, opsL=opsL, opsR=opsR, terms=terms)
    return sb, memL, memR


# ---------------- truncation (Algorithm 1, lines 4-7) ----------------

def _truncate(block, members, rho_blocks, m):
    cand = []      # (weight, sector, in-sector index, vector)
    for s, (mem, rho) in enumerate(zip(members, rho_blocks)):
        w, v = np.linalg.eigh(rho)
        for c in range(len(w)):
            cand.append((-w[c], s, c, v[:, c]))
    cand.sort(key=lambda z: (z[0], z[1], z[2]))
    keep = cand[:min(m, len(cand))]
    keep.sort(key=lambda z: (z[1], z[0], z[2]))
    P = np.zeros((block.dim, len(keep)))
    labels = []
    for col, (_, s, _, vec) in enumerate(keep):
        vec = vec.copy()
        if vec[np.argmax(np.abs(vec))] < 0:
            vec = -vec
        P[members[s], col] = vec
        labels.append(block.labels[members[s][0]])
    ops = {name: P.T @ M @ P for name, M in block.ops.items()}
    weight_kept = -sum(z[0] for z in keep)
    return Block(labels, ops), weight_kept


def target_for(model, N, filling=1.0):
    if model == "heisenberg":
        return (0,)
    n = int(round(filling * N / 2))
    return (n, n)


def infinite_dmrg(model: str, L: int, m: int, J=1.0, delta=1.0, t=1.0, U=4.0,
                  filling=1.0, seed: int = 0, tol: float = 1e-10, max_iter: int = 1000,
                  keep_last: bool = True, callback=None):
    """Grow a chain to L sites (L even, L >= 4).  Returns a dict with the energies per
    chain length, the last superblock and its ground state."""
    if model == "heisenberg":
        site = heisenberg_site()
        grow_l = lambda b: enlarge_left_heis(b, J, delta)
        grow_r = lambda b: enlarge_right_heis(b, J, delta)
    else:
        site = hubbard_site(U)
        grow_l = lambda b: enlarge_left_hub(b, t, U)
        grow_r = lambda b: enlarge_right_hub(b, t, U)
    left, right = site, site
    rng = np.random.default_rng(seed)
    energies = {}
    out = {}
    N = 4
    while N <= L:
        Lb, Rb = grow_l(left), grow_r(right)
        Q = target_for(model, N, filling)
        sb, memL, memR = build_superblock(Lb, Rb, Q, model, J=J, delta=delta, t=t)
        D = diagonal(sb)
        x0 = rng.uniform(-1.0, 1.0, sb.n)
        lam, x, info = davidson(lambda v: project_blocks(sb, v), D, x0, tol=tol,
                                max_iter=max_iter)
        energies[N] = lam
        if callback:
            callback(N, lam, info, sb)
        if N == L:
            out.update(superblock=sb, x=x, info=info)
            break
        # density matrices of the two enlarged blocks from the ground state (Alg. 1 l. 5)
        off = sb.offsets()
        rhoL = [np.zeros((len(mm), len(mm))) for mm in memL]
        rhoR = [np.zeros((len(mm), len(mm))) for mm in memR]
        for p, (i, k) in enumerate(sb.pairs):
            X = x[off[p]:off[p + 1]].reshape(len(memL[i]), len(memR[k]))
            rhoL[i] += X @ X.T
            rhoR[k] += X.T @ X
        # basis of each enlarged block re-ordered by sector for the truncation
        left, _ = _truncate(Lb, memL, rhoL, m)
        right, _ = _truncate(Rb, memR, rhoR, m)
        N += 2
    out["energies"] = energies
    return out
