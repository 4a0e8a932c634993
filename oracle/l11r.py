"""The projection X' = H_SB X in the l-1-1-r form (oracle; test infrastructure).

Sec. 4.2 writes the superblock Hamiltonian with one factor per subsystem (Eq. 12),

  H_SB = sum_a c_a  A_a^(l) (x) a_a (x) b_a (x) B_a^(r),

and evaluates the projection term by term with Algorithm 2: the vector, reshaped to the
four indices of (l, s1, s2, r), is multiplied by the factor of each index in turn -- the
last one (B of block r) first, then the two sites, then A of block l -- every reshape
being a change of the size descriptors only (Eq. 13 sums these over the terms).

Two independent restatements:

* ``superblock_dense`` / ``project_dense``: the plain definition, the sum of the
  four-fold Kronecker products restricted to the rows and columns whose quantum numbers
  add up to Q; a full index is ((l * q + s1) * q + s2) * dim_r + r.
* ``project_blocks``: Algorithm 2 for every term with the operators decomposed by
  quantum numbers (the paragraph after Eq. 13): for each block A_{i->j}, site elements
  a[s1' <- s1], b[s2' <- s2] and block B_{k->l} with valid input and output segments,
  the four stages applied to segment (i, s1, s2, k) and added to segment (j, s1', s2', l).

``diagonal`` gives diag(H_SB), the Davidson preconditioner input.
"""
from __future__ import annotations

import numpy as np

from dmrg_inputs.superblock import IDENTITY, SuperblockL11r


def _dense_block_op(d, op, identity: bool) -> np.ndarray:
    d = np.asarray(d, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(d)])
    if identity:
        return np.eye(int(off[-1]))
    M = np.zeros((int(off[-1]), int(off[-1])))
    for (i, j), blk in op.blocks.items():
        M[off[j]:off[j + 1], off[i]:off[i + 1]] = blk
    return M


def sector_indices(sb: SuperblockL11r) -> np.ndarray:
    """Full-space index of every entry of X in storage order."""
    offl = np.concatenate([[0], np.cumsum(sb.dl)])
    offr = np.concatenate([[0], np.cumsum(sb.dr)])
    q, dimr = sb.q, int(offr[-1])
    idx = []
    for i, s1, s2, k in sb.segs:
        a = np.arange(offl[i], offl[i + 1])
        b = np.arange(offr[k], offr[k + 1])
        idx.append((((a[:, None] * q + s1) * q + s2) * dimr + b[None, :]).ravel())
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def superblock_dense(sb: SuperblockL11r) -> np.ndarray:
    """Eq. 12 written out: sum_a c_a kron(A, a, b, B), restricted to sector Q."""
    idx = sector_indices(sb)
    q = sb.q
    dimr = int(np.sum(sb.dr))
    ir = idx % dimr
    rest = idx // dimr
    is2 = rest % q
    rest //= q
    is1 = rest % q
    il = rest // q
    H = np.zeros((len(idx), len(idx)))
    eye_q = np.eye(q)
    for coef, a, s1, s2, b in sb.terms:
        A = _dense_block_op(sb.dl, None if a == IDENTITY else sb.opsl[a], a == IDENTITY)
        S1 = eye_q if s1 == IDENTITY else sb.sops[s1]
        S2 = eye_q if s2 == IDENTITY else sb.sops[s2]
        B = _dense_block_op(sb.dr, None if b == IDENTITY else sb.opsr[b], b == IDENTITY)
        # entry (row, col) of the Kronecker product is the product of the factors' entries
        H += coef * (A[np.ix_(il, il)] * S1[np.ix_(is1, is1)] * S2[np.ix_(is2, is2)]
                     * B[np.ix_(ir, ir)])
    return H


def project_dense(sb: SuperblockL11r, x: np.ndarray) -> np.ndarray:
    return superblock_dense(sb) @ x


def _site_elements(sb: SuperblockL11r, o: int):
    """(s_in, s_out, value) of the non-zero elements of site operator o (identity: -1)."""
    if o == IDENTITY:
        return [(s, s, 1.0) for s in range(sb.q)]
    M = sb.sops[o]
    return [(s, t, float(M[t, s])) for s in range(sb.q) for t in range(sb.q) if M[t, s] != 0.0]


def project_blocks(sb: SuperblockL11r, x: np.ndarray) -> np.ndarray:
    """Algorithm 2 summed over the terms (Eq. 13), on the quantum-number blocks."""
    off = sb.offsets()
    where = sb.seg_index()
    y = np.zeros(off[-1])

    def seg(v, p):
        i, _, _, k = sb.segs[p]
        return v[off[p]:off[p + 1]].reshape(int(sb.dl[i]), int(sb.dr[k]))

    for coef, a, s1, s2, b in sb.terms:
        a_blocks = ({(i, i): None for i in range(len(sb.dl))} if a == IDENTITY
                    else sb.opsl[a].blocks)
        b_blocks = ({(k, k): None for k in range(len(sb.dr))} if b == IDENTITY
                    else sb.opsr[b].blocks)
        e1, e2 = _site_elements(sb, s1), _site_elements(sb, s2)
        for (i, j), A in a_blocks.items():
            for (k, l), B in b_blocks.items():
                for u1, v1, a1 in e1:
                    for u2, v2, a2 in e2:
                        pin, pout = where.get((i, u1, u2, k)), where.get((j, v1, v2, l))
                        if pin is None or pout is None:
                            continue
                        X = seg(x, pin)
                        Z = X if B is None else X @ B.T     # stage 1: the factor of block r
                        Z = a2 * Z                           # stage 2: site s2
                        Z = a1 * Z                           # stage 3: site s1
                        Z = Z if A is None else A @ Z        # stage 4: the factor of block l
                        seg(y, pout)[...] += coef * Z
    return y


def diagonal(sb: SuperblockL11r) -> np.ndarray:
    """diag(H_SB) in storage order: sum c diag(A_ii) (x) a[s1, s1] b[s2, s2] diag(B_kk)."""
    off = sb.offsets()
    D = np.zeros(off[-1])
    for coef, a, s1, s2, b in sb.terms:
        for p, (i, u1, u2, k) in enumerate(sb.segs):
            f1 = 1.0 if s1 == IDENTITY else float(sb.sops[s1][u1, u1])
            f2 = 1.0 if s2 == IDENTITY else float(sb.sops[s2][u2, u2])
            if f1 == 0.0 or f2 == 0.0:
                continue
            if a == IDENTITY:
                da = np.ones(int(sb.dl[i]))
            else:
                blk = sb.opsl[a].blocks.get((i, i))
                if blk is None:
                    continue
                da = np.diag(blk)
            if b == IDENTITY:
                db = np.ones(int(sb.dr[k]))
            else:
                blk = sb.opsr[b].blocks.get((k, k))
                if blk is None:
                    continue
                db = np.diag(blk)
            D[off[p]:off[p + 1]] += coef * f1 * f2 * np.outer(da, db).ravel()
    return D


def flop_count(sb: SuperblockL11r) -> dict:
    """Algorithmic FLOPs of one projection by Algorithm 2 on the blocks: per record the
    cheaper order of the two block products (site factors are scalars), identity factors
    skipped."""
    where = sb.seg_index()
    total = 0
    records = 0
    for coef, a, s1, s2, b in sb.terms:
        a_blocks = ({(i, i): None for i in range(len(sb.dl))} if a == IDENTITY
                    else sb.opsl[a].blocks)
        b_blocks = ({(k, k): None for k in range(len(sb.dr))} if b == IDENTITY
                    else sb.opsr[b].blocks)
        e1, e2 = _site_elements(sb, s1), _site_elements(sb, s2)
        for (i, j) in a_blocks:
            for (k, l) in b_blocks:
                for u1, v1, _ in e1:
                    for u2, v2, _ in e2:
                        if (i, u1, u2, k) not in where or (j, v1, v2, l) not in where:
                            continue
                        records += 1
                        di, dj, dk, dl = (int(sb.dl[i]), int(sb.dl[j]), int(sb.dr[k]),
                                          int(sb.dr[l]))
                        if a == IDENTITY and b == IDENTITY:
                            continue
                        if a == IDENTITY:
                            total += 2 * di * dk * dl
                        elif b == IDENTITY:
                            total += 2 * dj * di * dk
                        else:
                            total += min(2 * dj * di * dk + 2 * dj * dk * dl,
                                         2 * di * dk * dl + 2 * dj * di * dl)
    return {"flops": total, "records": records}
