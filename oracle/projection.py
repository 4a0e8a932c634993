"""The superblock projection X' = H_SB X (oracle; test infrastructure).

Two independent restatements:

* ``superblock_dense`` / ``project_dense``: the plain definition.  H_SB is the sum of
  Kronecker products coef * (A (x) B) of Eq. 9 over the full enlarged-block spaces,
  restricted to the rows and columns whose quantum numbers add up to the target Q
  (Sec. 3); a vector is indexed (left state) * dim_R + (right state), so the reshape of
  Eq. 10 is the row-major one (left index slow).
* ``project_blocks``: the sector-decomposed products of Eq. 11,
  X'_{jl} += coef * A_{i->j} X_{ik} B_{k->l}^T, over every transition pair whose input
  (i, k) and output (j, l) segments are both inside the sector (Sec. 4.1).

``diagonal`` gives diag(H_SB) from the diagonal blocks only; it is the preconditioner
input used by the Davidson correction step (Algorithm 3, "correct r").
"""
from __future__ import annotations

import numpy as np

from dmrg_inputs.superblock import IDENTITY, Superblock


def _dense_op(sb_d, op, identity: bool) -> np.ndarray:
    d = np.asarray(sb_d, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(d)])
    dim = int(off[-1])
    if identity:
        return np.eye(dim)
    M = np.zeros((dim, dim))
    for (i, j), blk in op.blocks.items():
        M[off[j]:off[j + 1], off[i]:off[i + 1]] = blk
    return M


def sector_indices(sb: Superblock) -> np.ndarray:
    """Full-space index (left * dim_R + right) of every entry of X in storage order."""
    offL = np.concatenate([[0], np.cumsum(sb.dL)])
    offR = np.concatenate([[0], np.cumsum(sb.dR)])
    dimR = int(offR[-1])
    idx = []
    for i, k in sb.pairs:
        a = np.arange(offL[i], offL[i + 1])
        b = np.arange(offR[k], offR[k + 1])
        idx.append((a[:, None] * dimR + b[None, :]).ravel())
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def superblock_dense(sb: Superblock) -> np.ndarray:
    """Eq. 9 written out: sum_a coef_a kron(A_a, B_a), restricted to sector Q.

    The entry of kron(A, B) at full indices (l*dimR + r, l'*dimR + r') is
    A[l, l'] * B[r, r'], so the restriction to the sector rows/columns is the
    elementwise product of A and B gathered at the sector's left and right indices."""
    idx = sector_indices(sb)
    dimR = int(np.sum(sb.dR))
    il, ir = idx // dimR, idx % dimR
    H = np.zeros((len(idx), len(idx)))
    for coef, a, b in sb.terms:
        A = _dense_op(sb.dL, None if a == IDENTITY else sb.opsL[a], a == IDENTITY)
        B = _dense_op(sb.dR, None if b == IDENTITY else sb.opsR[b], b == IDENTITY)
        H += coef * (A[np.ix_(il, il)] * B[np.ix_(ir, ir)])
    return H


def project_dense(sb: Superblock, x: np.ndarray) -> np.ndarray:
    return superblock_dense(sb) @ x


def leak_outside_sector(sb: Superblock, x: np.ndarray) -> float:
    """Norm of (sum coef A (x) B) x_full outside sector Q, for x zero outside Q.

    Sec. 3: H_SB commutes with the symmetry, so the result must vanish."""
    idx = sector_indices(sb)
    dimL, dimR = int(np.sum(sb.dL)), int(np.sum(sb.dR))
    xf = np.zeros(dimL * dimR)
    xf[idx] = x
    Xf = xf.reshape(dimL, dimR)
    Y = np.zeros_like(Xf)
    for coef, a, b in sb.terms:
        A = _dense_op(sb.dL, None if a == IDENTITY else sb.opsL[a], a == IDENTITY)
        B = _dense_op(sb.dR, None if b == IDENTITY else sb.opsR[b], b == IDENTITY)
        Y += coef * (A @ Xf @ B.T)          # Eq. 10 on the full spaces
    yf = Y.ravel().copy()
    yf[idx] = 0.0
    return float(np.linalg.norm(yf))


def project_blocks(sb: Superblock, x: np.ndarray) -> np.ndarray:
    """Eq. 11: X'_{jl} += coef A_{i->j} X_{ik} B_{k->l}^T over all transition pairs."""
    off = sb.offsets()
    where = sb.pair_index()
    y = np.zeros(off[-1])

    def seg(v, p):
        i, k = sb.pairs[p]
        return v[off[p]:off[p + 1]].reshape(int(sb.dL[i]), int(sb.dR[k]))

    for coef, a, b in sb.terms:
        # an identity operator contributes its single diagonal block i -> i
        a_blocks = ({(i, i): None for i in range(len(sb.dL))} if a == IDENTITY
                    else sb.opsL[a].blocks)
        b_blocks = ({(k, k): None for k in range(len(sb.dR))} if b == IDENTITY
                    else sb.opsR[b].blocks)
        for (i, j), A in a_blocks.items():
            for (k, l), B in b_blocks.items():
                pin, pout = where.get((i, k)), where.get((j, l))
                if pin is None or pout is None:
                    continue
                X = seg(x, pin)
                T = X if A is None else A @ X          # (A X)
                U = T if B is None else T @ B.T        # (A X) B^T
                seg(y, pout)[...] += coef * U
    return y


def diagonal(sb: Superblock) -> np.ndarray:
    """diag(H_SB) in storage order: sum coef diag(A_{i->i}) (x) diag(B_{k->k})."""
    off = sb.offsets()
    D = np.zeros(off[-1])
    for coef, a, b in sb.terms:
        for p, (i, k) in enumerate(sb.pairs):
            if a == IDENTITY:
                da = np.ones(int(sb.dL[i]))
            else:
                blk = sb.opsL[a].blocks.get((i, i))
                if blk is None:
                    continue
                da = np.diag(blk)
            if b == IDENTITY:
                db = np.ones(int(sb.dR[k]))
            else:
                blk = sb.opsR[b].blocks.get((k, k))
                if blk is None:
                    continue
                db = np.diag(blk)
            D[off[p]:off[p + 1]] += coef * np.outer(da, db).ravel()
    return D


def flop_count(sb: Superblock) -> dict:
    """Algorithmic FLOPs of one projection by Eq. 11, cheaper multiplication order per
    record, identity factors skipped (a record with one identity is one GEMM)."""
    where = sb.pair_index()
    total = 0
    records = 0
    for coef, a, b in sb.terms:
        a_blocks = ({(i, i): None for i in range(len(sb.dL))} if a == IDENTITY
                    else sb.opsL[a].blocks)
        b_blocks = ({(k, k): None for k in range(len(sb.dR))} if b == IDENTITY
                    else sb.opsR[b].blocks)
        for (i, j) in a_blocks:
            for (k, l) in b_blocks:
                if (i, k) not in where or (j, l) not in where:
                    continue
                di, dj, dk, dl = (int(sb.dL[i]), int(sb.dL[j]), int(sb.dR[k]), int(sb.dR[l]))
                records += 1
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
