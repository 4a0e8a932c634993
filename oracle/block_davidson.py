"""Block Davidson-Liu iteration for the lowest few eigenpairs (oracle; test infrastructure).

Sec. 6 remarks that the block extension of the Davidson method (Liu), which targets a
few of the lowest eigenvalues, adds several candidate vectors to the basis at once, so
that the vector work becomes matrix-matrix (BLAS-3) instead of matrix-vector; the paper's
own implementation computes only the lowest pair (Algorithm 3).  This restates that
extension in the terms of Algorithm 3, with a block of b >= nev vectors:

  W(:, new) = H V(:, new)                  projection of the columns added last (Eq. 11)
  B = V^T W                                (symmetric; the new columns and rows)
  (theta_i, y_i), i < b                    the b lowest eigenpairs of B
  X = V Y,  R = W Y - X diag(theta)        Ritz vectors and residuals
  stop if ||r_i|| <= tol for every i < nev
  t_i = r_i / (theta_i - D)                for every i < b with ||r_i|| > tol
  orthonormalise the t_i against V and each other; append them.

Readings where the paper is silent (beyond those of the single-vector oracle, which this
one follows: the diagonal correction with its 1e-8 guard, classical Gram-Schmidt twice,
||r||_2 <= tol on normalised vectors):

* block size b is an input (the number of start vectors), b >= nev; corrections are made
  for the unconverged ones among the b lowest Ritz pairs, in ascending order of theta;
* a correction whose norm after orthogonalisation falls below 1e-10 of its norm before is
  replaced by its raw residual, and dropped if that also collapses; if every correction of
  an iteration is dropped the iteration reports a breakdown;
* subspace limit max_subspace (24 here: 20 in Sec. 6.1 plus a block of 4): when the new
  corrections do not fit, the basis is first collapsed to the b current Ritz vectors and
  (restart_keep = 2, the default) as many of the previous iteration's b Ritz vectors as
  leave room for the corrections, orthonormalised against the current ones in coefficient
  space; W and B are replaced by the same combinations (the block form of the
  single-vector oracle's two-vector restart; keeping the current block alone stagnates
  when the limit is a small multiple of b);
* the start block is orthonormalised column by column (classical Gram-Schmidt twice).

With b = nev = 1 every step is the single-vector iteration of ``oracle.davidson`` with
the same restart_keep.
"""
from __future__ import annotations

import numpy as np

from .davidson import BREAKDOWN, correct


def _orth_against(Q: np.ndarray, t: np.ndarray) -> np.ndarray:
    for _ in range(2):
        t = t - Q @ (Q.T @ t)
    return t


def restart_block_coefficients(Y: np.ndarray, Y_prev, keep_prev: int) -> np.ndarray:
    """Columns C of the collapsed basis V C in the current basis (k rows): the b Ritz
    coefficient vectors Y, then up to keep_prev of the previous iteration's Ritz
    coefficients Y_prev (one or more rows shorter: padded with zeros for the columns added
    since), each orthogonalised (twice) against the columns already in C and normalised,
    and dropped if less than 1e-8 of it is left."""
    k = Y.shape[0]
    C = [Y[:, i] for i in range(Y.shape[1])]
    if Y_prev is not None:
        for i in range(min(keep_prev, Y_prev.shape[1])):
            c = np.zeros(k)
            c[:Y_prev.shape[0]] = Y_prev[:, i]
            for _ in range(2):
                for q in C:
                    c -= q * (q @ c)
            nc = np.linalg.norm(c)
            if nc > 1e-8:
                C.append(c / nc)
    return np.column_stack(C)


def collapse_block(V: np.ndarray, W: np.ndarray, B: np.ndarray, C: np.ndarray):
    """The collapsed basis V C, its projections W C = H V C and C^T B C."""
    return V @ C, W @ C, C.T @ B @ C


def block_davidson(matvec, D: np.ndarray, X0: np.ndarray, nev: int, tol: float = 1e-10,
                   max_iter: int = 1000, max_subspace: int = 24, restart_keep: int = 2):
    """Lowest ``nev`` eigenpairs of the symmetric operator ``matvec`` from the start block
    X0 (n x b, b >= nev).  Returns (theta[:nev], X[:, :nev], info)."""
    n, b = X0.shape
    if not (1 <= nev <= b and 2 * b <= max_subspace):
        raise ValueError("need 1 <= nev <= b and 2 b <= max_subspace")
    V = np.zeros((n, max_subspace))
    W = np.zeros((n, max_subspace))
    B = np.zeros((max_subspace, max_subspace))
    k = 0
    for j in range(b):
        t = _orth_against(V[:, :k], X0[:, j].astype(np.float64))
        nt = np.linalg.norm(t)
        if nt < BREAKDOWN * np.linalg.norm(X0[:, j]):
            raise ValueError("start block is rank deficient")
        V[:, k] = t / nt
        k += 1
    done = 0            # columns whose projection is in W
    history = []
    restarts = 0
    projections = 0
    theta = np.full(b, np.nan)
    Y_prev = None
    X = V[:, :b].copy()
    rn = np.full(b, np.inf)
    for it in range(1, max_iter + 1):
        for j in range(done, k):
            W[:, j] = matvec(V[:, j])
            projections += 1
        C = V[:, :k].T @ W[:, done:k]
        B[:k, done:k] = C
        B[done:k, :k] = C.T
        done = k
        evals, evecs = np.linalg.eigh(B[:k, :k])
        theta, Y = evals[:b], evecs[:, :b]
        X = V[:, :k] @ Y
        R = W[:, :k] @ Y - X * theta
        rn = np.linalg.norm(R, axis=0)
        history.append((theta.copy(), rn.copy()))
        if np.all(rn[:nev] <= tol):
            return theta[:nev], X[:, :nev], {"iters": it, "resnorm": rn[:nev], "converged": True,
                                             "history": history, "restarts": restarts,
                                             "projections": projections}
        idx = [i for i in range(b) if rn[i] > tol]
        T = [correct(R[:, i], theta[i], D) for i in idx]
        if k + len(T) > max_subspace:      # collapse to the Ritz block (and the previous one)
            keep_prev = (max_subspace - b - len(T)) if restart_keep == 2 else 0
            C = restart_block_coefficients(Y, Y_prev, keep_prev)
            Vn, Wn, Bn = collapse_block(V[:, :k], W[:, :k], B[:k, :k], C)
            k = done = C.shape[1]
            V[:, :k], W[:, :k] = Vn, Wn
            B[:, :] = 0.0
            B[:k, :k] = Bn
            Y = C.T @ Y            # the Ritz block in the new basis: the first b unit vectors
            restarts += 1
        Y_prev = Y
        added = 0
        for i, t in zip(idx, T):
            before = np.linalg.norm(t)
            t_o = _orth_against(V[:, :k], t)
            if np.linalg.norm(t_o) < BREAKDOWN * before:
                before = np.linalg.norm(R[:, i])
                t_o = _orth_against(V[:, :k], R[:, i])
                if np.linalg.norm(t_o) < BREAKDOWN * before:
                    continue
            V[:, k] = t_o / np.linalg.norm(t_o)
            k += 1
            added += 1
        if added == 0:
            return theta[:nev], X[:, :nev], {"iters": it, "resnorm": rn[:nev], "converged": False,
                                             "history": history, "breakdown": True,
                                             "restarts": restarts, "projections": projections}
    return theta[:nev], X[:, :nev], {"iters": max_iter, "resnorm": rn[:nev], "converged": False,
                                     "history": history, "restarts": restarts,
                                     "projections": projections}
