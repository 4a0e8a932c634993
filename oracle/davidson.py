"""The Davidson iteration of Algorithm 3 (oracle; test infrastructure).

One iteration, for a basis V of k orthonormal columns whose newest column has not yet
been projected (Algorithm 3, Sec. 5):

  W(:,k) = H V(:,k)                  projection (Eq. 11)
  B(:,k) = V^T W(:,k)                "asymmetric" matrix-vector product; B is symmetric,
                                     so the same numbers fill row k
  (lambda, y) = smallest eigenpair of B
  x = V y,  r = W y - lambda x
  stop if ||r|| <= tol
  correct r; orthonormalise it against V; append it to V.

Readings where the paper is silent (Sec. 6 names the Sadkane-Sidje variant only):

* correction: diagonal (Davidson) preconditioner t_e = r_e / (lambda - D_e) with
  D = diag(H_SB); where |lambda - D_e| < 1e-8 the denominator is replaced by
  +-1e-8 with the sign of lambda - D_e (plus when it is zero);
* orthogonalisation: classical Gram-Schmidt applied twice; if the norm left after it is
  below 1e-10 of the norm before, the raw residual r is used instead, and if that also
  collapses the iteration reports a breakdown;
* subspace limit: 20 columns (Sec. 6.1); when the basis is full it is collapsed, before
  the new direction is added, to the current Ritz vector x alone (restart_keep=1) or to x
  and the previous iteration's Ritz vector orthonormalised against it (restart_keep=2, the
  default, which is also the default of the CUDA library), with W and B replaced by the
  same combinations of their columns;
* convergence: ||r||_2 <= tol on a normalised x; at most ``max_iter`` iterations.
"""
from __future__ import annotations

import numpy as np

DENOM_GUARD = 1e-8
BREAKDOWN = 1e-10


def correct(r: np.ndarray, lam: float, D: np.ndarray) -> np.ndarray:
    den = lam - D
    small = np.abs(den) < DENOM_GUARD
    den = np.where(small, np.where(den >= 0.0, DENOM_GUARD, -DENOM_GUARD), den)
    return r / den


def _cgs2(V: np.ndarray, t: np.ndarray) -> np.ndarray:
    for _ in range(2):
        t = t - V @ (V.T @ t)
    return t


def restart_coefficients(y: np.ndarray, y_prev, keep: int) -> np.ndarray:
    """Columns C (k x 1 or k x 2) of the collapsed basis V C in the current basis.

    Column 0 is the Ritz vector's coefficient vector y.  With keep == 2, column 1 is the
    previous iteration's Ritz vector: its coefficients y_prev refer to the basis as it was
    one column shorter, so they are padded with a zero for the newest column, then
    orthogonalised against y (twice) and normalised; it is dropped if nothing is left."""
    k = y.shape[0]
    C = y[:, None]
    if keep == 2 and y_prev is not None:
        c2 = np.zeros(k)
        c2[:len(y_prev)] = y_prev
        c2 -= y * (y @ c2)
        c2 -= y * (y @ c2)
        if np.linalg.norm(c2) > 1e-8:
            C = np.column_stack([y, c2 / np.linalg.norm(c2)])
    return C


def collapse(V: np.ndarray, W: np.ndarray, B: np.ndarray, C: np.ndarray):
    """The collapsed basis V C, its projections W C = H V C and C^T B C (all in exact
    arithmetic consequences of W = H V and B = V^T H V)."""
    return V @ C, W @ C, C.T @ B @ C


def davidson(matvec, D: np.ndarray, x0: np.ndarray, tol: float = 1e-10,
             max_iter: int = 1000, max_subspace: int = 20, restart_keep: int = 2,
             on_restart=None):
    """Lowest eigenpair of the symmetric operator ``matvec``; returns (lam, x, info).

    ``on_restart(V, W, B, x_prev)``, if given, is called after every collapse of the basis
    with the new basis, its projections and small matrix (k = 1 or 2 columns) and the
    previous iteration's Ritz vector (None at the first iteration); tests use it to check
    the invariants of a restart."""
    n = x0.shape[0]
    V = np.zeros((n, max_subspace))
    W = np.zeros((n, max_subspace))
    B = np.zeros((max_subspace, max_subspace))
    V[:, 0] = x0 / np.linalg.norm(x0)
    k = 1
    history = []
    restarts = 0
    lam, x, rn = np.nan, V[:, 0].copy(), np.inf
    y_prev = None
    x_prev = None
    for it in range(1, max_iter + 1):
        W[:, k - 1] = matvec(V[:, k - 1])
        col = V[:, :k].T @ W[:, k - 1]
        B[:k, k - 1] = col
        B[k - 1, :k] = col
        evals, evecs = np.linalg.eigh(B[:k, :k])
        lam, y = float(evals[0]), evecs[:, 0]
        x = V[:, :k] @ y
        wy = W[:, :k] @ y
        r = wy - lam * x
        rn = float(np.linalg.norm(r))
        history.append((lam, rn))
        if rn <= tol:
            return lam, x, {"iters": it, "resnorm": rn, "converged": True, "history": history,
                            "restarts": restarts}
        t = correct(r, lam, D)
        if k == max_subspace:          # restart with the Ritz vector (and the previous one)
            C = restart_coefficients(y, y_prev, restart_keep)
            Vn, Wn, Bn = collapse(V[:, :k], W[:, :k], B[:k, :k], C)
            k = C.shape[1]
            V[:, :k], W[:, :k] = Vn, Wn
            B[:, :] = 0.0
            B[:k, :k] = Bn
            y = C.T @ y            # the Ritz vector in the new basis: e_1
            restarts += 1
            if on_restart is not None:
                on_restart(V[:, :k].copy(), W[:, :k].copy(), B[:k, :k].copy(),
                           None if x_prev is None else x_prev.copy())
        y_prev = y
        x_prev = x
        before = np.linalg.norm(t)
        t_o = _cgs2(V[:, :k], t)
        if np.linalg.norm(t_o) < BREAKDOWN * before:
            before = np.linalg.norm(r)
            t_o = _cgs2(V[:, :k], r)
            if np.linalg.norm(t_o) < BREAKDOWN * before:
                return lam, x, {"iters": it, "resnorm": rn, "converged": False,
                                "history": history, "breakdown": True, "restarts": restarts}
        V[:, k] = t_o / np.linalg.norm(t_o)
        k += 1
    return lam, x, {"iters": max_iter, "resnorm": rn, "converged": False, "history": history,
                    "restarts": restarts}
