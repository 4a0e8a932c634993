"""Site operators and full-chain Hamiltonians of Sec. 2 (oracle; test infrastructure).

Heisenberg (Sec. 2.1): basis (up, down); S+ = [[0,1],[0,0]], S- = [[0,0],[1,0]],
S^z = diag(1,-1)/2 (Eq. 3).  A one-site operator O on site j of an N-site chain is the
Kronecker product of identities with O in position j (Eq. 2).  The Hamiltonian is
H = 1/2 sum_j (S+_j S-_{j+1} + S-_j S+_{j+1}) + Delta sum_j S^z_j S^z_{j+1} (Eq. 1),
multiplied here by an overall exchange constant J (J = 1 reproduces Eq. 1).

Hubbard, spin 1/2 (Sec. 2.2): every site carries one two-state mode per spin
polarisation, ordered from sigma = -F to +F, i.e. down before up (Eq. 6).  A mode has
basis (empty, occupied) with c^dagger = [[0,0],[1,0]], c = [[0,1],[0,0]] (Eq. 8), and the
fermionic phase Phi = diag(1,-1) (Eq. 7) is applied to every mode that precedes the
acted-on mode in the global order (Eqs. 5, 6).  The Hamiltonian is
H = -t sum_{j,sigma} (c^dagger_{j,sigma} c_{j+1,sigma} + h.c.)
    + U/2 sum_j sum_{sigma != sigma'} n_{j,sigma} n_{j,sigma'}          (Eq. 4)
which for F = 1/2 equals U sum_j n_{j,up} n_{j,down}.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Eq. 3
S_PLUS = np.array([[0.0, 1.0], [0.0, 0.0]])
S_MINUS = np.array([[0.0, 0.0], [1.0, 0.0]])
S_Z = 0.5 * np.array([[1.0, 0.0], [0.0, -1.0]])
# Eq. 7 and Eq. 8
PHI = np.array([[1.0, 0.0], [0.0, -1.0]])
C_DAG = np.array([[0.0, 0.0], [1.0, 0.0]])
C_ANN = np.array([[0.0, 1.0], [0.0, 0.0]])
EYE2 = np.eye(2)


def _kron_all(factors):
    out = sp.identity(1, format="csr", dtype=np.float64)
    for f in factors:
        out = sp.kron(out, sp.csr_matrix(f), format="csr")
    return out


def chain_op(O: np.ndarray, j: int, N: int) -> sp.csr_matrix:
    """Eq. 2: identity on sites 1..j-1, O on site j, identity on j+1..N (j is 1-based)."""
    return _kron_all([EYE2] * (j - 1) + [O] + [EYE2] * (N - j))


def heisenberg_chain(N: int, delta: float = 1.0, J: float = 1.0) -> sp.csr_matrix:
    """Eq. 1 for an open chain of N spins, times the exchange constant J."""
    dim = 2 ** N
    H = sp.csr_matrix((dim, dim))
    for j in range(1, N):
        H = H + 0.5 * J * (chain_op(S_PLUS, j, N) @ chain_op(S_MINUS, j + 1, N)
                           + chain_op(S_MINUS, j, N) @ chain_op(S_PLUS, j + 1, N))
        H = H + J * delta * (chain_op(S_Z, j, N) @ chain_op(S_Z, j + 1, N))
    return H.tocsr()


def heisenberg_sz2(N: int) -> np.ndarray:
    """Diagonal of 2*S^z_total in the product basis (site 1 is the slowest index)."""
    diag = np.zeros(2 ** N, dtype=np.int64)
    for j in range(1, N + 1):
        diag += np.rint(2 * chain_op(S_Z, j, N).diagonal()).astype(np.int64)
    return diag


# ---- Hubbard: modes are (site j, sigma) with sigma index 0 = down, 1 = up (Eq. 6) ----

def fermion_mode_op(O: np.ndarray, j: int, sigma: int, N: int) -> sp.csr_matrix:
    """Eqs. 5-6: Phi on every mode before (j, sigma), O on it, identity after it.

    Modes are ordered site by site (j = 1..N) and, inside a site, down (sigma=0)
    before up (sigma=1)."""
    pos = 2 * (j - 1) + sigma
    nmodes = 2 * N
    return _kron_all([PHI] * pos + [O] + [EYE2] * (nmodes - pos - 1))


def hubbard_chain(N: int, t: float = 1.0, U: float = 4.0) -> sp.csr_matrix:
    """Eq. 4 for F = 1/2 on an open chain of N sites."""
    dim = 4 ** N
    H = sp.csr_matrix((dim, dim))
    for j in range(1, N):
        for s in (0, 1):
            hop = fermion_mode_op(C_DAG, j, s, N) @ fermion_mode_op(C_ANN, j + 1, s, N)
            H = H - t * (hop + hop.T)
    for j in range(1, N + 1):
        n_dn = fermion_mode_op(C_DAG, j, 0, N) @ fermion_mode_op(C_ANN, j, 0, N)
        n_up = fermion_mode_op(C_DAG, j, 1, N) @ fermion_mode_op(C_ANN, j, 1, N)
        # (U/2) sum_{sigma != sigma'} n n = (U/2)(n_dn n_up + n_up n_dn)
        H = H + 0.5 * U * (n_dn @ n_up + n_up @ n_dn)
    return H.tocsr()


def hubbard_numbers(N: int):
    """Diagonals of N_up and N_down (the conserved numbers of Sec. 3)."""
    nup = np.zeros(4 ** N, dtype=np.int64)
    ndn = np.zeros(4 ** N, dtype=np.int64)
    for j in range(1, N + 1):
        ndn += np.rint((fermion_mode_op(C_DAG, j, 0, N) @ fermion_mode_op(C_ANN, j, 0, N))
                       .diagonal()).astype(np.int64)
        nup += np.rint((fermion_mode_op(C_DAG, j, 1, N) @ fermion_mode_op(C_ANN, j, 1, N))
                       .diagonal()).astype(np.int64)
    return nup, ndn
