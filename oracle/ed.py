"""Exact diagonalisation inside one symmetry sector (oracle; test infrastructure).

Sec. 3: the Hamiltonian commutes with S^z_total (Heisenberg) and with N_up, N_down
(Hubbard), so it is block diagonal in their eigenvalues.  The lowest eigenvalue inside a
sector is found by restricting the full-chain matrix of Eqs. 1/4 to the basis states of
that sector and calling a dense symmetric eigensolver.
"""
from __future__ import annotations

import numpy as np

from . import sites


def lowest_in_sector(H, mask: np.ndarray, nev: int = 1):
    idx = np.nonzero(mask)[0]
    Hs = H[idx][:, idx].toarray()
    w, v = np.linalg.eigh(Hs)
    return w[:nev], v[:, :nev], idx


def heisenberg_ground_energy(N: int, sz2: int = 0, delta: float = 1.0, J: float = 1.0) -> float:
    H = sites.heisenberg_chain(N, delta=delta, J=J)
    w, _, _ = lowest_in_sector(H, sites.heisenberg_sz2(N) == sz2)
    return float(w[0])


def hubbard_ground_energy(N: int, n_up: int, n_dn: int, t: float = 1.0, U: float = 4.0) -> float:
    H = sites.hubbard_chain(N, t=t, U=U)
    nu, nd = sites.hubbard_numbers(N)
    w, _, _ = lowest_in_sector(H, (nu == n_up) & (nd == n_dn))
    return float(w[0])
