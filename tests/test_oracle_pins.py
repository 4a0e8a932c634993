"""Pins of the FP64 oracle against facts outside it (no GPU).

Each test ties one oracle function to a closed form, an exact diagonalisation built by
independent code, a textbook routine, an invariant of Sec. 3, or a known bulk energy.
The "planted mistake" tests at the end change one detail of the oracle on the CPU and
check that a pin catches it.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from dmrg_inputs import warmup
from dmrg_inputs.superblock import IDENTITY
from oracle import davidson as dav
from oracle import dmrg, ed, projection


# ---------------------------------------------------------------- closed forms (ED)
def test_heisenberg_closed_forms():
    # two spins: singlet energy -3/4; four spins, open chain: -3/4 - sqrt(3)/2
    assert ed.heisenberg_ground_energy(2) == pytest.approx(-0.75, abs=1e-13)
    assert ed.heisenberg_ground_energy(4) == pytest.approx(-0.75 - math.sqrt(3) / 2, abs=1e-13)


@pytest.mark.parametrize("U", [0.0, 1.0, 4.0, 8.0])
def test_hubbard_dimer_closed_form(U):
    # two sites at half filling, S_z = 0: E = (U - sqrt(U^2 + 16 t^2)) / 2
    assert ed.hubbard_ground_energy(2, 1, 1, t=1.0, U=U) == pytest.approx(
        (U - math.sqrt(U * U + 16.0)) / 2, abs=1e-13)


def test_xx_chain_free_fermions():
    # Delta = 0: Jordan-Wigner gives hopping 1/2, energies cos(k pi/(L+1)); S_z = 0 fills
    # the L/2 negative ones
    L = 8
    exact = -sum(math.cos(k * math.pi / (L + 1)) for k in range(1, L // 2 + 1))
    assert ed.heisenberg_ground_energy(L, delta=0.0) == pytest.approx(exact, abs=1e-12)


@pytest.mark.parametrize("L,nu,nd", [(4, 2, 2), (4, 1, 2), (5, 2, 1)])
def test_hubbard_u0_free_fermions(L, nu, nd):
    eps = sorted(-2.0 * math.cos(k * math.pi / (L + 1)) for k in range(1, L + 1))
    exact = sum(eps[:nu]) + sum(eps[:nd])
    assert ed.hubbard_ground_energy(L, nu, nd, t=1.0, U=0.0) == pytest.approx(exact, abs=1e-12)


# ---------------------------------------------------------------- DMRG vs ED
@pytest.mark.parametrize("L", [4, 6, 8])
def test_dmrg_untruncated_equals_ed_heisenberg(L):
    r = dmrg.infinite_dmrg("heisenberg", L, m=10 ** 6)
    assert r["energies"][L] == pytest.approx(ed.heisenberg_ground_energy(L), abs=1e-10)


@pytest.mark.parametrize("L,U", [(4, 4.0), (6, 4.0), (6, 0.0)])
def test_dmrg_untruncated_equals_ed_hubbard(L, U):
    r = dmrg.infinite_dmrg("hubbard", L, m=10 ** 6, U=U)
    assert r["energies"][L] == pytest.approx(
        ed.hubbard_ground_energy(L, L // 2, L // 2, U=U), abs=1e-10)


def test_dmrg_quarter_filling_equals_ed():
    r = dmrg.infinite_dmrg("hubbard", 8, m=10 ** 6, U=8.0, filling=0.5)
    assert r["superblock"].Q == (2, 2)
    assert r["energies"][8] == pytest.approx(ed.hubbard_ground_energy(8, 2, 2, U=8.0), abs=1e-10)


# ---------------------------------------------------------------- bulk energies
def test_bethe_ansatz_bulk_energy():
    # XXX chain: e_inf = 1/4 - ln 2 (Hulthen); the open-chain surface term cancels in
    # (E_L - E_{L-2}) / 2
    r = dmrg.infinite_dmrg("heisenberg", 100, m=64)
    E = r["energies"]
    assert (E[100] - E[98]) / 2 == pytest.approx(0.25 - math.log(2.0), abs=2e-4)


def lieb_wu_energy_per_site(U, t=1.0):
    f = lambda w: special.j0(w) * special.j1(w) / (w * (1.0 + math.exp(w * U / (2 * t))))
    val, _ = integrate.quad(f, 0.0, 60.0, limit=400)
    return -4.0 * t * val


def test_lieb_wu_bulk_energy():
    # quadrature of the Lieb-Wu integral at U = 4; the value is -0.57373 per site
    e_lw = lieb_wu_energy_per_site(4.0)
    assert e_lw == pytest.approx(-0.5737293679, abs=1e-8)
    r = dmrg.infinite_dmrg("hubbard", 40, m=96, U=4.0)
    E = r["energies"]
    assert (E[40] - E[38]) / 2 == pytest.approx(e_lw, abs=1e-3)


def test_dmrg_u0_truncated_free_fermions():
    L = 16
    eps = sorted(-2.0 * math.cos(k * math.pi / (L + 1)) for k in range(1, L + 1))
    exact = 2 * sum(eps[:L // 2])
    r = dmrg.infinite_dmrg("hubbard", L, m=64, U=0.0)
    assert r["energies"][L] == pytest.approx(exact, rel=1e-4)
    assert r["energies"][L] >= exact - 1e-10      # variational


# ---------------------------------------------------------------- projection
def _problems():
    out = []
    out.append(dmrg.infinite_dmrg("heisenberg", 8, m=10 ** 6)["superblock"])
    out.append(dmrg.infinite_dmrg("hubbard", 6, m=10 ** 6, U=4.0)["superblock"])
    out.append(warmup.warmup_superblock("heisenberg", 12, m=24))
    out.append(warmup.warmup_superblock("hubbard", 8, m=40, U=4.0))
    out.append(warmup.warmup_superblock("hubbard", 8, m=40, U=8.0, filling=0.5))
    return out


PROBLEMS = _problems()


@pytest.mark.parametrize("p", range(len(PROBLEMS)))
def test_decomposed_projection_equals_kron_definition(p):
    sb = PROBLEMS[p]
    rng = np.random.default_rng(p)
    x = rng.standard_normal(sb.n)
    y_def = projection.project_dense(sb, x)
    y_dec = projection.project_blocks(sb, x)
    assert np.linalg.norm(y_dec - y_def) <= 1e-14 * np.linalg.norm(y_def) * 10


@pytest.mark.parametrize("p", range(len(PROBLEMS)))
def test_hermiticity_and_closure(p):
    sb = PROBLEMS[p]
    rng = np.random.default_rng(100 + p)
    x, y = rng.standard_normal(sb.n), rng.standard_normal(sb.n)
    Hx, Hy = projection.project_blocks(sb, x), projection.project_blocks(sb, y)
    H = projection.superblock_dense(sb)
    scale = np.linalg.norm(H, 2) * np.linalg.norm(x) * np.linalg.norm(y)
    assert abs(x @ Hy - Hx @ y) <= 1e-12 * scale
    assert projection.leak_outside_sector(sb, x) <= 1e-13 * np.linalg.norm(Hx)
    np.testing.assert_allclose(projection.diagonal(sb), np.diag(H), atol=1e-14)


def test_flop_count_small_case():
    # one left and one right sector of size 3 and 2, terms H_L (x) 1, 1 (x) H_R and
    # A (x) B: records 2*3*3*2 (A X) + 2*3*2*2 (X B^T) + min(2*3*3*2 + 2*3*2*2, same) = 36+24+60
    from dmrg_inputs.superblock import BlockOp, Superblock
    rng = np.random.default_rng(0)
    A = BlockOp({(0, 0): rng.standard_normal((3, 3))})
    B = BlockOp({(0, 0): rng.standard_normal((2, 2))})
    sb = Superblock(qL=[(0,)], dL=np.array([3]), qR=[(0,)], dR=np.array([2]), Q=(0,),
                    pairs=[(0, 0)], opsL=[A], opsR=[B],
                    terms=[(1.0, 0, IDENTITY), (1.0, IDENTITY, 0), (0.5, 0, 0)])
    assert projection.flop_count(sb) == {"flops": 36 + 24 + 60, "records": 3}


# ---------------------------------------------------------------- Davidson
@pytest.mark.parametrize("keep", [1, 2])
@pytest.mark.parametrize("max_subspace", [20, 4])
def test_davidson_equals_eigh(max_subspace, keep):
    # both restart readings (Ritz vector alone, or with the previous Ritz vector) reach
    # LAPACK's lowest eigenpair; the problem needs several subspace-limit restarts
    sb = PROBLEMS[3]
    H = projection.superblock_dense(sb)
    w, v = np.linalg.eigh(H)
    x0 = warmup.start_vector(sb.n, seed=0)
    lam, x, info = dav.davidson(lambda z: H @ z, np.diag(H).copy(), x0, tol=1e-10,
                                max_subspace=max_subspace, restart_keep=keep)
    assert info["converged"] and info["restarts"] >= 2
    assert lam == pytest.approx(w[0], abs=1e-10)
    assert abs(x @ v[:, 0]) >= 1 - 1e-10
    assert np.linalg.norm(H @ x - lam * x) <= 1e-10 * 1.0001


def _random_operator(n=400, seed=1):
    # diagonally dominated symmetric matrix: the diagonal preconditioner helps, but the
    # iteration still needs several restarts at both subspace limits
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return np.diag(np.linspace(0.0, 20.0, n)) + 0.25 * (A + A.T)


class _RestartLog:
    """Collects, at every restart, how far the collapsed basis is from the invariants that
    hold in exact arithmetic: V^T V = I, W = H V, B = V^T H V, and (keeping two vectors)
    the previous Ritz vector lies in span(V)."""

    def __init__(self, H):
        self.H = H
        self.orth, self.w, self.b, self.prev, self.k = [], [], [], [], []

    def __call__(self, V, W, B, x_prev):
        H = self.H
        k = V.shape[1]
        self.k.append(k)
        self.orth.append(np.linalg.norm(V.T @ V - np.eye(k)))
        self.w.append(np.linalg.norm(W - H @ V) / np.linalg.norm(H, 2))
        self.b.append(np.linalg.norm(B - V.T @ H @ V) / np.linalg.norm(H, 2))
        if x_prev is not None and k == 2:
            self.prev.append(np.linalg.norm(x_prev - V @ (V.T @ x_prev)) / np.linalg.norm(x_prev))


@pytest.mark.parametrize("max_subspace", [4, 20])
@pytest.mark.parametrize("keep", [1, 2])
def test_davidson_restart_invariants(keep, max_subspace):
    H = _random_operator()
    w, v = np.linalg.eigh(H)
    log = _RestartLog(H)
    lam, x, info = dav.davidson(lambda z: H @ z, np.diag(H).copy(), warmup.start_vector(H.shape[0], 0),
                                tol=1e-10, max_subspace=max_subspace, restart_keep=keep,
                                on_restart=log)
    assert info["converged"] and info["restarts"] >= 3 and len(log.k) == info["restarts"]
    assert lam == pytest.approx(w[0], abs=1e-10)
    assert abs(x @ v[:, 0]) >= 1 - 1e-10
    assert max(log.orth) <= 1e-12
    assert max(log.w) <= 1e-12 and max(log.b) <= 1e-12
    if keep == 2:
        # two vectors kept at the restarts (one only where the previous Ritz vector has
        # become parallel to the current one, close to convergence), and the previous Ritz
        # vector lies in the span of the kept pair
        assert log.k.count(2) >= 3 and log.k[0] == 2
        assert max(log.prev) <= 1e-10
    else:
        assert set(log.k) == {1}


def test_planted_restart_w_not_recombined_is_caught(monkeypatch):
    # W kept as its first columns instead of W C: W = H V breaks after the first restart
    H = _random_operator()
    orig = dav.collapse

    def bad(V, W, B, C):
        Vn, _, Bn = orig(V, W, B, C)
        return Vn, W[:, :C.shape[1]].copy(), Bn

    monkeypatch.setattr(dav, "collapse", bad)
    log = _RestartLog(H)
    dav.davidson(lambda z: H @ z, np.diag(H).copy(), warmup.start_vector(H.shape[0], 0),
                 tol=1e-10, max_subspace=4, restart_keep=2, max_iter=60, on_restart=log)
    assert max(log.w) > 1e-3


def test_planted_restart_b_not_transformed_is_caught(monkeypatch):
    H = _random_operator()
    orig = dav.collapse

    def bad(V, W, B, C):
        Vn, Wn, _ = orig(V, W, B, C)
        m = C.shape[1]
        return Vn, Wn, B[:m, :m].copy()

    monkeypatch.setattr(dav, "collapse", bad)
    log = _RestartLog(H)
    dav.davidson(lambda z: H @ z, np.diag(H).copy(), warmup.start_vector(H.shape[0], 0),
                 tol=1e-10, max_subspace=4, restart_keep=2, max_iter=60, on_restart=log)
    assert max(log.b) > 1e-3


def test_planted_restart_previous_vector_misaligned_is_caught(monkeypatch):
    # the previous Ritz coefficients padded at the front instead of for the newest column:
    # the kept second vector is then not the previous Ritz vector
    H = _random_operator()

    def bad(y, y_prev, keep):
        k = y.shape[0]
        C = y[:, None]
        if keep == 2 and y_prev is not None:
            c2 = np.zeros(k)
            c2[k - len(y_prev):] = y_prev
            c2 -= y * (y @ c2)
            c2 -= y * (y @ c2)
            if np.linalg.norm(c2) > 1e-8:
                C = np.column_stack([y, c2 / np.linalg.norm(c2)])
        return C

    monkeypatch.setattr(dav, "restart_coefficients", bad)
    log = _RestartLog(H)
    dav.davidson(lambda z: H @ z, np.diag(H).copy(), warmup.start_vector(H.shape[0], 0),
                 tol=1e-10, max_subspace=4, restart_keep=2, max_iter=60, on_restart=log)
    assert max(log.prev) > 1e-3


def test_davidson_reports_nonconvergence():
    sb = PROBLEMS[3]
    H = projection.superblock_dense(sb)
    lam, x, info = dav.davidson(lambda z: H @ z, np.diag(H).copy(),
                                warmup.start_vector(sb.n, 1), tol=1e-14, max_iter=3)
    assert not info["converged"] and info["iters"] == 3


def test_correction_guard():
    r = np.array([1.0, 1.0, 1.0])
    D = np.array([0.5, 1.0, 2.0])
    t = dav.correct(r, 1.0, D)
    np.testing.assert_allclose(t, [2.0, 1e8, -1.0])


# ---------------------------------------------------------------- planted mistakes
def test_planted_wrong_fermion_string_is_caught(monkeypatch):
    # dropping the block parity from the hop across the superblock changes the energy
    orig = dmrg._parity

    def no_string(block):
        return np.eye(block.dim)

    monkeypatch.setattr(dmrg, "_parity", no_string)
    e_bad = dmrg.infinite_dmrg("hubbard", 6, m=10 ** 6, U=4.0)["energies"][6]
    monkeypatch.setattr(dmrg, "_parity", orig)
    assert abs(e_bad - ed.hubbard_ground_energy(6, 3, 3, U=4.0)) > 1e-3


def test_planted_column_major_segments_are_caught(monkeypatch):
    # Eq. 10 reshapes X; reading the segments column-major instead of row-major (the
    # ambiguity of the sizes printed after Eq. 10) must break agreement with Eq. 9
    sb = PROBLEMS[3]
    x = np.random.default_rng(5).standard_normal(sb.n)
    y_def = projection.project_dense(sb, x)
    off = sb.offsets()
    perm = np.concatenate([
        np.arange(off[p], off[p + 1]).reshape(int(sb.dR[k]), int(sb.dL[i])).T.ravel()
        for p, (i, k) in enumerate(sb.pairs)])
    y_bad = projection.project_blocks(sb, x[perm])[np.argsort(perm)]
    assert np.linalg.norm(y_bad - y_def) > 1e-6 * np.linalg.norm(y_def)


def test_planted_dropped_term_is_caught():
    sb = PROBLEMS[1]
    x = np.random.default_rng(6).standard_normal(sb.n)
    y_def = projection.project_dense(sb, x)
    saved = sb.terms
    sb.terms = saved[:-1]
    try:
        y_bad = projection.project_blocks(sb, x)
    finally:
        sb.terms = saved
    assert np.linalg.norm(y_bad - y_def) > 1e-6 * np.linalg.norm(y_def)
