"""Pins of the l-1-1-r oracle (Sec. 4.2, Eqs. 12-13, Algorithm 2) against facts outside
it (no GPU): the Kronecker definition, the LR form of the same superblock (same blocks,
same Hamiltonian, another basis: the spectra must agree), exact diagonalisation and the
closed forms of small chains, Hermiticity, and planted mistakes."""
import math

import numpy as np
import pytest

from dmrg_inputs import warmup
from oracle import davidson as dav
from oracle import ed, l11r
from oracle import projection as lr


def _problems():
    return {
        "heis_L6_exact": dict(model="heisenberg", L=6, m=1000),
        "heis_L12_m24": dict(model="heisenberg", L=12, m=24),
        "hub_L6_exact": dict(model="hubbard", L=6, m=1000, U=4.0),
        "hub_L8_m40": dict(model="hubbard", L=8, m=40, U=4.0),
        "hub_quarter_L8_m32": dict(model="hubbard", L=8, m=32, U=8.0, filling=0.5),
    }


PROBLEMS = _problems()
_cache = {}


def pair(name):
    if name not in _cache:
        kw = PROBLEMS[name]
        _cache[name] = (warmup.warmup_superblock_l11r(**kw), warmup.warmup_superblock(**kw))
    return _cache[name]


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_algorithm2_equals_kron_definition(name):
    sb, _ = pair(name)
    x = np.random.default_rng(1).standard_normal(sb.n)
    y_def = l11r.project_dense(sb, x)
    y_alg = l11r.project_blocks(sb, x)
    assert np.linalg.norm(y_alg - y_def) <= 1e-13 * np.linalg.norm(y_def)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_same_spectrum_as_the_lr_form(name):
    # the l-1-1-r and LR superblocks built from the same blocks l and r are one
    # Hamiltonian in two orderings of one basis
    sb, sb_lr = pair(name)
    assert sb.n == sb_lr.n
    w1 = np.linalg.eigvalsh(l11r.superblock_dense(sb))
    w2 = np.linalg.eigvalsh(lr.superblock_dense(sb_lr))
    np.testing.assert_allclose(w1, w2, atol=1e-10)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_hermitian_and_diagonal(name):
    sb, _ = pair(name)
    H = l11r.superblock_dense(sb)
    assert np.max(np.abs(H - H.T)) <= 1e-13 * np.max(np.abs(H))
    np.testing.assert_allclose(l11r.diagonal(sb), np.diag(H), atol=1e-14)


def test_exact_ground_energies():
    # untruncated blocks: the lowest eigenvalue is the chain's, from exact diagonalisation
    for name, exact in (("heis_L6_exact", ed.heisenberg_ground_energy(6)),
                        ("hub_L6_exact", ed.hubbard_ground_energy(6, 3, 3, U=4.0))):
        sb, _ = pair(name)
        assert np.linalg.eigvalsh(l11r.superblock_dense(sb))[0] == pytest.approx(exact, abs=1e-12)
    sb = warmup.warmup_superblock_l11r("heisenberg", 4, m=10)     # four spins: -3/4 - sqrt(3)/2
    assert np.linalg.eigvalsh(l11r.superblock_dense(sb))[0] == pytest.approx(-0.75 - math.sqrt(3) / 2, abs=1e-13)


def test_davidson_on_algorithm2_equals_eigh():
    sb, _ = pair("hub_L8_m40")
    H = l11r.superblock_dense(sb)
    w = np.linalg.eigvalsh(H)
    lam, x, info = dav.davidson(lambda v: l11r.project_blocks(sb, v), l11r.diagonal(sb),
                                warmup.start_vector(sb.n, 0))
    assert info["converged"] and lam == pytest.approx(w[0], abs=1e-10)


def test_flop_count_counts_every_record_once():
    # one record per (block pair, site elements) with valid segments; the identity-identity
    # terms cost nothing
    sb, _ = pair("heis_L6_exact")
    fc = l11r.flop_count(sb)
    assert fc["records"] > 0 and fc["flops"] > 0


def test_planted_missing_fermion_parity_is_caught():
    # the hop between the two sites without the parity of site s1: another Hamiltonian
    sb, sb_lr = pair("hub_L6_exact")
    bad_terms = []
    P = np.diag([1.0, -1.0, -1.0, 1.0])
    sops = list(sb.sops)
    for coef, a, s1, s2, b in sb.terms:
        if a == -1 and b == -1 and s1 != -1 and s2 != -1:
            # the first site's factor times P undoes its parity (P P = 1):
            # c^dag P -> c^dag, P c -> P c P
            M = sops[s1]
            sops.append(M @ P)
            bad_terms.append((coef, a, len(sops) - 1, s2, b))
        else:
            bad_terms.append((coef, a, s1, s2, b))
    bad = type(sb)(ql=sb.ql, dl=sb.dl, qs=sb.qs, qr=sb.qr, dr=sb.dr, Q=sb.Q, segs=sb.segs,
                   opsl=sb.opsl, sops=sops, opsr=sb.opsr, terms=bad_terms)
    w_bad = np.linalg.eigvalsh(l11r.superblock_dense(bad))
    w = np.linalg.eigvalsh(lr.superblock_dense(sb_lr))
    assert np.max(np.abs(w_bad - w)) > 1e-3


def test_planted_wrong_stage_order_is_caught():
    # block l's factor applied transposed where its blocks are square (stage 4 read with
    # the operator's indices swapped) breaks agreement with the definition
    sb, _ = pair("heis_L12_m24")
    x = np.random.default_rng(2).standard_normal(sb.n)
    y_def = l11r.project_dense(sb, x)
    saved = [op.blocks for op in sb.opsl]
    for op in sb.opsl:
        op.blocks = {(i, j): M.T.copy() if M.shape[0] == M.shape[1] else M for (i, j), M in op.blocks.items()}
    try:
        y_bad = l11r.project_blocks(sb, x)
    finally:
        for op, b in zip(sb.opsl, saved):
            op.blocks = b
    assert np.linalg.norm(y_bad - y_def) > 1e-6 * np.linalg.norm(y_def)
