"""The seeded input generator (dmrg_inputs) against exact diagonalisation (no GPU)."""
import numpy as np
import pytest

from dmrg_inputs import superblock as sbmod
from dmrg_inputs import warmup
from oracle import ed, projection


@pytest.mark.parametrize("L", [4, 6, 8])
def test_untruncated_heisenberg_superblock_equals_ed(L):
    sb = warmup.warmup_superblock("heisenberg", L, m=10 ** 6)
    sb.validate()
    w = np.linalg.eigvalsh(projection.superblock_dense(sb))[0]
    assert w == pytest.approx(ed.heisenberg_ground_energy(L), abs=1e-11)


@pytest.mark.parametrize("L,U,filling", [(4, 4.0, 1.0), (6, 4.0, 1.0), (6, 0.0, 1.0), (8, 8.0, 0.5)])
def test_untruncated_hubbard_superblock_equals_ed(L, U, filling):
    sb = warmup.warmup_superblock("hubbard", L, m=10 ** 6, U=U, filling=filling)
    sb.validate()
    n = int(round(filling * L / 2))
    assert sb.Q == (n, n)
    w = np.linalg.eigvalsh(projection.superblock_dense(sb))[0]
    assert w == pytest.approx(ed.hubbard_ground_energy(L, n, n, U=U), abs=1e-11)


@pytest.mark.parametrize("model,L,m", [("heisenberg", 12, 16), ("hubbard", 8, 40)])
def test_truncated_superblock_structure(model, L, m):
    sb = warmup.warmup_superblock(model, L, m=m)
    sb.validate()
    # H_L and H_R are symmetric block-diagonal; the hopping / spin-flip partners are
    # transposes of each other
    for ops in (sb.opsL, sb.opsR):
        for (i, j), blk in ops[0].blocks.items():
            assert i == j
            np.testing.assert_allclose(blk, blk.T, atol=1e-12)
    H = projection.superblock_dense(sb)
    np.testing.assert_allclose(H, H.T, atol=1e-12)
    # truncated enlarged blocks: at most m kept states times the site dimension
    q = 2 if model == "heisenberg" else 4
    assert sum(sb.dL) <= q * m and sum(sb.dR) <= q * m
    # variational: the truncated ground energy lies above the exact one
    w = np.linalg.eigvalsh(H)[0]
    exact = (ed.heisenberg_ground_energy(L) if model == "heisenberg"
             else ed.hubbard_ground_energy(L, L // 2, L // 2, U=4.0))
    assert w >= exact - 1e-10


def test_allocation_is_exact_and_bounded():
    d = [5, 40, 100, 40, 5]
    w = [0.1, 0.6, 1.0, 0.6, 0.1]
    for m in (1, 7, 64, 150, 190, 10 ** 6):
        keep = warmup.allocate(d, w, m)
        assert sum(keep) == min(m, sum(d))
        assert all(0 <= k <= di for k, di in zip(keep, d))


def test_start_vector_seeded_and_normalised():
    a, b = warmup.start_vector(1000, 3), warmup.start_vector(1000, 3)
    assert np.array_equal(a, b)
    assert np.linalg.norm(a) == pytest.approx(1.0, abs=1e-15)
    assert not np.array_equal(a, warmup.start_vector(1000, 4))


def test_npz_roundtrip(tmp_path):
    sb = warmup.warmup_superblock("hubbard", 8, m=20)
    path = str(tmp_path / "sb.npz")
    sbmod.save_npz(sb, path)
    sb2 = sbmod.load_npz(path)
    x = warmup.start_vector(sb.n, 0)
    np.testing.assert_array_equal(projection.project_blocks(sb, x), projection.project_blocks(sb2, x))
