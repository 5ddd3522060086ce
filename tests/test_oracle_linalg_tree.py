"""Pins of the oracle's QR, Krylov exponential, Hilbert curve and tree."""
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle.linalg import completion_order, krylov_expm, qr_complete, tridiag_expm_e1
from oracle.tree import Tree, hilbert_d2xy, leaf_atoms

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_qr_full_rank_matches_lapack_up_to_phases():
    rng = np.random.default_rng(0)
    A = _rand(rng, 40, 12)
    Q, R = qr_complete(A)
    Ql, Rl = np.linalg.qr(A)
    ph = np.diag(Rl) / abs(np.diag(Rl))          # LAPACK's diag(R) is not real-positive
    assert np.allclose(Q, Ql * ph.conj(), atol=1e-12)
    assert np.allclose(R, ph.conj()[:, None] * Rl, atol=1e-12)
    assert np.all(np.diag(R).real > 0) and np.allclose(np.diag(R).imag, 0)


def test_qr_rank_deficient_completion_rule():
    # A = [v, 2v, 0]: column 0 kept, columns 1 and 2 dependent.  With v = e_0
    # the candidates in (a+b, a) order for a 2x3 row grid are rows
    # (0,0), (0,1), (1,0), (0,2), (1,1), (1,2) -> e_0 is taken, so the
    # completion picks e_(0,1) = row 1 then e_(1,0) = row 3.
    M, D = 6, 3
    A = np.zeros((M, D), complex)
    A[0, 0] = 1.0
    A[0, 1] = 2.0
    order = completion_order(2, 3)
    assert order == [0, 1, 3, 2, 4, 5]
    Q, R = qr_complete(A, order)
    assert np.allclose(Q[:, 0], np.eye(M)[0])
    assert np.allclose(Q[:, 1], np.eye(M)[1])
    assert np.allclose(Q[:, 2], np.eye(M)[3])
    assert np.allclose(Q @ R, A, atol=1e-14)
    assert np.allclose(R[1:, 1:], 0) and abs(R[0, 1] - 2) < 1e-15


def test_qr_completion_skips_candidates_with_small_residual():
    # v = (e_0 + e_1)/sqrt2 kept; e_0 has residual 1/2 >= 1/4 -> accepted.
    # Then with Q = [v, e_0-part], e_1 lies in span -> residual 0 -> skipped.
    A = np.zeros((4, 3), complex)
    A[0, 0] = A[1, 0] = 1.0
    Q, R = qr_complete(A, [0, 1, 2, 3])
    assert np.allclose(Q.conj().T @ Q, np.eye(3), atol=1e-14)
    # the completed span must contain e_0, e_1 (from v and e_0) and then e_2
    P = Q @ Q.conj().T
    assert np.allclose(np.diag(P).real, [1, 1, 1, 0], atol=1e-14)


def test_qr_padding_leaf_restricts_candidates():
    # A padding leg allows only index 0: candidates (a, 0) only.
    order = completion_order(3, 3, None, [0])
    assert order == [0, 3, 6]


def test_tridiag_expm_matches_dense_expm():
    rng = np.random.default_rng(2)
    a = rng.normal(size=7)
    b = abs(rng.normal(size=6))
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    for z in (-0.3j, 0.8j):
        assert np.allclose(tridiag_expm_e1(a, b, z), expm(z * T)[:, 0], atol=1e-13)


def test_krylov_expm_matches_dense_expm():
    rng = np.random.default_rng(3)
    n = 60
    H = _rand(rng, n, n)
    H = (H + H.conj().T) / 2
    v = _rand(rng, n)
    for z in (-0.05j, 0.1j):
        got = krylov_expm(lambda x: H @ x, v, z)
        assert np.allclose(got, expm(z * H) @ v, atol=1e-12 * np.linalg.norm(v))


def test_krylov_happy_breakdown_on_eigenvector():
    H = np.diag([1.0, 2.0, 3.0]).astype(complex)
    v = np.array([0, 2.0, 0], complex)
    stats = []
    got = krylov_expm(lambda x: H @ x, v, -0.5j, stats=stats)
    assert np.allclose(got, v * np.exp(-1j)) and stats[0][0] == 1


def test_hilbert_curve_is_a_unit_step_space_filling_path():
    for side in (2, 4, 8):
        cells = [hilbert_d2xy(side, d) for d in range(side * side)]
        assert cells[0] == (0, 0)
        assert len(set(cells)) == side * side
        for (x0, y0), (x1, y1) in zip(cells, cells[1:]):
            assert abs(x0 - x1) + abs(y0 - y1) == 1
    assert [hilbert_d2xy(2, d) for d in range(4)] == [(0, 0), (0, 1), (1, 1), (1, 0)]


def test_leaf_order_and_padding():
    assert leaf_atoms(2, 2) == [0, 2, 3, 1]
    la = leaf_atoms(3, 3)
    assert len(la) == 16 and sorted(a for a in la if a >= 0) == list(range(9))
    assert la[9:] == [-1] * 7
    assert len(leaf_atoms(2, 3)) == 8


def test_tree_dims_golden():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "tree_dims_8x8.txt"))
            if l.strip() and not l.startswith("#")]
    trees = {}
    for chi, lev, count, d0, d1, d2 in rows:
        tr = trees.setdefault(chi, Tree(8, 8, chi))
        nodes = tr.level_nodes[lev]
        assert len(nodes) == count
        for k in nodes:
            assert tr.shape(k) == (d0, d1, d2)


def test_tree_bond_dims_are_consistent():
    for Lx, Ly, chi in ((3, 3, 5), (4, 4, 64), (5, 3, 20), (8, 8, 128), (2, 1, 4)):
        tr = Tree(Lx, Ly, chi)
        for k in range(tr.n_nodes):
            d0, d1, d2 = tr.shape(k)
            assert d2 <= d0 * d1 and d0 <= d1 * d2 and d1 <= d0 * d2
