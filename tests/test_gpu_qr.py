"""The GPU gauge-move QR (CGS2 with deterministic completion of dependent
columns) against the oracle's qr_complete, element by element, through the C
ABI (ttn_selftest_qr).

Shapes span several 128-row blocks with a ragged tail, full rank, low rank
with the structured completion (kept rank <= 64) and with the sequential one
(kept rank > 64), the zero matrix, a caller-given candidate order, the
degenerate 1 x 1 case, the largest node matricisation of an 8x8 chi=128 TTN
(16384 x 128), the widest one at chi = 256 (65536 x 256, one cooperative
launch with the smallest shared-memory option) and a tall matrix with more
row blocks than fit on the GPU at once (the multi-launch column loop).  Both sides work in FP64 and take every
dependence and candidate decision from values far from their thresholds, so
Q and R agree to rounding: 1e-11 of max|A| for R, 1e-10 absolute for Q.
"""
import numpy as np
import pytest

from oracle import linalg as OL

pytestmark = pytest.mark.gpu
Q_TOL = 1e-10
R_TOL = 1e-11


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    return nat


def _cmat(rng, m, n):
    return rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))


def _check(native, A, cand=None, expect_dep=None):
    Qg, Rg, nd, ms = native.selftest_qr(A, cand)
    Qo, Ro = OL.qr_complete(A, None if cand is None else list(cand))
    scale = max(np.max(abs(A)), 1e-300)
    assert np.max(abs(Rg - Ro)) <= R_TOL * scale, np.max(abs(Rg - Ro)) / scale
    assert np.max(abs(Qg - Qo)) <= Q_TOL, np.max(abs(Qg - Qo))
    D = A.shape[1]
    assert np.max(abs(Qg.conj().T @ Qg - np.eye(D))) < 1e-12
    assert np.max(abs(Qg @ Rg - A)) <= 1e-12 * scale * np.sqrt(D)
    ndo = int(np.sum(np.abs(np.diag(Ro)) == 0.0))
    assert nd == ndo
    if expect_dep is not None:
        assert nd == expect_dep
    return nd, ms


def test_full_rank_ragged(native):
    rng = np.random.default_rng(1)
    _check(native, _cmat(rng, 300, 40), expect_dep=0)


def test_low_rank_structured_completion(native):
    rng = np.random.default_rng(2)
    A = _cmat(rng, 500, 5) @ _cmat(rng, 5, 40)
    _check(native, A, expect_dep=35)


def test_rank_above_structured_limit(native):
    rng = np.random.default_rng(3)
    A = _cmat(rng, 2000, 100) @ _cmat(rng, 100, 128)
    _check(native, A, expect_dep=28)


def test_zero_matrix_and_candidate_order(native):
    rng = np.random.default_rng(4)
    A = np.zeros((90, 9), dtype=np.complex128)
    cand = rng.permutation(90)
    Qg, _, nd, _ = native.selftest_qr(A, cand)
    assert nd == 9
    # the first nine candidates are accepted in order
    for k in range(9):
        e = np.zeros(90)
        e[cand[k]] = 1.0
        assert np.max(abs(Qg[:, k] - e)) < 1e-15
    _check(native, A, cand, expect_dep=9)


def test_exact_zero_and_repeated_columns(native):
    rng = np.random.default_rng(5)
    B = _cmat(rng, 729, 3)
    A = np.concatenate([B[:, :1], np.zeros((729, 2)), B[:, :1] * (0.5 - 2j), B[:, 1:], B[:, :2]], axis=1)
    _check(native, A, cand=rng.permutation(729), expect_dep=5)


def test_square_low_rank(native):
    # the shapes of the gauge moves onto a padded parent leg (9 x 9 -> 81) and
    # of the root (128 x 128): square, so the completion runs out of clean
    # candidates and takes the largest-residual rule at the end
    rng = np.random.default_rng(8)
    x = (rng.normal(size=9) + 1j * rng.normal(size=9))
    prod = np.kron(x, x * np.exp(-0.5 * np.arange(9)))[:, None]
    A = prod @ (rng.normal(size=(1, 81)) + 1j * rng.normal(size=(1, 81)))
    _check(native, A, cand=OL.completion_order(9, 9), expect_dep=80)
    A = _cmat(rng, 128, 3) @ _cmat(rng, 3, 128)
    _check(native, A, expect_dep=125)


def test_widest_bond(native):
    rng = np.random.default_rng(9)
    _check(native, _cmat(rng, 1024, 256), expect_dep=0)
    A = _cmat(rng, 1024, 40) @ _cmat(rng, 40, 256)
    _check(native, A, expect_dep=216)


def test_one_by_one(native):
    _check(native, np.array([[2.0 - 1.0j]]), expect_dep=0)
    _check(native, np.zeros((1, 1), dtype=np.complex128), expect_dep=1)


def test_largest_node_matricisation(native):
    rng = np.random.default_rng(6)
    nd, ms = _check(native, _cmat(rng, 16384, 128), expect_dep=0)
    print("16384 x 128 full rank: %.3f ms" % ms)
    A = _cmat(rng, 16384, 3) @ _cmat(rng, 3, 128)
    nd, ms = _check(native, A, expect_dep=125)
    print("16384 x 128 rank 3: %.3f ms" % ms)


def test_widest_node_matricisation_one_launch(native):
    # 65536 x 256: the level-3/4 node of an 8x8, chi = 256 TTN.  512 row
    # blocks fit in one cooperative launch only with the smallest
    # shared-memory option (no cached columns, look-ahead window of 4).
    rng = np.random.default_rng(8)
    A = _cmat(rng, 65536, 2) @ _cmat(rng, 2, 256)
    nd, ms = _check(native, A, expect_dep=254)
    print("65536 x 256 rank 2: %.3f ms" % ms)
    nd, ms = _check(native, _cmat(rng, 65536, 256), expect_dep=0)
    print("65536 x 256 full rank: %.3f ms" % ms)


def test_more_row_blocks_than_resident(native):
    rng = np.random.default_rng(7)
    _check(native, _cmat(rng, 1 << 19, 3), expect_dep=0)


def test_invalid_arguments(native):
    with pytest.raises(native.TTNError):
        native.selftest_qr(np.zeros((3, 5), dtype=np.complex128))
    with pytest.raises(native.TTNError):
        native.selftest_qr(np.zeros((8, 2), dtype=np.complex128), cand=[0, 9])
