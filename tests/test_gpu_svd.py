"""Truncated SVD of a bond matrix on the GPU (ttn_svd_truncate) against
NumPy's LAPACK SVD and against what the mathematics fixes:

* singular values equal numpy.linalg.svd's to 1e-12 of sigma_max;
* U and V have orthonormal columns to 1e-12;
* Eckart-Young: the truncation error |A - U S Vh|_F^2 equals the sum of the
  discarded sigma^2, and the reported discarded weight is that sum over the
  total (1e-12);
* truncation by chi and by eps = sigma_i / sigma_max, odd N, tall and
  square, exactly rank-deficient inputs (zero singular values).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    return nat


def _matrix(M, N, rank, decay, seed):
    rng = np.random.default_rng(seed)
    Ua, _ = np.linalg.qr(rng.normal(size=(M, rank)) + 1j * rng.normal(size=(M, rank)))
    Va, _ = np.linalg.qr(rng.normal(size=(N, rank)) + 1j * rng.normal(size=(N, rank)))
    s = np.exp(-decay * np.arange(rank)) * (1 + 0.1 * rng.random(rank))
    return (Ua * s) @ Va.conj().T


@pytest.mark.parametrize("M,N,rank,chi,eps", [(64, 64, 64, 64, 0.0), (300, 37, 37, 20, 0.0), (1024, 128, 128, 32, 0.0),
                                              (81, 81, 12, 81, 1e-10), (500, 99, 99, 99, 1e-3),
                                              (16384, 128, 128, 100, 0.0), (9, 9, 9, 4, 0.0)])
def test_svd_truncate_matches_lapack(native, M, N, rank, chi, eps):
    A = _matrix(M, N, rank, 0.15, M + N + rank)
    U, S, Vh, disc = native.svd_truncate(A, chi, eps)
    s_ref = np.linalg.svd(A, compute_uv=False)
    smax = s_ref[0]
    keep = min(chi, int(np.sum(s_ref >= eps * smax)))
    assert len(S) == keep
    assert np.max(abs(S - s_ref[:keep])) <= 1e-12 * smax
    assert np.max(abs(U.conj().T @ U - np.eye(keep))) <= 1e-12
    assert np.max(abs(Vh @ Vh.conj().T - np.eye(keep))) <= 1e-12
    err2 = np.linalg.norm(A - (U * S) @ Vh) ** 2
    tail = np.sum(s_ref[keep:] ** 2)
    assert abs(err2 - tail) <= 1e-12 * np.sum(s_ref ** 2)
    assert abs(disc - tail / np.sum(s_ref ** 2)) <= 1e-12


def test_svd_rejects_bad_sizes(native):
    with pytest.raises(native.TTNError):
        native.svd_truncate(np.zeros((4, 8), complex), 2)        # M < N
    with pytest.raises(native.TTNError):
        native.svd_truncate(np.zeros((600, 300), complex), 2)    # N > 256
