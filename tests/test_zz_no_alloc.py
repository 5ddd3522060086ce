"""The allocation-free contraction (ttn_contract_split_noalloc) against the
existing ttn_apply_heff, through the C ABI, on two calls in a row.

It is meant for callers that cannot allocate device memory when they call it
(their memory belongs to their own pool or budget, or they must not
synchronise the device through cudaMalloc/cudaFree).  Set-up that makes the
root's H_eff a single contraction: C6 = 0 (no pair terms) and drives only on
atoms of the root's first subtree, so H_eff X = H_block(leg 0) x_0 X.  The
block Hamiltonian comes from the CPU oracle's environment of the same state;
the buffers are PyTorch device tensors.  Tolerance: the H_eff bound of the
split-precision tests (6e-6 of max|y|), which covers both contractions and the
split-precision environment inside ttn_apply_heff; against the host product
Hb0 @ X the single-contraction bound (1e-6 of max|y|).

Further cases, each against NumPy's complex128 A @ B: ragged and non-square
shapes run back to back (the FP64 kernel below the tensor-core tiles at
1e-12, the tensor-core path at 1e-6), and a pipeline wait made to run out,
which the call reports as TTN_ERR_TIMEOUT and clears for the next call.
"""
import ctypes

import numpy as np
import pytest

from oracle import ttn as ottn
from oracle.tree import Tree
from paper_2210_03763_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HEFF_TOL = 6e-6
CONTRACT_TOL = 1e-6


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    nat.inject(nat.INJECT_NONE)
    yield nat
    nat.inject(nat.INJECT_NONE)


def test_noalloc_contraction_matches_apply_heff(native):
    import torch
    Lx = Ly = 4
    chi = 64
    tr = Tree(Lx, Ly, chi)
    root = tr.root
    left_atoms = tr.leg_sites(root, 0)
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(Lx * Ly, 17, atoms=left_atoms)
    g = native.TTN(Lx, Ly, chi)
    g.set_precision(native.SPLIT_TF32X3)
    g.set_hamiltonian(xy, 0.0)
    g.apply_pulse(sched)
    Ts = W.random_ttn_tensors([tr.shape(k) for k in range(tr.n_nodes)], 23)
    for k, X in enumerate(Ts):
        g.set_node(k, X)
    g.refresh_envs()
    o = ottn.OracleTTN(Lx, Ly, chi, xy, 0.0)
    o.set_schedule(sched)
    o.set_tensors(Ts)
    Hb0 = ottn.block_hamiltonian(o.env(root, 0), o.coef(0.0))
    d0, d1, d2 = tr.shape(root)
    assert d2 == 1
    M, K, N = d0, d0, d1
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(Hb0.ravel(order="F").copy()).to(dev)
    rng = np.random.default_rng(4)
    for call in range(2):
        X = rng.normal(size=(d0, d1, d2)) + 1j * rng.normal(size=(d0, d1, d2))
        y_ref = g.apply_heff(root, X)[:, :, 0]
        B = torch.from_numpy(X.ravel(order="F").copy()).to(dev)
        C = torch.full((M * N,), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
        native.contract_split_noalloc(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K,
                                      torch.cuda.current_stream())
        torch.cuda.synchronize()
        y = C.cpu().numpy().reshape(M, N, order="F")
        err = np.max(abs(y - y_ref)) / np.max(abs(y_ref))
        assert err < HEFF_TOL, (call, err)
        host = Hb0 @ X[:, :, 0]
        err_host = np.max(abs(y - host)) / np.max(abs(host))
        assert 0.0 < err_host < CONTRACT_TOL, (call, err_host)
    g.close()


def _dev(torch, a):
    return torch.from_numpy(np.asfortranarray(a).ravel(order="F").copy()).to(torch.device("cuda", 0))


# (M, N, K): below the tensor-core tiles (FP64 kernel), K not a multiple of
# 16, N much larger than M (the swapped plan), and the reverse
RAGGED = [(8, 8, 8), (16, 300, 37), (300, 16, 130), (128, 96, 200)]


def test_noalloc_ragged_shapes_back_to_back(native):
    import torch
    rng = np.random.default_rng(8)
    cases = []
    for M, N, K in RAGGED:
        A = rng.normal(size=(M, K)) + 1j * rng.normal(size=(M, K))
        B = rng.normal(size=(K, N)) + 1j * rng.normal(size=(K, N))
        C = torch.full((M * N,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        cases.append((A, B, _dev(torch, A), _dev(torch, B), C))
    stream = torch.cuda.current_stream()
    for _ in range(2):
        for A, B, dA, dB, C in cases:
            M, K = A.shape
            N = B.shape[1]
            native.contract_split_noalloc(dA.data_ptr(), dB.data_ptr(), C.data_ptr(), M, N, K, stream)
        torch.cuda.synchronize()
        for A, B, dA, dB, C in cases:
            M, N = A.shape[0], B.shape[1]
            y = C.cpu().numpy().reshape(M, N, order="F")
            ref = A @ B
            err = np.max(abs(y - ref)) / np.max(abs(ref))
            tc = min(M, N) >= 16 and max(M, N) >= 64
            assert err < (CONTRACT_TOL if tc else 1e-12), (M, N, err)


def test_noalloc_reports_a_timeout_and_recovers(native):
    import torch
    rng = np.random.default_rng(9)
    M, N, K = 128, 96, 200
    A = rng.normal(size=(M, K)) + 1j * rng.normal(size=(M, K))
    B = rng.normal(size=(K, N)) + 1j * rng.normal(size=(K, N))
    dA, dB = _dev(torch, A), _dev(torch, B)
    C = torch.zeros((M * N,), dtype=torch.complex128, device="cuda")
    native.inject(native.INJECT_TC_STALL, 1)
    with pytest.raises(native.TTNError) as e:
        native.contract_split_noalloc(dA.data_ptr(), dB.data_ptr(), C.data_ptr(), M, N, K,
                                      torch.cuda.current_stream())
    assert e.value.code == 6      # TTN_ERR_TIMEOUT
    native.inject(native.INJECT_NONE)
    native.contract_split_noalloc(dA.data_ptr(), dB.data_ptr(), C.data_ptr(), M, N, K,
                                  torch.cuda.current_stream())
    y = C.cpu().numpy().reshape(M, N, order="F")
    assert np.max(abs(y - A @ B)) < CONTRACT_TOL * np.max(abs(A @ B))


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch(native):
    lib = native.load()
    p = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert lib.ttn_contract_split_noalloc(p, p, p, 2048, 2048, 2048, None) == 1
    assert lib.ttn_contract_split_noalloc(p, p, p, 0, 8, 8, None) == 1
