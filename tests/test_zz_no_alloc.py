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
split-precision environment inside ttn_apply_heff.
"""
import ctypes

import numpy as np
import pytest

from oracle import ttn as ottn
from oracle.tree import Tree
from paper_2210_03763_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HEFF_TOL = 6e-6


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    return nat


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
    g.close()


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch(native):
    lib = native.load()
    p = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert lib.ttn_contract_split_noalloc(p, p, p, 2048, 2048, 2048, None) == 1
    assert lib.ttn_contract_split_noalloc(p, p, p, 0, 8, 8, None) == 1
