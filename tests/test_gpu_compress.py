"""Truncation of a TTN to a smaller bond dimension on the GPU
(ttn_compress) against the oracle's truncation (oracle.ttn.compress, pinned
in tests/test_oracle_compress.py): same bond Schmidt bases, so the
truncated states agree (|1 - F| <= 1e-10 between the two) and so do the
discarded weights (1e-10); the GHZ state survives truncation to bond
dimension 2; the infidelity of the truncation respects
(sum_k sqrt(eps_k))^2 <= n_bonds * sum_k eps_k.
"""
import numpy as np
import pytest

from oracle import ttn as ottn
from paper_2210_03763_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    return nat


def test_compress_matches_oracle(native):
    Lx = Ly = 4
    o = ottn.OracleTTN(Lx, Ly, 32)
    Ts = W.random_ttn_tensors([o.tree.shape(k) for k in range(o.tree.n_nodes)], 21)
    o.set_tensors(Ts)
    g = native.TTN(Lx, Ly, 32)
    for k, X in enumerate(Ts):
        g.set_node(k, X)
    g.refresh_envs()
    small = native.TTN(Lx, Ly, 8)
    dsum, dmax = g.compress_into(small)
    ref, disc = ottn.compress(o, 8)
    assert abs(dsum - sum(disc.values())) < 1e-10
    assert abs(dmax - max(disc.values())) < 1e-10
    h = native.TTN(Lx, Ly, 8)
    for k in range(ref.tree.n_nodes):
        h.set_node(k, ref.T[k])
    h.refresh_envs()
    F = abs(small.overlap(h)) ** 2 / (small.norm() * h.norm())
    assert abs(1 - F) < 1e-10
    assert abs(small.norm() - ref.norm()) < 1e-10
    # truncation bound against the untruncated state
    inf = 1 - abs(small.overlap(g)) ** 2 / (small.norm() * g.norm())
    n_bonds = o.tree.n_nodes - 1
    assert 0 < inf <= n_bonds * dsum + 1e-12
    for x in (g, small, h):
        x.close()


def test_ghz_compresses_to_bond_dimension_two(native):
    g = native.TTN(8, 8, 16)
    g.set_ghz([1] * 64, 0.7)
    t = native.TTN(8, 8, 2)
    dsum, dmax = g.compress_into(t)
    assert dmax < 1e-12
    ref = native.TTN(8, 8, 2)
    ref.set_ghz([1] * 64, 0.7)
    assert abs(t.fidelity(ref) - 1) < 1e-12
    for x in (g, t, ref):
        x.close()


def test_compress_rejects_a_larger_target(native):
    g = native.TTN(4, 4, 8)
    big = native.TTN(4, 4, 32)
    with pytest.raises(native.TTNError):
        g.compress_into(big)
    g.close()
    big.close()
