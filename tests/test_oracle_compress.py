"""Pins of the oracle's bond truncation (oracle.ttn.compress: every bond
projected on the top eigenvectors of its bond Gram, i.e. its Schmidt basis;
bond dimension chi, Sec. "Tensor network simulations"):

* no truncation (chi' = chi) leaves the state unchanged;
* the GHZ state has bond dimension 2 exactly: truncating to 2 loses nothing;
* 2x2 lattice: the two root bonds cut the same bipartition, so truncating
  them to rank r is the best rank-r approximation (Eckart-Young), and the
  infidelity equals the discarded weight of that bond exactly;
* 3x3 lattice (exact state vector available): the infidelity of the
  truncated state is bounded by (sum_k sqrt(eps_k))^2 over the bonds.
"""
import numpy as np

from oracle import ttn as ottn
from paper_2210_03763_gb300 import workloads as W


def _random(Lx, Ly, chi, seed):
    o = ottn.OracleTTN(Lx, Ly, chi)
    o.set_tensors(W.random_ttn_tensors([o.tree.shape(k) for k in range(o.tree.n_nodes)], seed))
    return o


def _F(a, b):
    return abs(b.overlap(a)) ** 2 / (a.overlap(a).real * b.overlap(b).real)


def test_compress_without_truncation_is_identity():
    o = _random(3, 2, 9, 1)
    new, disc = ottn.compress(o, 9)
    assert abs(1 - _F(o, new)) < 1e-12
    assert max(disc.values()) < 1e-12


def test_ghz_is_bond_dimension_two():
    o = ottn.OracleTTN(3, 3, 16)
    o.set_ghz([1] * 9, 0.4)
    new, disc = ottn.compress(o, 2)
    assert abs(1 - _F(o, new)) < 1e-12
    assert max(disc.values()) < 1e-12


def test_single_cut_is_eckart_young():
    o = _random(2, 2, 9, 2)
    for r in (1, 3, 5):
        new, disc = ottn.compress(o, r)
        root = o.tree.root
        eps = [disc[c] for kind, c in o.tree.children[root] if kind == "node"]
        assert abs(eps[0] - eps[1]) < 1e-12
        assert abs((1 - _F(o, new)) - eps[0]) < 1e-12
        # the discarded weight is the tail of the Schmidt spectrum of that cut
        leaves = o.tree.leaf_atom
        left = [a for a in leaves[:2] if a >= 0]
        psi_t = o.dense().reshape([3] * 4, order="F")
        perm = left + [a for a in range(4) if a not in left]
        s = np.linalg.svd(np.transpose(psi_t, perm).reshape(9, 9, order="F"), compute_uv=False)
        assert abs(eps[0] - np.sum(s[r:] ** 2) / np.sum(s ** 2)) < 1e-12


def test_truncation_error_bounded_by_discarded_weights():
    o = _random(3, 3, 27, 3)
    new, disc = ottn.compress(o, 6)
    bound = sum(np.sqrt(e) for e in disc.values()) ** 2
    inf = 1 - _F(o, new)
    assert 0 < inf <= bound + 1e-12
    # the compressed state is in canonical form: its norm is the root's
    assert abs(new.norm() - new.overlap(new).real) < 1e-12
