"""Pins of the measurement samplers (oracle.sampling): inverse transform
sampling of the conditional marginals in the TTN's leaf order, with the
uniform random numbers as inputs.

* product states: each atom's outcome depends only on its own amplitudes,
  so the draw is the inverse CDF of |amps|^2 with that atom's uniform;
* the GHZ state: every shot is all-0 or all-1 (measured in |1>), decided by
  the first uniform alone;
* the TTN walk draws exactly the same outcomes as the state-vector
  definition for random TTN states (2x2, 2x3, 3x3 with padding leaves);
* histograms of many shots approach |psi|^2 (chi-square, 3x1 lattice).
"""
import numpy as np
import pytest

from oracle import exact, sampling, ttn as ottn
from paper_2210_03763_gb300 import workloads as W


def _order(tr):
    return [a for a in tr.leaf_atom if a >= 0]


def test_product_state_draws_are_independent_inverse_cdfs():
    amps = W.random_product_amps(6, 3)
    o = ottn.OracleTTN(3, 2, 9)
    o.set_product_state(amps)
    rng = np.random.default_rng(1)
    U = rng.random((200, 6))
    got = sampling.sample_ttn(o, U)
    order = _order(o.tree)
    for sh in range(200):
        for j, atom in enumerate(order):
            c = np.cumsum(abs(amps[atom]) ** 2)
            assert got[sh, atom] == int(np.searchsorted(c, U[sh, j], side="right"))


def test_ghz_shots_are_all_equal():
    o = ottn.OracleTTN(3, 3, 4)
    o.set_ghz([1] * 9, 0.3)
    U = np.random.default_rng(2).random((100, 9))
    got = sampling.sample_ttn(o, U)
    for sh in range(100):
        assert len(set(got[sh])) == 1
        assert got[sh, 0] == (0 if U[sh, 0] < 0.5 else 1)


def _entangled(Lx, Ly, chi, seed):
    """An entangled TTN whose padding leaves stay in |0> (the states the
    dynamics produce): a random product state evolved by a few TDVP steps
    under random drives and C6/a^6 = 20."""
    N = Lx * Ly
    o = ottn.OracleTTN(Lx, Ly, chi, W.square_lattice(Lx, Ly), 20.0)
    o.set_schedule(W.random_constant_schedule(N, seed))
    o.set_product_state(W.random_product_amps(N, seed + 1))
    for _ in range(3):
        o.step(0.1)
    return o


@pytest.mark.parametrize("Lx,Ly,chi,seed", [(2, 2, 9, 4), (2, 3, 27, 5), (3, 3, 27, 6)])
def test_ttn_walk_equals_state_vector_definition(Lx, Ly, chi, seed):
    o = _entangled(Lx, Ly, chi, seed)
    N = Lx * Ly
    U = np.random.default_rng(seed).random((60, N))
    a = sampling.sample_ttn(o, U)
    b = sampling.sample_dense(o.dense(), N, _order(o.tree), U)
    assert np.array_equal(a, b)


def test_histogram_matches_born_rule():
    o = _entangled(3, 1, 9, 7)
    psi = o.dense()
    p = abs(psi) ** 2 / np.vdot(psi, psi).real
    n = 20000
    got = sampling.sample_ttn(o, np.random.default_rng(8).random((n, 3)))
    idx = got[:, 0] + 3 * got[:, 1] + 9 * got[:, 2]
    counts = np.bincount(idx, minlength=27)
    m = p * n > 5
    chi2 = np.sum((counts[m] - n * p[m]) ** 2 / (n * p[m]))
    assert chi2 < 60          # 26 degrees of freedom at most: p ~ 1e-4
