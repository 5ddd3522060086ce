"""Projective measurement sampling on the GPU (ttn_sample) against the
oracle's samplers (oracle.sampling, pinned in tests/test_oracle_sampling.py
against the state-vector definition):

* identical states (the oracle's entangled TTNs copied into the GPU context)
  and identical uniforms give identical outcomes, shot by shot (FP64, both
  sides decide in double precision);
* product states: every atom's outcome is the inverse CDF of |amps|^2 at its
  own uniform (8x8, chi = 16, padding-free lattice);
* GHZ on 8x8: every shot is all 0 or all 1, decided by the first uniform;
* at the full 8x8 chi = 128 size after TDVP steps: per-atom outcome
  frequencies agree with <|s><s|_i> from ttn_measure within 5 sigma, and the
  split-precision walk draws the FP64 walk's outcomes (a flip needs a uniform
  within ~1e-7 of a boundary);
* argument errors.
"""
import numpy as np
import pytest

from oracle import sampling, ttn as ottn
from paper_2210_03763_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    return nat


def _entangled(Lx, Ly, chi, seed):
    N = Lx * Ly
    o = ottn.OracleTTN(Lx, Ly, chi, W.square_lattice(Lx, Ly), 20.0)
    o.set_schedule(W.random_constant_schedule(N, seed))
    o.set_product_state(W.random_product_amps(N, seed + 1))
    for _ in range(3):
        o.step(0.1)
    return o


@pytest.mark.parametrize("Lx,Ly,chi,seed", [(2, 2, 9, 4), (3, 3, 27, 6), (4, 4, 16, 8)])
def test_walk_equals_oracle_walk(native, Lx, Ly, chi, seed):
    o = _entangled(Lx, Ly, chi, seed)
    g = native.TTN(Lx, Ly, chi)
    g.set_precision(native.FP64)
    for k in range(o.tree.n_nodes):
        g.set_node(k, o.T[k])
    N = Lx * Ly
    U = np.random.default_rng(seed).random((80, N))
    want = sampling.sample_ttn(o, U)
    got = g.sample(U)
    assert np.array_equal(got, want)
    g.close()


def test_product_state_inverse_cdf(native):
    Lx = Ly = 8
    N = 64
    amps = W.random_product_amps(N, 12)
    g = native.TTN(Lx, Ly, 16)
    g.set_product_state(amps)
    order = [a for a in g.leaf_atoms() if a >= 0]
    U = np.random.default_rng(3).random((64, N))
    got = g.sample(U)
    for j, atom in enumerate(order):
        c = np.cumsum(abs(amps[atom]) ** 2)
        c = c / c[-1]
        want = np.searchsorted(c, U[:, j], side="right")
        assert np.array_equal(got[:, atom], np.minimum(want, 2))
    g.close()


def test_ghz_shots_are_all_equal(native):
    g = native.TTN(8, 8, 4)
    g.set_ghz([1] * 64, 0.4)
    U = np.random.default_rng(4).random((100, 64))
    got = g.sample(U)
    for sh in range(100):
        assert len(set(got[sh])) == 1
        assert got[sh, 0] == (0 if U[sh, 0] < 0.5 else 1)
    g.close()


def test_full_size_frequencies_and_split_agreement(native):
    Lx = Ly = 8
    N = 64
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(N, 21)
    runs = []
    for prec in (native.FP64, native.SPLIT_TF32X3):
        g = native.TTN(Lx, Ly, 128)
        g.set_precision(native.SPLIT_TF32X3)
        g.set_hamiltonian(xy, 20.0)
        g.apply_pulse(sched)
        g.set_product_state(W.random_product_amps(N, 22))
        for _ in range(3):
            g.step(0.02)
        g.set_precision(prec)
        runs.append(g)
    f, s = runs
    n = 400
    U = np.random.default_rng(23).random((n, N))
    a = f.sample(U)
    b = s.sample(U)
    assert np.mean(a == b) > 0.999
    P = np.stack([f.measure(w) for w in range(3)], axis=1) / f.norm()
    for lev in range(3):
        freq = np.mean(a == lev, axis=0)
        sig = np.sqrt(np.maximum(P[:, lev] * (1 - P[:, lev]), 1e-4) / n)
        assert np.all(abs(freq - P[:, lev]) < 5 * sig + 1e-9), lev
    f.close()
    s.close()


def test_sample_arguments(native):
    g = native.TTN(2, 2, 9)
    with pytest.raises(ValueError):
        g.sample(np.zeros((3, 5)))
    assert g.sample(np.zeros((0, 4))).shape == (0, 4)
    g.close()
