"""Pins of the two-tensor TDVP oracle (oracle.tdvp2, the paper's two-site
integrator with SVD truncation):

* exact regime (2x2 with chi = 16, 2x3 with chi = 27: every bond at full
  rank, no truncation): the TTN equals the exact state-vector propagation;
* truncation is the only norm loss: after a step, <psi|psi> equals its value
  before times prod over the step's splits of (1 - discarded weight), since
  every local exponential is unitary (time-independent Hermitian H);
* from a product state with |r> populated (3x3 lattice, truncated bonds) the
  two-site update follows the exact dynamics more closely than the
  single-site update at the same bond dimension (it grows the bonds from the
  dynamics instead of from fixed completion directions), and its error falls
  with chi (Table I's convergence in chi);
* a GHZ state at bond dimension 2 with no Hamiltonian stays itself.
"""
import numpy as np
import pytest

from oracle import exact, model, tdvp2, ttn as ottn
from paper_2210_03763_gb300 import workloads as W


def _run(cls, Lx, Ly, chi, steps, dt, seed=4):
    N = Lx * Ly
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(N, seed)
    amps = W.random_product_amps(N, seed + 1)
    o = cls(Lx, Ly, chi, xy, 20.0)
    o.set_schedule(sched)
    o.set_product_state(amps)
    for _ in range(steps):
        o.step(dt)
    psi = exact.evolve(exact.product_state(amps), model.pair_couplings(xy, 20.0), sched, 0.0, dt, steps)
    d = o.dense()
    infid = 1.0 - abs(np.vdot(psi, d)) ** 2 / np.vdot(d, d).real
    return infid, o


@pytest.mark.parametrize("Lx,Ly,chi", [(2, 2, 16), (2, 3, 27)])
def test_exact_regime_equals_state_vector(Lx, Ly, chi):
    infid, o = _run(tdvp2.OracleTTN2, Lx, Ly, chi, 3, 0.05)
    assert abs(infid) < 1e-11
    assert abs(o.norm() - 1.0) < 1e-11
    assert o.max_discarded < 1e-20


def test_norm_loss_is_the_discarded_weight():
    N = 9
    xy = W.square_lattice(3, 3)
    o = tdvp2.OracleTTN2(3, 3, 9, xy, 20.0)
    o.set_schedule(W.random_constant_schedule(N, 4))
    o.set_product_state(W.random_product_amps(N, 5))
    for _ in range(3):
        n0 = o.norm()
        o.step(0.05)
        expect = n0 * np.prod([1.0 - d for d in o.discarded])
        assert o.max_discarded > 1e-9            # the bonds do truncate
        assert abs(o.norm() - expect) < 1e-12 * n0, (o.norm(), expect)


def test_two_tensor_beats_single_site_and_converges_in_chi():
    errs = []
    for chi in (9, 27):
        e2, _ = _run(tdvp2.OracleTTN2, 3, 3, chi, 4, 0.05)
        e1, _ = _run(ottn.OracleTTN, 3, 3, chi, 4, 0.05)
        assert 0 < e2 < 0.7 * e1, (chi, e2, e1)
        errs.append(e2)
    assert errs[1] < 1e-2 * errs[0]


def test_ghz_at_bond_dimension_two_is_stationary_without_hamiltonian():
    o = tdvp2.OracleTTN2(3, 3, 2)
    o.set_ghz([1] * 9, 0.3)
    ref = tdvp2.OracleTTN2(3, 3, 2)
    ref.set_ghz([1] * 9, 0.3)
    o.step(0.1)
    assert tdvp2.convergence(o, ref) < 1e-13
