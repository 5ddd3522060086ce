"""Pins of Oracle-T (the CPU TTN-TDVP) against things other than itself.

P1  exact regime: every bond at its full rank bound -> TDVP = exact propagator.
P2  fixed-D 1TDVP conserves norm and <H> for a time-independent Hermitian H.
P3  C6 = 0 -> product of independent single-atom 3x3 exponentials.
P7  padding leaves and leaf order do not change the exact-regime result.
GHZ target: the chi = 2 construction equals the GHZ vector.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import exact, model, ttn
from oracle.tree import Tree
from paper_2210_03763_gb300 import workloads as W


def _exact_regime(Lx, Ly, chi, n_steps, dt, seed):
    N = Lx * Ly
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(N, seed)
    amps = W.random_product_amps(N, seed + 1)
    o = ttn.OracleTTN(Lx, Ly, chi, xy, 20.0)
    o.set_schedule(sched)
    o.set_product_state(amps)
    V = model.pair_couplings(xy, 20.0)
    psi = exact.product_state(amps)
    assert np.linalg.norm(o.dense() - psi) < 1e-13
    for s in range(n_steps):
        o.step(dt)
        psi = exact.step(psi, V, sched, s * dt, dt)
    return o, psi, V, sched


@pytest.mark.parametrize("Lx,Ly,chi", [(2, 2, 16), (2, 3, 81), (1, 3, 9)])
def test_p1_exact_regime_matches_state_vector(Lx, Ly, chi):
    o, psi, V, sched = _exact_regime(Lx, Ly, chi, 6, 0.02, 11)
    d = o.dense()
    F = abs(np.vdot(psi, d)) ** 2
    assert abs(1 - F) < 1e-11
    N = Lx * Ly
    assert np.allclose(o.measure(2), exact.expectation_local(psi, N, model.NR), atol=1e-11)
    assert np.allclose(o.measure(0), exact.expectation_local(psi, N, model.P0), atol=1e-11)
    assert np.allclose(o.measure(1), exact.expectation_local(psi, N, model.P1), atol=1e-11)
    assert abs(o.energy() - exact.energy(psi, V, sched, o.t)) < 1e-10


def test_p1_exact_regime_3x3_with_padding():
    # 9 atoms on 16 leaves (7 padding leaves) at chi = 81: every bond is at its
    # full rank bound, so TDVP reproduces exp(-iH dt) per step.
    o, psi, V, sched = _exact_regime(3, 3, 81, 2, 0.02, 21)
    assert abs(1 - abs(np.vdot(psi, o.dense())) ** 2) < 1e-11


def test_p1_time_dependent_schedule_ghz_2x2():
    # Config-1 style: GHZ-4 circuit (H + 3 CNOTs) as square and Jaksch pulses.
    xy = W.square_lattice(2, 2)
    layers = W.schedule_layers(W.ghz_circuit(2, 2, root=0), xy, None)[:4]
    sched, TL = W.layers_to_schedule(layers, 1.0)
    o = ttn.OracleTTN(2, 2, 16, xy, 20.0)
    o.set_schedule(sched)
    V = model.pair_couplings(xy, 20.0)
    psi = exact.product_state(np.tile([1, 0, 0], (4, 1)))
    dt = TL / 20
    for s in range(len(layers) * 20):
        o.step(dt)
        psi = exact.step(psi, V, sched, s * dt, dt)
    assert abs(1 - abs(np.vdot(psi, o.dense())) ** 2) < 1e-11


def test_p2_norm_energy_conservation_truncated():
    Lx = Ly = 4
    xy = W.square_lattice(Lx, Ly)
    o = ttn.OracleTTN(Lx, Ly, 8, xy, 20.0)
    o.set_schedule(W.random_constant_schedule(16, 3))
    o.set_product_state(W.random_product_amps(16, 5))
    e0, n0 = o.energy(), o.norm()
    for _ in range(3):
        o.step(0.02)
    assert abs(o.norm() - n0) < 1e-12
    assert abs(o.energy() - e0) < 1e-11 * max(1.0, abs(e0))


def test_p3_no_interaction_is_a_product():
    Lx = Ly = 4
    N = 16
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(N, 3)
    amps = W.random_product_amps(N, 5)
    o = ttn.OracleTTN(Lx, Ly, 4, xy, 0.0)
    o.set_schedule(sched)
    o.set_product_state(amps)
    t = 0.25
    for _ in range(5):
        o.step(t / 5)
    ox, oz, w, de = model.coefficients(sched, N, 0.1)
    states = []
    for i in range(N):
        h = model.local_term(ox[i], oz[i], w[i], de[i])
        states.append(expm(-1j * t * h) @ amps[i])
    states = np.array(states)
    assert np.allclose(o.measure(2), abs(states[:, 2]) ** 2, atol=1e-12)
    assert np.allclose(o.measure(1), abs(states[:, 1]) ** 2, atol=1e-12)
    tgt = ttn.OracleTTN(Lx, Ly, 4, xy, 0.0)
    tgt.set_product_state(states)
    assert abs(o.fidelity(tgt) - 1) < 1e-12


def test_p7_padding_and_leaf_order_invariance():
    # A 1x3 chain (4 leaves, 1 padding) and the same 3 atoms as a 3x1 chain
    # (other Hilbert order) give the same exact-regime state.
    o1, psi1, _, _ = _exact_regime(1, 3, 9, 4, 0.03, 31)
    o2, psi2, _, _ = _exact_regime(3, 1, 9, 4, 0.03, 31)
    assert abs(1 - abs(np.vdot(o1.dense(), o2.dense())) ** 2) < 1e-11


def test_ghz_target_is_the_ghz_vector():
    Lx, Ly = 2, 3
    N = 6
    mask = [1, 0, 1, 1, 0, 1]
    o = ttn.OracleTTN(Lx, Ly, 16)
    o.set_ghz(mask, phase=0.4)
    want = np.zeros(3 ** N, complex)
    want[0] = 1 / math.sqrt(2)
    want[exact.basis_index(mask)] = np.exp(0.4j) / math.sqrt(2)
    assert np.linalg.norm(o.dense() - want) < 1e-13
    assert abs(o.norm() - 1) < 1e-13


def test_tree_node_isometries_after_steps():
    o, _, _, _ = _exact_regime(2, 3, 9, 2, 0.02, 41)
    tr = o.tree
    for k in range(tr.n_nodes):
        if k == tr.root:
            continue
        X = o.T[k]
        M = X.reshape(-1, X.shape[2])
        assert np.allclose(M.conj().T @ M, np.eye(X.shape[2]), atol=1e-12)


def test_truncated_overlap_convergence_in_chi():
    # Convergence metric C(p1, p2) = 1 - |<psi(p1)|psi(p2)>|^2 (Table I) falls
    # as chi grows towards the exact regime (2x3: exact at chi = 9).
    Lx, Ly = 2, 3
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(6, 7)
    amps = W.random_product_amps(6, 8)
    runs = {}
    for chi in (2, 3, 9):
        o = ttn.OracleTTN(Lx, Ly, chi, xy, 20.0)
        o.set_schedule(sched)
        o.set_product_state(amps)
        for _ in range(8):
            o.step(0.05)
        runs[chi] = o.dense()
    c = {chi: 1 - abs(np.vdot(runs[chi], runs[9])) ** 2 for chi in (2, 3)}
    assert c[3] < c[2]
