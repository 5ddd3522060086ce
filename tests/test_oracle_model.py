"""Pins of the oracle's Hamiltonian (Eq. 1, Eq. 2) and exact propagator.

Every expected value here comes from a closed form, not from the oracle."""
import math

import numpy as np
import pytest

from oracle import exact, model

ATOL = 1e-12


def _one_atom(row, psi0, t):
    V = np.zeros((1, 1))
    sched = np.array([row], dtype=float)
    return exact.evolve(np.asarray(psi0, complex), V, sched, 0.0, t, 1)


def test_rabi_1_to_r_closed_form():
    # H = Omega (|r><1| + |1><r|): from |1>, P_r(t) = sin^2(Omega t), P_1 = cos^2
    om = 1.3
    for t in (0.1, 0.7, 1.9):
        psi = _one_atom([0, 0, 10, 0, 0, om, 0, 0], [0, 1, 0], t)
        assert abs(abs(psi[2]) ** 2 - math.sin(om * t) ** 2) < ATOL
        assert abs(abs(psi[1]) ** 2 - math.cos(om * t) ** 2) < ATOL


def test_rabi_phase_convention():
    # W = Omega e^{i phi}: exp(-i t (W|r><1| + h.c.)) |1> = cos(Ot)|1> - i e^{i phi} sin(Ot)|r>
    om, phi, t = 0.8, 0.9, 0.6
    psi = _one_atom([0, 0, 10, 0, 0, om, phi, 0], [0, 1, 0], t)
    assert abs(psi[1] - math.cos(om * t)) < ATOL
    assert abs(psi[2] - (-1j * np.exp(1j * phi) * math.sin(om * t))) < ATOL


def test_rx_rz_square_pulses_are_rotations():
    # R_X(theta) = exp(-i theta sx/2) needs Omega^x = theta/(2T); likewise R_Z.
    th, T = 0.77, 2.0
    c, s = math.cos(th / 2), math.sin(th / 2)
    psi = _one_atom([0, 0, 10, th / (2 * T), 0, 0, 0, 0], [1, 0, 0], T)
    assert np.allclose(psi, [c, -1j * s, 0], atol=ATOL)
    psi = _one_atom([0, 0, 10, 0, th / (2 * T), 0, 0, 0], [1, 1, 0], T)
    assert np.allclose(psi, [np.exp(-1j * th / 2), np.exp(1j * th / 2), 0], atol=ATOL)


def test_detuning_and_sigma_z_on_r():
    # -Delta n: |r> gains exp(+i Delta t); sz|r> = 0 (Pauli matrices act on the qubit only)
    de, t = 0.4, 1.7
    psi = _one_atom([0, 0, 10, 0, 0.9, 0, 0, de], [0, 0, 1], t)
    assert abs(psi[2] - np.exp(1j * de * t)) < ATOL


def test_pair_coupling_inverse_sixth_power():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    V = model.pair_couplings(xy, 20.0)
    assert V[0, 1] == pytest.approx(20.0, abs=1e-15)
    assert V[0, 2] == pytest.approx(20.0 / 64.0, abs=1e-15)
    assert V[1, 2] == pytest.approx(20.0 / 125.0, abs=1e-15)   # d^2 = 5
    assert np.all(np.diag(V) == 0) and np.allclose(V, V.T)
    Vc = model.pair_couplings(xy, 20.0, r_cut=2.1)
    assert Vc[1, 2] == 0.0 and Vc[0, 2] != 0.0


def test_diagonal_interaction_phases():
    # Omega = 0: each basis state only picks up exp(-i E_c t), E_c = sum_{i<j} V_ij [c_i=c_j=r]
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    V = model.pair_couplings(xy, 7.0)
    rng = np.random.default_rng(0)
    psi0 = rng.normal(size=27) + 1j * rng.normal(size=27)
    psi0 /= np.linalg.norm(psi0)
    t = 0.37
    psi = exact.evolve(psi0, V, None, 0.0, t, 1)
    for idx in range(27):
        s = [(idx // 3 ** i) % 3 for i in range(3)]
        E = 0.0
        for i in range(3):
            for j in range(i + 1, 3):
                if s[i] == 2 and s[j] == 2:
                    E += 7.0 / abs(i - j) ** 6
        assert abs(psi[idx] - psi0[idx] * np.exp(-1j * E * t)) < ATOL


def test_two_atom_blockade_sqrt2_rabi():
    # Both atoms driven 1<->r from |11>: symmetric subspace {|11>, |W>, |rr>},
    # <W|H|11> = sqrt2 Omega, <rr|H|W> = sqrt2 Omega, <rr|H|rr> = V.
    # As V -> inf, P_W(t) = sin^2(sqrt2 Omega t) (the sqrt2-enhanced blockaded Rabi).
    om = 1.0
    xy = np.array([[0.0, 0.0], [1.0, 0.0]])
    sched = np.array([[0, 0, 100, 0, 0, om, 0, 0], [1, 0, 100, 0, 0, om, 0, 0]], float)
    psi0 = np.zeros(9, complex)
    psi0[exact.basis_index([1, 1])] = 1.0
    for Vnn in (20.0, 3.0):
        V = model.pair_couplings(xy, Vnn)
        s2 = math.sqrt(2) * om
        H3 = np.array([[0, s2, 0], [s2, 0, s2], [0, s2, Vnn]])
        for t in (0.3, 1.1):
            w, U = np.linalg.eigh(H3)
            c = U @ (np.exp(-1j * w * t) * U[0, :])
            psi = exact.evolve(psi0, V, sched, 0.0, t, 1)
            pw = abs(psi[exact.basis_index([1, 2])]) ** 2 + abs(psi[exact.basis_index([2, 1])]) ** 2
            assert abs(pw - abs(c[1]) ** 2) < 1e-11
            assert abs(abs(psi[exact.basis_index([2, 2])]) ** 2 - abs(c[2]) ** 2) < 1e-11
    V = model.pair_couplings(xy, 1e7)
    for t in (0.3, 1.1):
        psi = exact.evolve(psi0, V, sched, 0.0, t, 1)
        pw = abs(psi[exact.basis_index([1, 2])]) ** 2 + abs(psi[exact.basis_index([2, 1])]) ** 2
        assert abs(pw - math.sin(math.sqrt(2) * om * t) ** 2) < 1e-6


def test_jaksch_cz_tends_to_cz_pi():
    # pi (control) - 2pi (target) - pi (control) on 1<->r with V >> Omega is
    # diag(1, -1, -1, -1) on the qubit space.  With the control in |r>, the
    # target's 1<->r transition is detuned by V, so during the 2pi pulse
    # (length pi/Omega) |11> picks up the light shift Omega^2/V: a phase error
    # pi Omega / V to first order; populations are off only at (Omega/V)^2.
    from paper_2210_03763_gb300 import workloads as W
    xy = np.array([[0.0, 0.0], [1.0, 0.0]])
    sched, TL = W.layers_to_schedule([[("cz", (0, 1), math.pi)]], 1.0)
    for Vnn in (200.0, 2000.0):
        V = model.pair_couplings(xy, Vnn)
        U = np.zeros((4, 4), complex)
        for k, (a, b) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
            psi0 = np.zeros(9, complex)
            psi0[exact.basis_index([a, b])] = 1.0
            psi = exact.evolve(psi0, V, sched, 0.0, TL / 400, 400)
            for l, (c, d) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
                U[l, k] = psi[exact.basis_index([c, d])]
        assert np.max(abs(U[:3, :3] - np.diag([1, -1, -1]))) < 1e-10
        assert abs(abs(U[3, 3]) - 1) < 2 * (1.0 / Vnn) ** 2
        phase_err = np.angle(-U[3, 3])
        assert abs(abs(phase_err) - math.pi / Vnn) < 0.05 * math.pi / Vnn


def test_exact_dense_vs_sparse_paths_agree():
    # N <= 6 uses eigh, larger N expm_multiply; a 7-atom run reduces to 6 when
    # atom 6 is idle and far away.
    xy = np.array([[i % 3, i // 3] for i in range(6)] + [[50.0, 50.0]], float)
    sched = np.array([[a, 0, 10, 0.3 * a, 0.2, 0.5, 0.1 * a, 0.1] for a in range(6)])
    rng = np.random.default_rng(1)
    amps = rng.normal(size=(7, 3)) + 1j * rng.normal(size=(7, 3))
    amps[6] = [1, 0, 0]
    amps /= np.linalg.norm(amps, axis=1, keepdims=True)
    V7 = model.pair_couplings(xy, 5.0)
    p7 = exact.evolve(exact.product_state(amps), V7, sched, 0.0, 0.05, 3)
    p6 = exact.evolve(exact.product_state(amps[:6]), V7[:6, :6], sched, 0.0, 0.05, 3)
    assert np.allclose(p7[:729], p6, atol=1e-12)
