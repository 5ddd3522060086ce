"""Pins of the synthetic circuit generator against the paper's gate identities
and printed circuit statistics (Table II)."""
import math
import os

import numpy as np

from paper_2210_03763_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
X = np.array([[0, 1], [1, 0]], complex)
Z = np.diag([1, -1]).astype(complex)


def _rot(P, th):
    return math.cos(th / 2) * np.eye(2) - 1j * math.sin(th / 2) * P


def _apply_qubit_circuit(gates, n):
    psi = np.zeros(2 ** n, complex)
    psi[0] = 1
    T = psi.reshape([2] * n, order="F")
    for kind, qs, th in gates:
        if kind == "cz":
            c, t = qs
            # CZ(pi) = diag(1, -1, -1, -1) on (c, t)
            idx = np.indices([2] * n)
            phase = np.where((idx[c] == 0) & (idx[t] == 0), 1.0, -1.0)
            T = T * phase
        else:
            U = _rot(X if kind == "rx" else Z, th)
            T = np.moveaxis(np.tensordot(U, T, axes=([1], [qs[0]])), 0, qs[0])
    return T.reshape(-1, order="F")


def _eq_up_to_phase(a, b):
    k = np.argmax(abs(b))
    ph = a[k] / b[k]
    return abs(abs(ph) - 1) < 1e-10 and np.allclose(a, ph * b, atol=1e-10)


def test_hadamard_decomposition():
    U = np.eye(2, dtype=complex)
    for kind, _, th in W.hadamard(0):
        U = _rot(Z if kind == "rz" else X, th) @ U
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    assert _eq_up_to_phase(U.ravel(), H.ravel())


def test_cnot_decomposition_with_cz_pi():
    for c, t in ((0, 1), (1, 0)):
        for inp in range(4):
            psi = np.zeros(4, complex)
            psi[inp] = 1
            T = psi.reshape(2, 2, order="F")
            for kind, qs, th in W.cnot(c, t):
                if kind == "cz":
                    T = T * np.array([[1, -1], [-1, -1]])
                else:
                    U = _rot(X if kind == "rx" else Z, th)
                    T = np.moveaxis(np.tensordot(U, T, axes=([1], [qs[0]])), 0, qs[0])
            bits = [(inp >> 0) & 1, (inp >> 1) & 1]
            bits[t] ^= bits[c]
            want = np.zeros(4, complex)
            want[bits[0] + 2 * bits[1]] = 1
            if inp == 0:
                ph = T.reshape(-1, order="F")[0]
            assert np.allclose(T.reshape(-1, order="F"), ph * want, atol=1e-12)


def test_ideal_gate_ghz_fidelity_is_one():
    for Lx, Ly in ((2, 2), (3, 3)):
        n = Lx * Ly
        psi = _apply_qubit_circuit(W.ghz_circuit(Lx, Ly), n)
        ghz = np.zeros(2 ** n, complex)
        ghz[0] = ghz[-1] = 1 / math.sqrt(2)
        assert abs(abs(np.vdot(ghz, psi)) ** 2 - 1) < 1e-12


def test_table2_serial_depths():
    for line in open(os.path.join(GOLDEN, "table2_circuit_stats.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        L, d_ser, d_czser = map(int, line.split())
        gates = W.ghz_circuit(L, L)
        assert len(gates) == d_ser
        assert len(W.schedule_layers(gates)) == d_ser
        assert d_ser == 11 * (L * L - 1) + 3
        n_cz = sum(1 for g in gates if g[0] == "cz")
        # serial-CZ layering (no two CZs together): at least one layer per CZ
        xy = W.square_lattice(L, L)
        depth = len(W.schedule_layers(gates, xy, 1e9))
        assert n_cz + 3 <= depth <= d_ser
        par = len(W.schedule_layers(gates, xy, 4.0))
        assert par <= depth


def test_parallel_layers_respect_cz_distance():
    L = 8
    xy = W.square_lattice(L, L)
    for layer in W.schedule_layers(W.ghz_circuit(L, L), xy, 4.0):
        czs = [g for g in layer if g[0] == "cz"]
        atoms = [q for g in layer for q in g[1]]
        assert len(atoms) == len(set(atoms))
        for i in range(len(czs)):
            for j in range(i + 1, len(czs)):
                for a in czs[i][1]:
                    for b in czs[j][1]:
                        assert np.hypot(*(xy[a] - xy[b])) >= 4.0 - 1e-12


def test_repetition_codes_fill_like_fig3():
    # Fig. 3: 3 codes (15 qubits) on 4x4, 12 codes (60 qubits) on 8x8.
    for L, n in ((4, 3), (8, 12)):
        groups = W.repetition_code_groups(L, L)
        assert len(groups) == n
        for g in groups:
            assert len(W.bfs_tree(L, L, g[2], g)) == 4          # connected
        gates = W.repetition_code_circuit(L, L)
        assert sum(1 for g in gates if g[0] == "cz") == 4 * n
        psi = _apply_qubit_circuit(gates, L * L) if L == 4 else None
        if psi is not None:
            # product of 3 five-qubit GHZ states, idle atom in |0>
            amp = abs(psi) ** 2
            assert abs(amp.sum() - 1) < 1e-12 and abs(amp.max() - 1 / 8) < 1e-12


def test_pulse_struct_layout():
    assert W.PULSE_DTYPE.itemsize == 64
    arr = W.to_pulse_array(np.array([[3, 0.5, 1.5, 1, 2, 3, 4, 5]]))
    assert arr["atom"][0] == 3 and arr["delta"][0] == 5.0
