"""Rydberg Hamiltonian of Eq. 1 / Eq. 2 (Sec. "Modeling 88Sr quantum computers").

Qutrit basis per atom: index 0 = |0>, 1 = |1>, 2 = |r>.

  H(t) = sum_i [ Ox_i(t) sx_i + Oz_i(t) sz_i
                 + (W_i(t) |r><1|_i + conj(W_i(t)) |1><r|_i)
                 - Delta_i(t) n_i ]
       + sum_{i<j} V_ij n_i n_j ,            V_ij = C6 / d_ij^6

* sx = |0><1| + |1><0|, sz = |0><0| - |1><1| act on the qubit subspace only
  (Eq. 1 and the Pauli definitions below it); sz|r> = 0.
* W_i = Omega^R_i exp(i phi_i) drives the single-photon 1<->r transition.
* The detuning term -Delta n is not printed in Eq. 1; the CZ pulse of
  Sec. "Compiler for global GHZ states" uses a detuning on |r>, so it is added
  here as -Delta n (the paper's pulse needs it; Eq. 1 omits it).
* Eq. 1 sums over all ordered pairs; we read it as unordered pairs i<j without
  self-interaction (Eq. 1's double sum read as unordered pairs).  Eq. 2 prints V = -C6/d^6; the caller passes
  the signed coefficient, V_ij = C6/d^6.
"""
import numpy as np

SX = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 0]], dtype=np.complex128)
SZ = np.diag([1.0, -1.0, 0.0]).astype(np.complex128)
RP = np.zeros((3, 3), dtype=np.complex128)
RP[2, 1] = 1.0                      # |r><1|
NR = np.diag([0.0, 0.0, 1.0]).astype(np.complex128)   # n = |r><r|
P0 = np.diag([1.0, 0.0, 0.0]).astype(np.complex128)
P1 = np.diag([0.0, 1.0, 0.0]).astype(np.complex128)

# column order of a pulse-schedule row (one piecewise-constant segment)
SEG_ATOM, SEG_T0, SEG_T1, SEG_OX, SEG_OZ, SEG_OR, SEG_PHI, SEG_DELTA = range(8)


def pair_couplings(xy, C6, r_cut=0.0):
    """V_ij = C6 / d_ij^6 for i != j (Eq. 2); zero on the diagonal.

    ``r_cut > 0`` drops pairs with d_ij > r_cut (the interaction radius
    r_I = r_G + d_off of Sec. "Tensor network simulations"); ``r_cut <= 0``
    keeps all pairs.
    """
    xy = np.asarray(xy, dtype=np.float64)
    n = xy.shape[0]
    V = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            d = np.hypot(xy[i, 0] - xy[j, 0], xy[i, 1] - xy[j, 1])
            if r_cut > 0 and d > r_cut:
                continue
            V[i, j] = C6 / d ** 6
    return V


def coefficients(schedule, n_atoms, t):
    """Drive coefficients of every atom at time t.

    ``schedule`` rows: (atom, t0, t1, omega_x, omega_z, omega_r, phase_r, delta);
    a row is active on [t0, t1).  Active rows of one atom add up.
    Returns (ox, oz, w, delta) arrays of length n_atoms with w complex.
    """
    ox = np.zeros(n_atoms)
    oz = np.zeros(n_atoms)
    w = np.zeros(n_atoms, dtype=np.complex128)
    de = np.zeros(n_atoms)
    if schedule is None:
        return ox, oz, w, de
    for row in np.asarray(schedule, dtype=np.float64).reshape(-1, 8):
        a = int(row[SEG_ATOM])
        if row[SEG_T0] <= t < row[SEG_T1]:
            ox[a] += row[SEG_OX]
            oz[a] += row[SEG_OZ]
            w[a] += row[SEG_OR] * np.exp(1j * row[SEG_PHI])
            de[a] += row[SEG_DELTA]
    return ox, oz, w, de


def local_term(ox, oz, w, delta):
    """Single-atom part of Eq. 1 (plus the detuning term -Delta n) as a 3x3 matrix."""
    return ox * SX + oz * SZ + w * RP + np.conj(w) * RP.conj().T - delta * NR
