"""Oracle-X: exact state-vector propagation of Eq. 1 for at most 9 atoms.

State psi in C^(3^N) with basis index sum_i s_i 3^i (s_i in {0:|0>, 1:|1>, 2:|r>}),
so atom 0 is the fastest index.  Time stepping is piecewise constant: step k
uses H(t_k + dt/2) and psi <- exp(-i H dt) psi, the same time discretisation
the TDVP step uses (H frozen at the step midpoint).  The exponential is NOT a Krylov method:

* N <= 6: dense Hermitian eigendecomposition (numpy.linalg.eigh),
* N <= 9: scipy.sparse.linalg.expm_multiply (Al-Mohy & Higham truncated Taylor).

Decay (Eq. 3, the open-system Hamiltonian of Sec. "Modeling 88Sr quantum
computers"): with ``gamma`` > 0 the generator is H_OQS = H - i gamma sum_i n_i
(the no-jump evolution of a decay out of the computational states); the
dense path then uses scipy.linalg.expm (the generator is not Hermitian).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model

MAX_ATOMS = 9


def basis_index(states):
    """Index of the product basis state with per-atom levels ``states``."""
    return int(sum(int(s) * 3 ** i for i, s in enumerate(states)))


def product_state(amps):
    """Kronecker product of per-atom 3-vectors (atom 0 fastest)."""
    amps = np.asarray(amps, dtype=np.complex128)
    psi = np.ones(1, dtype=np.complex128)
    for i in range(amps.shape[0]):
        # atom i has stride 3^i: it is the slower factor of kron(a_i, psi)
        psi = np.kron(amps[i], psi)
    return psi


def diagonal_interaction(V):
    """Diagonal of sum_{i<j} V_ij n_i n_j in the product basis."""
    n = V.shape[0]
    dim = 3 ** n
    idx = np.arange(dim)
    ryd = np.zeros((n, dim), dtype=bool)
    for i in range(n):
        ryd[i] = (idx // 3 ** i) % 3 == 2
    d = np.zeros(dim)
    for i in range(n):
        for j in range(i + 1, n):
            if V[i, j] != 0.0:
                d += V[i, j] * (ryd[i] & ryd[j])
    return d


def rydberg_count(n):
    """Number of atoms in |r> for every product basis state."""
    idx = np.arange(3 ** n)
    return sum(((idx // 3 ** i) % 3 == 2).astype(np.float64) for i in range(n))


def hamiltonian(V, schedule, t, gamma=0.0):
    """Sparse H(t) of Eq. 1 on the full 3^N space (minus i gamma sum_i n_i,
    Eq. 3, when gamma != 0)."""
    n = V.shape[0]
    if n > MAX_ATOMS:
        raise ValueError("exact oracle is limited to %d atoms" % MAX_ATOMS)
    ox, oz, w, de = model.coefficients(schedule, n, t)
    diag = diagonal_interaction(V).astype(np.complex128)
    if gamma != 0.0:
        diag = diag - 1j * gamma * rydberg_count(n)
    H = sp.diags(diag, format="csr")
    for i in range(n):
        h = model.local_term(ox[i], oz[i], w[i], de[i])
        if not np.any(h):
            continue
        # atom i has stride 3^i: kron(I_{3^(n-1-i)}, h, I_{3^i})
        op = sp.kron(sp.identity(3 ** (n - 1 - i), format="csr"),
                     sp.kron(sp.csr_matrix(h), sp.identity(3 ** i, format="csr")),
                     format="csr")
        H = H + op
    return H.tocsr()


def step(psi, V, schedule, t, dt, gamma=0.0):
    """One piecewise-constant step exp(-i H(t+dt/2) dt) psi."""
    H = hamiltonian(V, schedule, t + 0.5 * dt, gamma)
    n = V.shape[0]
    if n <= 6:
        if gamma != 0.0:
            from scipy.linalg import expm
            return expm(-1j * dt * H.toarray()) @ psi
        w, U = np.linalg.eigh(H.toarray())
        return U @ (np.exp(-1j * dt * w) * (U.conj().T @ psi))
    return spla.expm_multiply(-1j * dt * H, psi)


def evolve(psi, V, schedule, t0, dt, n_steps, gamma=0.0):
    t = t0
    for _ in range(n_steps):
        psi = step(psi, V, schedule, t, dt, gamma)
        t += dt
    return psi


def expectation_local(psi, n_atoms, op):
    """<psi| op_i |psi> for every atom i (op a 3x3 matrix)."""
    T = psi.reshape([3] * n_atoms, order="F")
    out = np.zeros(n_atoms)
    for i in range(n_atoms):
        opT = np.moveaxis(np.tensordot(op, T, axes=([1], [i])), 0, i)
        out[i] = np.real(np.vdot(T, opT))
    return out


def energy(psi, V, schedule, t):
    """<psi|H(t)|psi> of the Hermitian H of Eq. 1 (no decay term)."""
    H = hamiltonian(V, schedule, t)
    return float(np.real(np.vdot(psi, H @ psi)))
