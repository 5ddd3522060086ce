"""Oracle gradient of the final-state fidelity with respect to the
piecewise-constant pulse amplitudes, by exact reverse mode on the state
vector (Oracle-X).  Test infrastructure only (see the package docstring).

This is the reference for gradients of the discrete time-stepping map
(differentiate the discretised evolution, not the continuous one): with
steps U_n = exp(-i H(t_n + dt/2) dt) (the time discretisation of the TDVP
step: H frozen at the step midpoint) and

    F(theta) = |<target| U_N ... U_1 |psi_0>|^2,

theta the Rabi amplitude Omega_k (schedule field omega_r) or the detuning
Delta_k (field delta) of chosen schedule rows, H is linear in theta:

    dH/dOmega_k = e^{i phi_k} |r><1| + h.c.   on row k's atom,
    dH/dDelta_k = -|r><r|                      on row k's atom,

at the steps whose midpoint lies in row k's interval [t0, t1).  With
A = <target|psi_N> and chi_n = U_{n+1}^H ... U_N^H target,

    dF/dtheta = 2 Re( conj(A) sum_n <chi_n| D exp(-i dt H_n)[dH_n/dtheta] |psi_{n-1}> ),

where the derivative of the matrix exponential of the Hermitian H_n = W
diag(lambda) W^H is the Daleckii-Krein formula
D f(H)[E] = W (Gamma o (W^H E W)) W^H, Gamma_ab = (f(lambda_a) -
f(lambda_b)) / (lambda_a - lambda_b), and f'(lambda_a) on the diagonal and
for equal eigenvalues, with f(x) = exp(-i dt x).

Pins: central finite differences of the same discrete map, the single-atom
Rabi closed form dP_r/dOmega = T sin(2 Omega T), the vanishing derivative in
the detuning at zero detuning, and the TTN oracle in its exact regime
(tests/test_oracle_adjoint.py).
"""
import numpy as np

from . import exact, model

FIELDS = {"omega_r": model.SEG_OR, "delta": model.SEG_DELTA}


def _local(op, i, n):
    """Dense operator of the 3x3 `op` on atom i of n (atom 0 fastest)."""
    return np.kron(np.kron(np.eye(3 ** (n - 1 - i)), op), np.eye(3 ** i))


def fidelity(psi0, target, V, schedule, t0, dt, n_steps):
    """|<target|psi_N>|^2 after n_steps exact steps (exact.evolve)."""
    psi = exact.evolve(np.asarray(psi0, np.complex128), V, schedule, t0, dt, n_steps)
    return float(abs(np.vdot(target, psi)) ** 2)


def fidelity_gradient(psi0, target, V, schedule, params, t0, dt, n_steps):
    """(F, dF/dtheta) for theta = [schedule[row][field] for (row, field) in params],
    field "omega_r" or "delta".  Dense: at most 6 atoms."""
    n = V.shape[0]
    if n > 6:
        raise ValueError("the dense adjoint oracle is limited to 6 atoms")
    sched = np.asarray(schedule, dtype=np.float64).reshape(-1, 8)
    dops = []
    for row, field in params:
        if field not in FIELDS:
            raise ValueError("unknown parameter field %r" % (field,))
        a = int(sched[row, model.SEG_ATOM])
        if field == "omega_r":
            e = np.exp(1j * sched[row, model.SEG_PHI])
            op = e * model.RP + np.conj(e) * model.RP.conj().T
        else:
            op = -model.NR
        dops.append((row, _local(op, a, n)))
    # forward: states before every step and the eigendecompositions
    psi = np.asarray(psi0, np.complex128)
    before, eig = [], []
    for s in range(n_steps):
        tm = t0 + (s + 0.5) * dt
        lam, W = np.linalg.eigh(exact.hamiltonian(V, sched, tm).toarray())
        before.append(psi)
        eig.append((lam, W, tm))
        psi = W @ (np.exp(-1j * dt * lam) * (W.conj().T @ psi))
    A = np.vdot(target, psi)
    grad = np.zeros(len(params))
    chi = np.asarray(target, np.complex128)
    for s in reversed(range(n_steps)):
        lam, W, tm = eig[s]
        f = np.exp(-1j * dt * lam)
        dl = lam[:, None] - lam[None, :]
        close = np.abs(dl) <= 1e-12 * max(1.0, float(np.max(np.abs(lam))))
        gam = np.where(close, -1j * dt * f[:, None] * np.ones_like(dl),
                       (f[:, None] - f[None, :]) / np.where(close, 1.0, dl))
        cu = W.conj().T @ chi
        pu = W.conj().T @ before[s]
        for p, (row, E) in enumerate(dops):
            if not (sched[row, model.SEG_T0] <= tm < sched[row, model.SEG_T1]):
                continue
            term = np.vdot(cu, (gam * (W.conj().T @ E @ W)) @ pu)
            grad[p] += 2.0 * np.real(np.conj(A) * term)
        chi = W @ (np.conj(f) * cu)        # U_s^H chi
    return float(abs(A) ** 2), grad


def fd_gradient(psi0, target, V, schedule, params, t0, dt, n_steps, h=1e-6):
    """Central finite differences of the same discrete map (step h)."""
    sched = np.array(schedule, dtype=np.float64).reshape(-1, 8)
    g = np.zeros(len(params))
    for p, (row, field) in enumerate(params):
        col = FIELDS[field]
        plus, minus = sched.copy(), sched.copy()
        plus[row, col] += h
        minus[row, col] -= h
        g[p] = (fidelity(psi0, target, V, plus, t0, dt, n_steps) -
                fidelity(psi0, target, V, minus, t0, dt, n_steps)) / (2 * h)
    return g
