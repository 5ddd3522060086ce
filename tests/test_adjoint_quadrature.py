"""The GPU adjoint (ttn_fidelity_gradient) evaluates each step's derivative
<chi_n| dU_n |psi_{n-1}> = -i int_0^dt <chi(s)| dH |psi(s)> ds by Gauss-Legendre
quadrature on sub-steps of the step's own Hamiltonian.  This CPU test
restates that method on the state vector (exact sub-step exponentials from an
eigendecomposition, Gauss-Legendre nodes from numpy) and checks it against
the oracle's Daleckii-Krein derivative of the discrete map
(oracle.adjoint.fidelity_gradient): the quadrature error falls by orders of
magnitude per added node pair and reaches rounding at 8 nodes on two-atom
segmented CZ pulses with C6/a^6 = 20 (measured relative errors 2.8e-2,
5.7e-5, 1.5e-8 and 1.1e-12 with 2, 4, 6 and 8 nodes; the GPU uses 6 by
default and 8 in its exact-regime tests)."""
import math

import numpy as np
import pytest

from oracle import adjoint, exact, model
from paper_2210_03763_gb300 import workloads as W


def _local(op, i, n):
    return np.kron(np.kron(np.eye(3 ** (n - 1 - i)), op), np.eye(3 ** i))


def _quadrature_gradient(psi0, target, V, sched, params, dt, n_steps, q):
    n = V.shape[0]
    x, w = np.polynomial.legendre.leggauss(q)
    s_nodes, s_w = 0.5 * dt * (1.0 + x), 0.5 * dt * w
    dops = []
    for row, field in params:
        a = int(sched[row, model.SEG_ATOM])
        if field == "omega_r":
            e = np.exp(1j * sched[row, model.SEG_PHI])
            op = e * model.RP + np.conj(e) * model.RP.conj().T
        else:
            op = -model.NR
        dops.append((row, _local(op, a, n)))
    psis, eigs = [], []
    psi = psi0.copy()
    for k in range(n_steps):
        tm = (k + 0.5) * dt
        lam, Wm = np.linalg.eigh(exact.hamiltonian(V, sched, tm).toarray())
        psis.append(psi)
        eigs.append((lam, Wm, tm))
        psi = Wm @ (np.exp(-1j * dt * lam) * (Wm.conj().T @ psi))
    A = np.vdot(target, psi)
    grad = np.zeros(len(params))
    chi = target.copy()
    for k in reversed(range(n_steps)):
        lam, Wm, tm = eigs[k]
        pu, cu = Wm.conj().T @ psis[k], Wm.conj().T @ chi
        for p, (row, E) in enumerate(dops):
            if not (sched[row, model.SEG_T0] <= tm < sched[row, model.SEG_T1]):
                continue
            acc = 0.0
            for s, ws in zip(s_nodes, s_w):
                ps = Wm @ (np.exp(-1j * s * lam) * pu)
                cs = Wm @ (np.exp(1j * (dt - s) * lam) * cu)
                acc += ws * np.vdot(cs, E @ ps)
            grad[p] += 2.0 * np.real(np.conj(A) * (-1j) * acc)
        chi = Wm @ (np.exp(1j * dt * lam) * cu)
    return abs(A) ** 2, grad


def test_quadrature_converges_to_the_discrete_derivative():
    xy = W.square_lattice(2, 1)
    V = model.pair_couplings(xy, 20.0)
    sched, TG = W.segmented_cz_schedule([(0, 1)], 8, seed=7)
    dt = TG / 24
    plus = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    psi0 = exact.product_state(np.tile(plus, (2, 1)))
    target = exact.product_state(W.random_product_amps(2, 5))
    params = [(k, f) for k in range(len(sched)) for f in ("omega_r", "delta")]
    F0, g0 = adjoint.fidelity_gradient(psi0, target, V, sched, params, 0.0, dt, 24)
    errs = {}
    for q in (2, 4, 6, 8):
        F, g = _quadrature_gradient(psi0, target, V, sched, params, dt, 24, q)
        assert abs(F - F0) < 1e-14
        errs[q] = np.max(abs(g - g0)) / np.max(abs(g0))
    assert errs[8] < 1e-11, errs
    assert errs[2] > errs[4] > errs[6] >= errs[8] * 0.1, errs
