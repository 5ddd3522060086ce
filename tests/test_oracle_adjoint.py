"""Pins of the oracle gradient (oracle/adjoint.py): dF/dOmega_k, dF/dDelta_k
of the final-state fidelity of the discrete time-stepping map.

* single atom, |1> -> |r>: F = sin^2(Omega T), so the derivatives in the
  Rabi amplitudes of all segments add up to T sin(2 Omega T), and the
  derivative in a detuning vanishes at zero detuning (F is even in Delta);
* central finite differences of the same discrete map (h = 1e-6), held to
  1e-6 of the largest derivative (the bound asked of the gradients), on
  segmented CZ pulses of two and three interacting atoms;
* the TTN oracle in its exact regime (every bond at full rank): finite
  differences of its fidelity agree with the state-vector adjoint.
"""
import math

import numpy as np
import pytest

from oracle import adjoint, exact, model, ttn
from paper_2210_03763_gb300 import workloads as W

REL = 1e-6


def _cz_target(psi0, n, c, t):
    """Ideal CZ(pi) = diag(1, -1, -1, -1) on the qubit levels of atoms c, t."""
    T = psi0.reshape([3] * n, order="F").copy()
    idx = np.indices(T.shape)
    s = np.where((idx[c] == 1) | (idx[t] == 1), -1.0, 1.0)
    s = np.where((idx[c] == 2) | (idx[t] == 2), 0.0, s)
    out = (T * s).reshape(-1, order="F")
    return out / np.linalg.norm(out)


def test_single_atom_rabi_gradient_closed_form():
    V = np.zeros((1, 1))
    T, dt, Om = 1.3, 0.05, 0.7
    edges = np.linspace(0.0, T, 6)
    sched = np.array([[0, edges[k], edges[k + 1], 0, 0, Om, 0.3, 0.0] for k in range(5)])
    psi0 = exact.product_state([[0, 1, 0]])
    tgt = exact.product_state([[0, 0, 1]])
    params = [(k, "omega_r") for k in range(5)] + [(k, "delta") for k in range(5)]
    F, g = adjoint.fidelity_gradient(psi0, tgt, V, sched, params, 0.0, dt, int(round(T / dt)))
    assert abs(F - math.sin(Om * T) ** 2) < 1e-13
    assert abs(g[:5].sum() - T * math.sin(2 * Om * T)) < 1e-12
    assert np.max(np.abs(g[5:])) < 1e-13


@pytest.mark.parametrize("n_atoms,pairs", [(2, [(0, 1)]), (3, [(0, 1), (1, 2)])])
def test_adjoint_matches_central_differences(n_atoms, pairs):
    xy = W.square_lattice(n_atoms, 1)
    V = model.pair_couplings(xy, 20.0)
    sched, TG = W.segmented_cz_schedule(pairs, 8, seed=7)
    dt = TG / 24
    n_steps = 24 * len(pairs)
    plus = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    psi0 = exact.product_state(np.tile(plus, (n_atoms, 1)))
    tgt = psi0
    for c, t in pairs:
        tgt = _cz_target(tgt, n_atoms, c, t)
    params = [(k, f) for k in range(len(sched)) for f in ("omega_r", "delta")]
    F, g = adjoint.fidelity_gradient(psi0, tgt, V, sched, params, 0.0, dt, n_steps)
    fd = adjoint.fd_gradient(psi0, tgt, V, sched, params, 0.0, dt, n_steps)
    assert 0.0 < F <= 1.0
    assert np.max(np.abs(g - fd)) <= REL * np.max(np.abs(fd)), np.max(np.abs(g - fd)) / np.max(np.abs(fd))


def test_ttn_exact_regime_gradient_matches_adjoint():
    Lx, Ly, chi = 2, 2, 16                      # every bond at full rank: TDVP = exact steps
    xy = W.square_lattice(Lx, Ly)
    V = model.pair_couplings(xy, 20.0)
    sched, TG = W.segmented_cz_schedule([(0, 1)], 4, seed=3)
    dt = TG / 16
    n_steps = 16
    amps = np.tile(np.array([1.0, 1.0, 0.0]) / math.sqrt(2), (4, 1))
    psi0 = exact.product_state(amps)
    tgt = _cz_target(psi0, 4, 0, 1)
    params = [(0, "omega_r"), (1, "delta"), (2, "omega_r")]
    F, g = adjoint.fidelity_gradient(psi0, tgt, V, sched, params, 0.0, dt, n_steps)

    def ttn_fidelity(s):
        o = ttn.OracleTTN(Lx, Ly, chi, xy, 20.0)
        o.set_schedule(s)
        o.set_product_state(amps)
        for _ in range(n_steps):
            o.step(dt)
        return abs(np.vdot(tgt, o.dense())) ** 2

    h = 1e-6
    for p, (row, field) in enumerate(params):
        col = adjoint.FIELDS[field]
        sp, sm = sched.copy(), sched.copy()
        sp[row, col] += h
        sm[row, col] -= h
        fd = (ttn_fidelity(sp) - ttn_fidelity(sm)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(g[p])), (p, fd, g[p])
    assert abs(ttn_fidelity(sched) - F) < 1e-11
