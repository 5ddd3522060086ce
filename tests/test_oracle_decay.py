"""Pins of the open-system oracle (Eq. 3: H_OQS = H - i gamma sum n, the
no-jump evolution of a decay out of the computational states, Sec.
"Modeling 88Sr quantum computers").

* single driven atom: the closed form of exp(-i H t) on {|1>, |r>} with the
  non-Hermitian 2x2 generator [[0, W*], [W, -i gamma]];
* norm loss: d<psi|psi>/dt = -2 gamma sum_i <psi|n_i|psi> (the integrated
  Rydberg time T_R fixes the lost norm), by central differences on an
  interacting three-atom system;
* the TTN oracle with decay (Arnoldi) equals the exact state vector in the
  exact regime (every bond at full rank), and gamma = 0 is the closed system.
"""
import numpy as np
import pytest

from oracle import exact, model, ttn as ottn
from oracle.linalg import krylov_expm
from paper_2210_03763_gb300 import workloads as W


def test_single_atom_decay_closed_form():
    Om, gamma, phi = 0.9, 0.3, 0.4
    sched = np.array([[0, 0.0, 100.0, 0.0, 0.0, Om, phi, 0.0]])
    V = np.zeros((1, 1))
    psi0 = np.array([0, 1, 0], dtype=np.complex128)
    kappa = np.sqrt(Om ** 2 - gamma ** 2 / 4)
    for t in (0.3, 1.1, 2.7):
        psi = exact.step(psi0, V, sched, 0.0, t, gamma)
        e = np.exp(-gamma * t / 2)
        a1 = e * (np.cos(kappa * t) + gamma / (2 * kappa) * np.sin(kappa * t))
        ar = e * (-1j * Om * np.exp(1j * phi) * np.sin(kappa * t) / kappa)
        assert abs(psi[1] - a1) < 1e-13 and abs(psi[2] - ar) < 1e-13 and abs(psi[0]) < 1e-15


def test_norm_loss_equals_rydberg_population_rate():
    xy = W.square_lattice(3, 1)
    V = model.pair_couplings(xy, 2.0)
    sched = W.random_constant_schedule(3, 5)
    gamma = 0.07
    psi = exact.product_state(W.random_product_amps(3, 6))
    psi = exact.evolve(psi, V, sched, 0.0, 0.1, 5, gamma)
    h = 1e-4
    t = 0.5
    plus = exact.step(psi, V, sched, t, h, gamma)
    # backwards in time: exp(+i H h) psi, the inverse of one step of h
    H = exact.hamiltonian(V, sched, t, gamma).toarray()
    from scipy.linalg import expm
    minus = expm(1j * h * H) @ psi
    rate = (np.vdot(plus, plus).real - np.vdot(minus, minus).real) / (2 * h)
    nsum = exact.expectation_local(psi, 3, model.NR).sum()
    assert abs(rate + 2 * gamma * nsum) < 1e-8 * max(1.0, abs(rate))


def test_arnoldi_matches_dense_exponential():
    rng = np.random.default_rng(3)
    n = 40
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    H = (A + A.conj().T) / 2 - 0.2j * np.diag(rng.random(n))
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    from scipy.linalg import expm
    ref = expm(-0.05j * H) @ v
    got = krylov_expm(lambda x: H @ x, v, -0.05j, hermitian=False)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("Lx,Ly,chi", [(2, 2, 16), (2, 3, 81)])
def test_ttn_with_decay_equals_state_vector_in_exact_regime(Lx, Ly, chi):
    N = Lx * Ly
    xy = W.square_lattice(Lx, Ly)
    sched = W.random_constant_schedule(N, 2)
    amps = W.random_product_amps(N, 3)
    gamma = 0.2
    o = ottn.OracleTTN(Lx, Ly, chi, xy, 20.0)
    o.set_schedule(sched)
    o.set_decay(gamma)
    o.set_product_state(amps)
    V = model.pair_couplings(xy, 20.0)
    psi = exact.product_state(amps)
    dt = 0.02
    for s in range(3):
        o.step(dt)
        psi = exact.step(psi, V, sched, s * dt, dt, gamma)
    d = o.dense()
    nd, npsi = np.vdot(d, d).real, np.vdot(psi, psi).real
    # the exact-regime bound of the closed system (|1 - F| <= 1e-10, every
    # local exponential converged to 1e-13) on the normalised states, and
    # the norms, which the decay lowers, to the same level
    assert abs(1 - abs(np.vdot(psi, d)) ** 2 / (nd * npsi)) < 1e-10
    assert npsi < 1.0 - 1e-4
    assert abs(nd - npsi) < 1e-10
    assert abs(o.norm() - nd) < 1e-12
