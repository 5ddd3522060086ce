"""Gradients of the final-state fidelity with respect to piecewise-constant
pulse parameters on the GPU (ttn_fidelity_gradient, and its torch.autograd
binding) against the oracle:

* exact regime (2x2, chi = 16; 3x2, chi = 27: every bond complete, TDVP is
  the exact step exp(-i H dt)): F and dF/dOmega_k, dF/dDelta_k of two
  segmented CZ pulses (8 segments each, seed-random amplitudes, the
  adjoint config's recipe) against oracle.adjoint, the state-vector reverse
  pass with the Daleckii-Krein derivative of each step, held to 1e-8 of the
  largest derivative (8-point Gauss-Legendre in the step integral);
* the same gradient against central finite differences of the GPU's own
  discrete map (h = 1e-6);
* checkpointing every step and every sqrt(N) steps give the same gradient;
* truncated regime (4x4, chi = 16, one segmented CZ pulse, 48 steps): the
  adjoint of the projected dynamics against central differences of the
  discrete TDVP map, 2e-4 of the largest derivative (measured 6e-5 at
  chi = 16, 3e-5 at chi = 64: the difference is how the discrete map also
  moves through its gauge, completions and projectors, which the adjoint
  does not differentiate), and split precision against FP64, 5e-6 (measured
  8e-7 at chi = 64);
* the torch.autograd.Function returns the ABI gradient;
* argument errors (decay on, a row outside the schedule, a bad field).
"""
import math

import numpy as np
import pytest

from oracle import adjoint, exact, model
from paper_2210_03763_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    return nat


def _setup(native, Lx, Ly, chi, pairs):
    N = Lx * Ly
    xy = W.square_lattice(Lx, Ly)
    sched, TG = W.segmented_cz_schedule(pairs, 8, seed=7)
    dt = TG / 24
    n_steps = 24 * len(pairs)
    plus = np.tile(np.array([1.0, 1.0, 0.0]) / math.sqrt(2), (N, 1))
    tamps = W.random_product_amps(N, 5)
    g = native.TTN(Lx, Ly, chi)
    g.set_precision(native.FP64)
    g.set_hamiltonian(xy, 20.0)
    g.apply_pulse(sched)
    g.set_product_state(plus)
    t = native.TTN(Lx, Ly, chi)
    t.set_product_state(tamps)
    params = [(r, f) for r in range(len(sched)) for f in ("omega_r", "delta")]
    return g, t, xy, sched, dt, n_steps, plus, tamps, params


@pytest.mark.parametrize("Lx,Ly,chi,pairs", [(2, 2, 16, [(0, 1), (1, 3)]), (3, 2, 27, [(0, 1), (1, 4)])])
def test_exact_regime_gradient_matches_oracle(native, Lx, Ly, chi, pairs):
    g, t, xy, sched, dt, n_steps, plus, tamps, params = _setup(native, Lx, Ly, chi, pairs)
    F, grad = g.fidelity_gradient(t, dt, n_steps, params, n_quad=8)
    V = model.pair_couplings(xy, 20.0)
    Fo, go = adjoint.fidelity_gradient(exact.product_state(plus), exact.product_state(tamps), V, sched,
                                       params, 0.0, dt, n_steps)
    assert abs(F - Fo) < 1e-12
    assert np.max(abs(grad - go)) <= 1e-8 * np.max(abs(go)), np.max(abs(grad - go)) / np.max(abs(go))
    g.close()
    t.close()


def test_gradient_matches_central_differences_and_checkpointing(native):
    g, t, xy, sched, dt, n_steps, plus, tamps, params = _setup(native, 2, 2, 16, [(0, 1), (1, 3)])
    params = params[::5]
    F, grad = g.fidelity_gradient(t, dt, n_steps, params, n_quad=8)
    F1, grad1 = g.fidelity_gradient(t, dt, n_steps, params, n_quad=8, checkpoint_every=1)
    assert F1 == F
    assert np.max(abs(grad1 - grad)) <= 1e-13 * np.max(abs(grad))
    h = 1e-6
    fd = np.zeros(len(params))
    for p, (r, f) in enumerate(params):
        col = 5 if f == "omega_r" else 7
        vals = []
        for sgn in (1, -1):
            s2 = sched.copy()
            s2[r, col] += sgn * h
            g.apply_pulse(s2)
            g.set_product_state(plus)
            for _ in range(n_steps):
                g.step(dt)
            vals.append(g.fidelity(t))
        fd[p] = (vals[0] - vals[1]) / (2 * h)
    assert np.max(abs(grad - fd)) <= 1e-6 * np.max(abs(fd)), np.max(abs(grad - fd)) / np.max(abs(fd))
    g.close()
    t.close()


def _truncated(native, prec):
    Lx = Ly = 4
    N = 16
    xy = W.square_lattice(Lx, Ly)
    sched, TG = W.segmented_cz_schedule([(5, 6)], 8, seed=7)
    dt = TG / 48
    plus = np.tile(np.array([1.0, 1.0, 0.0]) / math.sqrt(2), (N, 1))
    tamps = W.random_product_amps(N, 5)
    tamps[:, 2] = 0.0
    tamps /= np.linalg.norm(tamps, axis=1, keepdims=True)
    g = native.TTN(Lx, Ly, 16)
    g.set_precision(prec)
    g.set_hamiltonian(xy, 20.0)
    g.apply_pulse(sched)
    g.set_product_state(plus)
    t = native.TTN(Lx, Ly, 16)
    t.set_product_state(tamps)
    return g, t, sched, dt, 48, plus


def test_truncated_regime_against_differences_and_split(native):
    params = [(0, "omega_r"), (1, "delta"), (3, "omega_r"), (4, "omega_r"), (5, "delta"), (7, "omega_r")]
    g, t, sched, dt, n_steps, plus = _truncated(native, native.FP64)
    F, grad = g.fidelity_gradient(t, dt, n_steps, params)
    h = 1e-6
    fd = np.zeros(len(params))
    for p, (r, f) in enumerate(params):
        col = 5 if f == "omega_r" else 7
        vals = []
        for sgn in (1, -1):
            s2 = sched.copy()
            s2[r, col] += sgn * h
            g.apply_pulse(s2)
            g.set_product_state(plus)
            for _ in range(n_steps):
                g.step(dt)
            vals.append(g.fidelity(t))
        fd[p] = (vals[0] - vals[1]) / (2 * h)
    assert np.max(abs(grad - fd)) <= 2e-4 * np.max(abs(fd)), np.max(abs(grad - fd)) / np.max(abs(fd))
    g.close()
    t.close()
    gs, ts, _, _, _, _ = _truncated(native, native.SPLIT_TF32X3)
    Fs, grads = gs.fidelity_gradient(ts, dt, n_steps, params)
    assert abs(Fs - F) <= 1e-5 * F
    assert np.max(abs(grads - grad)) <= 5e-6 * np.max(abs(grad)), np.max(abs(grads - grad)) / np.max(abs(grad))
    gs.close()
    ts.close()


def test_autograd_function_returns_the_abi_gradient(native):
    torch = pytest.importorskip("torch")
    from paper_2210_03763_gb300 import gradients
    g, t, xy, sched, dt, n_steps, plus, tamps, params = _setup(native, 2, 2, 16, [(0, 1)])
    params = params[:6]
    prob = gradients.PulseProblem(g, t, sched, params, dt, n_steps, plus, n_quad=8)
    theta = torch.tensor(prob.initial_theta(), dtype=torch.float64, requires_grad=True)
    F = gradients.fidelity(theta, prob)
    F.backward()
    g.apply_pulse(sched)
    g.set_product_state(plus)
    F0, g0 = g.fidelity_gradient(t, dt, n_steps, params, n_quad=8)
    assert abs(float(F.detach()) - F0) < 1e-14
    assert np.allclose(theta.grad.numpy(), g0, rtol=0, atol=1e-14)
    g.close()
    t.close()


def test_gradient_arguments(native):
    g, t, xy, sched, dt, n_steps, plus, tamps, params = _setup(native, 2, 2, 16, [(0, 1)])
    with pytest.raises(native.TTNError):
        g.fidelity_gradient(t, dt, n_steps, [(len(sched), "delta")])
    with pytest.raises(native.TTNError):
        g.fidelity_gradient(t, dt, n_steps, [(0, 7)])
    with pytest.raises(native.TTNError):
        g.fidelity_gradient(t, dt, n_steps, params[:2], n_quad=9)
    g.set_decay(0.1)
    with pytest.raises(native.TTNError):
        g.fidelity_gradient(t, dt, n_steps, params[:2])
    g.close()
    t.close()
