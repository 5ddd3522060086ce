"""Host logic of the autograd binding (paper_2210_03763_gb300.gradients), no
GPU: the parameter vector theta is read from and written to the schedule
columns of Omega_k (omega_r) and Delta_k (delta) of the chosen rows, and
unknown fields are rejected."""
import numpy as np
import pytest

from paper_2210_03763_gb300 import gradients, workloads as W


class _FakeCtx:
    """Records what the binding hands to the library."""

    def __init__(self):
        self.calls = []

    def apply_pulse(self, sched):
        self.calls.append(("apply_pulse", np.array(sched)))

    def set_product_state(self, amps):
        self.calls.append(("set_product_state", np.array(amps)))

    def fidelity_gradient(self, target, dt, n_steps, params, n_quad, checkpoint_every):
        self.calls.append(("fidelity_gradient", dt, n_steps, list(params), n_quad, checkpoint_every))
        return 0.5, np.arange(len(params), dtype=float)


def test_theta_maps_to_schedule_columns():
    sched, TG = W.segmented_cz_schedule([(0, 1)], 8, seed=7)
    params = [(0, "omega_r"), (3, "delta"), (5, "omega_r")]
    ctx = _FakeCtx()
    prob = gradients.PulseProblem(ctx, None, sched, params, TG / 24, 24, np.ones((2, 3)))
    th = prob.initial_theta()
    assert np.array_equal(th, [sched[0, 5], sched[3, 7], sched[5, 5]])
    F, g = prob.evaluate(th + 1.0)
    applied = ctx.calls[0][1]
    assert applied[0, 5] == sched[0, 5] + 1.0 and applied[3, 7] == sched[3, 7] + 1.0
    assert applied[5, 5] == sched[5, 5] + 1.0
    untouched = np.ones(sched.shape, dtype=bool)
    untouched[0, 5] = untouched[3, 7] = untouched[5, 5] = False
    assert np.array_equal(applied[untouched], sched[untouched])
    assert ctx.calls[1][0] == "set_product_state"
    assert ctx.calls[2][:3] == ("fidelity_gradient", TG / 24, 24)
    assert F == 0.5 and np.array_equal(g, [0.0, 1.0, 2.0])


def test_unknown_field_is_rejected():
    sched, _ = W.segmented_cz_schedule([(0, 1)], 8, seed=7)
    with pytest.raises(ValueError):
        gradients.PulseProblem(None, None, sched, [(0, "phase_r")], 0.1, 10, np.ones((2, 3)))


def test_autograd_backward_scales_the_stored_gradient():
    torch = pytest.importorskip("torch")
    sched, TG = W.segmented_cz_schedule([(0, 1)], 8, seed=7)
    params = [(0, "omega_r"), (1, "delta")]
    prob = gradients.PulseProblem(_FakeCtx(), None, sched, params, TG / 24, 24, np.ones((2, 3)))
    theta = torch.tensor(prob.initial_theta(), dtype=torch.float64, requires_grad=True)
    F = gradients.fidelity(theta, prob)
    (3.0 * F).backward()
    assert float(F.detach()) == 0.5
    assert np.array_equal(theta.grad.numpy(), [0.0, 3.0])
