"""torch.autograd access to the library's adjoint (ttn_fidelity_gradient):
the final-state fidelity F(theta) = |<target|psi(T)>|^2 of a pulse schedule
as a differentiable function of piecewise-constant pulse parameters theta
(Rabi amplitudes Omega_k and detunings Delta_k of chosen schedule rows).

Argument marshalling only: the forward pass writes theta into the schedule,
re-applies it, resets the initial state and calls the C ABI, which runs the
TDVP steps, the backward propagation and the gradient on the GPU; backward
returns the stored gradient times the incoming one.

    prob = PulseProblem(ctx, target, schedule, params, dt, n_steps, psi0_amps)
    theta = torch.tensor(prob.initial_theta(), dtype=torch.float64, requires_grad=True)
    F = fidelity(theta, prob)
    F.backward()          # theta.grad = dF/dtheta
"""
import numpy as np

from . import native

_COLUMN = {"omega_r": 5, "delta": 7}   # columns of a schedule row (atom, t0, t1, ox, oz, or, phi, delta)


class PulseProblem:
    """A TTN context, its target, a schedule (rows of 8 numbers) and the
    differentiated entries params = [(row, "omega_r" | "delta"), ...]."""

    def __init__(self, ctx, target, schedule, params, dt, n_steps, psi0_amps, n_quad=6, checkpoint_every=0):
        self.ctx = ctx
        self.target = target
        self.schedule = np.array(schedule, dtype=np.float64).reshape(-1, 8)
        self.params = [(int(r), f) for r, f in params]
        for _, f in self.params:
            if f not in _COLUMN:
                raise ValueError("unknown parameter field %r" % (f,))
        self.dt = float(dt)
        self.n_steps = int(n_steps)
        self.psi0 = np.asarray(psi0_amps, dtype=np.complex128)
        self.n_quad = n_quad
        self.checkpoint_every = checkpoint_every
        self.t0 = 0.0

    def initial_theta(self):
        return np.array([self.schedule[r, _COLUMN[f]] for r, f in self.params])

    def evaluate(self, theta):
        """(F, dF/dtheta) at theta (numpy, length len(params))."""
        sched = self.schedule.copy()
        for (r, f), v in zip(self.params, np.asarray(theta, dtype=np.float64)):
            sched[r, _COLUMN[f]] = v
        self.ctx.apply_pulse(sched)
        self.ctx.set_product_state(self.psi0)
        return self.ctx.fidelity_gradient(self.target, self.dt, self.n_steps, self.params, self.n_quad,
                                          self.checkpoint_every)


def _function():
    import torch

    class _Fidelity(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, problem):
            F, g = problem.evaluate(theta.detach().cpu().numpy())
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return theta.new_tensor(F)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None

    return _Fidelity


_FN = None


def fidelity(theta, problem):
    """F(theta) as a torch scalar with gradient support."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(theta, problem)
