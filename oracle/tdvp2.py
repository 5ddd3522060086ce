"""Oracle of the two-tensor TDVP (the paper's integrator, Sec. "Tensor network
simulations": the two-site update with truncation to the bond dimension chi).
TEST INFRASTRUCTURE ONLY, like the rest of this package.

The single-site oracle (ttn.OracleTTN) evolves every node forward and every
link backward.  Here every *edge* (c, k) between a node c and its parent k is
evolved forward as one two-site tensor

    Theta[a0, a1, o, p] = sum_b T_c[a0, a1, b] T_k[.. b on the leg of c ..]

(a0, a1: c's child legs; o: k's other child leg; p: k's parent leg) under the
two-site effective Hamiltonian of its four environments, and split again by a
singular value decomposition truncated to the edge's bond dimension D (and
to singular values sigma > eps sigma_max, eps = 1e-14).  Every node k is
evolved *backwards* (single site) once per edge it shares with the next edge
of the sweep: deg(k) - 1 times per half-sweep, deg(k) counting the edges at
k (node children and parent), so that the sequence of local exponentials is
the projector splitting of P = sum_edges P_edge - sum_nodes (deg - 1) P_node.

Half-sweeps (tau = dt / 2, H frozen at the step midpoint):
  forward  (post-order): for each node child c of k in order: move the
           centre to c, sweep c's subtree, evolve edge (c, k) forward and split
           with the centre on k, then evolve k backwards unless k is the root
           and c its last node child;
  reverse: the same local exponentials in the reverse order (each child in
           reverse order: backward step on k unless root and last child, edge
           forward with the centre going to c, sweep c's subtree backwards,
           move the centre back to k).
Splits: the isometry keeps the r <= D leading left singular vectors; when
r < D its remaining columns come from the deterministic completion rule of
linalg.qr_complete (candidates in (a+b, a) order, padding leaves offering
|0> only), so runs are reproducible; the other factor is the projection
Q^H Theta.  The discarded weight sum_{t >= r} sigma_t^2 / sum sigma^2 of
every split is recorded.
"""
import numpy as np

from .linalg import qr_complete, completion_order, krylov_expm
from .ttn import OracleTTN, apply_leg, block_hamiltonian, channel_list, renormalize, qr_leg

SVD_EPS = 1e-14


def _split(M, D, order):
    """M (m x n) = Q (Q^H M) with Q an m x D isometry spanning the r <= D
    leading left singular vectors of M (sigma > SVD_EPS sigma_max), completed
    deterministically; returns (Q, Q^H M, discarded weight)."""
    U, S, _ = np.linalg.svd(M, full_matrices=False)
    tot = float(np.sum(S ** 2))
    smax = S[0] if S.size else 0.0
    r = int(np.sum(S > SVD_EPS * smax)) if smax > 0 else 0
    r = max(1, min(D, r))
    A = np.zeros((M.shape[0], D), dtype=np.complex128)
    A[:, :r] = U[:, :r]
    Q, _ = qr_complete(A, order)
    disc = float(np.sum(S[r:] ** 2)) / tot if tot > 0 else 0.0
    return Q, Q.conj().T @ M, disc


class OracleTTN2(OracleTTN):
    """OracleTTN whose step() is the second-order two-tensor TDVP.  All
    observables, state setters and environments are the single-site
    oracle's; ``discarded`` collects the discarded weight of every split of
    the last step (``max_discarded`` its largest value)."""

    def __init__(self, *args, **kwargs):
        super().__init__(*args, **kwargs)
        self.discarded = []

    # ------------------------------------------------------------ edge maps
    def _leg_envs(self, c, k, u):
        """Environments of the four legs of Theta on edge (c, k), c = child u of k."""
        return [self.env(c, 0), self.env(c, 1), self.env(k, 1 - u), self.env(k, 2)]

    def _merge(self, c, k, u):
        Tk = np.moveaxis(self.T[k], u, 0)                 # (bond, other child, parent)
        return np.tensordot(self.T[c], Tk, axes=([2], [0]))

    def edge_heff_setup(self, c, k, u, coef):
        envs = self._leg_envs(c, k, u)
        Hb = [block_hamiltonian(e, coef, self.gamma) for e in envs]
        ch = []
        for x in range(4):
            for y in range(x + 1, 4):
                for n_i, G in channel_list(envs[x], envs[y], self.V):
                    ch.append((x, y, n_i, G))
        return Hb, ch

    @staticmethod
    def edge_heff_apply(Theta, Hb, ch):
        """H_eff Theta = sum_x H_block(x) x_x Theta + sum_{x<y} sum_i n_i x_x (G_i x_y Theta)."""
        Y = sum(apply_leg(Hb[x], Theta, x) for x in range(4))
        for x, y, n_i, G in ch:
            Y = Y + apply_leg(n_i, apply_leg(G, Theta, y), x)
        return Y

    def _edge_evolve(self, c, k, u, tau, coef, centre_on_parent):
        """exp(-i tau H_eff) on the two-site tensor of edge (c, k), split with
        the centre on k (forward sweep) or on c (reverse sweep)."""
        Th = self._merge(c, k, u)
        Hb, ch = self.edge_heff_setup(c, k, u, coef)
        shape = Th.shape
        f = lambda x: self.edge_heff_apply(x.reshape(shape), Hb, ch).ravel()
        Th = krylov_expm(f, Th.ravel(), -1j * tau, stats=self.krylov_stats,
                         hermitian=self.gamma == 0.0).reshape(shape)
        a0, a1, do, dp = shape
        D = self.tree.dim[c]
        if centre_on_parent:
            Q, rest, disc = _split(Th.reshape(a0 * a1, do * dp), D,
                                   completion_order(a0, a1, *self.allowed(c)))
            self.T[c] = Q.reshape(a0, a1, D)
            self.T[k] = np.moveaxis(rest.reshape(D, do, dp), 0, u)
            self.up[c] = renormalize(self.T[c], 2, self.env(c, 0), self.env(c, 1), self.V)
        else:
            M = Th.transpose(2, 3, 0, 1).reshape(do * dp, a0 * a1)
            Q, rest, disc = _split(M, D, completion_order(do, dp, self.allowed(k)[1 - u], None))
            self.T[k] = np.moveaxis(Q.reshape(do, dp, D), 2, u)
            self.T[c] = rest.T.reshape(a0, a1, D)
            o = [l for l in range(3) if l != u]
            self.down[c] = renormalize(self.T[k], u, self.env(k, o[0]), self.env(k, o[1]), self.V)
        self.discarded.append(disc)

    # ---------------------------------------------------------------- sweeps
    def _move_down(self, k, u, c):
        """Gauge move of the centre from k to its child c (leg u)."""
        self.T[k], R = qr_leg(self.T[k], u)
        o = [l for l in range(3) if l != u]
        self.down[c] = renormalize(self.T[k], u, self.env(k, o[0]), self.env(k, o[1]), self.V)
        self.T[c] = apply_leg(R, self.T[c], 2)

    def _move_up(self, c, k, u):
        """Gauge move of the centre from c back to its parent k."""
        self.T[c], R = qr_leg(self.T[c], 2, self.allowed(c))
        self.up[c] = renormalize(self.T[c], 2, self.env(c, 0), self.env(c, 1), self.V)
        self.T[k] = apply_leg(R, self.T[k], u)

    def _fwd2(self, k, tau, coef):
        kids = self._children_nodes(k)
        for i, (u, c) in enumerate(kids):
            self._move_down(k, u, c)
            self._fwd2(c, tau, coef)
            self._edge_evolve(c, k, u, tau, coef, centre_on_parent=True)
            if not (k == self.tree.root and i == len(kids) - 1):
                self.node_evolve(k, -tau, coef)              # backward single-site step

    def _rev2(self, k, tau, coef):
        kids = self._children_nodes(k)
        for i in reversed(range(len(kids))):
            u, c = kids[i]
            if not (k == self.tree.root and i == len(kids) - 1):
                self.node_evolve(k, -tau, coef)
            self._edge_evolve(c, k, u, tau, coef, centre_on_parent=False)
            self._rev2(c, tau, coef)
            self._move_up(c, k, u)

    def step(self, dt):
        """One second-order two-tensor TDVP step (centre at the root before
        and after)."""
        self.discarded = []
        coef = self.coef(self.t + 0.5 * dt)
        self._fwd2(self.tree.root, 0.5 * dt, coef)
        self._rev2(self.tree.root, 0.5 * dt, coef)
        self.t += dt

    @property
    def max_discarded(self):
        return max(self.discarded) if self.discarded else 0.0


def convergence(a, b):
    """C = 1 - |<a|b>|^2 / (<a|a> <b|b>) between two runs of the same circuit
    (Table I's convergence measure between bond dimensions or time steps)."""
    ov = a.overlap(b)
    return 1.0 - abs(ov) ** 2 / (a.norm() * b.norm())
