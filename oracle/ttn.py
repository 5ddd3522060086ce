"""Oracle-T: single-site TTN-TDVP for the Rydberg Hamiltonian, step by step.

Follows Sec. "Tensor network simulations": a binary TTN over the Hilbert-curve
ordering, evolved by the time-dependent variational principle, with the
Hamiltonian kept as a list of one-body terms and two-body n_i n_j terms
(a tensor product operator).  Readings of points the paper leaves open:

* A8  integrator: second-order symmetric recursive projector splitting.  One
      step of dt = a forward half-sweep with tau = dt/2 (post-order: children
      first, each child's link evolved backwards on the way up, the node
      evolved forwards last) followed by its exact reverse (pre-order,
      children in reverse order, links evolved backwards on the way down).
      H is frozen at the step midpoint t + dt/2.
* A9  single-site update at fixed bond dimensions D (the paper's two-tensor
      update is not the hot path).
* A10 rank-deficient bases are completed deterministically (linalg.qr_complete).
* A11 Krylov: linalg.krylov_expm, tol 1e-13, m_max 30.

Tensor conventions.  Node tensor X has shape (d0, d1, d2) for legs
(child 0, child 1, parent).  A leg matrix M acts as
Y[..a..] = sum_a' M[a, a'] X[..a'..].  Every environment stores, for the real
atoms S behind a leg, the static block Hamiltonian (all n_i n_j terms with
i, j in S) and the renormalised one-site operators n, sx, sz, |r><1| of every
atom in S; the time-dependent block Hamiltonian is assembled from them.

Parity note: the tensors are gauge dependent; only gauge-invariant outputs
(fidelity, overlaps, <n_i>, norm, energy) are compared across implementations,
unless both start from identical tensors.
"""
import numpy as np

from . import model
from .linalg import qr_complete, completion_order, krylov_expm
from .tree import Tree

KINDS = ("n", "sx", "sz", "rp")
BARE = {"n": model.NR, "sx": model.SX, "sz": model.SZ, "rp": model.RP}


class Env:
    def __init__(self, D):
        self.D = D
        self.H = np.zeros((D, D), dtype=np.complex128)
        self.sites = []
        self.ops = {}


def physical_env(atom, drive=True):
    """Leaf environment of one atom: n always; sx, sz, |r><1| unless
    ``drive`` is False (an atom that is never driven needs no drive operators;
    the sums they enter then have zero coefficients)."""
    e = Env(3)
    if atom >= 0:
        e.sites = [atom]
        for kind in KINDS if drive else ("n",):
            e.ops[(kind, atom)] = BARE[kind].copy()
    return e


def apply_leg(M, X, leg):
    """Y[..a..] = sum_a' M[a, a'] X[..a'..] on axis ``leg``."""
    return np.moveaxis(np.tensordot(M, X, axes=([1], [leg])), 0, leg)


def contract_conj(X, W, leg):
    """E[k, k'] = sum over the other legs of conj(X[..k..]) W[..k'..]."""
    others = [l for l in range(X.ndim) if l != leg]
    return np.tensordot(X.conj(), W, axes=(others, others))


def block_hamiltonian(env, coef, gamma=0.0):
    """H_block(t) = static part + sum over atoms of the drive terms of Eq. 1,
    and -i gamma n_i for every atom when the decay of Eq. 3 is on."""
    ox, oz, w, de = coef
    H = env.H.copy()
    for i in env.sites:
        if ("rp", i) not in env.ops:       # drive operators not kept: atom never driven
            assert ox[i] == 0 and oz[i] == 0 and w[i] == 0, "drive on atom %d without its operators" % i
            H -= (de[i] + 1j * gamma) * env.ops[("n", i)]
            continue
        rp = env.ops[("rp", i)]
        H += (ox[i] * env.ops[("sx", i)] + oz[i] * env.ops[("sz", i)]
              + w[i] * rp + np.conj(w[i]) * rp.conj().T
              - (de[i] + 1j * gamma) * env.ops[("n", i)])
    return H


def channel_list(env_u, env_v, V):
    """Cross terms between legs u and v: pairs (n_i^(u), G_i^(v)) with
    G_i^(v) = sum_{j in S_v} V_ij n_j^(v), one per atom i in S_u."""
    out = []
    for i in env_u.sites:
        G = np.zeros((env_v.D, env_v.D), dtype=np.complex128)
        nz = False
        for j in env_v.sites:
            if V[i, j] != 0.0:
                G += V[i, j] * env_v.ops[("n", j)]
                nz = True
        if nz:
            out.append((env_u.ops[("n", i)], G))
    return out


def renormalize(X, out_leg, env_u, env_v, V):
    """Environment seen through leg ``out_leg`` of X (X isometric w.r.t. that leg):
    E' = X^H (H_u + H_v + sum_{i in S_u, j in S_v} V_ij n_i n_j) X and
    E'_op = X^H op X for every stored one-site operator."""
    u, v = [l for l in range(3) if l != out_leg]
    W = apply_leg(env_u.H, X, u) + apply_leg(env_v.H, X, v)
    for n_i, G in channel_list(env_u, env_v, V):
        W = W + apply_leg(n_i, apply_leg(G, X, v), u)
    E = Env(X.shape[out_leg])
    E.H = contract_conj(X, W, out_leg)
    E.sites = list(env_u.sites) + list(env_v.sites)
    for leg, env in ((u, env_u), (v, env_v)):
        for key, op in env.ops.items():
            E.ops[key] = contract_conj(X, apply_leg(op, X, leg), out_leg)
    return E


def qr_leg(X, leg, allowed=(None, None)):
    """QR of X matricised with ``leg`` as columns; returns (Q as tensor, R).

    X[..a..] = sum_k Q[..k..] R[k, a].  ``allowed`` restricts the completion
    candidates of the two remaining legs (padding leaves: index 0 only)."""
    Xp = np.moveaxis(X, leg, 2)
    da, db, D = Xp.shape
    Q, R = qr_complete(Xp.reshape(da * db, D), completion_order(da, db, *allowed))
    return np.moveaxis(Q.reshape(da, db, D), 2, leg), R


class OracleTTN:
    def __init__(self, Lx, Ly, chi, xy=None, C6=0.0, r_cut=0.0, drive_atoms=None, amps=None):
        """``drive_atoms``: atoms whose drive operators (sx, sz, |r><1|) are
        carried through the environments; None keeps them for every atom.
        Restricting them only skips operators whose coefficients are zero (a
        drive on another atom is an error); measure(0) and measure(1) need
        every atom's sz.  ``amps``: the initial product state (N x 3), all
        atoms in |0> when None."""
        self.tree = Tree(Lx, Ly, chi)
        self.N = Lx * Ly
        if xy is None:
            xy = np.array([[i % Lx, i // Lx] for i in range(self.N)], dtype=float)
        self.V = model.pair_couplings(xy, C6, r_cut)
        self.schedule = None
        self.t = 0.0
        self.gamma = 0.0        # decay rate of Eq. 3 (0: closed system)
        keep = None if drive_atoms is None else set(int(a) for a in drive_atoms)
        self.phys = [physical_env(a, keep is None or a in keep) for a in self.tree.leaf_atom]
        self.T = [None] * self.tree.n_nodes
        self.up = [None] * self.tree.n_nodes
        self.down = [None] * self.tree.n_nodes
        self.krylov_stats = []
        self.set_product_state(np.tile([1.0, 0.0, 0.0], (self.N, 1)) if amps is None else amps)

    # ---------------------------------------------------------------- setup
    def set_hamiltonian(self, xy, C6, r_cut=0.0):
        self.V = model.pair_couplings(xy, C6, r_cut)
        self.rebuild_envs()

    def set_decay(self, gamma):
        """H_OQS = H - i gamma sum_i n_i (Eq. 3): the no-jump evolution of a
        decay out of the computational states; Krylov turns to Arnoldi."""
        self.gamma = float(gamma)

    def set_schedule(self, schedule):
        self.schedule = None if schedule is None else np.asarray(schedule, float).reshape(-1, 8)

    def coef(self, t):
        return model.coefficients(self.schedule, self.N, t)

    def allowed(self, k):
        """Completion candidates per child leg of node k: a padding leaf allows
        only |0>; any other leg allows every index."""
        out = []
        for kind, idx in self.tree.children[k]:
            out.append([0] if kind == "leaf" and self.tree.leaf_atom[idx] < 0 else None)
        return tuple(out)

    def env(self, k, leg):
        tr = self.tree
        if leg == 2:
            return Env(1) if k == tr.root else self.down[k]
        kind, idx = tr.children[k][leg]
        return self.phys[idx] if kind == "leaf" else self.up[idx]

    def _build_from_branches(self, leaf_branches, root_coef):
        """Node tensors from per-leaf branch vectors (3 x nb) combined with
        ``root_coef`` at the root; each node is the QR-completed isometry of its
        branch columns (the deterministic completion of rank-deficient bases)."""
        tr = self.tree
        B = {}
        for lev in tr.level_nodes:
            for k in lev:
                cols = []
                for leg in (0, 1):
                    kind, idx = tr.children[k][leg]
                    cols.append(leaf_branches[idx] if kind == "leaf" else B[k, idx])
                nb = cols[0].shape[1]
                d0, d1 = cols[0].shape[0], cols[1].shape[0]
                A = np.zeros((d0 * d1, nb), dtype=np.complex128)
                for b in range(nb):
                    A[:, b] = np.outer(cols[0][:, b], cols[1][:, b]).ravel()
                if k == tr.root:
                    self.T[k] = (A @ root_coef).reshape(d0, d1, 1)
                else:
                    D = tr.dim[k]
                    Af = np.zeros((d0 * d1, D), dtype=np.complex128)
                    Af[:, :min(nb, D)] = A[:, :min(nb, D)]
                    Q, R = qr_complete(Af, completion_order(d0, d1, *self.allowed(k)))
                    self.T[k] = Q.reshape(d0, d1, D)
                    Bk = np.zeros((D, nb), dtype=np.complex128)
                    Bk[:, :min(nb, D)] = R[:, :min(nb, D)]
                    if nb > D:          # branches beyond D are dependent here
                        Bk = Q.conj().T @ A
                    B[tr.parent[k], k] = Bk
        self.rebuild_envs()

    def set_product_state(self, amps):
        """Product state; amps[i] is the 3-vector of atom i, padding leaves in |0>."""
        amps = np.asarray(amps, dtype=np.complex128).reshape(self.N, 3)
        lb = []
        for a in self.tree.leaf_atom:
            v = amps[a] if a >= 0 else np.array([1, 0, 0], dtype=np.complex128)
            lb.append(v.reshape(3, 1))
        self._build_from_branches(lb, np.array([1.0 + 0j]))

    def set_ghz(self, mask, phase=0.0):
        """(|0..0> + e^{i phase} |1 on mask atoms, 0 elsewhere>)/sqrt(2) as an exact
        bond-dimension-2 TTN (Sec. "Tensor network simulations": GHZ has chi = 2)."""
        lb = []
        for a in self.tree.leaf_atom:
            m = np.zeros((3, 2), dtype=np.complex128)
            m[0, 0] = 1.0
            if a >= 0 and mask[a]:
                m[1, 1] = 1.0
            else:
                m[0, 1] = 1.0
            lb.append(m)
        self._build_from_branches(lb, np.array([1.0, np.exp(1j * phase)]) / np.sqrt(2.0))

    def set_tensors(self, tensors):
        self.T = [np.array(x, dtype=np.complex128) for x in tensors]
        self.rebuild_envs()

    def rebuild_envs(self):
        """All upward environments, bottom-up (centre at the root)."""
        tr = self.tree
        for lev in tr.level_nodes:
            for k in lev:
                if k != tr.root:
                    self.up[k] = renormalize(self.T[k], 2, self.env(k, 0),
                                             self.env(k, 1), self.V)

    # ------------------------------------------------------------ local maps
    def heff_setup(self, k, coef):
        envs = [self.env(k, u) for u in range(3)]
        Hb = [block_hamiltonian(e, coef, self.gamma) for e in envs]
        ch = []
        for u, v in ((0, 1), (0, 2), (1, 2)):
            for n_i, G in channel_list(envs[u], envs[v], self.V):
                ch.append((u, v, n_i, G))
        return Hb, ch

    @staticmethod
    def heff_apply(X, Hb, ch):
        """H_eff X = sum_u H_block(u) x_u X + sum_pairs sum_i n_i x_u (G_i x_v X)."""
        Y = apply_leg(Hb[0], X, 0) + apply_leg(Hb[1], X, 1) + apply_leg(Hb[2], X, 2)
        for u, v, n_i, G in ch:
            Y = Y + apply_leg(n_i, apply_leg(G, X, v), u)
        return Y

    def node_evolve(self, k, tau, coef):
        Hb, ch = self.heff_setup(k, coef)
        shape = self.T[k].shape
        f = lambda x: self.heff_apply(x.reshape(shape), Hb, ch).ravel()
        self.T[k] = krylov_expm(f, self.T[k].ravel(), -1j * tau, stats=self.krylov_stats,
                                hermitian=self.gamma == 0.0).reshape(shape)

    def link_evolve(self, R, env_r, env_c, tau, coef):
        """R <- exp(+i tau H_link) R, H_link R = Hr R + R Hc^T + sum_i n_i R G_i^T."""
        Hr = block_hamiltonian(env_r, coef, self.gamma)
        Hc = block_hamiltonian(env_c, coef, self.gamma)
        ch = channel_list(env_r, env_c, self.V)
        shape = R.shape

        def f(x):
            X = x.reshape(shape)
            Y = Hr @ X + X @ Hc.T
            for n_i, G in ch:
                Y = Y + n_i @ X @ G.T
            return Y.ravel()
        return krylov_expm(f, R.ravel(), 1j * tau, stats=self.krylov_stats,
                           hermitian=self.gamma == 0.0).reshape(shape)

    # ---------------------------------------------------------------- sweeps
    def _children_nodes(self, k):
        return [(u, idx) for u, (kind, idx) in enumerate(self.tree.children[k]) if kind == "node"]

    def _fwd(self, k, tau, coef):
        for u, c in self._children_nodes(k):
            self.T[k], R = qr_leg(self.T[k], u)                 # gauge move k -> c
            o = [l for l in range(3) if l != u]
            self.down[c] = renormalize(self.T[k], u, self.env(k, o[0]), self.env(k, o[1]), self.V)
            self.T[c] = apply_leg(R, self.T[c], 2)
            self._fwd(c, tau, coef)
            self.T[c], R = qr_leg(self.T[c], 2, self.allowed(c))  # c -> k
            self.up[c] = renormalize(self.T[c], 2, self.env(c, 0), self.env(c, 1), self.V)
            R = self.link_evolve(R, self.up[c], self.down[c], tau, coef)
            self.T[k] = apply_leg(R, self.T[k], u)
        self.node_evolve(k, tau, coef)

    def _rev(self, k, tau, coef):
        self.node_evolve(k, tau, coef)
        for u, c in reversed(self._children_nodes(k)):
            self.T[k], R = qr_leg(self.T[k], u)                 # k -> c
            o = [l for l in range(3) if l != u]
            self.down[c] = renormalize(self.T[k], u, self.env(k, o[0]), self.env(k, o[1]), self.V)
            R = self.link_evolve(R, self.down[c], self.up[c], tau, coef)
            self.T[c] = apply_leg(R, self.T[c], 2)
            self._rev(c, tau, coef)
            self.T[c], R = qr_leg(self.T[c], 2, self.allowed(c))  # gauge move c -> k
            self.up[c] = renormalize(self.T[c], 2, self.env(c, 0), self.env(c, 1), self.V)
            self.T[k] = apply_leg(R, self.T[k], u)

    def step(self, dt):
        coef = self.coef(self.t + 0.5 * dt)
        self._fwd(self.tree.root, 0.5 * dt, coef)
        self._rev(self.tree.root, 0.5 * dt, coef)
        self.t += dt

    # ----------------------------------------------------------- observables
    def norm(self):
        X = self.T[self.tree.root]
        return float(np.real(np.vdot(X, X)))

    def expect_op(self, kind):
        """<op_i> for every atom from the renormalised operators at the root."""
        out = np.zeros(self.N)
        r = self.tree.root
        X = self.T[r]
        for u in (0, 1):
            e = self.env(r, u)
            for i in e.sites:
                out[i] = np.real(np.vdot(X, apply_leg(e.ops[(kind, i)], X, u)))
        return out

    def measure(self, which):
        """which 0: <|0><0|>, 1: <|1><1|>, 2: <n> = <|r><r|> per atom.
        |0><0| = (1 - n + sz)/2 and |1><1| = (1 - n - sz)/2 on the qutrit."""
        n = self.expect_op("n")
        if which == 2:
            return n
        sz = self.expect_op("sz")
        nrm = self.norm()
        return 0.5 * (nrm - n + sz) if which == 0 else 0.5 * (nrm - n - sz)

    def energy(self, t=None):
        coef = self.coef(self.t if t is None else t)
        r = self.tree.root
        Hb, ch = self.heff_setup(r, coef)
        X = self.T[r]
        return float(np.real(np.vdot(X, self.heff_apply(X, Hb, ch))))

    def overlap(self, other):
        """<other|self> by bottom-up contraction of the two trees."""
        tr = self.tree
        M = {}
        for lev in tr.level_nodes:
            for k in lev:
                A, B = other.T[k], self.T[k]
                for leg in (0, 1):
                    kind, idx = tr.children[k][leg]
                    if kind == "node":
                        B = apply_leg(M[idx], B, leg)
                M[k] = np.tensordot(A.conj(), B, axes=([0, 1], [0, 1]))
        return complex(M[tr.root][0, 0])

    def fidelity(self, target):
        return abs(self.overlap(target)) ** 2

    def dense(self):
        """Full state vector, index sum_i s_i 3^i over atoms (padding leaves at |0>)."""
        tr = self.tree
        if self.N > 12:
            raise ValueError("dense() is for small lattices")
        V = {}
        for lev in tr.level_nodes:
            for k in lev:
                parts = []
                for leg in (0, 1):
                    kind, idx = tr.children[k][leg]
                    if kind == "leaf":
                        parts.append((np.eye(3), [idx]))
                    else:
                        parts.append(V[idx])
                (A, la), (Bm, lb) = parts
                X = self.T[k]
                # A: (leaves_a..., d0), Bm: (leaves_b..., d1)
                Y = np.tensordot(A, X, axes=([A.ndim - 1], [0]))       # la..., d1, D
                Y = np.tensordot(Bm, Y, axes=([Bm.ndim - 1], [len(la)]))  # lb..., la..., D
                na, nb = len(la), len(lb)
                perm = list(range(nb, nb + na)) + list(range(nb)) + [nb + na]
                V[k] = (np.transpose(Y, perm), la + lb)
        Y, leaves = V[tr.root]
        Y = Y[..., 0]
        # keep |0> on padding leaves, order axes by atom id (atom 0 fastest)
        idx = []
        keep = []
        for ax, leaf in enumerate(leaves):
            a = tr.leaf_atom[leaf]
            if a < 0:
                idx.append(0)
            else:
                idx.append(slice(None))
                keep.append(a)
        Y = Y[tuple(idx)]
        order = np.argsort(keep)
        Y = np.transpose(Y, order)
        return Y.reshape(-1, order="F")


# ------------------------------------------------------------- truncation
def bond_grams(o):
    """G_k(a, a') = <R_a|R_a'> for the parent bond of every non-root node k,
    where |psi> = sum_a |L_a> |R_a> with |L_a> the orthonormal subtree states
    (canonical form, centre at the root).  Top-down: the root's dummy leg
    has G = [[1]], and for node k, child u of p,
    G_k(a, a') = sum over p's other legs of conj(X_p(..a..)) (G_p x_2 X_p)(..a'..)."""
    tr = o.tree
    G = {tr.root: np.ones((1, 1), dtype=np.complex128)}
    for lev in reversed(tr.level_nodes):
        for p in lev:
            W = apply_leg(G[p], o.T[p], 2)
            for u, (kind, k) in enumerate(tr.children[p]):
                if kind == "node":
                    G[k] = contract_conj(o.T[p], W, u)
    return G


def compress(o, chi_new):
    """Truncation of every bond to the new tree's dimensions (bond dimension
    chi_new, Sec. "Tensor network simulations"): the kept basis of the parent
    bond of node k is the top eigenvectors U_k of its bond Gram G_k (the
    Schmidt basis of that bipartition); X_k <- U_c^H on its child legs, U_k
    on its parent leg (all bonds projected at once), then QR bottom-up
    restores the canonical form (centre at the root).  Returns the new
    OracleTTN and the discarded weight of every bond,
    sum of dropped eigenvalues / trace."""
    tr = o.tree
    new = OracleTTN(tr.Lx, tr.Ly, chi_new)
    new.V = o.V
    new.schedule = o.schedule
    new.gamma = o.gamma
    new.t = o.t
    nt = new.tree
    G = bond_grams(o)
    U, disc = {}, {}
    for k in range(tr.n_nodes):
        if k == tr.root:
            continue
        lam, vec = np.linalg.eigh(G[k])
        order = np.argsort(-lam, kind="stable")
        lam, vec = lam[order], vec[:, order]
        # G_k is the transpose of the bond's reduced density matrix: its
        # eigenvectors are the conjugates of the Schmidt vectors
        keep = nt.dim[k]
        U[k] = vec[:, :keep].conj()
        tot = np.sum(np.clip(lam, 0, None))
        disc[k] = float(np.sum(np.clip(lam[keep:], 0, None)) / tot) if tot > 0 else 0.0
    T = []
    for k in range(tr.n_nodes):
        X = o.T[k]
        for u, (kind, c) in enumerate(tr.children[k]):
            if kind == "node":
                X = apply_leg(U[c].conj().T, X, u)
        if k != tr.root:
            X = apply_leg(U[k].T, X, 2)
        T.append(X)
    # canonical form: QR of every non-root node towards its parent, bottom-up
    for lev in nt.level_nodes:
        for k in lev:
            if k == nt.root:
                continue
            T[k], R = qr_leg(T[k], 2, new.allowed(k))
            p = nt.parent[k]
            u = 0 if nt.children[p][0] == ("node", k) else 1
            T[p] = apply_leg(R, T[p], u)
    new.set_tensors(T)
    return new, disc
