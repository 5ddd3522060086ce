"""Projective measurement sampling (Sec. "Parallel quantum algorithms":
measurement histograms of 10^6 shots in the {|0>, |1>, |r>} basis of every
atom).  TEST INFRASTRUCTURE ONLY, like the rest of this package.

Every shot measures the atoms one after another in the TTN's leaf order
(Hilbert-curve order, padding leaves skipped) and draws atom i's outcome
from its conditional distribution given the outcomes already drawn, by
inverse transform sampling with the uniform number u[shot, i] in [0, 1):
outcome s is the first level with u < (P(0) + ... + P(s)) / (P(0) + P(1) +
P(2)).  The random numbers are inputs, so two implementations of the same
rule draw the same outcomes.

* ``sample_dense`` -- the definition: conditional marginals of |psi|^2 of
  the exact state vector (at most 9 atoms).
* ``sample_ttn``  -- the same rule on a TTN in canonical form (centre at the
  root): a depth-first walk where entering a subtree carries the Gram
  Gamma(a, a') = <R_a|R_a'> of the conditioned complement states of its
  parent bond, and leaving it returns the amplitude vector
  w(a) = <outcomes of the subtree|L_a> (parity with sample_dense is tested).
"""
import numpy as np


def _draw(p, u):
    p = np.clip(np.real(np.asarray(p, dtype=np.complex128)), 0.0, None)
    tot = p.sum()
    c = np.cumsum(p) / tot if tot > 0 else np.array([1.0, 1.0, 1.0])
    for s in range(len(p)):
        if u < c[s]:
            return s
    return len(p) - 1


def sample_dense(psi, n_atoms, order, uniforms):
    """Outcomes (shots x n_atoms, per atom id) from the state vector psi
    (index sum_i s_i 3^i), measuring the atoms in ``order``."""
    P = np.abs(psi.reshape([3] * n_atoms, order="F")) ** 2     # axis i = atom i
    shots = uniforms.shape[0]
    out = np.zeros((shots, n_atoms), dtype=np.int32)
    for sh in range(shots):
        Q = P
        fixed = {}
        for j, atom in enumerate(order):
            # marginal of `atom` given the fixed atoms: sum the others out
            idx = [slice(None)] * n_atoms
            for a, v in fixed.items():
                idx[a] = v
            sub = Q[tuple(idx)]
            remaining = [a for a in range(n_atoms) if a not in fixed]
            ax = remaining.index(atom)
            marg = np.moveaxis(sub, ax, 0).reshape(3, -1).sum(axis=1)
            s = _draw(marg, uniforms[sh, j])
            fixed[atom] = s
            out[sh, atom] = s
    return out


def sample_ttn(o, uniforms):
    """Outcomes (shots x N, per atom id) from the oracle TTN ``o`` (canonical
    form, centre at the root), atoms measured in leaf order."""
    tr = o.tree
    shots = uniforms.shape[0]
    out = np.zeros((shots, o.N), dtype=np.int32)
    for sh in range(shots):
        counter = [0]

        def leaf(idx, gamma):
            atom = tr.leaf_atom[idx]
            if atom < 0:                      # padding leaf: always |0>
                s = 0
            else:
                s = _draw(np.diag(gamma), uniforms[sh, counter[0]])
                counter[0] += 1
                out[sh, atom] = s
            w = np.zeros(3, dtype=np.complex128)
            w[s] = 1.0
            return w

        def visit(kind, idx, gamma):
            if kind == "leaf":
                return leaf(idx, gamma)
            X = o.T[idx]
            # Gamma of child 0's bond: sum over (c1, a, a') conj(X) Gamma X
            W = np.tensordot(X, gamma.T, axes=([2], [0]))        # W(c0', c1, a) = sum_a' X(c0',c1,a') G(a,a')
            g0 = np.tensordot(X.conj(), W, axes=([1, 2], [1, 2]))
            w0 = visit(*tr.children[idx][0], g0 / max(np.trace(g0).real, 1e-300))
            Y = np.tensordot(w0, X, axes=([0], [0]))             # Y(c1, a)
            g1 = (Y.conj() @ gamma) @ Y.T                         # G1(c1, c1') = sum conj(Y(c1,a)) G(a,a') Y(c1',a')
            w1 = visit(*tr.children[idx][1], g1 / max(np.trace(g1).real, 1e-300))
            w = w1 @ Y                                            # w(a) = sum_c1 w1(c1) Y(c1, a)
            n = np.linalg.norm(w)
            return w / n if n > 0 else w

        visit("node", tr.root, np.ones((1, 1), dtype=np.complex128))
    return out
