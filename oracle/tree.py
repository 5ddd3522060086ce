"""Binary tree over a Hilbert-curve ordering of the lattice (Sec. "Tensor network
simulations"; padding rule from Sec. "Parallel quantum algorithms").

* Leaves: the Lx*Ly atoms in the order the Hilbert curve of the smallest
  2^n x 2^n grid that holds the lattice visits them, followed by padding leaves
  up to the next power of two (>= 2).  Padding leaves hold no atom, sit in |0>,
  carry no Hamiltonian term and are never driven.
* Level-0 nodes pair leaves (2i, 2i+1); level-l nodes pair level-(l-1) nodes;
  the single top node is the root, whose parent leg is a dummy leg of dim 1
  (the paper does not fix the tree shape: a balanced binary tree is used).
* Bond dimension of the parent leg of a node whose subtree holds the atom set S:
  D = min(chi, 3^|S|, 3^|complement of S|) (only real atoms count).

Hilbert curve: the iterative index->(x, y) map, starting at the (0, 0) corner
(the paper does not fix the orientation).  Written here from the curve's recursive definition; the CUDA
library has its own copy and a test checks that the two agree.
"""
import numpy as np


def hilbert_d2xy(side, d):
    """Cell (x, y) visited at step d of the Hilbert curve on a side x side grid."""
    x = y = 0
    s = 1
    t = d
    while s < side:
        rx = 1 & (t // 2)
        ry = 1 & (t ^ rx)
        if ry == 0:                       # rotate the quadrant
            if rx == 1:
                x = s - 1 - x
                y = s - 1 - y
            x, y = y, x
        x += s * rx
        y += s * ry
        t //= 4
        s *= 2
    return x, y


def leaf_atoms(Lx, Ly):
    """Atom id (x + Lx*y) per leaf, -1 for padding leaves."""
    side = 1
    while side < max(Lx, Ly):
        side *= 2
    order = []
    for d in range(side * side):
        x, y = hilbert_d2xy(side, d)
        if x < Lx and y < Ly:
            order.append(x + Lx * y)
    n_leaves = 2
    while n_leaves < len(order):
        n_leaves *= 2
    return order + [-1] * (n_leaves - len(order))


def _pow3_capped(k, cap):
    v = 1
    for _ in range(k):
        v *= 3
        if v >= cap:
            return cap
    return v


class Tree:
    """Node k has ``children[k]`` = two entries, each ('leaf', leaf) or ('node', id),
    ``parent[k]`` (-1 for the root), ``sites[k]`` = real atoms under it in leaf order."""

    def __init__(self, Lx, Ly, chi):
        self.Lx, self.Ly, self.chi = Lx, Ly, chi
        self.leaf_atom = leaf_atoms(Lx, Ly)
        self.n_atoms = Lx * Ly
        self.children, self.parent, self.sites, self.level = [], [], [], []
        level_nodes = []
        cur = []
        for i in range(len(self.leaf_atom) // 2):
            k = self._add([("leaf", 2 * i), ("leaf", 2 * i + 1)], 0)
            cur.append(k)
        level_nodes.append(cur)
        lev = 0
        while len(cur) > 1:
            lev += 1
            nxt = []
            for i in range(len(cur) // 2):
                k = self._add([("node", cur[2 * i]), ("node", cur[2 * i + 1])], lev)
                nxt.append(k)
            cur = nxt
            level_nodes.append(cur)
        self.root = cur[0]
        self.level_nodes = level_nodes
        # bond dimension of every node's parent leg
        n_real = self.n_atoms
        self.dim = []
        for k in range(len(self.children)):
            a = len(self.sites[k])
            if k == self.root:
                self.dim.append(1)
            else:
                self.dim.append(min(chi, _pow3_capped(a, chi + 1),
                                    _pow3_capped(n_real - a, chi + 1)))

    def _add(self, ch, level):
        k = len(self.children)
        self.children.append(ch)
        self.parent.append(-1)
        self.level.append(level)
        s = []
        for kind, idx in ch:
            if kind == "leaf":
                if self.leaf_atom[idx] >= 0:
                    s.append(self.leaf_atom[idx])
            else:
                self.parent[idx] = k
                s.extend(self.sites[idx])
        self.sites.append(s)
        return k

    @property
    def n_nodes(self):
        return len(self.children)

    def leg_dim(self, k, leg):
        """Dimension of leg 0/1 (children) or 2 (parent) of node k."""
        if leg == 2:
            return self.dim[k]
        kind, idx = self.children[k][leg]
        return 3 if kind == "leaf" else self.dim[idx]

    def shape(self, k):
        return tuple(self.leg_dim(k, u) for u in range(3))

    def leg_sites(self, k, leg):
        """Real atoms behind leg ``leg`` of node k, in leaf order."""
        if leg == 2:
            inside = set(self.sites[k])
            return [a for a in self.leaf_atom if a >= 0 and a not in inside]
        kind, idx = self.children[k][leg]
        if kind == "leaf":
            a = self.leaf_atom[idx]
            return [a] if a >= 0 else []
        return list(self.sites[idx])
