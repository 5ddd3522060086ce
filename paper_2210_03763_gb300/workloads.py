"""Seeded synthetic inputs: lattices, gate circuits and pulse schedules.

This module produces inputs only (positions, schedules, random states); it
holds none of the TDVP arithmetic and serves the CUDA path and the oracle
alike.  The paper's compiled circuits and its optimal-control CZ pulse are not
available, so circuits are generated here in their shape:

* GHZ preparation: Hadamard on a centre atom, then CNOTs along a breadth-first
  spanning tree of the nearest-neighbour grid (Sec. "Compiler for global GHZ
  states": H = R_Z(pi/2) R_X(pi/2) R_Z(pi/2), CNOT = 10 rotations + CZ(phi)).
  The printed CNOT decomposition equals CNOT up to a global phase only at
  phi = pi; the synthetic CZ pulse implements exactly CZ(pi) = diag(1,-1,-1,-1),
  so phi = pi is used.  Gate count: 3 + 11 (N - 1) (696 on 8x8, 168 on 4x4,
  the serial depths of Table II).
* CZ pulse: Jaksch-type pi (control) - 2pi (target) - pi (control) square
  pulses on the 1<->r transition with Rabi frequency Omega; T_CZ = 2 pi/Omega.
* Square pulses for rotations: R_X(theta) = exp(-i theta sx/2) is
  Omega^x = theta / (2 T_L) held for the layer time T_L = T_CZ; likewise R_Z.
* Layers: serial (one gate per layer) or greedy as-soon-as-possible with the
  minimum distance r_G between atoms of different CZ gates in one layer
  (Sec. "Parallel quantum algorithms").
* Five-qubit repetition codes: 5-atom GHZ preparations on disjoint connected
  groups cut from a snake path over the grid (Fig. 3 packs 12 codes on 8x8,
  more than plus shapes allow).

Schedule rows: (atom, t0, t1, omega_x, omega_z, omega_r, phase_r, delta), a
piecewise-constant segment active on [t0, t1); active rows of an atom add up.
"""
import math
from collections import deque

import numpy as np

PULSE_DTYPE = np.dtype([("atom", np.int32), ("t0", np.float64), ("t1", np.float64),
                        ("omega_x", np.float64), ("omega_z", np.float64),
                        ("omega_r", np.float64), ("phase_r", np.float64),
                        ("delta", np.float64)], align=True)


# ------------------------------------------------------------------ lattices
def square_lattice(Lx, Ly, a=1.0, jitter=0.0, seed=None):
    """Positions (x, y) of atom i = x + Lx*y with spacing a and optional
    Gaussian jitter of relative size ``jitter`` (seeded)."""
    xy = np.array([[a * (i % Lx), a * (i // Lx)] for i in range(Lx * Ly)], dtype=np.float64)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        xy = xy + jitter * a * rng.normal(size=xy.shape)
    return xy


def blockade_radius(C6, omega):
    """r_B = (|C6| / Omega)^(1/6)."""
    return (abs(C6) / omega) ** (1.0 / 6.0)


def random_product_amps(n_atoms, seed, levels=3):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n_atoms, levels)) + 1j * rng.normal(size=(n_atoms, levels))
    return a / np.linalg.norm(a, axis=1, keepdims=True)


def plus_state_amps(n_atoms):
    """Every atom in (|0> + |1>)/sqrt(2)."""
    a = np.zeros((n_atoms, 3), dtype=np.complex128)
    a[:, 0] = a[:, 1] = 1.0 / np.sqrt(2.0)
    return a


def random_ttn_tensors(shapes, seed):
    """Random TTN in canonical form with the centre at the last node (the root):
    every other node is a random isometry w.r.t. its parent leg (NumPy QR of a
    Gaussian matrix), the root a random unit-norm tensor.  ``shapes`` are the
    (d0, d1, d2) node shapes in node order."""
    rng = np.random.default_rng(seed)
    out = []
    for k, (d0, d1, d2) in enumerate(shapes):
        G = rng.normal(size=(d0 * d1, d2)) + 1j * rng.normal(size=(d0 * d1, d2))
        if k == len(shapes) - 1:
            X = G / np.linalg.norm(G)
        else:
            X, _ = np.linalg.qr(G)
        out.append(X.reshape(d0, d1, d2))
    return out


# ------------------------------------------------------------------- circuits
def _rx(q, th):
    return ("rx", (q,), th)


def _rz(q, th):
    return ("rz", (q,), th)


def hadamard(q):
    return [_rz(q, math.pi / 2), _rx(q, math.pi / 2), _rz(q, math.pi / 2)]


def cnot(c, t, phi=math.pi):
    """Time-ordered native gates of the CNOT decomposition (rightmost factor of
    the printed operator product acts first)."""
    printed = [_rx(c, math.pi), _rx(t, math.pi / 2), _rz(t, -math.pi / 2), _rx(t, math.pi / 2),
               ("cz", (c, t), phi),
               _rz(c, phi - 3 * math.pi / 2), _rx(c, math.pi), _rz(c, 3 * math.pi / 2),
               _rz(t, -phi - 3 * math.pi / 2), _rx(t, math.pi / 2), _rz(t, 3 * math.pi / 2)]
    return printed[::-1]


def bfs_tree(Lx, Ly, root, atoms=None):
    """Breadth-first (parent, child) edges over nearest neighbours."""
    allowed = set(range(Lx * Ly)) if atoms is None else set(atoms)
    seen = {root}
    edges = []
    dq = deque([root])
    while dq:
        p = dq.popleft()
        x, y = p % Lx, p // Lx
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            nx, ny = x + dx, y + dy
            if 0 <= nx < Lx and 0 <= ny < Ly:
                c = nx + Lx * ny
                if c in allowed and c not in seen:
                    seen.add(c)
                    edges.append((p, c))
                    dq.append(c)
    return edges


def ghz_circuit(Lx, Ly, root=None):
    if root is None:
        root = (Lx // 2) + Lx * (Ly // 2)
    gates = hadamard(root)
    for p, c in bfs_tree(Lx, Ly, root):
        gates += cnot(p, c)
    return gates


def repetition_code_groups(Lx, Ly, n_codes=None):
    """Disjoint connected 5-atom groups: consecutive runs of 5 cells along the
    boustrophedon (snake) path through the rows.  Gives 3 codes on 4x4 and 12
    on 8x8 with 1 and 4 idle atoms, the densities of Fig. 3."""
    path = []
    for y in range(Ly):
        xs = range(Lx) if y % 2 == 0 else range(Lx - 1, -1, -1)
        path += [x + Lx * y for x in xs]
    groups = [path[5 * g:5 * g + 5] for g in range(len(path) // 5)]
    return groups if n_codes is None else groups[:n_codes]


def repetition_code_circuit(Lx, Ly, n_codes=None):
    """GHZ on each 5-atom group: Hadamard on the group's middle atom, then CNOTs
    along a breadth-first tree inside the group."""
    gates = []
    for grp in repetition_code_groups(Lx, Ly, n_codes):
        root = grp[2]
        gates += hadamard(root)
        for p, c in bfs_tree(Lx, Ly, root, grp):
            gates += cnot(p, c)
    return gates


def schedule_layers(gates, xy=None, r_G=None):
    """Serial (r_G None) or greedy ASAP layering with the CZ distance rule."""
    if r_G is None:
        return [[g] for g in gates]
    layers = []
    busy = {}
    for g in gates:
        lay = max((busy.get(q, -1) + 1 for q in g[1]), default=0)
        while True:
            while lay >= len(layers):
                layers.append([])
            ok = all(q not in h[1] for h in layers[lay] for q in g[1])
            if ok and g[0] == "cz":
                for h in layers[lay]:
                    if h[0] != "cz":
                        continue
                    for q in g[1]:
                        for r in h[1]:
                            if np.hypot(*(xy[q] - xy[r])) < r_G - 1e-12:
                                ok = False
            if ok:
                break
            lay += 1
        layers[lay].append(g)
        for q in g[1]:
            busy[q] = lay
    return layers


def layers_to_schedule(layers, omega=1.0, t0=0.0):
    """Pulse schedule (rows as in the module docstring) and the layer time."""
    TL = 2 * math.pi / omega
    rows = []
    for li, layer in enumerate(layers):
        s = t0 + li * TL
        for kind, qs, th in layer:
            if kind == "rx":
                rows.append([qs[0], s, s + TL, th / (2 * TL), 0, 0, 0, 0])
            elif kind == "rz":
                rows.append([qs[0], s, s + TL, 0, th / (2 * TL), 0, 0, 0])
            else:
                c, t = qs
                q = TL / 4
                rows.append([c, s, s + q, 0, 0, omega, 0, 0])
                rows.append([t, s + q, s + 3 * q, 0, 0, omega, 0, 0])
                rows.append([c, s + 3 * q, s + TL, 0, 0, omega, 0, 0])
    return np.array(rows, dtype=np.float64).reshape(-1, 8), TL


def to_pulse_array(schedule):
    """Schedule rows -> array of the C struct ttn_pulse."""
    sched = np.asarray(schedule, dtype=np.float64).reshape(-1, 8)
    out = np.zeros(sched.shape[0], dtype=PULSE_DTYPE)
    out["atom"] = sched[:, 0].astype(np.int32)
    for j, name in enumerate(PULSE_DTYPE.names[1:], start=1):
        out[name] = sched[:, j]
    return out


def segmented_cz_schedule(pairs, n_seg, seed, omega=1.0, t0=0.0):
    """CZ gates one after another, each as the Jaksch pulse sequence (pi on the
    control, 2 pi on the target, pi on the control; gate time 2 pi / omega)
    cut into n_seg equal piecewise-constant segments whose Rabi amplitudes are
    drawn from N(omega, 0.1 omega) and detunings from N(0, 0.1 omega), seeded:
    the inputs of gradient runs over pulse amplitudes.  n_seg must be a
    multiple of 4 so that segments do not straddle the sub-pulses.  Returns
    (rows, gate time); rows as in the module docstring."""
    if n_seg % 4:
        raise ValueError("n_seg must be a multiple of 4")
    rng = np.random.default_rng(seed)
    TG = 2 * math.pi / omega
    rows = []
    for g, (c, t) in enumerate(pairs):
        base = t0 + g * TG
        for k in range(n_seg):
            s0, s1 = base + k * TG / n_seg, base + (k + 1) * TG / n_seg
            atom = t if n_seg // 4 <= k < 3 * n_seg // 4 else c
            rows.append([atom, s0, s1, 0.0, 0.0, rng.normal(omega, 0.1 * omega), 0.0,
                         rng.normal(0.0, 0.1 * omega)])
    return np.array(rows, dtype=np.float64), TG


def random_constant_schedule(n_atoms, seed, t1=1e9, scale=1.0, atoms=None):
    """One constant segment per atom with seeded Gaussian amplitudes."""
    rng = np.random.default_rng(seed)
    rows = []
    for a in (range(n_atoms) if atoms is None else atoms):
        rows.append([a, 0.0, t1, scale * rng.normal(), scale * rng.normal(),
                     scale * rng.normal(), rng.uniform(0, 2 * math.pi), scale * rng.normal()])
    return np.array(rows, dtype=np.float64).reshape(-1, 8)


def cz_layer_workload(Lx, Ly, r_G, omega=1.0):
    """First layer of the greedy GHZ schedule that holds CZ gates, shifted to t = 0:
    a parallel CZ layer on a lattice (the steady state of the GHZ circuits)."""
    xy = square_lattice(Lx, Ly)
    layers = schedule_layers(ghz_circuit(Lx, Ly), xy, r_G)
    best = max(layers, key=lambda L: sum(1 for g in L if g[0] == "cz"))
    sched, TL = layers_to_schedule([best], omega)
    return sched, TL
