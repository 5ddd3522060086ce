"""Writes tests/golden/cfg2_trajectories.txt from the CPU oracle alone.

4x4 lattice, chi = 64, C6/a^6 = 20 with all 120 pairs: the GHZ circuit of
Sec. "Compiler for global GHZ states" scheduled serially and greedily with
the minimum CZ distance r_G = sqrt(8) a (Sec. "Parallel quantum algorithms").
Window: the serial schedule's first layer that holds a CZ gate, and the
greedy schedule's CZ layer with the most gates in parallel (at 4x4 and
r_G = sqrt(8) a no layer holds two CZ gates; rotations run beside the CZ),
each shifted so that the
24 steps straddle the end of the control atoms' pi pulse and the start of
the target atoms' 2 pi pulse (t = T_L/4 - 0.6 .. T_L/4 + 0.6 of the layer),
starting from a seeded random TTN with every bond at full rank (random
isometries, workloads.random_ttn_tensors): every pair interaction is active
and no QR of the sweep needs the completion of rank-deficient bases, whose
dependence decisions at the 1e-10 threshold make trajectories from product
states sensitive to rounding (reading A10).
24 single-site TDVP steps of dt = 0.05 (plain complex128 oracle).  Stored
per schedule: the return amplitude <psi(0)|psi(t)> (a gauge-invariant
functional of the whole state), <GHZ|psi> (GHZ target on
all 16 atoms, phase 0), the norm, the energy at the final time and
<|0><0|>, <|1><1|>, <n> per atom.

Usage: python tests/golden/make_cfg2_trajectories.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import ttn as ottn  # noqa: E402
from oracle.tree import Tree  # noqa: E402
from paper_2210_03763_gb300 import workloads as W  # noqa: E402

LX = LY = 4
CHI = 64
C6 = 20.0
DT = 0.05
STEPS = 24
SEED = 1234
SCHEDULES = (("serial", None), ("greedy", math.sqrt(8.0)))


def cfg2_schedule(r_G):
    xy = W.square_lattice(LX, LY)
    layers = W.schedule_layers(W.ghz_circuit(LX, LY), xy, r_G)
    ncz = [sum(1 for g in L if g[0] == "cz") for L in layers]
    if r_G is None:
        pick = next(i for i, n in enumerate(ncz) if n > 0)
    else:
        pick = max((i for i in range(len(layers)) if ncz[i] > 0), key=lambda i: (len(layers[i]), -i))
    TL = 2 * math.pi
    sched, _ = W.layers_to_schedule(layers[pick:pick + 2], 1.0, t0=-(TL / 4 - 0.5 * STEPS * DT))
    return xy, sched


def start_tensors():
    tr = Tree(LX, LY, CHI)
    return W.random_ttn_tensors([tr.shape(k) for k in range(tr.n_nodes)], SEED)


def main():
    lines = ["# cfg2 trajectories from oracle.ttn.OracleTTN (make_cfg2_trajectories.py)",
             "# lattice %dx%d chi %d C6 %g dt %g steps %d seed %d" % (LX, LY, CHI, C6, DT, STEPS, SEED)]
    Ts = start_tensors()
    for name, r_G in SCHEDULES:
        xy, sched = cfg2_schedule(r_G)
        o = ottn.OracleTTN(LX, LY, CHI, xy, C6)
        o.set_schedule(sched)
        o.set_tensors(Ts)
        for _ in range(STEPS):
            o.step(DT)
        start = ottn.OracleTTN(LX, LY, CHI, xy, C6)
        start.set_tensors(Ts)
        ret = o.overlap(start)
        tgt = ottn.OracleTTN(LX, LY, 2, xy, C6)
        tgt.set_ghz([1] * (LX * LY), 0.0)
        ov = o.overlap(tgt)
        lines.append("schedule %s" % name)
        lines.append("return %.17e %.17e" % (ret.real, ret.imag))
        lines.append("overlap %.17e %.17e" % (ov.real, ov.imag))
        lines.append("norm %.17e" % o.norm())
        lines.append("energy %.17e" % o.energy())
        for w in range(3):
            lines.append("measure%d %s" % (w, " ".join("%.17e" % v for v in o.measure(w))))
        lines.append("krylov_max_m %d" % max(m for m, _ in o.krylov_stats))
        print(name, ret, ov, o.norm(), o.energy(), flush=True)
    with open(os.path.join(HERE, "cfg2_trajectories.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
