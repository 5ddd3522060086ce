"""Writes oracle_regression.txt: the CPU oracle's own results on fixed-seed
cases, stored so that a later change to the oracle's arithmetic shows up as
a failing regression test (tests/test_oracle_regression.py).  Calls only the
oracle and the seeded input generators.

    python tests/golden/make_oracle_regression.py > tests/golden/oracle_regression.txt
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

from oracle import ttn  # noqa: E402
from paper_2210_03763_gb300 import workloads as W  # noqa: E402


def cases():
    """(name, OracleTTN after its steps, initial TTN)."""
    # 2x2, chi = 16 (exact regime): first four layers of the GHZ-4 pulse circuit
    xy = W.square_lattice(2, 2)
    layers = W.schedule_layers(W.ghz_circuit(2, 2, root=0), xy, None)[:4]
    sched, TL = W.layers_to_schedule(layers, 1.0)
    amps = np.tile([1.0, 0.0, 0.0], (4, 1))
    o = ttn.OracleTTN(2, 2, 16, xy, 20.0)
    o.set_schedule(sched)
    o.set_product_state(amps)
    o0 = ttn.OracleTTN(2, 2, 16, xy, 20.0)
    o0.set_product_state(amps)
    for _ in range(len(layers) * 20):
        o.step(TL / 20)
    yield "ghz4_2x2_chi16_4layers", o, o0
    # 4x4, chi = 16 (truncated): seeded constant drives, seeded product start
    for (Lx, Ly, chi, nst) in [(4, 4, 16, 5), (3, 3, 9, 5)]:
        xy = W.square_lattice(Lx, Ly)
        N = Lx * Ly
        amps = W.random_product_amps(N, 99)
        o = ttn.OracleTTN(Lx, Ly, chi, xy, 20.0)
        o.set_schedule(W.random_constant_schedule(N, 1234))
        o.set_product_state(amps)
        o0 = ttn.OracleTTN(Lx, Ly, chi, xy, 20.0)
        o0.set_product_state(amps)
        for _ in range(nst):
            o.step(0.02)
        yield "random_%dx%d_chi%d_%dsteps" % (Lx, Ly, chi, nst), o, o0


def values(o, o0):
    ov = o0.overlap(o)
    out = {"overlap_re": ov.real, "overlap_im": ov.imag, "norm": o.norm(), "energy": o.energy()}
    for i, p in enumerate(o.measure(2)):
        out["n_r_%d" % i] = p
    return out


if __name__ == "__main__":
    print("# CPU oracle (oracle/ttn.py) results on fixed-seed cases, written by")
    print("# tests/golden/make_oracle_regression.py; columns: case quantity value")
    for name, o, o0 in cases():
        for k, v in values(o, o0).items():
            print("%s %s %.17g" % (name, k, v))
