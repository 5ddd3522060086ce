"""Command-line self-tests of single kernels, for checking and profiling one
operation in isolation (no TTN context):

    python -m paper_2210_03763_gb300.selftest contract M N K [fp64|split] [reps]
        C = A B for seeded random complex A (M x K), B (K x N); prints the
        error of the chosen precision against the FP64 kernel.
    python -m paper_2210_03763_gb300.selftest qr M D [rank] [reps]
        the gauge-move QR of a seeded random M x D matrix of the given rank;
        prints the number of completed columns and the device time.

    python -m paper_2210_03763_gb300.selftest heff Lx Ly chi level [fp64|split] [reps]
        H_eff applied at the first node of tree level `level` of an Lx x Ly
        lattice (C6/a^6 = 20, all pairs, three driven atoms, seeded random
        isometric TTN); prints the per-launch records of the last call
        (index among its tensor-core launches, kind, shape, device ms).

`reps` repeats the call (the first one includes one-time set-up)."""
import sys

import numpy as np

from paper_2210_03763_gb300 import native


def main(argv):
    if len(argv) < 1 or argv[0] not in ("contract", "qr", "heff"):
        print(__doc__)
        return 2
    native.load()
    if argv[0] == "contract":
        M, N, K = (int(v) for v in argv[1:4])
        prec = native.FP64 if (len(argv) > 4 and argv[4] == "fp64") else native.SPLIT_TF32X3
        reps = int(argv[5]) if len(argv) > 5 else 1
        for _ in range(reps):
            err = native.selftest_contract(M, N, K, prec)
        print("contract %d x %d x %d %s: max rel err vs FP64 %.3e" %
              (M, N, K, "fp64" if prec == native.FP64 else "split", err))
        return 0
    if argv[0] == "heff":
        return heff(argv[1:])
    M, D = int(argv[1]), int(argv[2])
    rank = int(argv[3]) if len(argv) > 3 else D
    reps = int(argv[4]) if len(argv) > 4 else 1
    rng = np.random.default_rng(1)
    B = rng.normal(size=(M, rank)) + 1j * rng.normal(size=(M, rank))
    C = rng.normal(size=(rank, D)) + 1j * rng.normal(size=(rank, D))
    A = B @ C
    for _ in range(reps):
        Q, R, nd, ms = native.selftest_qr(A)
    print("qr %d x %d rank %d: %d completed columns, %.3f ms, max|Q^H Q - I| %.2e" %
          (M, D, rank, nd, ms, np.max(abs(Q.conj().T @ Q - np.eye(D)))))
    return 0


def heff(argv):
    from paper_2210_03763_gb300 import workloads as W
    Lx, Ly, chi, level = (int(v) for v in argv[:4])
    prec = native.FP64 if (len(argv) > 4 and argv[4] == "fp64") else native.SPLIT_TF32X3
    reps = int(argv[5]) if len(argv) > 5 else 2
    N = Lx * Ly
    g = native.TTN(Lx, Ly, chi)
    g.set_precision(prec)
    g.set_hamiltonian(W.square_lattice(Lx, Ly), 20.0)
    g.apply_pulse(W.random_constant_schedule(N, 31, atoms=[0, N // 2, N - 1]))
    nn = g.num_nodes()
    shapes = [g.node_info(k)[0] for k in range(nn)]
    for k, X in enumerate(W.random_ttn_tensors(shapes, 41)):
        g.set_node(k, X)
    g.refresh_envs()
    # node ids per level: level-0 nodes first, then level 1, ... (root last)
    levels, start, width = [], 0, nn + 1
    while start < nn:
        width //= 2
        levels.append(list(range(start, start + max(1, width))))
        start += max(1, width)
    k = levels[level][0]
    rng = np.random.default_rng(5)
    X = rng.normal(size=shapes[k]) + 1j * rng.normal(size=shapes[k])
    try:   # an NVTX range around the last call lets a profiler select it
        import torch
        nvtx = torch.cuda.nvtx
    except Exception:
        nvtx = None
    for r in range(reps):
        last = r == reps - 1
        if last:
            g.profile_begin()
            if nvtx:
                nvtx.range_push("heff_last")
        g.apply_heff(k, X)
        if last and nvtx:
            nvtx.range_pop()
    g.profile_end()
    kinds = g.PROFILE_KINDS
    tc = 0
    print("node %d shape %s, records of the last call:" % (k, shapes[k]))
    for rec in g.profile_records():
        kind = int(rec[0])
        tag = ("tc#%d" % tc) if kind == 0 else "   "
        if kind == 0:
            tc += 1
        print("  %-6s %-10s M %6d N %6d K %6d batches %5d  %.3f ms" % (tag, kinds[kind], *[int(v) for v in rec[1:5]],
                                                                      rec[5]))
    print("tensor-core launches per call: %d" % tc)
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
