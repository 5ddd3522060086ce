"""Command-line self-tests of single kernels, for checking and profiling one
operation in isolation (no TTN context):

    python -m paper_2210_03763_gb300.selftest contract M N K [fp64|split] [reps]
        C = A B for seeded random complex A (M x K), B (K x N); prints the
        error of the chosen precision against the FP64 kernel.
    python -m paper_2210_03763_gb300.selftest qr M D [rank] [reps]
        the gauge-move QR of a seeded random M x D matrix of the given rank;
        prints the number of completed columns and the device time.

`reps` repeats the call (the first one includes one-time set-up)."""
import sys

import numpy as np

from paper_2210_03763_gb300 import native


def main(argv):
    if len(argv) < 1 or argv[0] not in ("contract", "qr"):
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


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
