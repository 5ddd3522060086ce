"""Longer runs through the C ABI that back the numbers reported beside the
benchmark (each prints one JSON line; every input is seeded and synthetic):

    python -m paper_2210_03763_gb300.runs window Lx Ly chi steps [dt] [r_G]
        split-precision (3xTF32) and FP64 runs side by side from |+>^N
        through the greedy GHZ schedule (Sec. "Compiler for global GHZ
        states", minimum CZ distance r_G, default 4 a on 8x8 and sqrt(8) a
        otherwise), starting `steps // 2` steps before the end of the first
        layer that holds CZ gates so that the window crosses a layer boundary;
        reports the infidelity 1 - |<split|fp64>|^2 / (norms), |dE| and
        |dP_R| at checkpoints, and the steps/s of both precisions.
    python -m paper_2210_03763_gb300.runs repcode chi steps [dt]
        8x8 register holding the 12 five-atom repetition codes of Fig. 3
        (4 idle atoms in |0>, 2 % position jitter, seed 99), spacing
        a in {0.8, 1.0, 1.2} r_B with r_B = (C6 / Omega)^(1/6): the most
        parallel CZ layer of the codes' preparation (greedy layering with
        CZ gates at least 2 a apart) from every code atom in (|0> + |1>)/sqrt2,
        run once with every
        pair interaction and once with the codes moved far apart (no
        interaction between codes); the crosstalk infidelity is
        1 - |<isolated|full>|^2 / (norms) after `steps` steps, with the
        split-precision steps/s.
    python -m paper_2210_03763_gb300.runs sample Lx Ly chi shots
        projective measurement shots per second (ttn_sample, FP64 and split
        precision) on the state after 3 steps of the CZ-layer workload from
        |+>^N, and the fraction of shots both precisions draw alike.
"""
import json
import math
import sys
import time

import numpy as np

from paper_2210_03763_gb300 import native, workloads as W


def _ctx(Lx, Ly, chi, prec, xy, C6, sched, amps):
    g = native.TTN(Lx, Ly, chi)
    g.set_precision(prec)
    g.set_hamiltonian(xy, C6)
    g.apply_pulse(sched)
    g.set_product_state(amps)
    return g


def _sync_time():
    try:
        import torch
        torch.cuda.synchronize()
    except Exception:
        pass
    return time.perf_counter()


def window(Lx, Ly, chi, steps, dt=0.01, r_G=None):
    N = Lx * Ly
    if r_G is None:
        r_G = 4.0 if (Lx, Ly) == (8, 8) else math.sqrt(8.0)
    xy = W.square_lattice(Lx, Ly)
    layers = W.schedule_layers(W.ghz_circuit(Lx, Ly), xy, r_G)
    first = next(i for i, L in enumerate(layers) if any(g[0] == "cz" for g in L))
    TL = 2 * math.pi
    # the window [0, steps*dt) covers the end of layer `first` and the start
    # of the next one: shift the schedule so that the boundary sits mid-window
    shift = (first + 1) * TL - 0.5 * steps * dt
    sched, _ = W.layers_to_schedule(layers, 1.0, t0=-shift)
    amps = W.plus_state_amps(N)
    C6 = 20.0
    s = _ctx(Lx, Ly, chi, native.SPLIT_TF32X3, xy, C6, sched, amps)
    f = _ctx(Lx, Ly, chi, native.FP64, xy, C6, sched, amps)
    checkpoints = sorted({max(1, steps // 8), steps // 4, steps // 2, 3 * steps // 4, steps})
    out = {"run": "window", "lattice": "%dx%d" % (Lx, Ly), "chi": chi, "dt": dt, "steps": steps, "r_G": r_G,
           "layer_boundary_step": int(round(0.5 * steps)), "checkpoints": []}
    ts = tf = 0.0
    done = 0
    for cp in checkpoints:
        n = cp - done
        t0 = _sync_time()
        for _ in range(n):
            s.step(dt)
        t1 = _sync_time()
        for _ in range(n):
            f.step(dt)
        t2 = _sync_time()
        ts += t1 - t0
        tf += t2 - t1
        done = cp
        ov = s.overlap(f)
        infid = 1.0 - abs(ov) ** 2 / (s.norm() * f.norm())
        out["checkpoints"].append({"step": cp, "t": cp * dt, "infidelity_split_vs_fp64": infid,
                                   "abs_dE": abs(s.energy() - f.energy()),
                                   "abs_dP_R": float(abs(s.measure(2).sum() - f.measure(2).sum())),
                                   "norm_split": s.norm()})
        print(json.dumps(out["checkpoints"][-1]), file=sys.stderr, flush=True)
    out["split_steps_per_s"] = steps / ts
    out["fp64_steps_per_s"] = steps / tf
    out["max_infidelity"] = max(c["infidelity_split_vs_fp64"] for c in out["checkpoints"])
    s.close()
    f.close()
    return out


def repcode(chi, steps, dt=0.05):
    Lx = Ly = 8
    N = 64
    C6, omega = 20.0, 1.0
    rB = W.blockade_radius(C6, omega)
    groups = W.repetition_code_groups(Lx, Ly)
    gates = W.repetition_code_circuit(Lx, Ly)
    base = W.square_lattice(Lx, Ly, 1.0, jitter=0.02, seed=99)
    amps = np.zeros((N, 3), dtype=np.complex128)
    amps[:, 0] = 1.0
    code_of = {a: gi for gi, grp in enumerate(groups) for a in grp}
    # every code atom in (|0> + |1>)/sqrt2 (the single-qubit layers before the
    # CZ gates), idle atoms in |0>
    for grp in groups:
        for q in grp:
            amps[q] = [1 / math.sqrt(2), 1 / math.sqrt(2), 0.0]
    res = {"run": "repcode", "lattice": "8x8", "chi": chi, "dt": dt, "steps": steps, "codes": len(groups),
           "idle_atoms": N - 5 * len(groups), "jitter": 0.02, "r_B": rB, "spacings": []}
    for fac in (0.8, 1.0, 1.2):
        a = fac * rB
        xy = base * a
        layers = W.schedule_layers(gates, xy, 2.0 * a)
        best = max(layers, key=lambda L: sum(1 for g in L if g[0] == "cz"))
        sched, TL = W.layers_to_schedule([best], omega)
        far = xy.copy()
        for i in range(N):
            far[i, 0] += 1000.0 * a * (code_of.get(i, len(groups)) + 1)
        full = _ctx(Lx, Ly, chi, native.SPLIT_TF32X3, xy, C6, sched, amps)
        iso = _ctx(Lx, Ly, chi, native.SPLIT_TF32X3, far, C6, sched, amps)
        t0 = _sync_time()
        for _ in range(steps):
            full.step(dt)
        t1 = _sync_time()
        for _ in range(steps):
            iso.step(dt)
        ov = full.overlap(iso)
        infid = 1.0 - abs(ov) ** 2 / (full.norm() * iso.norm())
        n_cz = sum(1 for g in best if g[0] == "cz")
        rec = {"a_over_rB": fac, "cz_in_layer": n_cz, "crosstalk_infidelity": infid,
               "P_R_full": float(full.measure(2).sum()), "P_R_isolated": float(iso.measure(2).sum()),
               "split_steps_per_s": steps / (t1 - t0), "t": steps * dt}
        print(json.dumps(rec), file=sys.stderr, flush=True)
        res["spacings"].append(rec)
        full.close()
        iso.close()
    return res


def sample(Lx, Ly, chi, shots, steps=3, dt=0.01):
    """Shots/s of the projective measurement walk (ttn_sample) on the state
    after `steps` split-precision steps of the CZ-layer workload from |+>^N,
    in FP64 and in split precision, with the fraction of shots on which the
    two precisions draw the same outcomes from the same uniforms."""
    N = Lx * Ly
    xy = W.square_lattice(Lx, Ly)
    r_G = 4.0 if (Lx, Ly) == (8, 8) else math.sqrt(8.0)
    sched, _ = W.cz_layer_workload(Lx, Ly, r_G)
    g = _ctx(Lx, Ly, chi, native.SPLIT_TF32X3, xy, 20.0, sched, W.plus_state_amps(N))
    for _ in range(steps):
        g.step(dt)
    U = np.random.default_rng(7).random((shots, N))
    out = {"run": "sample", "lattice": "%dx%d" % (Lx, Ly), "chi": chi, "shots": shots, "steps_before": steps}
    res = {}
    for name, prec in (("fp64", native.FP64), ("split", native.SPLIT_TF32X3)):
        g.set_precision(prec)
        g.sample(U[:2])          # warm-up: workspaces
        t0 = _sync_time()
        res[name] = g.sample(U)
        t1 = _sync_time()
        out[name + "_shots_per_s"] = shots / (t1 - t0)
    out["same_outcomes"] = float(np.mean(np.all(res["fp64"] == res["split"], axis=1)))
    out["mean_rydberg_per_shot"] = float(np.mean(np.sum(res["fp64"] == 2, axis=1)))
    g.close()
    return out


def main(argv):
    if not argv or argv[0] not in ("window", "repcode", "sample"):
        print(__doc__)
        return 2
    native.load()
    if argv[0] == "window":
        Lx, Ly, chi, steps = (int(v) for v in argv[1:5])
        dt = float(argv[5]) if len(argv) > 5 else 0.01
        r_G = float(argv[6]) if len(argv) > 6 else None
        print(json.dumps(window(Lx, Ly, chi, steps, dt, r_G)))
    elif argv[0] == "sample":
        Lx, Ly, chi, shots = (int(v) for v in argv[1:5])
        print(json.dumps(sample(Lx, Ly, chi, shots)))
    else:
        chi, steps = int(argv[1]), int(argv[2])
        dt = float(argv[3]) if len(argv) > 3 else 0.05
        print(json.dumps(repcode(chi, steps, dt)))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
