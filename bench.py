"""TTN-TDVP steps/s at 8x8, chi = 128 on one GB300 (split-TF32x3 vs FP64).

Workload (synthetic, seeded): 8x8 square lattice of three-level atoms, spacing
a = 1, C6/a^6 = 20 with all 2016 van der Waals pairs, initial state
(|0> + |1>)/sqrt2 on every atom, pulses of the most parallel CZ layer of the
GHZ circuit scheduled with r_G = 4a (Jaksch pi-2pi-pi pulses, Omega = 1),
dt = 0.01.  One step = one second-order TDVP sweep over all 63 nodes.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs an independent replica (the TDVP sweep is
sequential; runs shard, the sweep does not); value = all ranks' steps / max
time.  Prints one JSON line on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LX = LY = 8
CHI = 128
C6 = 20.0
DT = 0.01
R_G = 4.0
METRIC = "TTN-TDVP steps/s at 8x8 chi=128 (split-TF32x3 tensor cores; FP64 reported beside)"
WORKLOAD = ("8x8 Rydberg lattice, chi=128, all-to-all vdW C6/a^6=20 (2016 pairs), initial |+>^64, "
            "most parallel CZ layer of the r_G=4a GHZ schedule (Jaksch pulses), dt=0.01")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def tc_traffic():
    """DRAM bytes per tc_gemm launch from the committed ncu summary, or None
    when the kernel source has changed since those counters were taken."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", "tc_gemm_8x8_chi128_slice.md")).read()
        kv = dict(l.strip().split(": ", 1) for l in txt.splitlines() if l.startswith("    ") and ": " in l)
        src = open(os.path.join(ROOT, kv["kernel_source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != kv["kernel_source_sha256_prefix"]:
            return None
        return float(kv["traffic_bytes_per_launch"])
    except Exception:
        return None


def workload():
    from paper_2210_03763_gb300 import workloads as W
    xy = W.square_lattice(LX, LY)
    sched, TL = W.cz_layer_workload(LX, LY, R_G)
    amps = W.plus_state_amps(LX * LY)
    return xy, sched, amps


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_ctx(native, precision, stream):
    xy, sched, amps = workload()
    g = native.TTN(LX, LY, CHI)
    g.set_stream(stream)
    g.set_precision(precision)
    g.set_hamiltonian(xy, C6)
    g.apply_pulse(sched)
    g.set_product_state(amps)
    return g


def time_steps(torch, g, stream, k, profile=False, tag="bench_step"):
    """K steps timed with CUDA events on the library's stream, each step in an
    NVTX range `tag` (the headline's steps in "bench_step", so that a
    profiler can capture exactly those)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if profile:
        g.profile_begin()
    g.reset_stats()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        torch.cuda.nvtx.range_push(tag)
        g.step(DT)
        torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = g.profile_end() if profile else None
    return e0.elapsed_time(e1) / 1000.0, g.stats(), prof


# ----------------------------------------------------------------- oracle leg
class OracleSampler:
    """Oracle (plain CPU complex128 TTN-TDVP) on the same workload, sampled.

    Built once (with drive operators only for the atoms the CZ layer drives;
    the others' coefficients are zero).  One sample = one node visit at a
    level-4 node (the heaviest level of the 8x8 tree: (128,128,128) tensors):
    Krylov exponential of H_eff, QR towards the parent, upward environment,
    backward link evolution.  A step visits every non-root node twice; the
    per-step time is extrapolated from the sample by the algorithmic flop
    model of a node visit (same Krylov count assumed for every node)."""

    def __init__(self):
        from oracle import ttn as ottn
        self.ottn = ottn
        xy, sched, amps = workload()
        drive = sorted({int(r[0]) for r in sched if r[3] != 0 or r[4] != 0 or r[5] != 0})
        o = ottn.OracleTTN(LX, LY, CHI, xy, C6, drive_atoms=drive, amps=amps)
        o.set_schedule(sched)
        tr = o.tree
        k = tr.level_nodes[-2][0]
        # gauge moves root -> k (not timed)
        path = []
        x = k
        while x != tr.root:
            path.append(x)
            x = tr.parent[x]
        cur = tr.root
        for ch in reversed(path):
            u = 0 if tr.children[cur][0] == ("node", ch) else 1
            o.T[cur], R = ottn.qr_leg(o.T[cur], u)
            oth = [l for l in range(3) if l != u]
            o.down[ch] = ottn.renormalize(o.T[cur], u, o.env(cur, oth[0]), o.env(cur, oth[1]), o.V)
            o.T[ch] = ottn.apply_leg(R, o.T[ch], 2)
            cur = ch
        self.o, self.k = o, k
        self.coef = o.coef(0.5 * DT)

    def sample(self):
        """Seconds of one node visit."""
        o, k, ottn = self.o, self.k, self.ottn
        t0 = time.perf_counter()
        o.node_evolve(k, 0.5 * DT, self.coef)
        o.T[k], R = ottn.qr_leg(o.T[k], 2, o.allowed(k))
        o.up[k] = ottn.renormalize(o.T[k], 2, o.env(k, 0), o.env(k, 1), o.V)
        R = o.link_evolve(R, o.up[k], o.down[k], 0.5 * DT, self.coef)
        t = time.perf_counter() - t0
        o.T[k] = ottn.apply_leg(R, o.T[k], 2)
        return t

    def step_factor(self):
        tr = self.o.tree
        m = self.o.krylov_stats[-2][0] if len(self.o.krylov_stats) >= 2 else 8

        def visit_flops(kk):
            d = tr.shape(kk)
            s = d[0] * d[1] * d[2]
            n = [len(tr.leg_sites(kk, u)) for u in range(3)]
            r = [min(n[0], n[1]), min(n[0], n[2]), min(n[1], n[2])]
            pair_d = [(d[0] + d[1]), (d[0] + d[2]), (d[1] + d[2])]
            heff = 8 * s * (sum(d) + sum(ri * pd for ri, pd in zip(r, pair_d)))
            qr = 16 * s * d[2]
            env = 8 * s * (d[0] + d[2]) * (n[0] + n[1]) * 4
            return m * heff + qr + env
        per_step = sum(2 * visit_flops(kk) for kk in range(tr.n_nodes) if kk != tr.root) + visit_flops(tr.root)
        return per_step / visit_flops(self.k), m


def oracle_sample(n_samples=1):
    """(steps/s extrapolated, seconds per sample, note) of the 8x8 workload."""
    smp = OracleSampler()
    t = min(smp.sample() for _ in range(n_samples))
    fac, m = smp.step_factor()
    note = ("oracle node visit at a (128,128,128) level-4 node (Krylov m=%d, QR, environment, link), "
            "%.1f s; step time extrapolated by the flop model x%.1f" % (m, t, fac))
    return 1.0 / (t * fac), t, note


SMALL_STEP_CODE = """
import json, sys, time
sys.path.insert(0, %r)
from oracle import ttn as ottn
from paper_2210_03763_gb300 import workloads as W
xy = W.square_lattice(4, 4)
sched, TL = W.cz_layer_workload(4, 4, 2.0 ** 1.5)
o = ottn.OracleTTN(4, 4, 64, xy, %r, amps=W.plus_state_amps(16))
o.set_schedule(sched)
o.step(%r)
t0 = time.perf_counter()
o.step(%r)
print(json.dumps({"s_per_step": time.perf_counter() - t0}))
"""


def oracle_small_step(threads):
    """Seconds of one real oracle step of the 4x4, chi = 64 CZ-layer workload
    (r_G = sqrt(8) a, |+>^16), in a fresh process whose BLAS uses `threads`
    threads (None: all cores).  A fresh interpreter, not a fork of this one."""
    env = dict(os.environ)
    if threads:
        for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
    code = SMALL_STEP_CODE % (ROOT, C6, DT, DT)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        return json.loads(r.stdout.strip().splitlines()[-1])["s_per_step"]
    except Exception:
        return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    smp = OracleSampler()
    fac, _ = smp.step_factor()
    for _ in range(args.warmup > 0 and 1 or 0):
        smp.sample()
    samples = [smp.sample() for _ in range(max(1, args.steps))]
    fac, m = smp.step_factor()
    t = statistics.median(samples)
    value = 1.0 / (t * fac)
    cores = os.cpu_count()
    note = ("each step: one oracle node visit at a (128,128,128) level-4 node (Krylov m=%d, QR, environment, "
            "link), median %.1f s; step time extrapolated by the flop model x%.1f" % (m, t, fac))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD, "lattice": "8x8", "chi": CHI},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": note},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- our arm
def replica_time(dist, secs, device):
    """The slowest rank's timed seconds (max over ranks; `dist` is
    torch.distributed after init_process_group, or None for one process)."""
    if dist is None:
        return secs
    import torch
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, steps, t_max):
    """Whole-job steps/s: every rank runs `steps` steps of its own replica."""
    return world * steps / t_max


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed FP64 steps (0: skip the FP64 leg)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--profile-steps", type=int, default=2, help="steps of the instrumented second pass")
    ap.add_argument("--full-rank-steps", type=int, default=2, help="timed steps from a full-rank start (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-out", default=None, help="write the kernel profile JSON here")
    ap.add_argument("--lattice", default=None, help="LXxLY of another case of the same recipe (profiling, chi=256); default 8x8")
    ap.add_argument("--chi", type=int, default=None, help="bond dimension of another case; default 128")
    args = ap.parse_args()
    global LX, LY, CHI, WORKLOAD
    if args.lattice or args.chi:
        if args.lattice:
            LX, LY = (int(v) for v in args.lattice.lower().split("x"))
        if args.chi:
            CHI = args.chi
        WORKLOAD = "%dx%d Rydberg lattice, chi=%d (another case of the same workload recipe: same pulses, |+> start, dt)" % (LX, LY, CHI)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as ge
    ge.build()
    from paper_2210_03763_gb300 import native

    stream = torch.cuda.current_stream()
    free0, total = torch.cuda.mem_get_info()
    g = make_ctx(native, native.SPLIT_TF32X3, stream)
    for _ in range(args.warmup):
        g.step(DT)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()   # after warm-up: workspaces have grown to size
    if dist:
        dist.barrier()
    # headline: K steps, no per-launch instrumentation
    clk = ClockSampler(local)
    clk.start()
    secs, stats, _ = time_steps(torch, g, stream, args.steps, profile=False)
    clocks = clk.stop()
    t_max = replica_time(dist, secs, "cuda")
    value = replica_value(world, args.steps, t_max)
    # second pass: the same steps with CUDA events around every contraction and
    # QR launch (kernel-class times for the roofline); not the headline
    n_prof = max(1, min(args.steps, args.profile_steps))
    p_secs, _, prof = time_steps(torch, g, stream, n_prof, profile=True, tag="profile_step")

    # e2e through the public API with host buffers: schedule in, populations out
    from paper_2210_03763_gb300 import workloads as W
    xy, sched, amps = workload()
    pulse_host = W.to_pulse_array(sched)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        g.apply_pulse(pulse_host)
        g.step(DT)
        pops = g.measure(2)
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    e2e = None
    if args.e2e_steps > 0:
        e2e = {"value": args.e2e_steps / e2e_secs, "unit": "steps/s",
               "h2d_bytes_per_step": int(pulse_host.nbytes), "d2h_bytes_per_step": int(pops.nbytes)}

    pk, peak_kind = peaks()
    tc = prof["tc_gemm"]
    # a kernel timed inside seconds-long steps: the sustained BF16 rate, scaled
    # by the nominal TF32 : BF16 ratio
    tf32_peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * 1.1 / 2.25
    dominant = max(prof.items(), key=lambda kv: kv[1]["ms"])
    roof = None
    if tc["launches"] > 0 and tc["ms"] > 0:
        ach = tc["flops"] / (tc["ms"] * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "tc_gemm_kernel (tcgen05 kind::tf32, 3xTF32)",
                "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak,
                "peak_source": "%s bf16_tflops_sustained x 1.1/2.25 (nominal TF32:BF16), of %s" % (
                    peak_kind, peak_kind),
                "traffic": tc_traffic(), "launches": tc["launches"] / n_prof,
                "traffic_source": "ncu dram__bytes_read+write per launch, mean over the first 2500 tc_gemm "
                                  "launches of the timed 8x8 chi=128 step (profiles/tc_gemm_8x8_chi128_slice.md)",
                "share_of_step": tc["ms"] / (p_secs * 1e3),
                "flops_counted": "algorithmic 8*M*N*K per complex contraction; tensor pipe executes 3x"}
    pack = prof["split_pack"]
    pack_line = None
    if pack["launches"] > 0 and pack["ms"] > 0:
        gbs = pack["bytes"] / (pack["ms"] * 1e-3) / 1e9
        pack_line = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / pk["hbm_gbs"], "ms_per_step": pack["ms"] / n_prof,
                     "bytes_per_step": pack["bytes"] / n_prof,
                     "bytes_counted": "16 B read per complex operand element + hi/lo FP32 planes written"}

    result = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64 state, 3xtf32 contractions",
              "data": "synthetic",
              "config": {"workload": WORKLOAD, "lattice": "%dx%d" % (LX, LY), "chi": CHI, "dt": DT,
                         "parallelism": "replicas" if world > 1 else "single",
                         "l2": "working set (node tensors, environments, Krylov basis) > 129 MB L2",
                         "device_mem_gb": round((free0 - free1) / 1e9, 2)},
              "gpu_launches": int(stats["launches"]), "launches_per_step": stats["launches"] / args.steps,
              "clocks": clocks, "e2e": e2e, "roofline": roof, "split_pack": pack_line,
              "profile": {k: {"launches": v["launches"] / n_prof, "ms_per_step": round(v["ms"] / n_prof, 3)}
                          for k, v in prof.items()},
              "profile_pass": {"steps": n_prof, "ms_per_step_instrumented": 1e3 * p_secs / n_prof,
                               "ms_per_step_outside_classes": round(1e3 * p_secs / n_prof - sum(
                                   v["ms"] for v in prof.values()) / n_prof, 3)},
              "dominant_kernel_class": dominant[0],
              "krylov_matvecs_per_step": stats["matvecs"] / max(1, args.steps)}

    if args.full_rank_steps > 0 and rank == 0:
        # the same workload from a random full-rank isometric TTN: every QR is
        # full rank (the |+>^64 start keeps most bonds rank-deficient early on)
        h = make_ctx(native, native.SPLIT_TF32X3, stream)
        Ts = W.random_ttn_tensors([h.node_info(k)[0] for k in range(h.num_nodes())], 77)
        for k, X in enumerate(Ts):
            h.set_node(k, X)
        h.refresh_envs()
        h.step(DT)
        fr_secs, _, _ = time_steps(torch, h, stream, args.full_rank_steps, profile=False, tag="full_rank_step")
        result["full_rank_start"] = {"value": args.full_rank_steps / fr_secs, "unit": "steps/s",
                                     "steps": args.full_rank_steps}
        h.close()

    if args.fp64_steps > 0 and rank == 0:
        f = make_ctx(native, native.FP64, stream)
        s2 = make_ctx(native, native.SPLIT_TF32X3, stream)
        f.step(DT)                      # warm-up step (also the first comparison step)
        s2.step(DT)
        f_secs, f_stats, f_prof = time_steps(torch, f, stream, args.fp64_steps, profile=True, tag="fp64_step")
        for _ in range(args.fp64_steps):
            s2.step(DT)
        ov = s2.overlap(f)
        infid = 1.0 - abs(ov) ** 2 / (s2.norm() * f.norm())
        fa = f_prof["f64_gemm"]
        dfma = native.fp64_peak(0)
        dmma = native.fp64_peak(1)
        result["fp64"] = {"value": args.fp64_steps / f_secs, "unit": "steps/s",
                          "speedup_split_over_fp64": value / (args.fp64_steps / f_secs),
                          "f64_gemm_tflops": fa["flops"] / max(1e-9, fa["ms"] * 1e-3) / 1e12,
                          "f64_peak_tflops": max(dfma, dmma),
                          "f64_peak_source": "measured in this run: DFMA chains %.3f, DMMA m8n8k4 %.3f TFLOP/s"
                                             % (dfma, dmma)}
        result["fidelity_err"] = {"steps": 1 + args.fp64_steps,
                                  "infidelity_split_vs_fp64": infid,
                                  "abs_dE": abs(s2.energy() - f.energy()),
                                  "abs_dP_R": float(abs(s2.measure(2).sum() - f.measure(2).sum()))}
        f.close()
        s2.close()

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        v, t, note = oracle_sample(1)
        cores = os.cpu_count()
        small_all = oracle_small_step(None)
        small_one = oracle_small_step(1)
        result["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                                  "sample": note,
                                  "oracle_step_4x4_chi64": {
                                      "workload": "4x4, chi=64, CZ layer of the r_G=sqrt(8)a schedule, |+>^16, "
                                                  "one full oracle step, timed",
                                      "s_per_step_all_cores": small_all, "cores": cores,
                                      "s_per_step_1_core": small_one}}
    if args.profile_out and rank == 0:
        with open(args.profile_out, "w") as fo:
            json.dump({"prof": prof, "profile_steps": n_prof, "stats": stats,
                       "records": {"columns": ["kind", "M", "N", "K", "batches", "ms", "flops"],
                                   "kinds": ["tc_gemm", "split_pack", "f64_gemm", "qr"],
                                   "rows": g.profile_records().tolist()}}, fo)
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


if __name__ == "__main__":
    main()
