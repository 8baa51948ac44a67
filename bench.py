#!/usr/bin/env python
"""Throughput benchmark of the GB300 Stokeslet + stresslet treecode.

Workload (one "step" = the whole hot path over one particle system):
  N = 1,000,000 particles uniform in the unit cube, f and h uniform in
  [-1, 1]^3, nu uniform random unit vectors (seeded); tree build with leaf
  size N0 = 2000, cluster moments of order p = 8, and the treecode velocity
  at every particle with MAC theta = 0.5 (Algorithm 1), mixed precision.
  Metric: targets/s = N / (time of one step), inputs resident in HBM.

Prints ONE JSON line (rank 0).  Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own seeded system of the same
size (replicas, weak scaling); there is no data-path collective.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "targets/s at N=1M, p=8 (rel-L2<=1e-6 vs FP64 direct); fwd+adjoint s/step"
UNIT = "targets/s"
L2_FLUSH_BYTES = 256 << 20
# nominal GB300 arithmetic peaks (152 SMs at 2070 MHz): FP64 2 FMA/clk/SM,
# FP32 128 FMA/clk/SM; the roofline fractions are taken against the peaks
# measured in the run itself (tc_fma_peak) and reported beside these
PEAK_FP64_TFLOPS = 1.25
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def ncoef(n):
    return (n + 1) * (n + 2) * (n + 3) // 6


def far_flops_per_interaction(p):
    """Algorithmic flops of one (target, cluster) far-field interaction of the
    far kernel (FMA = 2): the Coulomb recurrence on the harmonic subset k1 <= 1
    (first product 1 flop, each further product an FMA, additions of the
    second sum, the closing FMA) and the FP32 contraction (12 FMA per
    coefficient, 12 FMA per level for the level factor, 18 for d'.B)."""
    P = p + 2
    rec = 0
    ncoefs = 0
    for n in range(1, P + 1):
        for k1 in (0, 1):
            for k3 in range(0, n - k1 + 1):
                k2 = n - k1 - k3
                t1 = sum(1 for v in (k1, k2, k3) if v >= 1)
                t2 = sum(1 for v in (k2, k3) if v >= 2)
                rec += (2 * t1 - 1) + max(t2 - 1, 0) + 2
                ncoefs += 1
    con = 24 * (ncoefs + 1) + 24 * P + 18
    return float(rec), float(con)


def folded_coefficients(P):
    """Coefficients with k1 <= 1 of orders 0..P (the harmonic subset the
    folded tables keep): (P + 1)^2."""
    return (P + 1) ** 2


# Algorithmic flops of the adjoint's per-unit work (FMA = 2), from the
# formulas of the adjoint (the header of csrc/tc_adjoint.cu):
# near field, target side, per (target, source) pair: d 3, r^2 5, 1/r 1,
# r^-2, r^-3, r^-5, r^-7 4, the dot products g.f, g.d, d.f, d.h, d.nu 25,
# s and t 3 and their sum 1, c3, c4, c5 5, c1 8, the gradient
# d c1 + g (s + t) + f c3 + h c4 + nu c5 27, its accumulation 3: 85;
# near field, source side, per pair: the same 85 for dL/dy plus dL/df
# (g / r + d c3: 9, accumulated 3), dL/dh (d c4: 3 + 3) and dL/dnu
# (d c5: 3 + 3): 109;
# far field, target side, per (target, cluster) interaction: the recurrence
# one order further (to p + 3) and, per coefficient k, alpha^k = g.(A^k +
# d' B^k) 30, beta_l^k = sum_i g_i B_il^k 18, the sums b^k beta^k 6 and
# (k_l + 1) b^{k+e_l} alpha^k 9: 63.
# regularized pair terms per (target, source) pair: d 3, r^2 5, s 1, 1/sqrt(s)
# 1, q^2 1, d.f, d.h, d.nu 15, f coefficient q (1 + eps^2 q^2) 3, (d.h)(d.nu)
# + (eps^2/2)(h.nu) 3, the d coefficient 4, the h and nu coefficient 5, the
# three components (f, d, h, nu terms) 24: 65
REG_NEAR_PAIR_FLOPS = 65
NEAR_ADJ_TARGET_FLOPS = 85.0
NEAR_ADJ_SOURCE_FLOPS = 109.0
FAR_ADJ_PER_COEF_FLOPS = 45.0


def far_adj_target_flops(p):
    """(folded, unfolded) flops of one far interaction of the adjoint's
    target side: on the harmonic subset the kernel works on (recurrence as in
    far_flops_per_interaction, one order further), and on the full set of
    C(p+5, 3) coefficients with the unfolded recurrence 11 C(p+6, 3)."""
    rec_next, _ = far_flops_per_interaction(p + 1)
    folded = rec_next + FAR_ADJ_PER_COEF_FLOPS * folded_coefficients(p + 2)
    unfolded = 11 * ncoef(p + 3) + FAR_ADJ_PER_COEF_FLOPS * ncoef(p + 2)
    return float(folded), float(unfolded)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--N0", type=int, default=2000)
    ap.add_argument("--cpu-sample", type=int, default=16384, help="targets the oracle evaluates for cpu_baseline")
    ap.add_argument("--cpu-sample-1t", type=int, default=1024,
                    help="targets the oracle evaluates for the one-thread cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=2048, help="targets per step of the reference arm")
    ap.add_argument("--error-samples", type=int, default=10000, help="targets of the FP64 direct-sum error check")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the accuracy-against-time sweep on the 4M-point sphere")
    ap.add_argument("--only-extra", choices=["fwd_adjoint", "batched", "sphere_sweep", "table1_sphere",
                                             "fig3_sphere", "regularized"],
                    help="run just this extra measurement and print it as one JSON line (for profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the forward+adjoint (Gaussian clusters) and batched (64 systems) measurements")
    return ap.parse_args()


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the slowest rank's time); dist is
    torch.distributed or None for one process."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_per_rank, world, ms):
    """Targets per second of the whole job: every rank evaluates its own
    n_per_rank-particle replica in the slowest rank's time ms."""
    return n_per_rank * world / (ms / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if re.match(r"^[0-9.]+$", r[1])]
        mx = [float(r[2]) for r in rows if re.match(r"^[0-9.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# the files that hold each profiled kernel's code
NEAR_SOURCES = ("tc_near.cu", "tc_nearpair.cuh")
FAR_SOURCES = ("tc_far.cu", "tc_recurrence.cuh")


def source_sha(sources):
    """sha256 over the kernel's source files (csrc/), concatenated in order."""
    hsh = hashlib.sha256()
    for f in sources:
        hsh.update(open(os.path.join(ROOT, "paper_1811_12498_gb300", "csrc", f), "rb").read())
    return hsh.hexdigest()


def kernel_traffic(sources, profile, profiles_dir=None):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if the
    summary was taken on the current kernel sources (source_sha); else None."""
    prof = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), profile)
    if not os.path.exists(prof):
        return None
    text = open(prof).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != source_sha(sources):
        return None
    return float(m_b.group(1))


def cpu_baseline(x, f, h, nu, args, sample, threads=0):
    """The oracle as it stands, on this host's cores (threads = 0: all of
    them): tree + moments over all N particles, the treecode at `sample`
    seeded targets; the evaluation time extrapolated to N targets."""
    import oracle
    from paper_1811_12498_gb300 import inputs
    N = x.shape[0]
    idx = inputs.sample_indices(N, sample, 4242)
    oracle.set_threads(threads)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    tree = oracle.Tree(x, args.N0, True)
    t1 = time.perf_counter()
    tree.set_moments(f, h, nu, args.p)
    t2 = time.perf_counter()
    u = tree.treecode(x[idx], args.theta, args.p)
    t3 = time.perf_counter()
    oracle.set_threads(0)
    full = (t1 - t0) + (t2 - t1) + (t3 - t2) * N / len(idx)
    return {"value": N / full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle tree + order-%d moments over all %d particles (%.1f s), treecode at %d seeded "
                      "targets (%.1f s), extrapolated to %d targets; %d thread(s)"
                      % (args.p, N, t2 - t0, len(idx), t3 - t2, N, cores),
            "seconds": t3 - t0}, idx, u


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1811_12498_gb300 import inputs
    x, f, h, nu = inputs.uniform_cube(args.N, inputs.SEED_BASE + 1)
    vals = []
    for k in range(args.warmup + args.steps):
        r, _, _ = cpu_baseline(x, f, h, nu, args, args.ref_sample)
        if k >= args.warmup:
            vals.append(r)
    v = statistics.mean(r["value"] for r in vals)
    ms = args.N / v * 1e3
    cfg = config(args)
    cfg["reference_timing"] = ("extrapolated: each step times the oracle's tree and moments over all %d particles "
                               "and its treecode at %d sampled targets, scaled to %d targets"
                               % (args.N, args.ref_sample, args.N))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _events(stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    return e0, e1


def bench_fwd_adjoint(flush, stream, steps=3):
    """Forward + adjoint step on 262,144 particles in 8 Gaussian clusters
    (sigma 0.05), p = 8, theta = 0.5, N0 = 2000, mixed precision: tc_build,
    tc_moments, tc_eval and tc_adjoint for dL/df, dL/dh, dL/dnu, dL/dx."""
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs
    N, N0, p, theta = 262_144, 2000, 8, 0.5
    x, f, h, nu = inputs.gaussian_clusters(N, inputs.SEED_BASE + 4)
    d = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]
    g = torch.from_numpy(np.ascontiguousarray(np.random.default_rng(5).standard_normal((N, 3)).T)).cuda()
    tc = api.Treecode("mixed", True, stream)
    u = torch.empty((3, N), dtype=torch.float64, device="cuda")
    fwd, tot = [], []
    for k in range(steps + 1):
        flush.fill_(1)
        e0, e1 = _events(stream)
        tc.build(d[0], N0).moments(d[1], d[2], d[3], p)
        tc.eval(theta, p, out=u)
        em = torch.cuda.Event(enable_timing=True)
        em.record(stream)
        tc.adjoint(g)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            fwd.append(e0.elapsed_time(em))
            tot.append(e0.elapsed_time(e1))
    # each adjoint kernel's own duration (phase events, one more step with
    # everything serialised), and its counted work against the measured FP32
    # peak
    tc.profile(2)
    flush.fill_(1)
    tc.build(d[0], N0).moments(d[1], d[2], d[3], p)
    tc.eval(theta, p, out=u)
    tc.adjoint(g)
    ph = tc.phase_times()
    tc.profile(False)
    st = tc.stats()
    tc.close()
    peak = api.fma_peak("mixed", stream)
    far_f, far_u = far_adj_target_flops(p)

    def roof(kernel, flops, ms_k, unit):
        tf = flops / (ms_k / 1e3) / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                "flops_per_launch": flops, "launch_ms": ms_k, "work_unit": unit}

    rooflines = [
        roof("k_near_leaf<NearOpG> (near field, target side)", NEAR_ADJ_TARGET_FLOPS * st["near_pairs"],
             ph["adj_near_target"],
             "%g flops per near pair" % NEAR_ADJ_TARGET_FLOPS),
        roof("k_near_adj_source_units (near field, source side)", NEAR_ADJ_SOURCE_FLOPS * st["near_pairs"],
             ph["adj_near_source"],
             "%g flops per near pair" % NEAR_ADJ_SOURCE_FLOPS),
        roof("k_far_adj_target32p<10> (far field, target side)", far_f * st["far_interactions"], ph["adj_far_target"],
             "%g flops per far interaction on the folded coefficients (%g on all C(p+5,3))" % (far_f, far_u)),
    ]
    ms = statistics.mean(tot)
    return {"workload": "8 Gaussian clusters N=262144, sigma=0.05, p=8, theta=0.5, N0=2000, mixed",
            "s_per_step": ms / 1e3, "fwd_ms": statistics.mean(fwd), "adjoint_ms": ms - statistics.mean(fwd),
            "steps": steps, "grads": "f, h, nu, x",
            "adjoint_phases_ms": {k: v for k, v in ph.items() if k.startswith("adj_")},
            "interactions": {"near_pairs": st["near_pairs"], "far": st["far_interactions"]},
            "roofline": rooflines,
            "peak_kind": "measured FP32 FMA peak (tc_fma_peak)"}


def bench_sphere_sweep(flush, stream):
    """Accuracy against time on 4,000,000 quasi-uniform points of the unit
    sphere (nu = outward normal, f, h ~ N(0,1)), p in {4, 6, 8, 10}, theta in
    {0.5, 0.7}, N0 = 2000: per point, the time of build + moments + eval
    (mixed, FP32 recurrence; and with the FP64 recurrence for p >= 8) and E
    against the FP64 direct sum on 10,000 sampled targets."""
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs
    N, N0 = 4_000_000, 2000
    x, f, h, nu = inputs.fibonacci_sphere(N, inputs.SEED_BASE + 3)
    d = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]
    eidx = inputs.sample_indices(N, 10_000, 778)
    tgt = torch.from_numpy(np.ascontiguousarray(x[eidx].T)).cuda()
    ud = api.direct(d[0], d[1], d[2], d[3], targets=tgt, precision="fp64").cpu().numpy().T
    u = torch.empty((3, N), dtype=torch.float64, device="cuda")
    rows = []
    for rec64 in (False, True):
        tc = api.Treecode("mixed", True, stream, rec64=rec64)
        for p in (4, 6, 8, 10):
            if rec64 and p < 8:
                continue
            for theta in (0.5, 0.7):
                times = []
                for k in range(3):
                    flush.fill_(1)
                    e0, e1 = _events(stream)
                    tc.build(d[0], N0).moments(d[1], d[2], d[3], p)
                    tc.eval(theta, p, out=u)
                    e1.record(stream)
                    e1.synchronize()
                    if k > 0:
                        times.append(e0.elapsed_time(e1))
                uh = u.cpu().numpy().T[eidx]
                E = float(np.sqrt(np.sum((uh - ud) ** 2) / np.sum(ud ** 2)))
                ms = statistics.mean(times)
                rows.append({"p": p, "theta": theta, "recurrence": "fp64" if rec64 else "fp32", "ms": ms,
                             "targets_per_s": N / (ms / 1e3), "E_vs_fp64_direct": E})
        tc.close()
    return {"workload": "Fibonacci sphere N=4000000, nu = outward normal, f, h ~ N(0,1), N0=2000, mixed",
            "E_samples": int(len(eidx)), "points": rows}


def bench_table1(flush, stream):
    """Test case 1 of the paper at its Table 1(b) size: Stokeslets and
    stresslets at the N = 327680 centroids of a 7-times refined icosahedron
    on the unit sphere, weights uniform in [-1, 1], shrunk clusters, N0 =
    2000, theta in {0.2, 0.5, 0.8}, p in {0, 2, ..., 10}, mixed precision:
    per point the time t of build + moments + eval, E over all targets
    against the FP64 direct sum, and the speedup d/t over the mixed-precision
    direct sum on the same GPU (the paper's d/t column is CPU against CPU)."""
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs
    x, f, h, nu = inputs.icosahedral_sphere(7, inputs.SEED_BASE + 101)
    N, N0 = x.shape[0], 2000
    d = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]
    ud = api.direct(*d, precision="fp64", stream=stream)
    u = torch.empty((3, N), dtype=torch.float64, device="cuda")
    dms = []
    for k in range(3):
        flush.fill_(1)
        e0, e1 = _events(stream)
        api.direct(*d, precision="mixed", out=u, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            dms.append(e0.elapsed_time(e1))
    d_ms = statistics.mean(dms)
    tc = api.Treecode("mixed", True, stream)
    rows = []
    for theta in (0.2, 0.5, 0.8):
        for p in range(0, 11, 2):
            times = []
            for k in range(3):
                flush.fill_(1)
                e0, e1 = _events(stream)
                tc.build(d[0], N0).moments(d[1], d[2], d[3], p)
                tc.eval(theta, p, out=u)
                e1.record(stream)
                e1.synchronize()
                if k > 0:
                    times.append(e0.elapsed_time(e1))
            E = float(torch.linalg.norm(u - ud) / torch.linalg.norm(ud))
            ms = statistics.mean(times)
            rows.append({"theta": theta, "p": p, "ms": ms, "d_over_t": d_ms / ms, "E": E})
    tc.close()
    return {"workload": "icosahedral sphere N=327680 (Table 1(b) size), f, h, nu uniform in [-1,1], N0=2000, "
                        "shrink, mixed; E over all targets vs FP64 direct (mixed floor ~3e-7)",
            "direct_mixed_ms": d_ms, "points": rows}


def bench_fig3(flush, stream):
    """Fig. 3 of the paper: test case 1 (icosahedral sphere, weights uniform
    in [-1, 1], shrunk clusters, N0 = 2000) at theta = 0.5, p = 0, 2, ..., 10,
    N = 20 * 4^L for L = 5..8 (20480 ... 1310720), mixed precision: per point
    the time of build + moments + eval and E over 20000 sampled targets
    (all at N = 20480) against the FP64 direct sum; per N the time of the
    mixed direct sum; and the slopes of log time against log N (the paper:
    direct O(N^2), treecode consistent with O(N log N))."""
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs

    def timed(fn, reps=2):
        out = []
        for k in range(reps + 1):
            flush.fill_(1)
            e0, e1 = _events(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                out.append(e0.elapsed_time(e1))
        return statistics.mean(out)

    rows, direct = [], {}
    for L in (5, 6, 7, 8):
        x, f, h, nu = inputs.icosahedral_sphere(L, inputs.SEED_BASE + 101)
        N = x.shape[0]
        d = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]
        idx = inputs.sample_indices(N, min(N, 20000), 5)
        tgt = torch.from_numpy(np.ascontiguousarray(x[idx].T)).cuda()
        ud = api.direct(*d, targets=tgt, precision="fp64", stream=stream)
        it = torch.from_numpy(idx).cuda()
        u = torch.empty((3, N), dtype=torch.float64, device="cuda")
        direct[N] = timed(lambda: api.direct(*d, precision="mixed", out=u, stream=stream))
        tc = api.Treecode("mixed", True, stream)
        for p in range(0, 11, 2):
            ms = timed(lambda: (tc.build(d[0], 2000).moments(d[1], d[2], d[3], p), tc.eval(0.5, p, out=u)))
            E = float(torch.linalg.norm(u[:, it] - ud) / torch.linalg.norm(ud))
            rows.append({"N": N, "p": p, "ms": ms, "E": E, "d_over_t": direct[N] / ms})
        tc.close()
    Ns = sorted(direct)
    lnN = np.log(np.array(Ns, dtype=np.float64))
    slopes = {"direct": float(np.polyfit(lnN, np.log([direct[n] for n in Ns]), 1)[0])}
    for p in range(0, 11, 2):
        t = [r["ms"] for n in Ns for r in rows if r["N"] == n and r["p"] == p]
        slopes["treecode_p%d" % p] = float(np.polyfit(lnN, np.log(t), 1)[0])
    return {"workload": "icosahedral sphere N=20480..1310720, theta=0.5, p=0..10, N0=2000, shrink, mixed; E on "
                        "20000 sampled targets vs FP64 direct",
            "direct_mixed_ms": {str(n): direct[n] for n in Ns}, "points": rows,
            "loglog_slopes_time_vs_N": slopes}


def bench_regularized(flush, stream):
    """Regularized Stokeslet and stresslet (tc_config.reg_eps) on the headline
    workload: N = 1,000,000 uniform in the unit cube, p = 8, theta = 0.5,
    N0 = 2000, eps = 1e-3 (a tenth of the mean spacing), mixed precision (FP32
    far and near fields): time of build + moments + eval, the far and near
    phases alone, and E against the FP64 regularized direct sum on 2000
    sampled targets."""
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs
    N, N0, p, theta, eps = 1_000_000, 2000, 8, 0.5, 1e-3
    x, f, h, nu = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    d = [torch.from_numpy(np.ascontiguousarray(a.T)).cuda() for a in (x, f, h, nu)]
    tc = api.Treecode("mixed", True, stream, reg_eps=eps)
    u = torch.empty((3, N), dtype=torch.float64, device="cuda")
    times = []
    for k in range(3):
        flush.fill_(1)
        e0, e1 = _events(stream)
        tc.build(d[0], N0).moments(d[1], d[2], d[3], p)
        tc.eval(theta, p, out=u)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            times.append(e0.elapsed_time(e1))
    tc.profile(2)
    tc.build(d[0], N0).moments(d[1], d[2], d[3], p)
    tc.eval(theta, p, out=u)
    ph = tc.phase_times()
    tc.profile(False)
    st = tc.stats()
    tc.close()
    idx = inputs.sample_indices(N, 2000, 983)
    tgt = torch.from_numpy(np.ascontiguousarray(x[idx].T)).cuda()
    ud = api.direct_reg(*d, eps, targets=tgt, precision="fp64", stream=stream)
    it = torch.from_numpy(idx).cuda()
    E = float(torch.linalg.norm(u[:, it] - ud) / torch.linalg.norm(ud))
    ms = statistics.mean(times)
    peak32 = api.fma_peak("mixed", stream)
    # far field per interaction: the recurrences of G_1/2 (orders <= p+2) and
    # G_3/2 (orders <= p+1) at 11 flops per coefficient, the contractions at
    # 24 and 6 flops per coefficient, d'.B 18
    far_unit = 35 * ncoef(p + 2) + 17 * ncoef(p + 1) + 18
    far_tf = far_unit * st["far_interactions"] / (ph["far"] / 1e3) / 1e12
    near_tf = REG_NEAR_PAIR_FLOPS * st["near_pairs"] / (ph["near"] / 1e3) / 1e12
    return {"workload": "regularized kernels, eps=1e-3, uniform cube N=1000000, p=8, theta=0.5, N0=2000, mixed "
                        "(FP32 far and near fields)",
            "ms_per_step": ms, "targets_per_s": N / (ms / 1e3), "far_ms": ph["far"], "near_ms": ph["near"],
            "far_interactions": st["far_interactions"], "near_pairs": st["near_pairs"],
            "E_vs_fp64_regularized_direct": E, "E_samples": int(len(idx)),
            "roofline": [
                {"kernel": "k_far_reg32r<10>", "bound": "alu", "achieved": far_tf, "peak": peak32, "unit": "TFLOP/s",
                 "frac": far_tf / peak32, "work_unit": "%d flops per far interaction" % far_unit},
                {"kernel": "k_near_leaf<NearOpReg>", "bound": "alu", "achieved": near_tf, "peak": peak32,
                 "unit": "TFLOP/s", "frac": near_tf / peak32,
                 "work_unit": "%d flops per near pair" % REG_NEAR_PAIR_FLOPS}]}


def bench_batched(flush, stream, reps=3):
    """64 independent systems, sizes log-uniform in [1e4, 5e5] (even: uniform
    cube, odd: Fibonacci sphere), p = 6, theta = 0.6, N0 = 2000, mixed: one
    batched evaluation (persistent kernels from a CUDA graph, autotuned
    shapes) against 64 separate tc_eval calls; trees and moments built once."""
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs
    sizes = inputs.batch_sizes(64, inputs.SEED_BASE + 5)
    parts = []
    for k, n in enumerate(sizes):
        gen = inputs.uniform_cube if k % 2 == 0 else inputs.fibonacci_sphere
        parts.append(gen(int(n), inputs.SEED_BASE + 500 + k))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    seg = [torch.from_numpy(np.ascontiguousarray(np.concatenate([pp[c] for pp in parts]).T)).cuda() for c in range(4)]
    b = api.Batch("mixed", True, stream)
    b.build(seg[0], off, 2000).moments(seg[1], seg[2], seg[3], 6)
    u = b.eval(0.6, 6)  # tunes and captures the graph
    outs = b.eval_separate(0.6, 6)
    tb, ts = [], []
    for _ in range(reps):
        flush.fill_(1)
        e0, e1 = _events(stream)
        b.eval(0.6, 6, out=u)
        e1.record(stream)
        e1.synchronize()
        tb.append(e0.elapsed_time(e1))
        flush.fill_(1)
        e0, e1 = _events(stream)
        b.eval_separate(0.6, 6, outs)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    same = all(torch.equal(u[:, int(off[s]):int(off[s + 1])], outs[s]) for s in range(len(sizes)))
    info = b.info()
    b.close()
    ntot = int(off[-1])
    return {"workload": "64 systems, log-uniform N in [1e4, 5e5], cube/sphere, p=6, theta=0.6, N0=2000, mixed",
            "total_targets": ntot, "batched_ms": statistics.mean(tb), "separate_ms": statistics.mean(ts),
            "batched_targets_per_s": ntot / (statistics.mean(tb) / 1e3),
            "separate_targets_per_s": ntot / (statistics.mean(ts) / 1e3),
            "identical_results": bool(same), "tuned_shape": info}


def run_only_extra(name):
    """One extra measurement alone (its JSON object on one line), so that a
    profiler can be pointed at exactly that workload."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    fn = {"fwd_adjoint": bench_fwd_adjoint, "batched": bench_batched, "sphere_sweep": bench_sphere_sweep,
          "table1_sphere": bench_table1, "fig3_sphere": bench_fig3, "regularized": bench_regularized}[name]
    print(json.dumps({"extra": name, **fn(flush, stream)}), flush=True)


def config(args):
    return {"workload": "uniform cube N=%d, Stokeslet+stresslet, p=%d, theta=%g, N0=%d, %s precision, "
                        "clusters shrunk to their boxes" % (args.N, args.p, args.theta, args.N0, args.precision),
            "N": args.N, "p": args.p, "theta": args.theta, "N0": args.N0, "precision": args.precision,
            "l2": "flushed before every timed step (256 MiB write)", "targets": "all N particles"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only_extra:
        return run_only_extra(args.only_extra)
    import numpy as np
    import torch

    from paper_1811_12498_gb300 import api, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    N, p, theta, N0 = args.N, args.p, args.theta, args.N0
    x, f, h, nu = inputs.uniform_cube(N, inputs.SEED_BASE + 1 + rank)
    hx = [torch.from_numpy(np.ascontiguousarray(a.T)).pin_memory() for a in (x, f, h, nu)]
    dx = [a.cuda() for a in hx]
    stream = torch.cuda.current_stream()
    tc = api.Treecode(args.precision, True, stream)
    u = torch.empty((3, N), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step(inputs_dev):
        tc.build(inputs_dev[0], N0)
        tc.moments(inputs_dev[1], inputs_dev[2], inputs_dev[3], p)
        tc.eval(theta, p, out=u)

    for _ in range(args.warmup):
        step(dx)
    torch.cuda.synchronize()
    peaks = {"fp32": [api.fma_peak("mixed", stream)], "fp64": [api.fma_peak("fp64", stream)]}
    tc.profile(True)
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    launches0 = api.kernel_launches()
    clocks.start()
    times, phases = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(dx)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        phases.append(tc.phase_times())
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = api.kernel_launches() - launches0
    peaks["fp32"].append(api.fma_peak("mixed", stream))
    peaks["fp64"].append(api.fma_peak("fp64", stream))
    ms = max_over_ranks(statistics.mean(times), dist, "cuda")
    value = whole_job_value(N, world, ms)
    st = tc.stats()
    ls = tc.list_stats()
    ph_overlap = {k: statistics.mean(pp[k] for pp in phases if pp[k] is not None)
                  for k in phases[0] if phases[0][k] is not None}
    # per-kernel durations for the rooflines: the same step with the far and
    # near fields serialised (the timed steps above run them concurrently)
    tc.profile(2)
    serial = []
    for _ in range(2):
        flush.fill_(1)
        step(dx)
        torch.cuda.synchronize()
        serial.append(tc.phase_times())
    tc.profile(False)
    ph = {k: statistics.mean(pp[k] for pp in serial if pp[k] is not None)
          for k in serial[0] if serial[0][k] is not None}

    # end to end through the C ABI's host-buffer call (tc_velocity_host): the
    # pinned host inputs are copied in, the step runs, u is copied back to a
    # pinned host array, all inside the one call and the timed region
    uh = torch.empty((3, N), dtype=torch.float64).pin_memory()
    e2e_times = []
    for k in range(args.steps + 1):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tc.velocity_host(hx[0], hx[1], hx[2], hx[3], N0, theta, p, out=uh)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.mean(e2e_times), dist, "cuda")
    e2e_same = bool(torch.equal(uh, u.cpu()))

    if rank != 0:
        tc.close()
        if dist is not None:
            dist.destroy_process_group()
        return

    # accuracy: E against the FP64 direct sum on sampled targets (eq. 6.1)
    u_host = u.cpu().numpy().T
    eidx = inputs.sample_indices(N, args.error_samples, 777)
    tgt = torch.from_numpy(np.ascontiguousarray(x[eidx].T)).cuda()
    ud = api.direct(dx[0], dx[1], dx[2], dx[3], targets=tgt, precision="fp64").cpu().numpy().T
    E = float(np.sqrt(np.sum((u_host[eidx] - ud) ** 2) / np.sum(ud ** 2)))

    # roofline of the dominant kernel (the near field at this configuration):
    # algorithmic flops per launch (43 per Stokeslet + stresslet pair: d 3,
    # r^2 5, 1/r 1, powers 3, three dot products 15, s and t 4, accumulation 12)
    # over its phase time; the far kernel beside it
    n_far = st["far_interactions"]
    fp64 = args.precision == "fp64"
    far_ms = ph.get("far")
    near_ms = ph.get("near")
    # measured peak of the run (best of the FMA-chain probes before and after
    # the timed steps), the nominal one beside it
    peak = max(peaks["fp64" if fp64 else "fp32"])
    nominal = PEAK_FP64_TFLOPS if fp64 else PEAK_FP32_TFLOPS
    peak_kind = ("measured FP64 FMA peak of this run (tc_fma_peak); nominal 1.25 (152 SMs x 2 FMA/clk x 2.07 GHz)"
                 if fp64 else "measured FP32 FMA peak of this run (tc_fma_peak); nominal 80.5 (152 SMs x 128 "
                              "FMA/clk x 2.07 GHz)")
    near_flops = 43.0 * st["near_pairs"]
    near_tf = near_flops / (near_ms / 1e3) / 1e12
    rec_unit, con_unit = far_flops_per_interaction(p)
    rec_flops = rec_unit * n_far
    con_flops = con_unit * n_far
    far_tf = (rec_flops + con_flops) / (far_ms / 1e3) / 1e12
    # the unfolded form: recurrence 11 and contraction 24 flops per coefficient
    # of order <= p+2, plus 18 for d.B
    unfolded_far_flops = (11 + 24) * ncoef(p + 2) + 18
    near_kernel = "k_near_fp64" if fp64 else "k_near_leaf<NearOpU>"
    dominant_near = near_ms >= far_ms
    if dominant_near:
        roof = {"bound": "alu", "kernel": near_kernel + " (near field, 43 flops per pair)", "achieved": near_tf,
                "peak": peak, "unit": "TFLOP/s", "peak_kind": peak_kind, "frac": near_tf / peak,
                "nominal_peak": nominal, "frac_of_nominal": near_tf / nominal,
                "traffic": None if fp64 else kernel_traffic(NEAR_SOURCES, "near_field_uniform_cube_1M.md"),
                "flops_per_launch": near_flops, "launch_ms": near_ms}
    else:
        roof = {"bound": "alu", "kernel": "k_far (far field, folded recurrence + contraction)", "achieved": far_tf,
                "peak": peak, "unit": "TFLOP/s", "peak_kind": peak_kind, "frac": far_tf / peak,
                "nominal_peak": nominal, "frac_of_nominal": far_tf / nominal,
                "traffic": None if fp64 else kernel_traffic(FAR_SOURCES, "far_field_uniform_cube_524k.md"),
                "flops_per_launch": rec_flops + con_flops, "launch_ms": far_ms}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": config(args),
        "roofline": roof,
        "e2e": {"value": N / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(sum(a.numel() * 8 for a in hx)),
                "d2h_bytes_per_step": int(uh.numel() * 8), "ms_per_step": e2e_ms,
                "call": "tc_velocity_host (pinned host arrays in and out, copies inside the call)",
                "same_result_as_device_path": e2e_same},
        "measured_peaks_tflops": {"fp32": peaks["fp32"], "fp64": peaks["fp64"],
                                  "how": "tc_fma_peak before and after the timed steps (FMA chains, 8 blocks of 256 "
                                         "threads per SM, best of 5 launches)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "phases_ms": ph,
        "phases_ms_note": "each phase alone (far and near serialised); the timed steps run the far and near "
                          "fields concurrently",
        "phases_ms_concurrent": ph_overlap,
        "interactions": {"far": n_far, "near_pairs": st["near_pairs"], "clusters": st["clusters"],
                         "far_entries": ls["far_entries"], "near_entries": ls["near_entries"],
                         "far_lane_use": ls["far_lane_use"], "near_lane_use": ls["near_lane_use"]},
        "secondary": {"near_tflops": near_tf, "near_frac": near_tf / peak,
                      "far_tflops_folded_count": far_tf, "far_frac_folded_count": far_tf / peak,
                      "far_flops_per_interaction_folded": rec_unit + con_unit,
                      "far_tflops_unfolded_count": unfolded_far_flops * n_far / (far_ms / 1e3) / 1e12,
                      "far_flops_per_interaction_unfolded": unfolded_far_flops,
                      "near_plus_far_frac_unfolded_count":
                          (near_flops + unfolded_far_flops * n_far) / ((near_ms + far_ms) / 1e3) / 1e12 / peak,
                      # the whole timed step against the FP32 peak, counting the work per target as
                      # 43 flops per near pair plus the unfolded FP32 contraction (24 C(p+5,3) + 18)
                      # per far interaction, without and with the unfolded recurrence (11 C(p+5,3))
                      "step_frac_fp32_count":
                          (near_flops + (24 * ncoef(p + 2) + 18) * n_far) / (ms / 1e3) / 1e12 / peak,
                      "step_frac_fp32_count_with_recurrence":
                          (near_flops + unfolded_far_flops * n_far) / (ms / 1e3) / 1e12 / peak},
        "accuracy": {"E_vs_fp64_direct": E, "E_samples": int(len(eidx))},
    }
    if not args.no_fp64_compare and args.precision == "mixed":
        def other_path(precision, rec64):
            t2 = api.Treecode(precision, True, stream, rec64=rec64)
            t2.build(dx[0], N0).moments(dx[1], dx[2], dx[3], p)
            u2 = t2.eval(theta, p)
            torch.cuda.synchronize()
            times = []
            for _ in range(2):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                t2.build(dx[0], N0).moments(dx[1], dx[2], dx[3], p)
                t2.eval(theta, p, out=u2)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            t2.close()
            return statistics.mean(times), u2.cpu().numpy().T

        def rel(a, b):
            return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))

        ms64, u64h = other_path("fp64", False)
        line["fp64_path"] = {"ms_per_step": ms64, "value": N / (ms64 / 1e3), "mixed_vs_fp64_rel_l2": rel(u_host, u64h)}
        msr, urh = other_path("mixed", True)
        line["mixed_fp64_recurrence_path"] = {"ms_per_step": msr, "value": N / (msr / 1e3),
                                              "vs_fp64_rel_l2": rel(urh, u64h),
                                              "note": "tc_config.rec64: far-field recurrence in FP64 for p >= 8"}
    if not args.no_cpu_baseline:
        cb, idx, uo = cpu_baseline(x, f, h, nu, args, args.cpu_sample)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cb1, _, _ = cpu_baseline(x, f, h, nu, args, args.cpu_sample_1t, threads=1)
        line["cpu_baseline"]["one_thread"] = {k: cb1[k] for k in ("value", "unit", "cores", "sample")}
        line["accuracy"]["vs_oracle_treecode"] = float(np.sqrt(np.sum((u_host[idx] - uo) ** 2) / np.sum(uo ** 2)))
        line["accuracy"]["oracle_samples"] = int(len(idx))
    if not args.no_extras:
        line["fwd_adjoint"] = bench_fwd_adjoint(flush, stream)
        line["batched"] = bench_batched(flush, stream)
        line["table1_sphere"] = bench_table1(flush, stream)
        line["fig3_sphere"] = bench_fig3(flush, stream)
        line["regularized"] = bench_regularized(flush, stream)
        if not args.no_sweep:
            line["sphere_sweep"] = bench_sphere_sweep(flush, stream)
    print(json.dumps(line), flush=True)
    tc.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
