#!/usr/bin/env python
"""Benchmark of the grouped Barnes-Hut force calculation on GB300.

Workload: Plummer sphere, N = 1,048,576 equal masses, theta = 0.5, N_leaf = 16,
eps = 0.01, G = 1 (synthetic, seeded). One step = one tree walk + evaluation
of all N particles (the fused sm_103a kernel) on the tree already resident in
HBM; L2 is flushed (256 MiB write) before every timed step, outside the timed
events. The line also reports:
  e2e           the same metric through the one-shot C-ABI call with host
                buffers and the tree built on the host in FP64, the paper's
                split (octgrav_forces_ex), with its phases; beside it the
                one-shot call that builds the same tree on the GPU
                (octgrav_forces_gpu, pinned buffers);
  roofline      paper-convention flops (38 per particle-particle, 70 per
                particle-cell interaction, Sec. 3.3) per launch / kernel time,
                against the FP32 CUDA-core peak (SMs x 128 lanes x 2 x max clock);
  cpu_baseline  the FP64 CPU oracle on the host cores (full tree build plus a
                bounded sample of groups, scaled to N);
  accuracy      FP32 kernel vs FP64 oracle on sampled groups (relative RMS) and
                vs direct summation on sampled particles (median / p99 Delta a/a).

Multi-GPU (torchrun): every rank computes its own independent system
(seed + rank); value = total particles over all ranks / max time over ranks.
--impl reference times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

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

from paper_1005_5384_gb300 import ranks as RK  # noqa: E402
from paper_1005_5384_gb300 import workloads as W  # noqa: E402

METRIC = "particle forces/sec and GFLOP/s (frac of FP32 peak) at N=1M θ=0.5, at median rel err 1e-3"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="octgrav", choices=["octgrav", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--n-leaf", type=int, default=16)
    ap.add_argument("--n-group", type=int, default=0, help="0 = chosen by the autotuner")
    ap.add_argument("--ppl", type=int, default=0, help="0 = chosen by the autotuner")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the theta scan, clustered and ensemble legs")
    ap.add_argument("--no-balance", action="store_true",
                    help="keep the default work-item order (most particles first) instead of longest first "
                         "by the costs of the first warm-up launch")
    ap.add_argument("--sweep-n", default="30000,100000,300000,1000000",
                    help="particle numbers of --leg accuracy (comma separated)")
    ap.add_argument("--leg", default="", choices=["", "learned", "build", "accuracy", "small"],
                    help="learned: train the criterion on the 1M sphere+disc and launch the learned walk "
                         "twice (a small driver for profilers; prints the interaction counts); build: "
                         "--warmup + --steps GPU tree builds of the workload (prints their wall times); "
                         "accuracy: error distribution and throughput over theta, N and N_leaf on the "
                         "galaxy stand-in (one JSON line per configuration, then the fitted theta slopes); "
                         "small: C1 with the autotuner's launch shape, one launch then four (a profiler driver)")
    return ap.parse_args()


def workload_name(a):
    return ("plummer N=%d theta=%g N_leaf=%d N_group=%d eps=%g G=1" %
            (a.n, a.theta, a.n_leaf, a.n_group, a.eps))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()  # let the sampler produce its first row before the timed region
            while not self.rows and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.rows.clear()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def fp32_peak_tflops(torch):
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flops (FMA) x max SM clock."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU (MEASURED_PEAKS.json), else the profiling fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def kernel_sources_sha256():
    """sha256 of the kernel source and of the header holding the work-item rule:
    the DRAM traffic of a launch depends on both."""
    import hashlib
    h = hashlib.sha256()
    for f in ("octgrav_kernels.cu", "octgrav_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1005_5384_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(a):
    """DRAM bytes per launch from the committed ncu summary, if it matches this kernel and workload."""
    try:
        sha, table = None, {}
        for line in open(os.path.join(ROOT, "profiles", "walk_eval_traffic.txt")):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("kernel_sources_sha256_prefix:"):
                sha = line.split(":", 1)[1].strip()
            elif " = " in line:
                k, v = line.rsplit(" = ", 1)
                table[k.strip()] = int(v)
        if kernel_sources_sha256()[:16] != sha:
            return None
        return table.get(workload_name(a))
    except (OSError, ValueError):
        return None


def cpu_baseline(pos, m, a, budget_s, acc=None):
    """The oracle timed on all host cores, defined as the GPU's value is: forces
    of the tree walk and evaluation with the tree already built (the FP64 tree
    build is timed and reported apart, t_build_s). A random sample of groups
    sized to budget_s; value = particles evaluated / time. With the kernel's
    accelerations (acc, input order) it also reports their deviation from the
    oracle's FP64 forces on that sample: the global relative RMS and the
    per-particle median and 99th percentile of |a_gpu - a_oracle| / |a_oracle|."""
    import oracle as O
    threads = O.default_threads()
    t0 = time.perf_counter()
    R = O.Tree(pos, m, a.n_leaf, a.n_group)
    t_build = time.perf_counter() - t0
    # calibrate on a small sample, then size the timed sample to the budget
    rng = np.random.default_rng(123)
    probe = np.sort(rng.choice(R.n_groups, size=min(R.n_groups, 64), replace=False))
    t0 = time.perf_counter()
    R.forces(a.eps, a.theta, groups=probe, nthreads=threads, counts=False)
    t_probe = max(1e-6, time.perf_counter() - t0)
    ng = int(min(R.n_groups, max(64, 64 * budget_s / t_probe)))
    gs = np.sort(rng.choice(R.n_groups, size=ng, replace=False))
    npart = int(R.count[R.groups[gs]].sum())
    t0 = time.perf_counter()
    ra, _, _, _, _ = R.forces(a.eps, a.theta, groups=gs, nthreads=threads, counts=False)
    t_forces = time.perf_counter() - t0
    line = {"value": npart / t_forces, "unit": "forces/s", "cores": threads, "kind": "oracle",
            "sample": "forces of %d random groups (%d of N=%d particles, %.2fs), tree already built"
                      % (ng, npart, a.n, t_forces),
            "t_build_s": t_build, "t_forces_sample_s": t_forces}
    # the same on one core, a smaller sample
    g1 = gs[:: max(1, min(4 * threads, len(gs) // 8))]  # every k-th sampled group
    n1 = int(R.count[R.groups[g1]].sum())
    t0 = time.perf_counter()
    R.forces(a.eps, a.theta, groups=g1, nthreads=1, counts=False)
    t1 = time.perf_counter() - t0
    line["one_core"] = {"value": n1 / t1, "unit": "forces/s", "cores": 1,
                        "sample": "forces of %d groups (%d particles, %.2fs) on 1 thread, tree already built"
                                  % (len(g1), n1, t1)}
    if acc is not None:
        idx = np.concatenate([R.cell_members(int(R.groups[g])) for g in gs])
        e = O.rel_err(acc[idx], ra[idx])
        line["kernel_vs_oracle_rel_rms"] = O.rel_rms(acc[idx], ra[idx])
        line["kernel_vs_oracle_median_rel"] = float(np.median(e))
        line["kernel_vs_oracle_p99_rel"] = float(np.percentile(e, 99))
        line["kernel_vs_oracle_max_rel"] = float(np.max(e))
        line["kernel_vs_oracle_particles"] = int(len(idx))
    return line


def accuracy(G, acc, pos, m, a):
    """Delta a/a of the kernel against FP64 direct sums (on the GPU) at 1024 sampled particles."""
    samp = W.sample_indices(a.n, 1024, seed=17)
    ad, _ = G.direct(pos, m, a.eps, targets=samp)
    e = G.rel_err(acc[samp], ad)
    return {"median_rel_err_vs_direct": float(np.median(e)), "p99_rel_err_vs_direct": float(np.percentile(e, 99)),
            "direct_sample": int(len(samp)), "direct": "FP64 direct summation on the GPU (octgrav_direct)"}


def time_kernel(torch, launch, flush, steps, stream):
    """Median CUDA-event time (ms) of `launch()` over `steps` runs, L2 flushed before each."""
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launch()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def device_acc(torch, T, out, n):
    acc = np.empty((n, 3))
    acc[T.perm()] = out.cpu().numpy()[:, :3]
    return acc


def theta_for_median(torch, G, T, out, eps, samp, ad, target=1e-3, lo=0.5, hi=2.5, iters=9):
    """Bisect theta so that the median Delta a/a over the sampled particles hits target."""

    def med(th):
        T.forces_device(eps, th, out)
        torch.cuda.synchronize()
        acc = device_acc(torch, T, out, T.n)
        return float(np.median(G.rel_err(acc[samp], ad)))
    m_lo, m_hi = med(lo), med(hi)
    if not (m_lo < target < m_hi):
        return None, None
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        mm = med(mid)
        if mm < target:
            lo, m_lo = mid, mm
        else:
            hi, m_hi = mid, mm
    return lo, m_lo


def extras(torch, G, a, pos, m, T, out, flush, stream, peak, steps):
    res = {}
    # tree build: the host FP64 build against the same tree built on the GPU
    xd = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    md = torch.from_numpy(np.ascontiguousarray(m)).cuda()
    gb, hb = [], []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B = G.Tree.build_gpu(xd, md, a.n_leaf, a.n_group, stream=stream)
        gb.append(1e3 * (time.perf_counter() - t0))
    for _ in range(3):
        t0 = time.perf_counter()
        H = G.Tree.build(pos, m, a.n_leaf, a.n_group)
        hb.append(1e3 * (time.perf_counter() - t0))
    res["tree_build"] = {"n": a.n, "gpu_ms": statistics.median(gb[1:]), "host_ms": statistics.median(hb[1:]),
                         "host_threads": os.cpu_count(),
                         "identical": bool(np.array_equal(B.cell_keys(), H.cell_keys())
                                           and np.array_equal(B.perm(), H.perm()))}
    del B, H, xd, md
    # time integration: leapfrog steps of a 1M Plummer sphere in equilibrium, the
    # tree rebuilt on the GPU for every force evaluation, state on the device
    xs, vs, ms_ = W.plummer_pv(a.n, seed=a.seed)
    S = G.Sim(xs, vs, ms_, a.eps, a.theta, n_leaf=a.n_leaf, n_group=a.n_group, stream=stream)
    e0 = sum(S.energy(stream=stream))
    S.step(1.0 / 128, 1, stream=stream)
    nsteps = 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.step(1.0 / 128, nsteps, stream=stream)
    dt_wall = time.perf_counter() - t0
    e1 = sum(S.energy(stream=stream))
    # the same with a full build every 4th step and refits in between
    S.set_rebuild(4)
    S.step(1.0 / 128, 4, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.step(1.0 / 128, nsteps, stream=stream)
    dt_refit = time.perf_counter() - t0
    e2 = sum(S.energy(stream=stream))
    res["leapfrog_plummer_1M"] = {"dt": 1.0 / 128, "steps": nsteps, "ms_per_step": 1e3 * dt_wall / nsteps,
                                  "particle_steps_per_s": a.n * nsteps / dt_wall,
                                  "rel_energy_change_9_steps": (e1 - e0) / abs(e0),
                                  "per_step": "kick+drift, GPU tree build, walk+evaluation, unpermute, kick",
                                  "rebuild_every_4": {"ms_per_step": 1e3 * dt_refit / nsteps,
                                                      "particle_steps_per_s": a.n * nsteps / dt_refit,
                                                      "rel_energy_change_21_steps": (e2 - e0) / abs(e0)}}
    del S
    # C1: the 16,384-particle Plummer sphere (the parity workload), theta 0.5
    spos, sm = W.plummer(16384, seed=1)
    stuned = G.autotune([(spos, sm)], n_leaf=a.n_leaf, eps=a.eps, theta=0.5, candidates=(16, 32, 64, 128),
                        stream=stream)
    ST = G.Tree.build(spos, sm, a.n_leaf, stuned["n_group"])
    ST.set_launch(stuned["particles_per_lane"])
    ST.set_split(stuned["split"])
    ST.set_staging(stuned["staging"])
    sout = torch.empty((ST.n, 4), dtype=torch.float32, device="cuda")
    ST.forces_device(a.eps, 0.5, sout, stream=stream)
    ST.balance(stream=stream)
    ms = time_kernel(torch, lambda: ST.forces_device(a.eps, 0.5, sout, stream=stream), flush, steps, stream)
    c = ST.interaction_counts()
    res["plummer_16k"] = {"autotuned": stuned, "forces_per_s": ST.n / (ms * 1e-3), "ms": ms,
                          "frac_fp32_peak": c["flops"] / ms / 1e9 / peak, "flops_per_particle": c["flops"] / ST.n}
    del ST, sout
    # C2 (theta 0.5) with each staging mode of the accepted cell records, the
    # same tree and item order; results are bitwise identical across modes
    ref_bits = None
    stag = {}
    for mode, name in ((1, "cp.async per lane"), (2, "TMA tile::gather4"), (0, "cp.async.bulk per record")):
        T.set_staging(mode)
        T.forces_device(a.eps, a.theta, out, stream=stream)
        torch.cuda.synchronize()
        bits = out.view(torch.int32).clone()
        if ref_bits is None:
            ref_bits = bits
        stag[name] = {"mode": mode, "ms": time_kernel(torch, lambda: T.forces_device(a.eps, a.theta, out, stream=stream),
                                                         flush, steps, stream),
                      "bitwise_equal_to_cp_async": bool(torch.equal(bits, ref_bits))}
    T.set_staging(1)
    res["staging_modes_plummer_1M"] = stag
    # C2 at theta = 0.75
    T.forces_device(a.eps, 0.75, out, stream=stream)
    ms = time_kernel(torch, lambda: T.forces_device(a.eps, 0.75, out, stream=stream), flush, steps, stream)
    c = T.interaction_counts()
    res["plummer_theta0.75"] = {"forces_per_s": a.n / (ms * 1e-3), "ms": ms, "frac_fp32_peak": c["flops"] / ms / 1e9 / peak,
                                "flops_per_particle": c["flops"] / a.n}
    # C2 at the theta whose median Delta a/a vs direct summation is 1e-3
    samp = W.sample_indices(a.n, 1024, seed=17)
    ad, _ = G.direct(pos, m, a.eps, targets=samp)
    th, md = theta_for_median(torch, G, T, out, a.eps, samp, ad)
    if th is not None:
        ms = time_kernel(torch, lambda: T.forces_device(a.eps, th, out, stream=stream), flush, steps, stream)
        c = T.interaction_counts()
        res["plummer_median_1e-3"] = {"theta": th, "median_rel_err": md, "forces_per_s": a.n / (ms * 1e-3),
                                      "ms": ms, "frac_fp32_peak": c["flops"] / ms / 1e9 / peak,
                                      "flops_per_particle": c["flops"] / a.n, "n_group": a.n_group}
        # the group size is part of the operating point: the same search at N_group 256
        T2 = G.Tree.build(pos, m, a.n_leaf, 256)
        T2.forces_device(a.eps, th, out, stream=stream)
        T2.balance(stream=stream)
        th2, md2 = theta_for_median(torch, G, T2, out, a.eps, samp, ad)
        if th2 is not None:
            ms2 = time_kernel(torch, lambda: T2.forces_device(a.eps, th2, out, stream=stream), flush, steps, stream)
            c2 = T2.interaction_counts()
            res["plummer_median_1e-3"]["at_n_group_256"] = {
                "theta": th2, "median_rel_err": md2, "forces_per_s": a.n / (ms2 * 1e-3), "ms": ms2,
                "frac_fp32_peak": c2["flops"] / ms2 / 1e9 / peak, "flops_per_particle": c2["flops"] / a.n}
        del T2
    # C3: clustered, 4,194,304 particles, theta 0.5, eps 0.001
    cpos, cm = W.clustered(4_194_304, 64, seed=3)
    CT = G.Tree.build(cpos, cm, a.n_leaf, a.n_group)
    cout = torch.empty((CT.n, 4), dtype=torch.float32, device="cuda")
    CT.forces_device(0.001, 0.5, cout, stream=stream)
    CT.balance(stream=stream)
    ms = time_kernel(torch, lambda: CT.forces_device(0.001, 0.5, cout, stream=stream), flush, steps, stream)
    c = CT.interaction_counts()
    cacc = device_acc(torch, CT, cout, CT.n)
    csamp = W.sample_indices(CT.n, 1024, seed=19)
    cad, _ = G.direct(cpos, cm, 0.001, targets=csamp)
    ce = G.rel_err(cacc[csamp], cad)
    res["clustered_4M"] = {"workload": "64 Plummer spheres N=4194304 theta=0.5 eps=0.001 N_leaf=%d N_group=%d"
                                       % (a.n_leaf, a.n_group),
                           "forces_per_s": CT.n / (ms * 1e-3), "ms": ms,
                           "frac_fp32_peak": c["flops"] / ms / 1e9 / peak,
                           "median_rel_err_vs_direct": float(np.median(ce)),
                           "p99_rel_err_vs_direct": float(np.percentile(ce, 99))}
    del CT, cout
    # C4: 256-system ensemble, one graph-captured persistent launch, autotuned
    systems = W.ensemble(256, seed=4)
    best = G.autotune(systems, n_leaf=a.n_leaf, eps=0.01, theta=0.6, candidates=(16, 32, 64, 128, 256, 512),
                      stream=stream)
    ET = G.Tree.build_batch(systems, a.n_leaf, best["n_group"])
    ET.set_launch(best["particles_per_lane"])
    ET.set_split(best["split"])
    ET.set_staging(best["staging"])
    eout = torch.empty((ET.n, 4), dtype=torch.float32, device="cuda")
    gstream = torch.cuda.Stream()
    with torch.cuda.stream(gstream):
        ET.forces_device(0.01, 0.6, eout, stream=gstream)
        ET.balance(stream=gstream)  # the captured launch takes the items longest first
        ET.capture_graph(0.01, 0.6, eout, stream=gstream)
        ET.launch_graph(stream=gstream)
        gstream.synchronize()
        ms = time_kernel(torch, lambda: ET.launch_graph(stream=gstream), flush, steps, gstream)
    c = ET.interaction_counts(stream=gstream)
    eacc = device_acc(torch, ET, eout, ET.n)
    errs = []
    for s in range(0, 256, 37):  # Delta a/a against direct sums inside each sampled system
        pos_s, m_s = systems[s]
        sa = W.sample_indices(len(m_s), 256, seed=s)
        ds, _ = G.direct(pos_s, m_s, 0.01, targets=sa)
        errs.append(float(np.median(G.rel_err(eacc[ET.offsets[s]:ET.offsets[s + 1]][sa], ds))))
    res["ensemble_256"] = {"workload": "256 Plummer systems, N log-uniform in [1024, 65536], total N=%d, theta=0.6 "
                                       "eps=0.01 N_leaf=%d" % (ET.n, a.n_leaf),
                           "autotuned": best, "launch": "CUDA graph replay of one persistent launch",
                           "forces_per_s": ET.n / (ms * 1e-3), "ms": ms,
                           "frac_fp32_peak": c["flops"] / ms / 1e9 / peak,
                           "median_rel_err_vs_direct_7_systems": errs}
    del ET, eout
    # C4 end to end through the one-shot batched call: pinned host arrays in,
    # FP64 input-order results out (copies, GPU builds, one launch, unpermute)
    off = np.zeros(len(systems) + 1, np.int64)
    off[1:] = np.cumsum([len(m_s) for _, m_s in systems])
    ntot = int(off[-1])
    hpos = torch.empty((ntot, 3), dtype=torch.float64).pin_memory()
    hmass = torch.empty(ntot, dtype=torch.float64).pin_memory()
    hpos.numpy()[:] = np.concatenate([p_s for p_s, _ in systems])
    hmass.numpy()[:] = np.concatenate([m_s for _, m_s in systems])
    hacc = torch.empty((ntot, 3), dtype=torch.float64).pin_memory()
    hpot = torch.empty(ntot, dtype=torch.float64).pin_memory()
    args = ((off, hpos.numpy(), hmass.numpy()), np.full(len(systems), 0.01), np.full(len(systems), 0.6))
    kw = dict(n_leaf=a.n_leaf, n_group=best["n_group"], out=(hacc.numpy(), hpot.numpy()))
    G.forces_batched(*args, **kw)  # first call: per-thread device buffers, build graph
    ts = []
    for _ in range(max(3, min(steps, 10))):
        t0 = time.perf_counter()
        G.forces_batched(*args, **kw)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    res["ensemble_256"]["e2e_forces_batched"] = {
        "value": ntot / t, "unit": "forces/s", "seconds_per_call": t, "h2d_bytes_per_call": 32 * ntot,
        "d2h_bytes_per_call": 32 * ntot,
        "path": "octgrav_forces_batched_ex (pinned host arrays, per-system eps/theta; H2D, GPU builds of all "
                "systems, one launch, device unpermute, FP64 D2H), host wall clock per call"}
    del hpos, hmass, hacc, hpot
    # N_group 256: the fastest group size for both walks here (64: 403 / 454 M forces/s,
    # 512: 439 / 491 M with 96 training groups)
    res["learned_criterion_sphere_disc_1M"] = learned_leg(torch, G, a, flush, stream, peak, steps, ng=256,
                                                          train_groups=256)
    return res


def near_band(f, lab, theta_lo):
    """The training samples whose cell size over distance (input 3) is at least
    0.7 theta_lo: well below the band the plain test accepts the cell and the
    network never sees it, so those pairs only dilute the training (measured:
    1.197-1.202x over the theta walk against 1.174-1.191x with every sample,
    four training seeds)."""
    keep = f[:, 3] >= 0.7 * theta_lo
    return np.ascontiguousarray(f[keep]), np.ascontiguousarray(lab[keep])


def learned_leg(torch, G, a, flush, stream, peak, steps, ng=64, train_groups=128):
    """C5: sphere + disc, N = 1,048,576; the plain theta walk and the learned
    criterion, each tuned to a median Delta a/a of 1e-3 against direct sums
    (groups of at most ng particles; the network trains on train_groups of them)."""
    n = 1_048_576
    # the band measured fastest at equal error on this workload (sweep over
    # (theta_lo, theta_hi) and N_group 128 / 256 / 512, see the design notes)
    band = dict(theta_lo=0.85, theta_hi=1.5, theta_fb=1.0)
    t0 = time.perf_counter()
    tpos, tm = W.sphere_disc(n, seed=6)                 # training system (another seed)
    TT = G.Tree.build(tpos, tm, a.n_leaf, ng)
    groups = np.sort(np.random.default_rng(0).choice(TT.stats["n_groups"], train_groups, replace=False))
    f, lab, _ = TT.mlp_samples(groups, 0.35, 0.01, stream=stream)
    n_all = len(lab)
    f, lab = near_band(f, lab, band["theta_lo"])
    rec, loss = G.mlp_train(f, lab, steps=3000, batch=4096, lr=2e-3, seed=3, stream=stream)
    t_train = time.perf_counter() - t0
    del TT
    pos, m = W.sphere_disc(n, seed=5)
    T = G.Tree.build(pos, m, a.n_leaf, ng)
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    samp = W.sample_indices(n, 1024, seed=23)
    ad, _ = G.direct(pos, m, 0.01, targets=samp)

    def med(theta):
        T.forces_device(0.01, theta, out, stream=stream)
        torch.cuda.synchronize()
        return float(np.median(G.rel_err(device_acc(torch, T, out, n)[samp], ad)))

    def bisect(fn, lo, hi, iters=10):
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            if fn(mid) < 1e-3:
                lo = mid
            else:
                hi = mid
        return lo
    th = bisect(med, 0.3, 2.0)
    e_th = med(th)
    c_th = T.interaction_counts()
    ni_th = T.stats["n_items"]  # 33..48-particle rests cut 32 + rest
    T.balance(stream=stream)  # both walks timed longest first, from their own last launch
    ms_th = time_kernel(torch, lambda: T.forces_device(0.01, th, out, stream=stream), flush, steps, stream)
    T.balance(0)

    def med_tau(tau):
        T.set_criterion(rec, tau=tau, **band)
        return med(0.5)
    tau = bisect(med_tau, -6.0, -1.0)
    e_ml = med_tau(tau)
    c_ml = T.interaction_counts()
    ni_ml = T.stats["n_items"]  # set_criterion cut the items again, rests whole
    T.balance(stream=stream)
    ms_ml = time_kernel(torch, lambda: T.forces_device(0.01, 0.5, out, stream=stream), flush, steps, stream)
    return {"workload": "sphere (r=1) + exponential disc (R_d=0.3, z_d=0.03), N=1048576, eps=0.01, "
                        "N_leaf=%d N_group=%d" % (a.n_leaf, ng),
            "training": {"system": "same recipe, seed 6", "groups": train_groups, "samples": int(len(lab)),
                         "samples_of_the_walk": n_all, "kept": "l/d >= 0.7 theta_lo",
                         "steps": 3000, "final_loss": loss, "seconds": t_train},
            "theta_walk": {"theta": th, "median_rel_err": e_th, "forces_per_s": n / (ms_th * 1e-3), "ms": ms_th,
                           "flops_per_particle": c_th["flops"] / n, "work_items": ni_th,
                           "frac_fp32_peak": c_th["flops"] / ms_th / 1e9 / peak},
            "learned_walk": {"tau": tau, "band": band, "median_rel_err": e_ml, "forces_per_s": n / (ms_ml * 1e-3),
                             "ms": ms_ml, "flops_per_particle": c_ml["flops"] / n, "work_items": ni_ml,
                             "frac_fp32_peak": c_ml["flops"] / ms_ml / 1e9 / peak},
            "speedup_learned_over_theta": ms_th / ms_ml}


def run_small_driver():
    """C1 as the autotuner launches it (16k Plummer, N_group 128, one particle per
    lane, lists split over 4 warps): one launch, the order by its costs, then four
    more (a small driver for profilers)."""
    import torch
    from paper_1005_5384_gb300 import octgrav as G
    n = 16384
    pos, m = W.plummer(n, seed=1)
    T = G.Tree.build(pos, m, 16, 128)
    T.set_launch(1)
    T.set_split(4)
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.5, out)
    T.balance()
    for _ in range(4):
        T.forces_device(0.01, 0.5, out)
    torch.cuda.synchronize()
    print(json.dumps({"leg": "small", "status": T.status(), "counts": T.interaction_counts()}), flush=True)


def run_learned_driver():
    """Train on the sphere+disc (seed 6); on seed 5 launch the plain walk at
    theta 0.93 (its median-1e-3 point) once, then the learned walk twice."""
    import torch
    from paper_1005_5384_gb300 import octgrav as G
    n = 1_048_576
    pos, m = W.sphere_disc(n, seed=6)
    TT = G.Tree.build(pos, m, 16, 256)
    groups = np.sort(np.random.default_rng(0).choice(TT.stats["n_groups"], 64, replace=False))
    f, lab, _ = TT.mlp_samples(groups, 0.35, 0.01)      # includes one plain-test launch
    f, lab = near_band(f, lab, 0.85)
    rec, _ = G.mlp_train(f, lab, steps=3000, batch=4096, lr=2e-3, seed=3)
    del TT
    pos, m = W.sphere_disc(n, seed=5)
    T = G.Tree.build(pos, m, 16, 256)
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    T.forces_device(0.01, 0.93, out)
    torch.cuda.synchronize()
    plain = T.interaction_counts()
    T.set_criterion(rec, tau=-3.6, theta_lo=0.85, theta_hi=1.5, theta_fb=1.0)  # the C5 leg's band and tau
    for _ in range(2):
        T.forces_device(0.01, 0.5, out)
    torch.cuda.synchronize()
    print(json.dumps({"status": T.status(), "counts_theta_0.93": plain, "counts_learned": T.interaction_counts()}),
          flush=True)


def run_build_driver(a):
    """The GPU tree build alone: warm-up builds, then --steps builds of the
    workload's tree from device-resident positions (profiling driver)."""
    import torch
    from paper_1005_5384_gb300 import octgrav as G
    pos, m = W.plummer(a.n, seed=a.seed)
    xd = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    md = torch.from_numpy(np.ascontiguousarray(m)).cuda()
    ng = a.n_group if a.n_group > 0 else 512
    ms = []
    for k in range(a.warmup + a.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B = G.Tree.build_gpu(xd, md, a.n_leaf, ng)
        if k >= a.warmup:
            ms.append(1e3 * (time.perf_counter() - t0))
        del B
    print(json.dumps({"leg": "build", "n": a.n, "n_group": ng, "ms": ms}), flush=True)


def run_accuracy_driver(a):
    """The paper's accuracy study (Sec. 3.1): Delta a/a of the tree against FP64
    direct sums at 1024 sampled particles, for theta = 0.2 ... 0.7, several N
    and N_leaf in {8, 16, 64} (N_group = max(64, N_leaf), the paper's 64), on
    the galaxy stand-in (bulge : disc : halo = 1 : 1 : 4), eps = 0.01; the
    kernel time is the median of 3 CUDA-event timings (no L2 flush)."""
    import torch
    from paper_1005_5384_gb300 import octgrav as G
    G.load()
    thetas = (0.2, 0.3, 0.4, 0.5, 0.6, 0.7)
    eps = 0.01
    peak, _, _ = fp32_peak_tflops(torch)
    fits = []
    for n in (int(v) for v in a.sweep_n.split(",")):
        pos, m = W.galaxy(n, seed=9)
        samp = W.sample_indices(n, 1024, seed=31)
        ad, _ = G.direct(pos, m, eps, targets=samp)
        xd = torch.from_numpy(pos).cuda()
        md = torch.from_numpy(m).cuda()
        for nl in (8, 16, 64):
            ng = max(64, nl)
            T = G.Tree.build_gpu(xd, md, nl, ng)
            perm = T.perm()
            out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
            meds = []
            for th in thetas:
                T.forces_device(eps, th, out)
                torch.cuda.synchronize()
                ts = []
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    T.forces_device(eps, th, out)
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                if T.status() != G.OK:
                    raise SystemExit("device status %d" % T.status())
                acc = np.empty((n, 3))
                acc[perm] = out.cpu().numpy()[:, :3]
                err = G.rel_err(acc[samp], ad)
                c = T.interaction_counts()
                meds.append(float(np.median(err)))
                print(json.dumps({"n": n, "n_leaf": nl, "n_group": ng, "theta": th,
                                  "median": float(np.median(err)), "p90": float(np.percentile(err, 90)),
                                  "p99": float(np.percentile(err, 99)), "ms": ms, "forces_per_s": n / (ms * 1e-3),
                                  "flops_per_particle": c["flops"] / n,
                                  "frac_fp32_peak": c["flops"] / ms / 1e9 / peak}), flush=True)
            slope = float(np.polyfit(np.log(thetas), np.log(meds), 1)[0])
            fits.append({"n": n, "n_leaf": nl, "median_theta_slope": slope})
            del T, out
    print(json.dumps({"leg": "accuracy", "workload": "galaxy stand-in (bulge:disc:halo 1:1:4), eps=0.01",
                      "fits": fits}), flush=True)


def run_reference(a, rank, world):
    """The oracle arm: the FP64 CPU tree code on the host's cores, on the
    headline workload, defined as the GPU's value is (forces of the walk and
    evaluation with the tree built beforehand; the build is timed apart). A
    timed step evaluates all N particles when --steps such steps fit in about
    four minutes, else a fixed random sample of groups sized to fit (the
    line's ms_per_step is then the sample's measured time and
    full_n_step_ms_estimate the extrapolation). Warm-up steps (nothing to warm
    in a CPU program) evaluate a small sample."""
    if rank != 0:
        return
    import oracle as O
    pos, m = W.plummer(a.n, seed=a.seed)
    threads = O.default_threads()
    if a.n_group <= 0:
        a.n_group = 256  # the group size the GPU autotuner selects for this workload on GB300
    t0 = time.perf_counter()
    R = O.Tree(pos, m, a.n_leaf, a.n_group)
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(5)
    probe = np.sort(rng.choice(R.n_groups, size=min(R.n_groups, 256), replace=False))
    t0 = time.perf_counter()
    R.forces(a.eps, a.theta, groups=probe, counts=False)
    tp = max(1e-6, time.perf_counter() - t0)
    full_est = tp * a.n / int(R.count[R.groups[probe]].sum())
    budget = 240.0 / max(1, a.steps)  # seconds per timed step
    if full_est <= budget:
        gs_timed = None
        npart = a.n
        what = "all N=%d particles per step" % a.n
    else:
        ng = int(max(16, R.n_groups * budget / full_est))
        gs_timed = np.sort(rng.choice(R.n_groups, size=ng, replace=False))
        npart = int(R.count[R.groups[gs_timed]].sum())
        what = "%d random groups (%d of N=%d particles) per step" % (ng, npart, a.n)
    gs_warm = np.sort(rng.choice(R.n_groups, size=max(1, R.n_groups // 32), replace=False))
    for _ in range(a.warmup):
        R.forces(a.eps, a.theta, groups=gs_warm, counts=False)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        R.forces(a.eps, a.theta, groups=gs_timed, counts=False)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = npart / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "forces/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "l2": "n/a (CPU)"},
            "t_build_s": t_build,
            "cpu_baseline": {"value": value, "unit": "forces/s", "cores": threads, "kind": "oracle",
                             "sample": "forces of %s, tree built beforehand (%.2fs); warm-up steps "
                                       "%d groups each" % (what, t_build, len(gs_warm))},
            "e2e": {"value": value, "unit": "forces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if gs_timed is not None:
        line["full_n_step_ms_estimate"] = ms * a.n / npart
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.leg == "learned":
        run_learned_driver()
        return
    if a.leg == "small":
        run_small_driver()
        return
    if a.leg == "build":
        run_build_driver(a)
        return
    if a.leg == "accuracy":
        run_accuracy_driver(a)
        return

    import torch
    from paper_1005_5384_gb300 import octgrav as G

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    pos, m = W.plummer(a.n, seed=RK.rank_seed(a.seed, rank))
    G.load()
    tuned = None
    if a.n_group <= 0 or a.ppl <= 0:
        tuned = G.autotune([(pos, m)], n_leaf=a.n_leaf, eps=a.eps, theta=a.theta,
                           candidates=(16, 32, 64, 128, 256, 512))
        a.n_group = a.n_group if a.n_group > 0 else tuned["n_group"]
        a.ppl = a.ppl if a.ppl > 0 else tuned["particles_per_lane"]
    T = G.Tree.build(pos, m, a.n_leaf, a.n_group)
    T.set_launch(a.ppl)
    if tuned is not None and tuned["n_group"] == a.n_group and tuned["particles_per_lane"] == a.ppl:
        T.set_split(tuned["split"])
        T.set_staging(tuned["staging"])
    T.upload()
    out = torch.empty((T.n, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    for k in range(a.warmup):
        T.forces_device(a.eps, a.theta, out, stream=stream)
        if k == 0 and not a.no_balance:
            T.balance(stream=stream)  # later launches take the items longest first (costs of launch 0)
    torch.cuda.synchronize()
    st = T.status()
    if st != G.OK:
        raise SystemExit("device status %d: %s" % (st, G.load().octgrav_last_error().decode()))
    counts = T.interaction_counts()

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    w0 = time.perf_counter()
    for k in range(a.steps):
        flush.zero_()
        ev[k][0].record(stream)
        T.forces_device(a.eps, a.theta, out, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = [s.elapsed_time(e) for s, e in ev]
    ms_local = statistics.mean(ms)
    ms_step = RK.max_over_ranks(dist, ms_local, device="cuda")  # the slowest rank
    st = T.status()
    if st != G.OK:
        raise SystemExit("device status %d after timing" % st)

    value = RK.job_rate(dist, a.n, ms_local * 1e-3, device="cuda")  # all ranks' particles / slowest time
    peak, sms, mhz = fp32_peak_tflops(torch)
    achieved = counts["flops"] / (ms_step * 1e-3) / 1e12

    # e2e through the one-shot C-ABI calls with pinned host buffers, every step
    # inside the timed region: octgrav_forces_ex (tree built on the host, its
    # arrays copied in) and octgrav_forces_gpu (inputs copied in, tree built on
    # the GPU); both unpermute on the device and copy the FP64 results out
    pin_x = torch.from_numpy(np.ascontiguousarray(pos)).pin_memory()
    pin_m = torch.from_numpy(np.ascontiguousarray(m)).pin_memory()
    pin_a = torch.empty((a.n, 3), dtype=torch.float64).pin_memory()
    pin_p = torch.empty(a.n, dtype=torch.float64).pin_memory()
    e2e_t, host_t = [], []
    for k in range(a.e2e_steps + 1 if a.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.forces_gpu(pin_x.numpy(), pin_m.numpy(), a.eps, a.theta, a.n_leaf, a.n_group, stream=stream,
                     out=(pin_a.numpy(), pin_p.numpy()))
        e2e_t.append(time.perf_counter() - t0)
    for k in range(a.e2e_steps + 1 if a.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.forces(pin_x.numpy(), pin_m.numpy(), a.eps, a.theta, a.n_leaf, a.n_group, stream=stream,
                 out=(pin_a.numpy(), pin_p.numpy()))
        host_t.append(time.perf_counter() - t0)
    host_phases = G.oneshot_phases() if host_t else None  # the last call's breakdown (ms)
    e2e_s = statistics.mean(e2e_t[1:]) if len(e2e_t) > 1 else float("nan")
    host_s = statistics.mean(host_t[1:]) if len(host_t) > 1 else float("nan")
    if dist and len(e2e_t) > 1:  # the slowest rank's time, as for the headline
        e2e_s = RK.max_over_ranks(dist, e2e_s, device="cuda")
        host_s = RK.max_over_ranks(dist, host_s, device="cuda")
    s = T.stats
    # host-build path: the tree's device arrays go up (particles 32 B + the int32 permutation,
    # cells 16 + 8 + 64 B, items 16 + 64 B + the 4-byte processing order) and the FP64
    # results, unpermuted on the device, come back (24 + 8 B per particle)
    h2d = 36 * a.n + 88 * s["n_cells"] + 84 * s["n_items"]
    d2h = 32 * a.n
    h2d_gpu = 32 * a.n  # GPU-build path: positions (24 B) and masses (8 B)
    d2h_gpu = 32 * a.n  # accelerations (24 B) and potentials (8 B), FP64

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    traffic = measured_traffic(a)
    hbm_peak, hbm_src = hbm_peak_gbs()
    line = {
        "metric": METRIC, "value": value, "unit": "forces/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "seed": a.seed, "particles_per_lane": a.ppl,
                   "autotuner": tuned,
                   "item_order": "most particles first (default)" if a.no_balance else
                   "longest first, from the interaction counts of the first warm-up launch (octgrav_balance)",
                   "l2": "flushed (256 MiB write) before every timed step, outside the events",
                   "parallelism": "replica per GPU" if world > 1 else "1 GPU"},
        "gflops": achieved * 1e3, "frac_fp32_peak": achieved / peak,
        # the paper's own figures, same flop convention (abstract, Sec. 3.3): context only --
        # a G80 GPU, another model (Milky Way), N_leaf = N_group = 64
        "paper_context": {"gflops": 100.0, "seconds_per_million_particles": 1.0, "theta": 0.5,
                          "hardware": "GeForce 8800 Ultra (G80)"},
        "interactions": {"n_pp": counts["n_pp"], "n_pc": counts["n_pc"], "flops_per_step": counts["flops"],
                         "flops_per_particle": counts["flops"] / a.n},
        "e2e": None if host_s != host_s else {
            "value": world * a.n / host_s, "unit": "forces/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "seconds_per_step": host_s,
            "path": "octgrav_forces_ex (the paper's split, Sec. 2: host FP64 tree build, upload, kernel, device "
                    "unpermute, FP64 download)",
            "phases_ms": host_phases,
            "gpu_build_path": None if e2e_s != e2e_s else {
                "value": world * a.n / e2e_s, "unit": "forces/s", "h2d_bytes_per_step": h2d_gpu,
                "d2h_bytes_per_step": d2h_gpu, "seconds_per_step": e2e_s,
                "path": "octgrav_forces_gpu: pinned H2D of positions and masses, GPU tree build (the host "
                        "build's tree, byte for byte), kernel, device unpermute, pinned FP64 D2H"}},
        "gpu_launches": a.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (sms, mhz),
                     "kernel": "walk_eval_kernel (fused walk + evaluation)",
                     # the tree sits in L2: DRAM sees each array about once per launch
                     "hbm": None if traffic is None else {
                         "achieved_gbs": traffic / (ms_step * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                         "frac": traffic / (ms_step * 1e-3) / 1e9 / hbm_peak, "peak_source": hbm_src}},
        "clocks": clk,
        "wall_s_timed_loop_incl_flush": wall,
        "tree": s,
    }
    acc = np.empty((a.n, 3))
    acc[T.perm()] = out.cpu().numpy()[:, :3]
    # the oracle baseline, the accuracy check and the extra workloads run at N = 1 only: at N > 1
    # the GPUs are held for the headline line alone
    if not a.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(pos, m, a, a.cpu_seconds, acc)
    if not a.no_accuracy and world == 1:
        line["accuracy"] = accuracy(G, acc, pos, m, a)
    if not a.no_extras and world == 1:
        line["extras"] = extras(torch, G, a, pos, m, T, out, flush, stream, peak, min(a.steps, 10))
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
