#!/usr/bin/env python
"""Benchmark of the batched-volume FBP workload on B300 GPUs.

Workload (per GPU): a 1024-slice stack of raw uint16 radiographies
[2000 angles][1024 slices][2048 bins] with seeded flat/dark fields, phantom =
200 random ellipsoids in a unit cylinder with exact line integrals and
Poisson counts; output 1024 x 2048 x 2048 float32.  The whole stack and the
output stay resident in HBM; a step reconstructs the next 64 slices of the
stack (normalise + Ram-Lak filter + back-projection) through pyhst_fbp.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "backproj Gupd/s (voxel·angle) + FBP slices/s; TV vs learned-prox s/slice @PSNR"
N_SLICES, N_PIX, N_ANG, N_BINS = 1024, 2048, 2000, 2048
WORKLOAD = ("batched volume FBP: 1024 slices x 2048x2048 float32 output, 2000 angles over 180 deg, 2048 bins, "
            "raw uint16 radiographies with seeded flat (3e4 +-5% smooth) / dark (100 +-3) fields; "
            "phantom = 200 random ellipsoids (density 0-1) in a unit cylinder")
DATA = ("synthetic: seeded ellipsoid phantom, exact (closed-form) line integrals, Poisson counts + dark, "
        "uint16; random numbers drawn once at set-up")
UPD_PER_SLICE = N_PIX * N_PIX * N_ANG
# Reduced-dose TV workload: beta per slice size, frozen from a seeded PSNR
# calibration (4 training foams per size disjoint from the benchmark's,
# 13-point log grid 1e-4..1e-1, 200 x 20 iterations, PSNR over the inscribed
# disk; maxima 30.3 / 30.4 / 30.2 dB).
TV_BETA = {256: 1.7783e-3, 512: 1.7783e-3, 1024: 1.0e-3}
TV_WORKLOAD = ("reduced-dose iterative TV: FISTA + Chambolle TV prox (20 inner steps), 200 outer iterations, "
               "128 slices of mixed size 256^2/512^2/1024^2 with 50/100/200 angles over 180 deg (43/43/42, "
               "shuffled) in one batched solve; Poisson 1e4 photons; seeded Voronoi foams with 4 density levels")
OPS_PER_UPDATE = 4          # coordinate FMA, floor add, interpolation FMA, accumulate add
SMEM_BYTES_PER_UPDATE = 8   # one float32 (dq, c0) window entry read from shared memory
SMEM_BYTES_PER_CLK = 128    # shared-memory data pipe per SM per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--slices-per-step", type=int, default=64)
    ap.add_argument("--slices-per-pass", type=int, default=16,
                    help="slices filtered and back-projected per pass of pyhst_fbp (the workspace holds their "
                         "filtered rows); 16 slices give 16,384 back-projection CTAs, 36.9 waves of 444")
    ap.add_argument("--volume-slices", type=int, default=N_SLICES)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunk", type=int, default=16, help="largest chunk of the host-buffer call, in slices")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the baseline sample")
    ap.add_argument("--no-tv", action="store_true", help="skip the reduced-dose TV measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-slice and mixed-precision FBP measurements")
    ap.add_argument("--patch-study", action="store_true",
                    help="overlapping-patch prior on a 2048^2 phantom with 150 projections (Sec. 3.2.1)")
    ap.add_argument("--precision-study", action="store_true",
                    help="mixed-precision FBP study (4096^2, 4000 angles; f32/f16/bf16 storage vs the FP64 oracle)")
    ap.add_argument("--precision-slices", type=int, default=4, help="slices checked against the oracle")
    ap.add_argument("--tv-only", action="store_true", help="only the reduced-dose TV measurement (for profilers)")
    ap.add_argument("--pre-study", action="store_true",
                    help="cost of the Sec. 2.3 preprocessing variants on the batched-volume geometry")
    ap.add_argument("--beta-study", action="store_true",
                    help="beta estimators (Sec. 4) on a 2048^2 foam with 150 projections vs its ground truth")
    ap.add_argument("--kernel-slices", type=int, default=4, help="slices per launch of --kernel-case")
    ap.add_argument("--kernel-case", choices=["backproject", "project", "filter", "cnn", "project-sparse", "project-tv", "tvprox",
                                              "patch"],
                    help="run only a few launches of one kernel at the workload's slice geometry (for profilers)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# DRAM bytes (read + write) of one back-projection launch of BP_DRAM_SLICES
# slices (2048^2, 2000 angles) from an ncu capture of bp_kernel, and the hash
# of the kernel source it was taken on: the figure is reported only while the
# source is unchanged.
BP_DRAM_BYTES = 502970368
BP_DRAM_SLICES = 16
BP_DRAM_SOURCE_SHA16 = "28dcc8ce9243e080"


def bp_traffic(slices):
    """DRAM bytes per back-projection launch of `slices` slices if the capture
    above was taken on the current kernel source (scaled by the slice count:
    every slice reads its own filtered rows and writes its own image), else
    None."""
    src = os.path.join(ROOT, "paper_1306_1392_b300", "csrc", "backproject.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return BP_DRAM_BYTES * slices // BP_DRAM_SLICES if sha == BP_DRAM_SOURCE_SHA16 else None


def cpu_sample_fbp(orc, raw_slice, flat, dark, angles, axis, target_s):
    """Oracle FBP of one slice restricted to a band of rows, sized to about
    target_s seconds: normalise + filter all angle rows, back-project R image
    rows.  Returns (updates, prorated seconds, R, threads).  The filter is
    per-slice work; R/N of its time is charged to the R rows."""
    import numpy as np
    n = N_PIX
    t0 = time.perf_counter()
    p = orc.normalise(raw_slice, flat, dark)
    q = orc.ramlak_filter(p)
    t_filter = time.perf_counter() - t0
    cy = (n - 1) / 2.0
    # pilot band wide enough to keep every OpenMP thread busy (rows are split among threads)
    pilot = 64
    t0 = time.perf_counter()
    orc.backproject(q, angles, axis, n, pilot, orc.fbp_weight(N_ANG, 2.0 / n), cy=cy - (n - pilot) // 2)
    per_row = (time.perf_counter() - t0) / pilot
    R = int(max(4, min(n, (target_s - t_filter) / max(per_row, 1e-6))))
    # a whole slice is shorter than the target: repeat its back-projection
    # until the measured time reaches the target (at most 16 times)
    r0 = (n - R) // 2
    reps, t_bp = 0, 0.0
    while reps == 0 or (R == n and reps < 16 and t_bp + t_filter * reps < target_s):
        t0 = time.perf_counter()
        orc.backproject(q, angles, axis, n, R, orc.fbp_weight(N_ANG, 2.0 / n), cy=cy - r0)
        t_bp += time.perf_counter() - t0
        reps += 1
    secs = t_bp + t_filter * reps * R / n
    return reps * R * n * N_ANG, secs, R * reps, orc.num_threads()


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    import numpy as np
    import torch
    import oracle as orc
    from synth import acquisition as acq
    if rank != 0:
        return
    orc.build()
    z = args.volume_slices // 2
    vol = acq.ellipsoid_volume(n_slices=args.volume_slices, n=N_PIX, n_angles=N_ANG, seed=1000, device="cpu",
                               slices=[z], dtype=torch.float32, compact=True)
    raw = vol.raw[:, 0, :].double().numpy()
    fl, dk = vol.flat[0].double().numpy(), vol.dark[0].double().numpy()
    ang, ax = vol.angles.double().numpy(), vol.axis.double().numpy()
    per_step_s = max(1.0, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_sample_fbp(orc, raw, fl, dk, ang, ax, per_step_s)
    upd_total, secs_total, rows = 0, 0.0, []
    for _ in range(args.steps):
        u, s, R, threads = cpu_sample_fbp(orc, raw, fl, dk, ang, ax, per_step_s)
        upd_total += u
        secs_total += s
        rows.append(R)
    value = upd_total / secs_total / 1e9
    sample = (f"each step: one slice of the workload (2000 x 2048 uint16 counts): normalise + filter all rows, "
              f"back-project {min(rows)}-{max(rows)} image rows (a band of its 2048 rows, the whole slice "
              f"repeated when the step needs more); filter time prorated by rows/2048")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gupd/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA,
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "Gupd/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gupd/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ reduced-dose TV
def psnr(x, truth):
    """PSNR over the inscribed disk r <= N/2 - 1, peak = truth range."""
    import numpy as np
    n = truth.shape[0]
    yy, xx = np.meshgrid(np.arange(n) - (n - 1) / 2, np.arange(n) - (n - 1) / 2, indexing="ij")
    m = np.hypot(xx, yy) <= n / 2 - 1
    mse = float(np.mean((x[m] - truth[m]) ** 2))
    return 10 * math.log10((truth.max() - truth.min()) ** 2 / mse)


def tv_kernel_rates(P, plan, n_iter, n_inner, n_power_iter, kern, peaks, props):
    """Per-kernel rates of one batched solve from its event-timed launches:
    algorithmic units per solve (projector and back-projector: voxel-angle
    updates; Chambolle: pixel-steps) over the kernel's summed launch time."""
    sizes = sorted({(n, na) for n, na in plan})
    upd_all = sum(n * n * na for n, na in plan)
    upd_rep = sum(n * n * na for n, na in sizes)          # one representative per geometry
    units = {"project": n_iter * upd_all + (n_power_iter + 1) * upd_rep,
             "backproject": n_iter * upd_all + n_power_iter * upd_rep,
             "chambolle": n_iter * n_inner * sum(n * n for n, _ in plan)}
    out = {}
    for k, (ms, n) in kern.items():
        out[k] = {"launches": n, "total_ms": ms, "units": units[k],
                  "unit": "pixel-steps" if k == "chambolle" else "voxel-angle updates",
                  "g_units_per_s": units[k] / (ms * 1e-3) / 1e9 if ms > 0 else None}
    sm_max = float(peaks.get("sm_max_mhz") or 2032.0)
    peak_smem = props.multi_processor_count * SMEM_BYTES_PER_CLK * sm_max * 1e6 / 1e12
    top = max(kern, key=lambda k: kern[k][0])
    roof = None
    if top in ("project", "backproject") and kern[top][0] > 0:
        achieved = SMEM_BYTES_PER_UPDATE * units[top] / (kern[top][0] * 1e-3) / 1e12
        roof = {"kernel": {"project": "proj_batch_kernel", "backproject": "bp_batch_kernel"}[top],
                "bound": "smem", "achieved": achieved, "peak": peak_smem, "unit": "TB/s", "frac": achieved / peak_smem,
                "traffic": None, "tupd_per_s": units[top] / (kern[top][0] * 1e-3) / 1e12,
                "share_of_solve_kernels": kern[top][0] / sum(v[0] for v in kern.values()),
                "peak_basis": f"shared-memory data pipe: {props.multi_processor_count} SMs x {SMEM_BYTES_PER_CLK} "
                              f"B/clk x {sm_max:.0f} MHz; {SMEM_BYTES_PER_UPDATE} B per voxel-angle update (the "
                              "matched back-projector's window entry; the projector makes the same updates); "
                              "units: every projection of the solve (power iteration on one slice per geometry, "
                              "then one projection of every slice per iteration) over the summed launch times"}
    return out, roof


def tv_cpu_baseline(plan, n_iter, n_inner, n_power_iter, target_s):
    """The FP64 oracle's FISTA-TV on one seeded slice of each size of the
    reduced-dose batch, for a bounded number of outer iterations: s/slice =
    power iteration + n_iter x the measured time per iteration, weighted by
    the batch's size mix."""
    import numpy as np
    import oracle as orc
    from synth import acquisition as acq
    orc.build()
    per, done = {}, {}
    first = {}
    for k, (n, na) in enumerate(plan):
        first.setdefault((n, na), k)
    budget = target_s / len(first)
    for (n, na), k in sorted(first.items()):
        fs = acq.foam_slice(n, na, seed=3000 + k, truth=False)
        og = orc.Geometry(fs.angles.double().numpy(), fs.axis.double().numpy(), n, n, n, fs.pixel_size)
        sino = fs.extra["sino"].double().numpy()
        t0 = time.perf_counter()
        L = 1.01 * orc.power_iteration(og, np.ones((n, n)), 2)[0]
        t_pow = (time.perf_counter() - t0) / 2 * n_power_iter
        t0 = time.perf_counter()
        orc.fista(og, sino, TV_BETA[n], L, 1, n_inner=n_inner)
        t1 = time.perf_counter() - t0
        its = int(max(1, min(n_iter, (budget - t1 - t_pow * 2 / n_power_iter) / max(t1, 1e-6))))
        t0 = time.perf_counter()
        orc.fista(og, sino, TV_BETA[n], L, its, n_inner=n_inner)
        t_it = (time.perf_counter() - t0) / its
        per[f"{n}^2/{na}"] = t_pow + n_iter * t_it
        done[f"{n}^2/{na}"] = its
    counts = {}
    for n, na in plan:
        counts[f"{n}^2/{na}"] = counts.get(f"{n}^2/{na}", 0) + 1
    mean = sum(per[k] * c for k, c in counts.items()) / len(plan)
    return {"value": mean, "unit": "s/slice", "cores": orc.num_threads(), "kind": "oracle",
            "per_size_s_per_slice": per,
            "sample": "one seeded slice per size (the batch's first of each); FISTA-TV with 20 Chambolle steps "
                      f"timed over {done} outer iterations, power iteration over 2 of its {n_power_iter}, "
                      f"extrapolated to {n_iter} iterations and weighted by the batch's size mix"}


def run_tv(dev, n_slices=128, n_iter=200, n_inner=20, cpu_seconds=20.0):
    """One batched FISTA-TV solve of the mixed reduced-dose set, event-timed
    (power iteration, table upload and graph capture included); then the same
    solve with per-kernel events (the kernels' rates and the roofline of the
    dominant one) and once more reporting the prox duality gaps."""
    import numpy as np
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    plan = acq.mixed_tv_batch_plan(n_slices, seed=3000)
    geos, items, truths = {}, [], []
    for k, (n, na) in enumerate(plan):
        fs = acq.foam_slice(n, na, seed=3000 + k, device=dev)
        if n not in geos:
            geos[n] = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), n, n, n, fs.pixel_size)
        items.append((geos[n], fs.extra["sino"].to(dev).contiguous(), None, TV_BETA[n]))
        truths.append(fs.truth.double().cpu().numpy())
    n_power_iter = 50
    opts = P.TvOptions(beta=1e-3, n_iter=n_iter, n_inner=n_inner, n_power_iter=n_power_iter)
    # autotune the Chambolle steps fused per launch for each slice size (results
    # do not depend on it); outside the timed region
    tuned, tuned_bp, tuned_pw = {}, {}, {}
    for n in sorted(geos):
        z = torch.randn((4, n, n), device=dev, generator=torch.Generator(device=dev).manual_seed(n))
        tuned[str(n)] = P.pyhst_autotune_tv_prox(z, 0.01, n_inner)
        # the back-projector's angle block for this geometry (identical results), on 16 of its sinograms
        sinos = torch.stack([it[1] for it in items if it[0] is geos[n]][:16]).contiguous()
        tuned_bp[str(n)] = P.pyhst_autotune_backproject(geos[n], sinos)
        # and the projector's staging width (identical results), on 16 images of that size
        imgs = torch.rand((16, n, n), device=dev, generator=torch.Generator(device=dev).manual_seed(n + 1))
        tuned_pw[str(n)] = P.pyhst_autotune_project(geos[n], imgs)
    P.pyhst_tv_solve_batch(items, P.TvOptions(beta=1e-3, n_iter=2, n_inner=n_inner, n_power_iter=2))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    xs, es, lip = P.pyhst_tv_solve_batch(items, opts)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the same solve, every projector / back-projector / Chambolle launch bracketed by events
    for k in ("project", "backproject", "chambolle"):
        P.pyhst_profile_read(k)
    P.pyhst_profile_enable(True)
    e0.record()
    xs_p, _, _ = P.pyhst_tv_solve_batch(items, opts, energy=False)
    e1.record()
    torch.cuda.synchronize()
    P.pyhst_profile_enable(False)
    ms_prof = e0.elapsed_time(e1)
    kern = {k: P.pyhst_profile_read(k) for k in ("project", "backproject", "chambolle")}
    same = all(torch.equal(a, b) for a, b in zip(xs, xs_p))
    rates, roof = tv_kernel_rates(P, plan, n_iter, n_inner, n_power_iter, kern, measured_peaks(),
                                  torch.cuda.get_device_properties(dev))
    # the prox duality gaps of the same solve (extra reductions, not timed)
    gaps = [torch.empty(n_iter, dtype=torch.float64, device=dev) for _ in items]
    xs_g, _, lip_g = P.pyhst_tv_solve_batch(items, opts, energy=False, gaps=gaps)
    torch.cuda.synchronize()
    gap_by = {}
    for (n, na), g, x, Lk, it in zip(plan, gaps, xs_g, lip_g.tolist(), items):
        xd = x.double()
        tvx = float(torch.sqrt(torch.nn.functional.pad(xd[1:] - xd[:-1], (0, 0, 0, 1)) ** 2 +
                               torch.nn.functional.pad(xd[:, 1:] - xd[:, :-1], (0, 1)) ** 2).sum())
        lam = it[3] / Lk
        gl = float(g[-1])
        gap_by.setdefault(f"{n}^2/{na}", []).append((float(g[0]), gl, gl / (lam * tvx)))
    gap_rep = {k: {"first_iteration_mean": float(np.mean([v[0] for v in vs])),
                   "last_iteration_mean": float(np.mean([v[1] for v in vs])),
                   "last_relative_to_lam_tv_mean": float(np.mean([v[2] for v in vs])),
                   "min": float(min(v[1] for v in vs))} for k, vs in gap_by.items()}
    ps_tv = [psnr(x.double().cpu().numpy(), t) for x, t in zip(xs, truths)]
    ps_fbp = []
    for (g, sino, _, _b), t in zip(items, truths):
        ps_fbp.append(psnr(P.pyhst_fbp(g, sino[None], "f32_sino")[0].double().cpu().numpy(), t))
    mono = float(np.mean([float((e[-1] <= e[n_iter // 2]).item()) for e in es]))
    by = {}
    for (n, na), p in zip(plan, ps_tv):
        by.setdefault(f"{n}^2/{na}", []).append(p)
    res = {"workload": TV_WORKLOAD, "slices": n_slices, "n_iter": n_iter, "n_inner": n_inner,
           "total_s": ms * 1e-3, "s_per_slice": ms * 1e-3 / n_slices,
           "psnr_tv_mean": float(np.mean(ps_tv)), "psnr_fbp_mean": float(np.mean(ps_fbp)),
           "psnr_tv_by_size": {k: float(np.mean(v)) for k, v in by.items()},
           "energy_lower_at_end_fraction": mono, "beta": {str(k): v for k, v in TV_BETA.items()},
           "chambolle_steps_per_launch": tuned, "backproject_angles_per_block": tuned_bp,
           "project_staging_columns": tuned_pw,
           "kernels": rates, "roofline": roof,
           "profiled_solve_s": ms_prof * 1e-3, "profiled_iterates_equal": same,
           "prox_gap_after_n_inner": gap_rep}
    if cpu_seconds > 0:
        res["cpu_baseline"] = tv_cpu_baseline(plan, n_iter, n_inner, n_power_iter, cpu_seconds)
    res["learned_prox"] = run_learned_prox(dev)
    return res


def run_c1(dev, reps=200, batch=64, cpu=True):
    """The single-slice FBP workload (256^2, 180 angles over 180 deg, 256
    bins, axis 127.5, Poisson counts at 1e5 photons, flat 1e5, dark 0,
    Ram-Lak, padding 512): event-timed one slice per call (latency) and
    `batch` slices of the same geometry per call (throughput), inputs
    resident; the result's relative L2 error against the FP64 oracle; the
    oracle's own time for the slice."""
    import numpy as np
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    sl = acq.single_slice_fbp(seed=0)
    geo = P.Geometry(sl.angles.to(dev), sl.axis.to(dev), sl.n_bins, sl.nx, sl.ny, sl.pixel_size)
    raw = sl.extra["raw"].to(dev)                        # [180, 1, 256] float32 counts
    fl, dk = sl.extra["flat"].to(dev), sl.extra["dark"].to(dev)
    out = torch.empty((1, sl.ny, sl.nx), device=dev)
    ws = torch.empty(P.pyhst_fbp_workspace_size(geo, 1, 512, 1), dtype=torch.uint8, device=dev)
    call = lambda: P.pyhst_fbp(geo, raw, "f32_raw", fl, dk, pad_len=512, out=out, workspace=ws)   # noqa: E731
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / reps
    rawb = raw.expand(-1, batch, -1).contiguous()
    flb, dkb = fl.expand(batch, -1).contiguous(), dk.expand(batch, -1).contiguous()
    outb = torch.empty((batch, sl.ny, sl.nx), device=dev)
    wsb = torch.empty(P.pyhst_fbp_workspace_size(geo, batch, 512, 16), dtype=torch.uint8, device=dev)
    callb = lambda: P.pyhst_fbp(geo, rawb, "f32_raw", flb, dkb, pad_len=512, out=outb, workspace=wsb)  # noqa: E731
    callb()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        callb()
    e1.record()
    torch.cuda.synchronize()
    msb = e0.elapsed_time(e1) / 20
    upd = sl.nx * sl.ny * len(sl.angles)
    res = {"workload": "single-slice FBP: 256^2 float32 grid, 180 angles over 180 deg, 256 bins, axis 127.5; "
                       "head-like 10-ellipse phantom, Poisson counts at 1e5 photons, flat 1e5, dark 0; Ram-Lak, "
                       "zero-padded to 512",
           "one_slice_per_call": {"ms_per_slice": ms1, "slices_per_s": 1e3 / ms1, "gupd_per_s": upd / ms1 / 1e6},
           f"{batch}_slices_per_call": {"ms_per_slice": msb / batch, "slices_per_s": 1e3 * batch / msb,
                                        "gupd_per_s": upd * batch / msb / 1e6}}
    if cpu:
        import oracle as orc
        orc.build()
        args = (sl.extra["raw"][:, 0, :].double().numpy(), sl.extra["flat"][0].double().numpy(),
                sl.extra["dark"][0].double().numpy(), sl.angles.double().numpy(), sl.axis.double().numpy(),
                sl.nx, sl.ny, sl.pixel_size)
        orc.fbp_from_raw(*args)
        t0 = time.perf_counter()
        k = 0
        while k == 0 or time.perf_counter() - t0 < 2.0:
            ref = orc.fbp_from_raw(*args)
            k += 1
        t = (time.perf_counter() - t0) / k
        g = out[0].double().cpu().numpy()
        res["rel_l2_vs_oracle"] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        res["cpu_baseline"] = {"value": 1.0 / t, "unit": "slices/s", "cores": orc.num_threads(), "kind": "oracle",
                               "sample": f"the whole slice, {k} repetitions"}
    return res


def run_c4(dev, n_slices=32):
    """The mixed-precision FBP workload's geometry (4096^2, 4000 angles over
    180 deg, 4096 bins; exact line integrals of 200 random ellipsoids stored
    as f32 / f16 / bf16, float32 arithmetic): `n_slices` central slices of
    its 256-slice stack per storage type, event-timed, inputs resident."""
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    n, na, ns_all = 4096, 4000, 256
    z0 = ns_all // 2 - n_slices // 2
    ang = acq.uniform_angles(na)
    geo = P.Geometry(ang.to(dev), torch.full((na,), (n - 1) / 2.0, device=dev), n, n, n, 2.0 / n)
    p = torch.empty((n_slices, na, n), dtype=torch.float32, device=dev)
    for a in range(0, n_slices, 16):
        p[a:a + 16] = acq.ellipsoid_sinograms(ns_all, n, na, seed=4000, device=dev,
                                              slices=range(z0 + a, z0 + min(n_slices, a + 16)))
    out = torch.empty((n_slices, n, n), dtype=torch.float32, device=dev)
    ws = torch.empty(P.pyhst_fbp_workspace_size(geo, n_slices, 0, 4), dtype=torch.uint8, device=dev)
    res = {"workload": f"mixed-precision FBP: slices {z0}..{z0 + n_slices - 1} of 256 x 4096^2, 4000 angles over "
                       "180 deg, 4096 bins; exact line integrals of 200 random ellipsoids stored as f32/f16/bf16, "
                       "float32 arithmetic"}
    for kind, dt in (("f32_sino", torch.float32), ("f16_sino", torch.float16), ("bf16_sino", torch.bfloat16)):
        stored = p.to(dt)
        P.pyhst_fbp(geo, stored, kind, out=out[:4], workspace=ws, slices=(0, 4))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.pyhst_fbp(geo, stored, kind, out=out, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[kind[:-5]] = {"fbp_slices_per_s": n_slices / (ms * 1e-3),
                          "gupd_per_s": n_slices * n * n * na / (ms * 1e-3) / 1e9,
                          "input_bytes_per_slice": na * n * stored.element_size()}
        del stored
    return res


PROX_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1306_1392_b300", "weights",
                            "prox_cnn_foam512.npy")


def run_learned_prox(dev, n_eval=64):
    """Plain TV vs the learned solve (FBP, K_T FISTA-TV iterations, K_L ISTA
    steps with the trained CNN prox; the fastest (K_T, K_L) of a small grid
    that reaches plain TV's PSNR) at equal PSNR on 64 held-out seeded 512^2
    foams (100 angles, Poisson 1e4), against the fastest plain TV solve that
    reaches it: with the paper's prox (20 Chambolle steps from a zero dual
    field; from zero or the FBP) for ``speedup``, and among those and the
    warm-started proxes (5-20 steps) for ``speedup_vs_any_tv``; the learned
    solve's own TV phase may use warm-started proxes too.  Everything
    event-timed on the GPU."""
    import numpy as np
    import torch
    from paper_1306_1392_b300 import train_prox
    params = torch.from_numpy(np.load(PROX_WEIGHTS).astype(np.float32)).to(dev)
    r = train_prox.evaluate(params, dev, n_eval=n_eval, ks=(), tv_long=0, hybrid_kt=(75, 100, 125, 150, 200),
                            tv_first=(25, 28, 30, 35, 40), learned_steps=(2, 3, 4, 5),
                            tv_zero=(100, 125, 150, 175),
                            tv_warm_dual=tuple((n_in, k) for n_in in (5, 10, 15, 20) for k in (80, 90, 100, 110, 125)),
                            learned_warm_dual=tuple((n_in, k, 4) for n_in in (10, 15) for k in (22, 25, 28)))
    r["weights"] = "paper_1306_1392_b300/weights/prox_cnn_foam512.npy (train_prox.py)"
    return r


# ------------------------------------------------------------------ overlapping-patch prior
def run_patch_study(n=2048, na=150, m=8, stride=4, k=12, n_iter=400, betas=(3e-4, 1e-3, 3e-3)):
    """The paper's validation setting for the patch prior: a 2048^2 phantom
    (seeded foam), 150 projections, Gaussian white noise on the line
    integrals (sigma = 1 % of their maximum); 8x8 patches on a stride-4 grid,
    144-atom over-complete DCT, rho = 1, FISTA from zero.  Event-timed
    gradient evaluation and solves; PSNR over the inscribed disk."""
    import numpy as np
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    from synth.patches import overcomplete_dct
    dev = torch.device("cuda", 0)
    fs = acq.foam_slice(n, na, seed=7000, photons=1e4, device=dev)
    g = torch.Generator(device=dev).manual_seed(7001)
    p = fs.p.to(torch.float32)
    sino = (p + 0.01 * p.max() * torch.randn(p.shape, device=dev, generator=g)).contiguous()
    truth = fs.truth.double().cpu().numpy()
    geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), n, n, n, fs.pixel_size)
    D = torch.from_numpy(overcomplete_dct(m, k).astype(np.float32)).to(dev)
    pp = P.PatchProblem(n, n, m, stride, D, 1.0)
    kr, kc = pp.grid()
    W0 = torch.zeros((kr * kc, k * k), device=dev)
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    P.pyhst_patch_gradient(pp, geo, W0, sino)
    torch.cuda.synchronize()
    e0, e1 = ev()
    e0.record()
    for _ in range(5):
        P.pyhst_patch_gradient(pp, geo, W0, sino)
    e1.record()
    torch.cuda.synchronize()
    grad_ms = e0.elapsed_time(e1) / 5
    _, _, _, lip = P.pyhst_patch_solve(pp, geo, sino, 0.0, 1, n_power_iter=30, energy=False)
    L = float(lip.item())
    runs = []
    for beta in betas:
        e0, e1 = ev()
        e0.record()
        W, x, _, _ = P.pyhst_patch_solve(pp, geo, sino, beta, n_iter, lipschitz=L, energy=False)
        e1.record()
        torch.cuda.synchronize()
        runs.append({"beta": beta, "solve_s": e0.elapsed_time(e1) * 1e-3,
                     "ms_per_iter": e0.elapsed_time(e1) / n_iter,
                     "psnr": psnr(x.double().cpu().numpy(), truth),
                     "nonzero_coef_fraction": float((W != 0).float().mean().item())})
    fbp = P.pyhst_fbp(geo, sino[None], "f32_sino")[0]
    print(json.dumps({"patch_study": {
        "workload": f"{n}^2 foam, {na} projections, Gaussian noise 1 % of max p; {m}x{m} patches, stride "
                    f"{stride} ({kr}x{kc} = {kr * kc} patches), {k * k}-atom over-complete DCT, rho 1, FISTA "
                    f"{n_iter} iterations from zero",
        "gradient_ms": grad_ms, "lipschitz": L, "runs": runs,
        "psnr_fbp": psnr(fbp.double().cpu().numpy(), truth)}}), flush=True)


# ------------------------------------------------------------------ precision study
def run_precision_study(args):
    """256 slices x 4096^2, 4000 angles, 4096 bins: FBP throughput with the
    sinogram stored as float32 / float16 / bfloat16 (float32 arithmetic), and
    the error of each against the FP64 oracle run on the exact float64 line
    integrals, at sampled pixels of a few seeded slices."""
    import numpy as np
    import torch
    import oracle as orc
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    orc.build()
    dev = torch.device("cuda", 0)
    n, na, ns = 4096, 4000, 256
    ang = acq.uniform_angles(na)
    geo = P.Geometry(ang.to(dev), torch.full((na,), (n - 1) / 2.0, device=dev), n, n, n, 2.0 / n)
    p = torch.empty((ns, na, n), dtype=torch.float32, device=dev)
    for z0 in range(0, ns, 16):
        p[z0:z0 + 16] = acq.ellipsoid_sinograms(ns, n, na, seed=4000, device=dev, slices=range(z0, min(ns, z0 + 16)))
    out = torch.empty((ns, n, n), dtype=torch.float32, device=dev)
    check = [int(z) for z in np.linspace(ns // 5, 4 * ns // 5, args.precision_slices).round()]
    rng = np.random.default_rng(7)
    ii = rng.integers(0, n, 2000)
    jj = rng.integers(0, n, 2000)
    refs = {}
    for z in check:
        q = orc.ramlak_filter(acq.ellipsoid_sinograms(ns, n, na, seed=4000, slices=[z])[0].numpy())
        refs[z] = orc.backproject_at(q, ang.double().numpy(), (n - 1) / 2.0, n, n, ii, jj, orc.fbp_weight(na, 2.0 / n))
    res = {}
    for kind, dt in (("f32_sino", torch.float32), ("f16_sino", torch.float16), ("bf16_sino", torch.bfloat16)):
        stored = p.to(dt)
        ws = torch.empty(P.pyhst_fbp_workspace_size(geo, ns, 0, 4), dtype=torch.uint8, device=dev)
        P.pyhst_fbp(geo, stored, kind, out=out[:4], workspace=ws, slices=(0, 4))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.pyhst_fbp(geo, stored, kind, out=out, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        errs = []
        for z in check:
            g = out[z].cpu().numpy()[ii, jj].astype(np.float64)
            r = refs[z]
            errs.append((np.linalg.norm(g - r) / np.linalg.norm(r), np.abs(g - r).max() / np.abs(r).max()))
        res[kind[:-5]] = {"rel_l2": max(e[0] for e in errs), "max_abs_over_max": max(e[1] for e in errs),
                          "fbp_slices_per_s": ns / (ms * 1e-3), "gupd_per_s": ns * n * n * na / (ms * 1e-3) / 1e9,
                          "input_bytes_per_slice": na * n * stored.element_size()}
        del stored
    print(json.dumps({"precision_study": res, "workload": "256 slices x 4096^2, 4000 angles over 180 deg, 4096 bins; "
                      "exact line integrals of 200 random ellipsoids stored as f32/f16/bf16; float32 arithmetic",
                      "reference": f"FP64 oracle on the exact float64 line integrals, {len(ii)} sampled pixels of "
                                   f"slices {check}, worst slice reported"}), flush=True)


# ------------------------------------------------------------------ beta estimators
def run_beta_study(n=2048, n_angles=150, n_iter=200, seed=5150):
    """The paper's validation setting (Sec. 4): a synthetic 2k x 2k phantom
    with 150 projections; cross-validation and E_cohe over a beta grid in one
    scan, against the ground-truth PSNR of each reconstruction."""
    import numpy as np
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    dev = torch.device("cuda", 0)
    fs = acq.foam_slice(n, n_angles, seed=seed, device=dev)
    geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), n, n, n, fs.pixel_size)
    betas = [1e-5] + [float(b) for b in np.logspace(-4, -1, 13)]
    opts = P.TvOptions(beta=0.0, n_iter=n_iter, n_inner=20)
    sino = fs.extra["sino"].to(dev)
    P.pyhst_beta_scan(geo, sino, betas[:2], P.TvOptions(beta=0.0, n_iter=2, n_inner=20), held_out=n_angles // 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x, cv, ec = P.pyhst_beta_scan(geo, sino, betas, opts, held_out=n_angles // 2)
    e1.record()
    torch.cuda.synchronize()
    truth = fs.truth.double().cpu().numpy()
    ps = [psnr(x[k].double().cpu().numpy(), truth) for k in range(len(betas))]
    cvv, ecv = cv.cpu().numpy(), ec.cpu().numpy()
    k_gt, k_cv = int(np.argmax(ps[1:])) + 1, int(np.argmin(cvv[1:])) + 1
    k_ec = int(np.nanargmin(np.abs(ecv[1:]))) + 1
    print(json.dumps({"beta_study": {
        "workload": f"foam phantom {n}^2, {n_angles} projections over 180 deg, Poisson 1e4 photons; "
                    f"FISTA {n_iter} x Chambolle 20 per beta; held-out angle {n_angles // 2}",
        "betas": betas, "psnr": ps, "cv": cvv.tolist(), "ecohe": ecv.tolist(),
        "beta_best_psnr": betas[k_gt], "beta_min_cv": betas[k_cv], "beta_min_abs_ecohe": betas[k_ec],
        "psnr_at": {"best": ps[k_gt], "min_cv": ps[k_cv], "min_abs_ecohe": ps[k_ec]},
        "scan_s": e0.elapsed_time(e1) * 1e-3}}), flush=True)


# ------------------------------------------------------------------ preprocessing cost
def run_pre_study(ns=64):
    """pyhst_fbp against pyhst_fbp_pre (three flats interpolated in time,
    hot-spot filter, ring filter) on 64 slices of the batched-volume geometry."""
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    dev = torch.device("cuda", 0)
    vol = acq.ellipsoid_volume(n_slices=ns, n=N_PIX, n_angles=N_ANG, seed=1000, device=dev)
    geo = P.Geometry(vol.angles.to(dev), vol.axis.to(dev), N_BINS, N_PIX, N_PIX, vol.pixel_size)
    flats = torch.stack([vol.flat * 0.99, vol.flat, vol.flat * 1.02])
    pos = torch.linspace(0, 2, N_ANG, device=dev)
    out = torch.empty((ns, N_PIX, N_PIX), device=dev)
    runs = {"fbp": lambda: P.pyhst_fbp(geo, vol.raw, "u16_raw", vol.flat, vol.dark, out=out),
            "fbp_pre_flats": lambda: P.pyhst_fbp_pre(geo, vol.raw, "u16_raw", flats, vol.dark, flat_pos=pos, out=out),
            "fbp_pre_all": lambda: P.pyhst_fbp_pre(geo, vol.raw, "u16_raw", flats, vol.dark, flat_pos=pos,
                                                   hotspot_threshold=0.2, ring_window=9, out=out)}
    res = {}
    for k, fn in runs.items():
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[k] = {"slices_per_s": ns / (ms * 1e-3), "gupd_per_s": ns * UPD_PER_SLICE / (ms * 1e-3) / 1e9}
    print(json.dumps({"pre_study": res, "workload": f"{ns} slices of 2048^2, 2000 angles, 2048 bins, uint16 raw"}),
          flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_1306_1392_b300 as P
    from paper_1306_1392_b300.shard import reduce_throughput
    from synth import acquisition as acq

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    S, NZ = args.slices_per_step, args.volume_slices
    # inputs: this rank's shard (seeded per rank), generated on the device
    vol = acq.ellipsoid_volume(n_slices=NZ, n=N_PIX, n_angles=N_ANG, seed=1000 + rank, device=dev)
    raw, flat, dark = vol.raw, vol.flat, vol.dark
    geo = P.Geometry(vol.angles.to(dev), vol.axis.to(dev), N_BINS, N_PIX, N_PIX, vol.pixel_size)
    out = torch.empty((NZ, N_PIX, N_PIX), dtype=torch.float32, device=dev)
    SP = max(1, min(args.slices_per_pass, S))
    ws = torch.empty(P.pyhst_fbp_workspace_size(geo, S, 0, SP), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step(k):
        z0 = (k * S) % NZ
        z1 = min(z0 + S, NZ)
        P.pyhst_fbp(geo, raw, "u16_raw", flat, dark, out=out[z0:z1], workspace=ws, slices=(z0, z1))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for k in range(args.warmup):
        step(k)
    barrier()
    P.pyhst_profile_read("backproject"), P.pyhst_profile_read("filter")
    P.pyhst_profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        ev0.record()
        for k in range(args.steps):
            step(args.warmup + k)
        ev1.record()
        barrier()
    P.pyhst_profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    bp_ms, bp_n = P.pyhst_profile_read("backproject")
    fl_ms, fl_n = P.pyhst_profile_read("filter")
    slices_done = sum(min(((args.warmup + k) * S) % NZ + S, NZ) - ((args.warmup + k) * S) % NZ
                      for k in range(args.steps))
    ms_max, n_slices_all = reduce_throughput(ms, slices_done, device=dev)
    value = n_slices_all * UPD_PER_SLICE / (ms_max * 1e-3) / 1e9

    # ---- end to end through the host-buffer C-ABI call (same metric)
    e2e = None
    if not args.no_e2e:
        z0 = NZ // 2 - S // 2
        host_raw = torch.empty((N_ANG, S, N_BINS), dtype=torch.uint16, pin_memory=True)
        host_raw.copy_(raw[:, z0:z0 + S, :].cpu())
        host_flat = flat[z0:z0 + S].cpu().pin_memory()
        host_dark = dark[z0:z0 + S].cpu().pin_memory()
        host_out = torch.empty((S, N_PIX, N_PIX), dtype=torch.float32, pin_memory=True)
        chunk = args.e2e_chunk
        hws = torch.empty(P.pyhst_fbp_host_workspace_size(geo, "u16_raw", S, 0, chunk), dtype=torch.uint8,
                          device=dev)

        def estep():
            P.pyhst_fbp_host(geo, host_raw, "u16_raw", host_flat, host_dark, out=host_out,
                             slices_per_chunk=chunk, workspace=hws)

        for _ in range(max(1, min(args.warmup, 3))):
            estep()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            estep()
        e1.record()
        barrier()
        ems, e_slices = reduce_throughput(e0.elapsed_time(e1), args.steps * S, device=dev)
        e2e = {"value": e_slices * UPD_PER_SLICE / (ems * 1e-3) / 1e9, "unit": "Gupd/s",
               "h2d_bytes_per_step": int(host_raw.numel() * 2 + 2 * host_flat.numel() * 4),
               "d2h_bytes_per_step": int(host_out.numel() * 4),
               "call": f"pyhst_fbp_host (pinned host in/out, chunks of up to {chunk} slices ramped 1, 4, .. at "
                       "both ends, double-buffered)"}

    # ---- roofline of the back-projection kernel (dominant)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz") or 2032.0)
    peak_ops = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12      # T FP32 lane-ops/s
    per_launch_upd = SP * UPD_PER_SLICE
    bp_avg_s = bp_ms / max(1, bp_n) * 1e-3
    peak_smem = props.multi_processor_count * SMEM_BYTES_PER_CLK * sm_max * 1e6 / 1e12   # TB/s
    achieved = SMEM_BYTES_PER_UPDATE * per_launch_upd / bp_avg_s / 1e12
    alu = OPS_PER_UPDATE * per_launch_upd / bp_avg_s / 1e12
    roofline = {"bound": "smem", "achieved": achieved, "peak": peak_smem, "unit": "TB/s",
                "frac": achieved / peak_smem, "traffic": bp_traffic(SP),
                "kernel": "bp_kernel", "launches": bp_n, "avg_launch_ms": bp_avg_s * 1e3,
                "gupd_per_s": per_launch_upd / bp_avg_s / 1e9,
                "peak_basis": f"shared-memory data pipe: {props.multi_processor_count} SMs x "
                              f"{SMEM_BYTES_PER_CLK} B/clk x {sm_max:.0f} MHz (measured max SM clock); "
                              f"{SMEM_BYTES_PER_UPDATE} B (one float32 (dq, c0) pair) per voxel-angle update; "
                              "traffic = DRAM bytes per launch from an ncu capture of the same kernel source",
                "alu": {"achieved": alu, "peak": peak_ops, "unit": "T FP32 lane-ops/s", "frac": alu / peak_ops,
                        "basis": f"{props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz; "
                                 f"{OPS_PER_UPDATE} FP32 ops per update"},
                "filter_share_of_step": fl_ms / ms,
                "peak_check": peak_check(peak_smem, peak_ops)}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as orc
        orc.build()
        z = NZ // 2
        rs = raw[:, z, :].double().cpu().numpy()
        u, secs, R, threads = cpu_sample_fbp(orc, rs, flat[z].double().cpu().numpy(),
                                             dark[z].double().cpu().numpy(), vol.angles.double().numpy(),
                                             vol.axis.double().numpy(), args.cpu_seconds)
        cpu = {"value": u / secs / 1e9, "unit": "Gupd/s", "cores": threads, "kind": "oracle",
               "sample": f"slice {z}: normalise + filter all 2000 rows, back-project {R} image rows "
                         f"(2048 per slice; a whole slice repeated when the target needs more; filter time "
                         f"prorated by rows); {secs:.1f} s"}

    tv = c1 = c4 = None
    raw_gb = raw.numel() * 2 / 1e9
    if rank == 0 and not (args.no_tv and args.no_configs):
        del out, raw
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_configs:
        c1 = run_c1(dev, cpu=world == 1 and not args.no_cpu_baseline)
        c4 = run_c4(dev)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_tv:
        tv = run_tv(dev, cpu_seconds=0.0 if (world > 1 or args.no_cpu_baseline) else args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gupd/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": DATA,
                "config": {"workload": WORKLOAD, "slices_per_step": S, "volume_slices_per_gpu": NZ,
                           "parallelism": f"slice shards, {world} GPU(s), no collective on the data path",
                           "l2": f"inputs larger than L2: {S * N_ANG * N_BINS * 2 / 1e6:.0f} MB of raw counts "
                                 f"per step; the whole {NZ}-slice stack ({raw_gb:.1f} GB) resident",
                           "pad_len": 4096, "slices_per_pass": SP},
                "fbp_slices_per_s": n_slices_all / (ms_max * 1e-3),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "tv": tv,
                "single_slice_fbp": c1, "mixed_precision_fbp": c4,
                "gpu_launches": int(bp_n + fl_n + 3 * args.steps),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def peak_check(peak_smem_tbs, peak_ops_t):
    """The derived on-chip peaks against the library's microbenchmarks on
    this GPU, run after the timed region (pyhst_microbench on every SM:
    conflict-free 8-byte shared-memory loads; independent FP32 fma chains,
    scalar and paired; approximate reciprocal and square-root chains, the
    MUFU operations of the XU pipe, 16 per clock and SM, that bound the
    Chambolle steps)."""
    import paper_1306_1392_b300 as P
    smem = P.pyhst_microbench("smem_read", iters=8192) / 1e12
    fma = P.pyhst_microbench("fp32_fma", iters=8192) / 1e12
    fma2 = P.pyhst_microbench("fp32_fma2", iters=8192) / 1e12
    mufu = P.pyhst_microbench("mufu", iters=4096) / 1e12
    return {"smem_read_tbs": smem, "smem_frac_of_derived": smem / peak_smem_tbs,
            "fp32_fma_tflops": fma, "fp32_fma2_tflops": fma2,
            "fma_lane_ops_frac_of_derived": fma / 2 / peak_ops_t,
            "mufu_tops": mufu, "mufu_frac_of_derived": mufu / (peak_ops_t / 8),   # 16 of 128 lanes per clock
            "basis": "one launch each of 4 CTAs x 256 threads per SM, event-timed after a warm-up launch"}


def run_kernel_case(args):
    """A few launches of one kernel on the workload's slice geometry
    (--kernel-slices slices per launch, 4 by default; the timed FBP's passes
    hold 16), inputs resident: a small, fixed case for profilers.  Prints one
    JSON line with the event-timed launches."""
    import torch
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    dev = torch.device("cuda", 0)
    S = args.kernel_slices
    ang = acq.uniform_angles(N_ANG).to(dev)
    geo = P.Geometry(ang, torch.full((N_ANG,), (N_BINS - 1) / 2.0, device=dev), N_BINS, N_PIX, N_PIX, 2.0 / N_PIX)
    g = torch.Generator(device=dev).manual_seed(5)
    if args.kernel_case == "backproject":
        q = torch.randn((S, N_ANG, N_BINS), device=dev, generator=g)
        out = torch.empty((S, N_PIX, N_PIX), device=dev)
        ws = torch.empty(P.pyhst_workspace_size(geo, P.PYHST_OP_BACKPROJECT, S), dtype=torch.uint8, device=dev)
        fn = lambda: P.pyhst_backproject(geo, q, 1.0, out=out, workspace=ws)
        upd = S * UPD_PER_SLICE
    elif args.kernel_case == "project":
        img = torch.randn((S, N_PIX, N_PIX), device=dev, generator=g)
        out = torch.empty((S, N_ANG, N_BINS), device=dev)
        ws = torch.empty(P.pyhst_workspace_size(geo, P.PYHST_OP_PROJECT, S), dtype=torch.uint8, device=dev)
        fn = lambda: P.pyhst_project(geo, img, out=out, workspace=ws)
        upd = S * UPD_PER_SLICE
    elif args.kernel_case == "project-sparse":
        # one 2048^2 slice, 150 angles: the 512-column staging variant with row segments
        ang150 = acq.uniform_angles(150).to(dev)
        geo150 = P.Geometry(ang150, torch.full((150,), (N_BINS - 1) / 2.0, device=dev), N_BINS, N_PIX, N_PIX,
                            2.0 / N_PIX)
        img = torch.randn((1, N_PIX, N_PIX), device=dev, generator=g)
        out = torch.empty((1, 150, N_BINS), device=dev)
        ws = torch.empty(P.pyhst_workspace_size(geo150, P.PYHST_OP_PROJECT, 1), dtype=torch.uint8, device=dev)
        fn = lambda: P.pyhst_project(geo150, img, out=out, workspace=ws)
        upd = N_PIX * N_PIX * 150
    elif args.kernel_case == "project-tv":
        # the reduced-dose TV batch's largest geometry: 42 slices of 1024^2, 200 angles, 1024 bins
        n, na, ns = 1024, 200, 42
        angt = acq.uniform_angles(na).to(dev)
        geot = P.Geometry(angt, torch.full((na,), (n - 1) / 2.0, device=dev), n, n, n, 2.0 / n)
        img = torch.randn((ns, n, n), device=dev, generator=g)
        out = torch.empty((ns, na, n), device=dev)
        ws = torch.empty(P.pyhst_workspace_size(geot, P.PYHST_OP_PROJECT, ns), dtype=torch.uint8, device=dev)
        fn = lambda: P.pyhst_project(geot, img, out=out, workspace=ws)
        upd = ns * n * n * na
    elif args.kernel_case == "tvprox":
        # 20 Chambolle steps on 16 images of 1024^2 (default fusion depth)
        z = torch.randn((16, 1024, 1024), device=dev, generator=g)
        out = torch.empty_like(z)
        fn = lambda: P.pyhst_tv_prox(z, 0.05, 20, out=out)
        upd = 16 * 1024 * 1024 * 20
    elif args.kernel_case == "patch":
        # one gradient of the overlapping-patch functional: 2048^2, 150 angles, 8x8 patches, stride 4, 144 atoms
        import numpy as np
        from synth.patches import overcomplete_dct
        ang150 = acq.uniform_angles(150).to(dev)
        geo150 = P.Geometry(ang150, torch.full((150,), (N_BINS - 1) / 2.0, device=dev), N_BINS, N_PIX, N_PIX,
                            2.0 / N_PIX)
        D = torch.from_numpy(overcomplete_dct(8, 12).astype(np.float32)).to(dev)
        pp = P.PatchProblem(N_PIX, N_PIX, 8, 4, D, 1.0)
        W = torch.randn(pp.coef_shape(), device=dev, generator=g)
        y = torch.randn((150, N_BINS), device=dev, generator=g)
        fn = lambda: P.pyhst_patch_gradient(pp, geo150, W, y)
        upd = pp.coef_shape()[0]
    elif args.kernel_case == "cnn":
        # CNN prox forward pass on 16 images of 512^2 (seeded initial weights)
        from synth.cnn_init import init_params
        params = torch.from_numpy(init_params(1)).to(dev)
        z = torch.rand((16, 512, 512), device=dev, generator=g)
        out = torch.empty_like(z)
        ws = torch.empty(P._lib.lib.pyhst_cnn_workspace_size(16, 512, 512), dtype=torch.uint8, device=dev)
        fn = lambda: P.pyhst_cnn_forward(params, z, out=out, workspace=ws)
        upd = 16 * 512 * 512
    else:
        raw = torch.randint(1000, 30000, (N_ANG, S, N_BINS), device=dev, generator=g, dtype=torch.int32).to(torch.uint16)
        fl = torch.full((S, N_BINS), 3e4, device=dev)
        dk = torch.full((S, N_BINS), 100.0, device=dev)
        out = torch.empty((S, N_ANG, N_BINS), device=dev)
        fn = lambda: P.pyhst_filter(geo, raw, "u16_raw", fl, dk, out=out)
        upd = S * N_ANG * N_BINS
    fn()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ms = []
    for k in range(3):
        ev[0].record()
        fn()
        ev[1].record()
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
    print(json.dumps({"kernel_case": args.kernel_case, "ms": ms, "units_per_launch": upd,
                      "g_units_per_s": upd / min(ms) / 1e6}), flush=True)


def main():
    args = parse()
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.precision_study:
        run_precision_study(args)
        return
    if args.pre_study:
        run_pre_study()
        return
    if args.beta_study:
        run_beta_study()
        return
    if args.patch_study:
        run_patch_study()
        return
    if args.tv_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"tv": run_tv(torch.device("cuda", 0))}), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
