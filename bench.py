#!/usr/bin/env python
"""Benchmark of the list-mode OS-LM-MLEM attenuation-and-scatter-compensated
reconstruction on one GB300.

One step is one pass of the whole hot path on the 128 x 128 DaT-like brain
workload (1,000,000 events, 120 angles, 8 subsets x 10 iterations):
attenuation tables, subset sensitivities, the per-event path-sum model
build, the model cache in the chosen format, the initial image, ten OSEM
iterations and the FP64 log-likelihood of the result, all through the C ABI
with the events resident on the device.  The chosen form caches the model
as FP16 with per-event FP32 scales; the exact form (FP32 model) is timed
beside it on the same events.

Printed (rank 0, one JSON line): the event-pixel model evals/s of the whole
step (J * N_nz per step / step time) for the chosen form and, under
"exact", for the FP32 form; seconds per OSEM iteration with the model cached;
each form's error against the FP64 oracle on a frozen 20,000-event subset of
the same events and the chosen form's error against the exact form on all
events; the end-to-end rate through host buffers; the roofline of the
dominant kernel (timed live with CUDA events on the library's stream); the
CPU oracle baseline; SM clocks sampled during the timed region and the
number of kernel launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload dat128|dat64|batch64|surrogate128|windows64|binned64]
                  [--fmt fp16|bf16|fp32]

Under torchrun every rank reconstructs its own noise realisation (weak
scaling, no collective on the data path); rank 0 prints the aggregate.
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

METRIC = "event-pixel model evals/s & LM-OSEM s/iter on 1 GB300, exact vs chosen @ error"
UNIT = "evals/s"
WORKLOADS = {
    "dat64": ("2-D DaT-like brain, 64x64 pixels at 4 mm, 120 angles x 64 bins x 4 mm, R = 150 mm, "
              "200,000 list-mode events (100-175 keV, 10% FWHM at 159 keV), 8 subsets x 10 "
              "iterations, FP32 model and accumulation"),
    "dat128": ("2-D DaT-like brain, 128x128 pixels at 2 mm, 120 angles x 128 bins x 2 mm, R = 150 mm, "
               "1,000,000 list-mode events (100-175 keV, 10% FWHM at 159 keV), 8 subsets x 10 "
               "iterations, model cached in the chosen format, FP32 accumulation"),
    "surrogate128": ("scatter surrogate on the 128x128 DaT-like family (2 mm, 120 angles x 128 bins x 2 mm, "
                     "R = 150 mm): MLP 8 -> 4 x 256 -> 1 with BF16 weights and FP32 accumulation trained "
                     "on exact scatter path sums of 32 jittered phantoms (~6M event-pixel pairs each), exact rows below an "
                     "energy cut chosen by the exact judge; "
                     "one step = sensitivity, surrogate model build, 8 subsets x 10 iterations on "
                     "2,000,000 events of a held-out phantom"),
    "windows64": ("energy-window variants (photopeak [143, 175], [120, 175], full [100, 175] keV) of the "
                  "64 noise realisations of the 64x64 DaT phantom, each window reconstructed in one persistent "
                  "launch, 8 subsets x 10 iterations; ROI-mean NRMSE over realisations"),
    "binned64": ("binned attributes (paper Sec. 4): the 64 noise realisations of the 64x64 DaT phantom "
                 "binned into the detector's 64 position bins and 2 ([100, 143, 175] keV) or 3 "
                 "([100, 120, 143, 175] keV) energy bins, reconstructed from the bin-integrated model with "
                 "count-weighted EM, against list mode; 8 subsets x 10 iterations; ROI-mean NRMSE"),
    "ex2_peak": ("throughput of the exponential unit (ex2.approx.ftz.f32), the bound of the path sum: every SM "
                 "runs 4 CTAs x 512 threads of 8 independent chains (one ex2 and one FP32 add per step)"),
    "mlp_infer": ("scatter-surrogate inference alone: MLP 8 -> 4 x 256 -> 1, BF16 operands, FP32 accumulation, "
                  "2,000,000 rows of standard-normal inputs (He-initialised weights; the kernel's work does not "
                  "depend on their values), one lmosem_surrogate_infer call per step"),
    "mlp_train": ("scatter-surrogate training alone: MLP 8 -> 4 x 256 -> 1, BF16 products on the tcgen05 "
                  "tensor cores with FP32 accumulation, Adam on FP32 parameters; minibatches of 8,192 rows "
                  "drawn from 4,000,000 standard-normal samples; one step = one Adam step (the whole "
                  "lmosem_surrogate_train call of --steps steps is timed)"),
    "batch64": ("64 independent noise realisations of the 64x64 DaT phantom (120 angles, R = 150 mm), "
                "event counts Poisson with means uniform in [50k, 400k], 8 subsets x 10 iterations, "
                "all realisations in one persistent launch, FP32 model"),
}
WORKLOAD = "dat128"
WORKLOAD_DESC = WORKLOADS[WORKLOAD]
# event seeds of the single-set workloads (rank r adds r): the same event sets
# the parity tests and the frozen oracle subset are drawn from
SEEDS = {"dat64": 2, "dat128": 3}
# the chosen model format of each single-set workload; the exact FP32 form is
# timed beside any other
CHOSEN_FMT = {"dat64": "fp32", "dat128": "fp16"}
# MUFU ex2 throughput of a GB300 SM, measured with independent ex2.approx.ftz.f32
# chains (4 CTAs x 512 threads per SM): 31.8 per clock, i.e. 32 (twice the 16 of
# compute capability 10.0).  Each path term needs one ex2 and three FP32 FMAs,
# so the term rate of the path-sum kernel is bounded by 32 per clock per SM.
MUFU_EX2_PER_CLK_SM = 32
SM_MAX_MHZ_FALLBACK = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for the dat64 GPU arm, about 0.6 s; 5 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fmt", choices=["fp32", "fp16", "bf16"], default=None,
                    help="chosen model format (default: fp16 at 128x128, fp32 at 64x64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--events", type=int, default=0,
                    help="override the event count (small cases for profiling)")
    ap.add_argument("--table-budget-mb", type=int, default=0,
                    help="device budget of the scatter-weight tables (0: the library's 4 GiB); "
                         "small profiling captures keep one angle group resident")
    ap.add_argument("--e-sigma", type=float, default=0.0,
                    help="energy cut of the path sum in energy sigmas (0: the library's 6; "
                         "negative: every term, the exact sum)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dat128")
    args = ap.parse_args()
    if args.fmt is None:
        args.fmt = CHOSEN_FMT.get(args.workload, "fp32")
    if args.steps is None:
        args.steps = 20 if args.workload == "dat64" and args.impl == "ours" else 5
    global WORKLOAD, WORKLOAD_DESC
    WORKLOAD, WORKLOAD_DESC = args.workload, WORKLOADS[args.workload]
    return args


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": SM_MAX_MHZ_FALLBACK}, "fallback"


# ------------------------------------------------------------------ inputs

def make_inputs(seed, events=0):
    from paper_2002_12471_gb300 import synthetic as S
    ph, g, J, ns, ni = S.workload(WORKLOAD)
    J = events or J
    ev = S.simulate_events(ph, g, J, seed=seed)
    return ph, g, ev, ns, ni


def strip_terms(ph, g, ev, k_sigma=6.0):
    """Algorithmic count of the model build: sum over events of N_nz (primary)
    plus N_nz per scatter pixel m with |u_j - u_a(m)| <= k_sigma sigma_u(m)."""
    mu = ph.mu.reshape(-1)
    ny, nx = ph.mu.shape
    scat = np.nonzero(mu > 0)[0]
    n_nz = len(scat)
    x = (scat % nx + 0.5 - 0.5 * nx) * ph.pixel_mm
    y = (scat // nx + 0.5 - 0.5 * ny) * ph.pixel_mm
    total = 0
    for a in range(g["n_angles"]):
        th = g["angle0_rad"] + 2 * np.pi * a / g["n_angles"]
        um = -x * np.sin(th) + y * np.cos(th)
        sig = (g["coll_fwhm0_mm"] + g["coll_fwhm_slope"] * (g["radius_mm"] - (x * np.cos(th) + y * np.sin(th)))) / 2.3548200450309493
        lo, hi = um - k_sigma * sig, um + k_sigma * sig
        uj = np.sort(ev.u_mm[ev.angle == a].astype(np.float64))
        # events inside [lo_m, hi_m] for every m
        cnt = np.searchsorted(uj, hi, side="right") - np.searchsorted(uj, lo, side="left")
        total += int(cnt.sum()) + len(uj)
    return total * n_nz, n_nz


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ OS vs MLEM

def os_vs_mlem(L, ph, g, a, u, e, ns, ni, stream, dev, T=1.0):
    """Ordered subsets against plain LM-MLEM (N_s = 1) on the same events
    (paper Sec. 4: similar images, about N_s times faster, quoted there for
    N_s = 4): seconds per iteration of each (CUDA events, model cached, no
    log-likelihood pass), and the MLEM iterations needed to reach the
    log-likelihood that `ni` OS iterations reach.  One entry per subset
    count: 4 (the paper's) and `ns` (the benchmark's)."""
    import torch
    counts = sorted({4, ns})
    res = {}
    for n_sub, iters in [(k, ni) for k in counts] + [(1, 8 * ni)]:
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
        try:
            nsup = L.lmosem_n_support(ctx)
            L.lmosem_sensitivity(ctx, n_sub)
            L.lmosem_build_model(ctx, a, u, e, n_sub, "fp32")
            f = torch.empty(nsup, dtype=torch.float32, device=dev)
            ll = torch.empty(iters, dtype=torch.float64, device=dev)
            L.lmosem_init_image(ctx, T, f)
            L.lmosem_iterate(ctx, iters, T, f, ll)
            curve = ll.cpu().numpy()
            L.lmosem_init_image(ctx, T, f)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lmosem_iterate(ctx, iters, T, f)
            e1.record(stream)
            e1.synchronize()
            res[n_sub] = (e0.elapsed_time(e1) / iters * 1e-3, curve)
        finally:
            L.lmosem_destroy(ctx)
    t_ml, ll_ml = res[1]
    out = []
    for k in counts:
        t_os, ll_os = res[k]
        reached = np.nonzero(ll_ml >= ll_os[-1])[0]
        need = int(reached[0]) + 1 if len(reached) else None
        out.append({"subsets": k, "os_iters": ni, "os_s_per_iter": t_os, "mlem_s_per_iter": t_ml,
                    "mlem_iters_to_match": need, "mlem_iters_run": 8 * ni,
                    "speedup_to_same_loglik": (need * t_ml) / (ni * t_os) if need else None})
    return out


# ------------------------------------------------------------------ ranks

def max_over_ranks(t_ms, world, dev):
    """The slowest rank's timed total (all ranks receive it); weak scaling
    reports the units all ranks processed divided by this time."""
    if world <= 1:
        return t_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def aggregate_rate(units_per_rank, world, ms_per_step):
    """Whole-job throughput: every rank processes units_per_rank per step."""
    return world * units_per_rank / (ms_per_step * 1e-3)


# ------------------------------------------------------------------ our arm

EXACT_FMT = "fp32"
GOLDEN_128 = os.path.join(ROOT, "tests", "golden", "dat128_subset_oracle.npz")


def workload_config(J, n_nz, chosen, world):
    """The config block both arms print (same keys, same values)."""
    cfg = {"workload": WORKLOAD_DESC, "events": J, "support_pixels": n_nz,
           "model_format": chosen, "parallelism": "replicas" if world > 1 else "1 GPU",
           "l2": "model larger than L2 (129 MB); 256 MB L2 flush before every step"}
    if chosen != EXACT_FMT:
        cfg["exact_format"] = EXACT_FMT
    return cfg


def roi_means(img_full, rois):
    return {k: float(np.dot(w.reshape(-1), img_full) / w.sum()) for k, w in rois.items()}


def oracle_subset_errors(L, stream, dev, fmts=("fp32", "fp16", "bf16"), T=1.0):
    """Every model format reconstructs the frozen 20,000-event subset of the
    128 x 128 workload (tests/golden, written by the FP64 oracle alone);
    returns each image's rel-L2 and striatal ROI-mean errors against the
    oracle's image, and the FP32 form's log-likelihood error."""
    import torch
    G = np.load(GOLDEN_128)
    g = {k: float(v) for k, v in zip(G["geometry_keys"], G["geometry_values"])}
    g["n_angles"], g["n_bins"] = int(g["n_angles"]), int(g["n_bins"])
    ns, ni = int(G["n_subsets"]), int(G["n_iters"])
    mu, sup = G["mu"], G["support"]
    rois = {"caudate": G["roi_caudate"].astype(np.float64), "putamen": G["roi_putamen"].astype(np.float64)}
    ref = np.zeros(mu.size)
    ref[sup] = G["image"]
    ref_roi = roi_means(ref, rois)
    a = torch.from_numpy(G["angle"].astype(np.int32)).to(dev)
    u = torch.from_numpy(G["u_mm"]).to(dev)
    e = torch.from_numpy(G["e_kev"]).to(dev)
    out = {"subset": "%d of the 1,000,000 events (seeded pick), 8 subsets x 10 iterations; "
                     "the FP64 oracle's image from tests/golden" % len(G["angle"])}
    for fmt in fmts:
        ctx = L.lmosem_create(mu, float(G["pixel_mm"]), g, stream=stream)
        try:
            nsup = L.lmosem_n_support(ctx)
            if not np.array_equal(L.lmosem_support(ctx), sup):
                raise RuntimeError("support differs from the oracle's")
            L.lmosem_sensitivity(ctx, ns)
            L.lmosem_build_model(ctx, a, u, e, ns, fmt)
            f = torch.empty(nsup, dtype=torch.float32, device=dev)
            ll = torch.empty(ni, dtype=torch.float64, device=dev)
            L.lmosem_init_image(ctx, T, f)
            L.lmosem_iterate(ctx, ni, T, f, ll)
            img = np.zeros(mu.size)
            img[sup] = f.cpu().numpy()
            r = roi_means(img, rois)
            out[fmt] = {"rel_l2": float(np.linalg.norm(img - ref) / np.linalg.norm(ref)),
                        "roi_rel": {k: r[k] / ref_roi[k] - 1.0 for k in r},
                        "loglik_rel": abs(float(ll[-1].item()) / float(G["loglik"][-1]) - 1.0)}
        finally:
            L.lmosem_destroy(ctx)
    return out


def run_ours(args, rank, world, local_rank):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # a dedicated (non-default) stream: the library replays OSEM iterations as
    # CUDA graphs on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ph, g, ev, ns, ni = make_inputs(seed=SEEDS[WORKLOAD] + rank, events=args.events)
    J = len(ev)
    chosen = args.fmt
    forms = [chosen] + ([EXACT_FMT] if chosen != EXACT_FMT else [])
    a_h = torch.from_numpy(ev.angle).pin_memory()
    u_h = torch.from_numpy(ev.u_mm).pin_memory()
    e_h = torch.from_numpy(ev.e_kev).pin_memory()
    a_d, u_d, e_d = a_h.to(dev), u_h.to(dev), e_h.to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB of L2
    T = 1.0

    budget = args.table_budget_mb << 20

    kept_terms = {}

    def step(fmt, a, u, e, profile=0, count=False):
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, e_sigma=args.e_sigma, profile=profile,
                              table_budget_bytes=budget)
        try:
            nsup = L.lmosem_n_support(ctx)
            L.lmosem_sensitivity(ctx, ns)
            L.lmosem_build_model(ctx, a, u, e, ns, fmt)
            if count:   # untimed steps only: the count synchronises the stream
                kept_terms[fmt] = L.lmosem_model_terms(ctx)
            f = torch.empty(nsup, dtype=torch.float32, device=dev)
            ll = torch.empty(1, dtype=torch.float64, device=dev)
            L.lmosem_init_image(ctx, T, f)
            L.lmosem_iterate(ctx, ni, T, f)
            L.lmosem_loglik(ctx, T, f, ll)
            prof = L.lmosem_profile_read(ctx) if profile else None
            launches = L.lmosem_launch_count(ctx)
            return nsup, prof, launches, f, ll
        finally:
            L.lmosem_destroy(ctx)

    for fmt in forms:
        for w in range(max(1, args.warmup)):   # the first untimed step also counts the path terms
            step(fmt, a_d, u_d, e_d, count=w == 0)
    torch.cuda.synchronize()

    # ---- device-resident timed region, one block of steps per model format
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001 - the clock sampler then takes every line
        uuid = None
    clocks = ClockSampler(uuid)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    runs = {}
    for fmt in forms:
        times, profs, launches = [], [], 0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            # kernel timing of everything but the graph-replayed OSEM iterations
            nsup, prof, nl, f, ll = step(fmt, a_d, u_d, e_d, profile=2)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            profs.append(prof)
            launches += nl
        runs[fmt] = dict(times=times, profs=profs, launches=launches,
                         f=f.cpu().numpy().astype(np.float64), ll=float(ll.item()))
    torch.cuda.synchronize()
    clk = clocks.stop()
    for fmt in forms:
        runs[fmt]["t_total_ms"] = max_over_ranks(sum(runs[fmt]["times"]), world, dev)
    ll_final = runs[chosen]["ll"]

    # ---- end to end through the host-buffer call: lmosem_create, then
    # lmosem_reconstruct copies the pinned events in and the image and the
    # log-likelihood out on the context stream
    f_h = torch.empty(nsup, dtype=torch.float32).pin_memory()
    ll_h = torch.empty(1, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, e_sigma=args.e_sigma)
        try:
            L.lmosem_reconstruct(ctx, a_h, u_h, e_h, ns, ni, T, chosen, f_h, ll_h)
        finally:
            L.lmosem_destroy(ctx)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    if abs(float(ll_h[0]) - ll_final) > 1e-6 * abs(ll_final):
        raise RuntimeError("the host-buffer call's log-likelihood differs from the device path's")

    # ---- seconds per OSEM iteration with the model cached (graph replay), and
    # the per-kernel times of the pass and the update from a profiled context
    for fmt in forms:
        it_times = []
        for prof_level in (0, 1):
            ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, e_sigma=args.e_sigma, profile=prof_level)
            try:
                L.lmosem_sensitivity(ctx, ns)
                L.lmosem_build_model(ctx, a_d, u_d, e_d, ns, fmt)
                f = torch.empty(nsup, dtype=torch.float32, device=dev)
                L.lmosem_init_image(ctx, T, f)
                L.lmosem_iterate(ctx, 2, T, f)
                if prof_level:
                    L.lmosem_profile_read(ctx)
                    L.lmosem_iterate(ctx, 10, T, f)
                    runs[fmt]["it_prof"] = L.lmosem_profile_read(ctx)
                else:
                    runs[fmt]["model_bytes"] = L.lmosem_model_bytes(ctx)
                    for _ in range(10):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        L.lmosem_iterate(ctx, 1, T, f)
                        e1.record(stream)
                        e1.synchronize()
                        it_times.append(e0.elapsed_time(e1))
                    # count conservation of the last sub-iteration (Eq. 7), FP64
                    tot = torch.zeros(ns, dtype=torch.float64, device=dev)
                    L.lmosem_subset_totals(ctx, T, f, tot)
                    n_last = int(np.sum(ev.angle % ns == ns - 1))
                    runs[fmt]["count_resid"] = abs(float(tot[ns - 1].item()) - n_last) / max(1, n_last)
            finally:
                L.lmosem_destroy(ctx)
        runs[fmt]["s_per_iter"] = statistics.mean(it_times) * 1e-3

    # ---- the paper's structure: the model recomputed for every iteration (no
    # cache).  One iteration = scatter tables + path sums (lmosem_build_model
    # without a preceding sensitivity pass builds the tables itself) + the
    # subset passes and updates.
    otf_times = []
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, e_sigma=args.e_sigma)
    try:
        L.lmosem_sensitivity(ctx, ns)
        L.lmosem_build_model(ctx, a_d, u_d, e_d, ns, chosen)
        f_otf = torch.empty(nsup, dtype=torch.float32, device=dev)
        L.lmosem_init_image(ctx, T, f_otf)
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lmosem_build_model(ctx, a_d, u_d, e_d, ns, chosen)
            L.lmosem_iterate(ctx, 1, T, f_otf)
            e1.record(stream)
            e1.synchronize()
            otf_times.append(e0.elapsed_time(e1))
    finally:
        L.lmosem_destroy(ctx)

    osml = (os_vs_mlem(L, ph, g, a_d, u_d, e_d, ns, ni, stream, dev)
            if rank == 0 and WORKLOAD == "dat64" else None)
    errors = (oracle_subset_errors(L, stream, dev)
              if rank == 0 and WORKLOAD == "dat128" and os.path.exists(GOLDEN_128) else None)
    # path terms: those of the exact sum (host enumeration of the position
    # strips) and those the kernels formed after the energy cut (device count)
    terms_exact, n_nz = strip_terms(ph, g, ev)
    terms = kept_terms[chosen]
    evals = J * n_nz
    pk, pk_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = (clk or {}).get("sm_max_mhz") or pk.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK)

    def summary(fmt):
        R = runs[fmt]
        agg = {}
        for p in R["profs"]:
            for k, (ms, n) in p.items():
                a = agg.setdefault(k, [0.0, 0])
                a[0] += ms
                a[1] += n
        # when the timed steps replayed the OSEM iterations as CUDA graphs
        # (untimed per kernel), their pass and update kernels enter the
        # breakdown from the profiled context (10 iterations), scaled to the
        # step's iterations; the persistent launch is timed in the steps
        coop = R["it_prof"]["pass"][1] < 10   # one launch for the 10 profiled iterations
        if not coop:
            for k in ("pass", "update"):
                ms, n = R["it_prof"][k]
                a = agg.setdefault(k, [0.0, 0])
                a[0] += ms * ni / 10 * args.steps
                a[1] += int(round(n * ni / 10 * args.steps))
        # the profiled 10 iterations: one persistent launch (passes and updates of
        # every subset), or one pass kernel per subset with its update apart
        pass_ms, pass_n = R["it_prof"]["pass"]
        iter_bytes = R["model_bytes"] + ns * n_nz * 4          # model rows once + image reads
        pass_gbs = 10 * iter_bytes / (pass_ms * 1e-3) / 1e9
        ms_step = R["t_total_ms"] / args.steps
        return agg, pass_ms, pass_n, pass_gbs, ms_step

    agg, pass_ms, pass_n, pass_gbs, ms_step = summary(chosen)
    tot_kernel_ms = sum(v[0] for v in agg.values())
    ps_ms, ps_n = agg["pathsum"]
    ps_launch_ms = ps_ms / max(1, ps_n)
    terms_per_launch = terms / max(1, ps_n / args.steps)
    achieved = terms_per_launch / (ps_launch_ms * 1e-3) / 1e9          # Gterm/s
    peak = MUFU_EX2_PER_CLK_SM * sms * sm_max * 1e6 / 1e9             # Gterm/s (1 ex2 / term)
    traffic = read_traffic("k_pathsum", "%s_%gM" % (WORKLOAD, J / 1e6))
    value = aggregate_rate(evals, world, ms_step)
    e2e_ms = statistics.mean(e2e_times)
    R = runs[chosen]
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if chosen == "fp32" else chosen + "+f32",
        "data": "synthetic (seeded ellipse phantom, photon Monte-Carlo list-mode events)",
        "config": workload_config(J, n_nz, chosen, world),
        "s_per_iter": R["s_per_iter"],
        "s_per_iter_on_the_fly": statistics.median(otf_times) * 1e-3,
        "count_conservation_rel_residual": R["count_resid"],
        "s_per_iter_detail": {"pass_class_ms_per_iteration": pass_ms / 10, "pass_class_launches_per_10_iterations": pass_n,
                              "pass_gbs": pass_gbs, "hbm_peak_gbs": pk["hbm_gbs"],
                              "pass_frac_of_%s_hbm" % pk_kind: pass_gbs / pk["hbm_gbs"],
                              "model_bytes": R["model_bytes"]},
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in agg.items() if v[1]},
        "kernel_share": {k: v[0] / tot_kernel_ms for k, v in agg.items() if v[1]},
        "model_build_evals_per_s": evals / (ps_launch_ms * ps_n / args.steps * 1e-3),
        "path_terms_per_step": terms,
        "path_terms_exact_sum_per_step": terms_exact,
        "energy_cut_kept_frac": terms / terms_exact,
        "energy_cut_sigma": (args.e_sigma if args.e_sigma > 0 else 6.0) if args.e_sigma >= 0 else None,
        "os_vs_mlem": osml,
        "loglik_final": ll_final,
        "e2e": {"value": world * evals / (e2e_ms * 1e-3), "unit": UNIT,
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(J * 12),
                "d2h_bytes_per_step": int(nsup * 4 + 8)},
        "roofline": {"bound": "alu", "kernel": "k_pathsum", "achieved": achieved, "peak": peak,
                     "unit": "Gterm/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": "%d MUFU ex2 per clock per SM x %d SMs x %.0f MHz; one ex2 and "
                                   "three FP32 FMAs per path term" % (MUFU_EX2_PER_CLK_SM, sms, sm_max),
                     "units": "path terms the position and energy cuts keep (counted by the kernels)",
                     "exact_sum_terms_frac": achieved * (terms_exact / terms) / peak,
                     "exact_sum_terms_note": "the exact sum's terms (position strip only) per second of "
                                             "the same kernel time, over the same peak: the rate at "
                                             "which the cut delivers the exact sum's result"},
        "roofline_pass": {"bound": "hbm", "kernel": "k_osem_coop" if pass_n < 10 else "k_pass",
                          "units": "model rows once per iteration plus the image once per subset",
                          "achieved": pass_gbs,
                          "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": pass_gbs / pk["hbm_gbs"],
                          "peak_kind": pk_kind},
        "clocks": clk,
        "gpu_launches": sum(runs[f]["launches"] for f in forms),
    }
    if chosen != EXACT_FMT:
        _, x_pass_ms, x_pass_n, x_pass_gbs, x_ms_step = summary(EXACT_FMT)
        X = runs[EXACT_FMT]
        out["exact"] = {"model_format": EXACT_FMT, "value": aggregate_rate(evals, world, x_ms_step),
                        "unit": UNIT, "ms_per_step": x_ms_step, "s_per_iter": X["s_per_iter"],
                        "pass_gbs": x_pass_gbs, "pass_frac_of_%s_hbm" % pk_kind: x_pass_gbs / pk["hbm_gbs"],
                        "model_bytes": X["model_bytes"], "loglik_final": X["ll"]}
        fc, fx = np.zeros(ph.mu.size), np.zeros(ph.mu.size)
        sup = np.nonzero(ph.mu.reshape(-1) > 0)[0]
        fc[sup], fx[sup] = R["f"], X["f"]
        rc, rx = roi_means(fc, ph.rois), roi_means(fx, ph.rois)
        out["chosen_vs_exact"] = {
            "what": "the chosen form's image against the exact FP32 form's, all %d events" % J,
            "rel_l2": float(np.linalg.norm(fc - fx) / np.linalg.norm(fx)),
            "roi_rel": {k: rc[k] / rx[k] - 1.0 for k in rc},
            "s_per_iter_ratio": R["s_per_iter"] / X["s_per_iter"]}
    if errors is not None:
        out["error_vs_fp64_oracle"] = errors
    return out


def kernel_source_sha1():
    """Hash of the path-sum kernel's source text (its argument block through
    the end of the kernel), so that edits elsewhere in the file keep the
    committed traffic figure valid."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2002_12471_gb300", "csrc", "model.cu"), "rb").read()
    i = src.find(b"struct PathSumArgs {")
    j = src.find(b"\n// Row scaling and rounding", i)
    return hashlib.sha1(src[i:j] if i >= 0 and j > i else src).hexdigest()[:12]


def read_traffic(kernel, workload):
    """DRAM bytes per launch of a kernel on a workload (name and event count,
    e.g. dat128_1M) from the committed ncu summary, if the kernel's source has
    not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_source_sha1()
    for ln in open(path):
        parts = dict(p.split("=", 1) for p in ln.split() if "=" in p)
        if (parts.get("kernel") == kernel and parts.get("source_sha1") == h
                and parts.get("workload", "") == workload):
            try:
                return float(parts["dram_bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


# ------------------------------------------------------------------ oracle arm

# Angles in the oracle sample: all of them at 64 x 64; every 15th at 128 x 128
# (8 of 120, one per subset), where the full tables and sensitivity alone take
# minutes of CPU.
ORACLE_ANGLE_STRIDE = {"dat64": 1, "dat128": 15}


def oracle_sample_run(ph, g, ev, ns, ni, per_angle, stride=1, P=None):
    """The FP64 oracle on a bounded sample: attenuation tables, subset
    sensitivity, then model rows and OSEM for `per_angle` events of every
    `stride`-th angle.  With stride > 1 the sample runs on a scanner with
    only those angles (the same physical angles, a -> a / stride), so its
    sensitivity and per-angle table cost are 1/stride of the workload's.
    Returns phase times in seconds (tables 0 when a built problem P is
    passed in) and the problem."""
    import oracle
    gs = dict(g, n_angles=g["n_angles"] // stride, pixel_mm=ph.pixel_mm)
    rng = np.random.default_rng(per_angle)
    idx = np.concatenate([rng.choice(np.nonzero(ev.angle == a)[0],
                                     min(per_angle, int(np.sum(ev.angle == a))), replace=False)
                          for a in range(0, g["n_angles"], stride) if np.any(ev.angle == a)])
    a_s = (ev.angle[idx] // stride).astype(np.int32)
    t0 = time.perf_counter()
    tables = 0.0
    if P is None:
        P = oracle.Problem(gs, ph.mu)
        tables = time.perf_counter() - t0
    t1 = time.perf_counter()
    s = P.sensitivity(min(ns, gs["n_angles"]))
    t2 = time.perf_counter()
    p = P.model(a_s, ev.u_mm[idx], ev.e_kev[idx])
    t3 = time.perf_counter()
    f, _ = oracle.osem(p, a_s, s, ni, oracle.initial_image(len(idx), s.sum(0)))
    oracle.loglik(p, f, s.sum(0))
    t4 = time.perf_counter()
    return dict(tables=tables, sens=t2 - t1, model=t3 - t2, osem=t4 - t3, n=len(idx), n_nz=P.n_sup,
                stride=stride, P=P)


def oracle_rate(ph, g, ev, ns, ni, fit=None):
    """Oracle evals/s extrapolated to the whole workload: tables + sensitivity
    x stride + per-angle model tables x stride + (model + OSEM per event) x J.
    The model time is fitted as a per-angle table cost plus a per-event cost
    from two sample sizes; a given fit (with its problem) is reused and only
    the larger sample is run again."""
    J = len(ev)
    stride = ORACLE_ANGLE_STRIDE.get(WORKLOAD, 1)
    small, large = (3, 6) if stride == 1 else (2, 10)
    if fit is None:
        r1 = oracle_sample_run(ph, g, ev, ns, ni, small, stride)
        r2 = oracle_sample_run(ph, g, ev, ns, ni, large, stride, P=r1["P"])
        b = max(0.0, (r2["model"] - r1["model"]) / (r2["n"] - r1["n"]))
        a = max(0.0, r2["model"] - b * r2["n"])
        fit = dict(model_fixed=a, model_per_event=b, tables=r1["tables"], P=r1["P"])
        wall = sum(r[k] for r in (r1, r2) for k in ("tables", "sens", "model", "osem"))
        run = r2
    else:
        run = oracle_sample_run(ph, g, ev, ns, ni, large, stride, P=fit["P"])
        wall = run["sens"] + run["model"] + run["osem"]
    t_full = (fit["tables"] + stride * (run["sens"] + fit["model_fixed"])
              + (fit["model_per_event"] + run["osem"] / run["n"]) * J)
    value = J * run["n_nz"] / t_full
    return value, fit, run, wall


def cores_used():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n and n.isdigit() else (os.cpu_count() or 1)


def cpu_baseline_block(value, run, wall, J):
    st, na = run["stride"], run["P"].geom.n_angles
    where = ("every angle" if st == 1 else
             "every %d-th angle (%d of %d, on a scanner with only those angles; sensitivity and "
             "per-angle table time x %d)" % (st, na, na * st, st))
    return {"value": value, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
            "sample": ("FP64 C/OpenMP oracle on %s: attenuation tables, subset sensitivity, model rows "
                       "and 10 OSEM iterations for %d of the %d events; the whole workload's time "
                       "extrapolated linearly in J and in the angle count (model time fitted as a "
                       "per-angle table cost plus a per-event cost from two sample sizes); %.1f s of "
                       "CPU wall time measured" % (where, run["n"], J, wall))}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    ph, g, ev, ns, ni = make_inputs(seed=SEEDS[WORKLOAD])
    J = len(ev)
    stride = ORACLE_ANGLE_STRIDE.get(WORKLOAD, 1)
    P = None
    for _ in range(args.warmup):
        P = oracle_sample_run(ph, g, ev, ns, ni, 1, stride, P=P)["P"]
    v0, fit, run0, wall0 = oracle_rate(ph, g, ev, ns, ni)
    vals, walls = [], []
    run = run0
    for _ in range(args.steps):
        v, _, run, wall = oracle_rate(ph, g, ev, ns, ni, fit)
        vals.append(v)
        walls.append(wall)
    value = statistics.mean(vals)
    ms = J * run["n_nz"] / value * 1e3
    cpu = cpu_baseline_block(value, run, statistics.mean(walls), J)
    cpu["sample"] += ("; each timed step reran the larger sample on the problem the fit built "
                      "(its %.1f s of tables counted once in every extrapolation)" % fit["tables"])
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "ms_per_step_kind": "extrapolated to the whole workload from the measured sample",
            "sample_wall_ms_per_step": statistics.mean(walls) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded ellipse phantom, photon Monte-Carlo list-mode events)",
            "config": workload_config(J, run["n_nz"], args.fmt, world),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ batching form

def _realisation_events(args):
    """Worker: events of one realisation (numpy only, no CUDA)."""
    r, n = args
    from paper_2002_12471_gb300 import synthetic as S
    ph, g, _, _, _ = S.workload("dat64")
    ev = S.simulate_events(ph, g, int(n), seed=4000 + r)
    return ev.angle, ev.u_mm, ev.e_kev


def run_batch_bench(args):
    """64 noise realisations of the 64x64 DaT phantom with Poisson event counts
    (lambda uniform in [50k, 400k]) reconstructed together: one step = model
    build for all realisations + 10 batched iterations (one persistent
    launch), tiles chosen by the autotuner."""
    import multiprocessing as mp

    from paper_2002_12471_gb300 import synthetic as S
    counts = S.realisation_counts(64, seed=4)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:   # before any CUDA call
        parts = pool.map(_realisation_events, list(enumerate(counts)))
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    ph, g, _, ns, ni = S.workload("dat64")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    a = torch.from_numpy(np.concatenate([p[0] for p in parts])).to(dev)
    u = torch.from_numpy(np.concatenate([p[1] for p in parts])).to(dev)
    e = torch.from_numpy(np.concatenate([p[2] for p in parts])).to(dev)
    J = int(off[-1])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    choice = None

    def step(tune=False):
        nonlocal choice
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, profile=2)
        try:
            nsup = L.lmosem_n_support(ctx)
            L.lmosem_sensitivity(ctx, ns)
            L.lmosem_build_model_batch(ctx, a, u, e, off, ns)
            f = torch.empty((len(counts), nsup), dtype=torch.float32, device=dev)
            L.lmosem_init_image_batch(ctx, 1.0, f)
            if tune:
                choice = L.lmosem_autotune_batch(ctx, 1.0, f)
            L.lmosem_set_batch_tiles(ctx, *choice)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lmosem_iterate_batch(ctx, ni, 1.0, f)
            e1.record(stream)
            e1.synchronize()
            prof = L.lmosem_profile_read(ctx)
            return nsup, e0.elapsed_time(e1), prof, L.lmosem_model_bytes(ctx), L.lmosem_launch_count(ctx)
        finally:
            L.lmosem_destroy(ctx)

    step(tune=True)
    for _ in range(max(0, args.warmup - 1)):
        step()
    clocks = ClockSampler(None)
    torch.cuda.synchronize()
    clocks.start()
    times, it_ms, launches = [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        nsup, ims, prof, model_bytes, nl = step()
        t1.record(stream)
        t1.synchronize()
        times.append(t0.elapsed_time(t1))
        it_ms.append(ims)
        launches += nl
    clk = clocks.stop()
    pk, pk_kind = peaks()
    ms_step = statistics.mean(times)
    s_iter = statistics.mean(it_ms) / ni * 1e-3
    gbs = model_bytes / s_iter / 1e9
    return {
        "metric": METRIC, "value": J * nsup / (ms_step * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipse phantom, photon Monte-Carlo list-mode events)",
        "config": {"workload": WORKLOAD_DESC, "events": J, "realisations": len(counts),
                   "events_min_max": [int(min(counts)), int(max(counts))], "support_pixels": nsup,
                   "tiles": {"chunk_rows": choice[0], "ctas_per_sm": choice[1]},
                   "l2": "model (%.1f GB) larger than L2; 256 MB flush before every step" % (model_bytes / 1e9)},
        "s_per_iter": s_iter,
        "batched_iteration": {"gbs": gbs, "frac_of_%s_hbm" % pk_kind: gbs / pk["hbm_gbs"],
                              "model_bytes": model_bytes, "persistent_launches_per_call": 1},
        "breakdown_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]},
        "clocks": clk, "gpu_launches": launches,
    }


# ------------------------------------------------------------------ surrogate form

SURR_TRAIN_SEEDS = tuple(range(1000, 1032))
SURR_TRAIN_EVENTS = 1000           # x ~5,900 support pixels = ~6M (event, pixel) pairs per phantom
SURR_GATE_ROW_TOL = 1e-2           # energy gate: bins whose sampled mean row error exceeds this are exact
SURR_CHECK_ROWS = 512              # rows the library's exact judge samples (its default)
SURR_EVAL_SEED = 2000
SURR_EVAL_EVENTS = 2_000_000
SURR_EVAL_CHUNKS = 16
MLP_FLOPS_PER_PAIR = 2 * (8 * 256 + 3 * 256 * 256 + 256)   # the network's multiply-adds x 2


def surrogate_phantom(seed):
    from paper_2002_12471_gb300 import synthetic as S
    return S.brain_phantom(128, 2.0, jitter=np.random.default_rng(seed))


def _surrogate_events(job):
    """Worker: events of one jittered 128 x 128 phantom (numpy only, no CUDA)."""
    phantom_seed, n, event_seed = job
    from paper_2002_12471_gb300 import synthetic as S
    g = S.workload("dat128")[1]
    ev = S.simulate_events(surrogate_phantom(phantom_seed), g, int(n), seed=event_seed)
    return ev.angle, ev.u_mm, ev.e_kev


def surrogate_jobs(eval_events):
    per = -(-eval_events // SURR_EVAL_CHUNKS)
    sizes = [min(per, eval_events - k * per) for k in range(SURR_EVAL_CHUNKS)]
    return ([(s, SURR_TRAIN_EVENTS, s) for s in SURR_TRAIN_SEEDS]
            + [(SURR_EVAL_SEED, n, SURR_EVAL_SEED * 100 + k) for k, n in enumerate(sizes) if n > 0])


def run_ex2_bench(args):
    """The MUFU ex2 rate that the path sum's ALU roofline divides by, measured
    by the library (lmosem_measure_ex2_rate) under the clock sampler; also
    the rate with other launch shapes, to show where it saturates."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for _ in range(args.warmup):
        L.lmosem_measure_ex2_rate(None, 4, 512, 1 << 14)
    clocks = ClockSampler(None)
    clocks.start()
    rates = [L.lmosem_measure_ex2_rate(None, 4, 512, 1 << 16) for _ in range(args.steps)]
    clk = clocks.stop()
    shapes = {}
    for cps, nt in ((1, 128), (1, 512), (2, 512), (4, 256), (4, 512), (8, 256)):
        shapes["%dx%d" % (cps, nt)] = L.lmosem_measure_ex2_rate(None, cps, nt, 1 << 15)
    mhz = (clk or {}).get("sm_mhz") or SM_MAX_MHZ_FALLBACK
    rate = statistics.median(rates)
    per_clk = lambda r: r / (sms * mhz * 1e6)
    return {"metric": "ex2.approx.ftz.f32 per second", "value": rate, "unit": "ex2/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "config": {"workload": WORKLOAD_DESC, "sms": sms},
            "per_clock_per_sm": per_clk(rate), "clock_mhz_used": mhz,
            "per_clock_per_sm_by_launch_shape": {k: per_clk(v) for k, v in shapes.items()},
            "clocks": clk}


def run_mlp_bench(args):
    """The tcgen05 inference kernel alone (the tensor roofline of form 4):
    each step is one lmosem_surrogate_infer call on `--events` rows (default
    2M); the network's own time comes from the library's per-kernel profile."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    from paper_2002_12471_gb300 import synthetic as S
    rows = args.events or 2_000_000
    ph, g, *_ = S.workload("tiny16")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    rng = np.random.default_rng(1)
    blob = torch.from_numpy(L.surrogate_init(seed=2)).to(dev)
    X = torch.from_numpy(rng.standard_normal((rows, 8)).astype(np.float32)).to(dev)
    y = torch.empty(rows, dtype=torch.float32, device=dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, profile=1)
    try:
        for _ in range(args.warmup):
            L.lmosem_surrogate_infer(ctx, blob, X, y)
        L.lmosem_profile_read(ctx)
        clocks = ClockSampler(None)
        clocks.start()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lmosem_surrogate_infer(ctx, blob, X, y)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        clk = clocks.stop()
        prof = L.lmosem_profile_read(ctx)
        launches = L.lmosem_launch_count(ctx)
    finally:
        L.lmosem_destroy(ctx)
    if not bool(torch.isfinite(y).all()):
        raise RuntimeError("non-finite network output")
    mlp_ms = prof["mlp"][0] / args.steps
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    achieved = rows * MLP_FLOPS_PER_PAIR / (mlp_ms * 1e-3) / 1e12
    return {"metric": METRIC, "value": rows / (statistics.mean(ms) * 1e-3), "unit": "rows/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
            "data": "synthetic (standard-normal inputs, He-initialised weights)",
            "config": {"workload": WORKLOAD_DESC, "rows": rows},
            "network_ms_per_step": mlp_ms,
            "roofline": {"bound": "tensor", "kernel": "k_mlp_tc", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "peak_kind": pk_kind + " sustained BF16"},
            "clocks": clk, "gpu_launches": launches}


# flops of one training step per minibatch row: the forward products
# (16 -> 256, 3 x 256 -> 256), the input-gradient products of the three hidden
# layers and the weight-gradient products of all four, 2 flops per
# multiply-add (the 256 -> 1 output layer is not a tensor-core product)
MLP_TRAIN_FLOPS_PER_ROW = 2 * (2 * (16 * 256 + 3 * 256 * 256) + 3 * 256 * 256)


def run_mlp_train_bench(args):
    """The surrogate's training loop alone: --steps Adam steps of 8,192 rows
    in one lmosem_surrogate_train call (its CUDA-graph replay of a captured
    step), timed with CUDA events; TFLOP/s of the products against the
    measured sustained BF16 peak."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    from paper_2002_12471_gb300 import synthetic as S
    n, B = 4_000_000, 8192
    steps = max(1, args.steps) * 500
    ph, g, *_ = S.workload("tiny16")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    rng = np.random.default_rng(1)
    feat = torch.from_numpy(rng.standard_normal((n, 8)).astype(np.float32)).to(dev)
    targ = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
    try:
        blob = torch.from_numpy(L.surrogate_init(seed=3)).to(dev)
        L.lmosem_surrogate_train(ctx, feat, targ, blob, steps=max(1, args.warmup) * 100, batch=B, lr=1e-3, seed=5)
        blob = torch.from_numpy(L.surrogate_init(seed=3)).to(dev)
        clocks = ClockSampler(None)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        curve = L.lmosem_surrogate_train(ctx, feat, targ, blob, steps=steps, batch=B, lr=1e-3, seed=5)
        e1.record(stream)
        e1.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        launches = L.lmosem_launch_count(ctx)
    finally:
        L.lmosem_destroy(ctx)
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    tflops = steps * B * MLP_TRAIN_FLOPS_PER_ROW / (ms * 1e-3) / 1e12
    return {"metric": "surrogate training steps/s", "value": steps / (ms * 1e-3), "unit": "steps/s", "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
            "data": "synthetic (standard-normal features and targets)",
            "config": {"workload": WORKLOAD_DESC, "batch": B, "samples": n},
            "loss_first": float(curve[0]), "loss_last": float(np.mean(curve[-50:])),
            "roofline": {"bound": "tensor", "kernel": "training step (tcgen05 products, transposes, Adam)",
                         "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                         "traffic": None, "peak_kind": pk_kind + " sustained BF16"},
            "clocks": clk, "gpu_launches": launches}


def surrogate_baseline(blob, x):
    """The blob's quadratic baseline c . phi(x) of the log scatter at scaled
    inputs x (n x 8 torch tensor): phi = (1, x_i, x_i x_k for i <= k <= 6), the
    first six inputs only."""
    import torch
    nb = 28
    coef = torch.as_tensor(np.asarray(blob[-2 - nb:-2], dtype=np.float64), device=x.device)
    cols = [torch.ones_like(x[:, 0])] + [x[:, i] for i in range(6)]
    cols += [x[:, i] * x[:, k] for i in range(6) for k in range(i, 6)]
    return torch.stack(cols, 1) @ coef


def run_surrogate_bench(args):
    """Form (4): the scatter term of the model from the MLP surrogate.  The
    network is trained (untimed) on exact scatter path sums of 32 jittered
    128 x 128 phantoms; one timed step is the whole hot path on 2M events of
    a held-out phantom with the surrogate scatter term: sensitivity, model
    build (fused tcgen05 inference), 8 subsets x 10 OSEM iterations and the
    log-likelihood.  The exact model is built and reconstructed beside it, and
    the surrogate's error is measured against it on model rows, on held-out
    log scatter values and on the reconstructed image."""
    import multiprocessing as mp

    from paper_2002_12471_gb300 import synthetic as S
    n_eval = args.events or SURR_EVAL_EVENTS
    jobs = surrogate_jobs(n_eval)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:   # before any CUDA call
        parts = pool.map(_surrogate_events, jobs)
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    g = S.workload("dat128")[1]
    ns, ni = 8, 10
    T = 1.0
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # ---- training set: exact log scatter of every (event, support pixel)
    t_samples = time.perf_counter()
    feats, targs, rels = [], [], []
    for (seed, _, _), (a, u, e) in zip(jobs[:len(SURR_TRAIN_SEEDS)], parts):
        ph = surrogate_phantom(seed)
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
        try:
            nsup = L.lmosem_n_support(ctx)
            feat = torch.empty((len(a) * nsup, L.SURROGATE_INPUTS), dtype=torch.float32, device=dev)
            targ = torch.empty(len(a) * nsup, dtype=torch.float32, device=dev)
            rel = torch.empty(len(a) * nsup, dtype=torch.float32, device=dev)
            L.lmosem_surrogate_samples(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(u).to(dev),
                                       torch.from_numpy(e).to(dev), feat, targ, rel)
            feats.append(feat)
            targs.append(targ)
            rels.append(rel)
        finally:
            L.lmosem_destroy(ctx)
    feat = torch.cat(feats)
    targ = torch.cat(targs)
    rel = torch.cat(rels)
    n_train_pairs = int(targ.numel())
    del feats, targs, rels
    torch.cuda.synchronize()
    t_samples = time.perf_counter() - t_samples

    ph = surrogate_phantom(SURR_EVAL_SEED)
    ev_parts = parts[len(SURR_TRAIN_SEEDS):]
    a_h = torch.from_numpy(np.concatenate([p[0] for p in ev_parts])).pin_memory()
    u_h = torch.from_numpy(np.concatenate([p[1] for p in ev_parts])).pin_memory()
    e_h = torch.from_numpy(np.concatenate([p[2] for p in ev_parts])).pin_memory()
    J = len(a_h)
    a_d, u_d, e_d = a_h.to(dev), u_h.to(dev), e_h.to(dev)

    # pairs drawn in proportion to (scatter / its row's largest scatter)^1
    train_steps, train_batch, train_floor, train_power = 60000, 8192, 14.0, 1.0
    blob = torch.from_numpy(L.surrogate_init(seed=3)).to(dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
    try:
        t_train = time.perf_counter()
        curve = L.lmosem_surrogate_train(ctx, feat, targ, blob, steps=train_steps, batch=train_batch,
                                         lr=1e-3, seed=5, target_floor=train_floor, residual_fit=True,
                                         d_rel_log=rel, magnitude_power=train_power)
        t_train = time.perf_counter() - t_train
        # held out: exact log scatter of 200 events of the evaluation phantom
        nsup = L.lmosem_n_support(ctx)
        hold = 200
        hf = torch.empty((hold * nsup, L.SURROGATE_INPUTS), dtype=torch.float32, device=dev)
        ht = torch.empty(hold * nsup, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_samples(ctx, a_d[:hold].contiguous(), u_d[:hold].contiguous(),
                                   e_d[:hold].contiguous(), hf, ht)
        hy = torch.empty(hold * nsup, dtype=torch.float32, device=dev)
        L.lmosem_surrogate_infer(ctx, blob, hf, hy)
        _, mu_t, sigma_t = L.unpack_surrogate(blob.cpu().numpy())
        pred = surrogate_baseline(blob.cpu().numpy(), hf.double()) + mu_t + sigma_t * hy.double()
        err = (pred - ht.double()).cpu().numpy()
        w_ho = ht.double().exp()
        ho_lin = float(torch.linalg.vector_norm(pred.exp() - w_ho) / torch.linalg.vector_norm(w_ho))
        ho_wabs = float((w_ho * (pred - ht.double()).abs()).sum() / w_ho.sum())
    finally:
        L.lmosem_destroy(ctx)
    del feat, targ
    torch.cuda.empty_cache()

    support = None
    last_check = [None]
    rows_ids = torch.arange(0, J, max(1, J // 2000), dtype=torch.int64, device=dev)

    last_gate = [None]

    def step(surrogate, a, u, e, profile=0, rows=None, host_out=None, gate=SURR_GATE_ROW_TOL):
        nonlocal support
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream, profile=profile)
        try:
            nsup = L.lmosem_n_support(ctx)
            if support is None:
                support = L.lmosem_support(ctx)
            if surrogate:
                L.lmosem_surrogate_load(ctx, blob)
                L.lmosem_set_surrogate_gate(ctx, gate)
            L.lmosem_sensitivity(ctx, ns)
            L.lmosem_build_model(ctx, a, u, e, ns, "surrogate" if surrogate else "fp32")
            if surrogate:
                last_check[0] = L.lmosem_surrogate_check(ctx)
                last_gate[0] = L.lmosem_surrogate_gate(ctx)
            f = torch.empty(nsup, dtype=torch.float32, device=dev)
            ll = torch.empty(1, dtype=torch.float64, device=dev)
            L.lmosem_init_image(ctx, T, f)
            L.lmosem_iterate(ctx, ni, T, f)
            L.lmosem_loglik(ctx, T, f, ll)
            if host_out is not None:
                host_out[0].copy_(f, non_blocking=True)
                host_out[1].copy_(ll, non_blocking=True)
            if rows is not None:
                rows.append(torch.empty((rows_ids.numel(), nsup), dtype=torch.float32, device=dev))
                L.lmosem_model_rows(ctx, rows_ids, rows[-1])
            prof = L.lmosem_profile_read(ctx) if profile else None
            return f, ll, prof, L.lmosem_launch_count(ctx)
        finally:
            L.lmosem_destroy(ctx)

    def timed(fn):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    # ---- exact model beside it (same events): image, sampled rows, build time
    rows_exact, rows_sur = [], []
    ex_ms, (f_exact, _, prof_ex, _) = timed(lambda: step(False, a_d, u_d, e_d, profile=2, rows=rows_exact))
    f_exact = f_exact.double().cpu().numpy()

    for _ in range(args.warmup):
        step(True, a_d, u_d, e_d)
    torch.cuda.synchronize()
    clocks = ClockSampler(None)
    clocks.start()
    times, profs, launches = [], [], 0
    for _ in range(args.steps):
        ms, (f_sur, ll, prof, nl) = timed(lambda: step(True, a_d, u_d, e_d, profile=2))
        times.append(ms)
        profs.append(prof)
        launches += nl
    clk = clocks.stop()
    _, (f_sur, ll, _, _) = timed(lambda: step(True, a_d, u_d, e_d, rows=rows_sur))
    f_sur_np = f_sur.double().cpu().numpy()
    check_gated, gate_gated = last_check[0], last_gate[0]
    # the network alone (gate off), for the error it leaves without the exact rows
    rows_net = []
    _, (f_net, _, _, _) = timed(lambda: step(True, a_d, u_d, e_d, rows=rows_net, gate=0.0))
    f_net_np = f_net.double().cpu().numpy()
    check_net = last_check[0]

    # ---- end to end through host buffers
    nsup = len(support)
    f_h = torch.empty(nsup, dtype=torch.float32).pin_memory()
    ll_h = torch.empty(1, dtype=torch.float64).pin_memory()
    e2e = []
    for _ in range(max(1, min(args.steps, 2))):
        ms, _ = timed(lambda: step(True, a_h.to(dev, non_blocking=True), u_h.to(dev, non_blocking=True),
                                   e_h.to(dev, non_blocking=True), host_out=(f_h, ll_h)))
        e2e.append(ms)

    # ---- errors of the surrogate form against the exact model
    re = rows_exact[0].double()
    rs = rows_sur[0].double()
    row_err = float(torch.linalg.vector_norm(rs - re) / torch.linalg.vector_norm(re))
    row_err_net = float(torch.linalg.vector_norm(rows_net[0].double() - re) / torch.linalg.vector_norm(re))
    img = lambda f: np.bincount(support, weights=f, minlength=ph.mu.size)

    def roi_err(f):
        out = {}
        for name, w in ph.rois.items():
            w = w.reshape(-1)
            ref = float(np.dot(w, img(f_exact)) / w.sum())
            out[name] = (float(np.dot(w, img(f)) / w.sum()) - ref) / ref
        return out
    roi = roi_err(f_sur_np)
    img_err = float(np.linalg.norm(f_sur_np - f_exact) / np.linalg.norm(f_exact))
    img_err_net = float(np.linalg.norm(f_net_np - f_exact) / np.linalg.norm(f_exact))

    agg = {}
    for p in profs:
        for k, (ms, n) in p.items():
            a = agg.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n
    mlp_ms, mlp_n = agg["mlp"]
    pairs = J * nsup
    # the network evaluates the judge's sampled rows, then the rows at or
    # above the gate's cut (the exact path sum builds the others)
    n_exact_rows = int(round(gate_gated[1] * J))
    net_pairs = (min(J, SURR_CHECK_ROWS) + (J - n_exact_rows)) * nsup
    pk, pk_kind = peaks()
    achieved = net_pairs * MLP_FLOPS_PER_PAIR / (mlp_ms / args.steps * 1e-3) / 1e12
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    ms_step = statistics.mean(times)
    ex_build_ms = prof_ex["pathsum"][0] + prof_ex["wtable"][0]
    sur_build_ms = (agg["mlp"][0] + agg["surrogate"][0]) / args.steps
    terms, _ = strip_terms(ph, g, type("E", (), {"u_mm": u_h.numpy(), "angle": a_h.numpy()})())
    kernel_ms = sum(v[0] for v in agg.values())
    return {
        "metric": METRIC, "value": pairs / (ms_step * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
        "data": "synthetic (seeded jittered ellipse phantoms, photon Monte-Carlo list-mode events)",
        "config": {"workload": WORKLOAD_DESC, "events": J, "support_pixels": nsup,
                   "train_pairs": n_train_pairs, "train_phantoms": len(SURR_TRAIN_SEEDS),
                   "train_steps": train_steps, "train_batch": train_batch,
                   "train_target_floor": train_floor, "train_residual_of_quadratic_baseline": True,
                   "train_sampling": "pairs drawn with probability proportional to (scatter / row maximum)^%g"
                                     % train_power,
                   "l2": "model (%.1f GB) larger than L2; 256 MB flush before every step" % (J * nsup * 4 / 1e9)},
        "model_build_evals_per_s": {"surrogate": pairs / (sur_build_ms * 1e-3),
                                    "exact": pairs / (ex_build_ms * 1e-3),
                                    "exact_path_terms": terms},
        "exact_step_ms": ex_ms,
        "exact_check": {"what": "the library's exact judge of every surrogate build: 512 evenly spaced rows "
                                "recomputed with the exact path sum; the energy gate gives the rows of every "
                                "5 keV bin up to the highest one whose sampled mean row error exceeds its "
                                "tolerance exact rows; above the check's tolerance the whole build falls back "
                                "to the exact model", "tol": 1e-2, "gate_row_tol": SURR_GATE_ROW_TOL,
                        "gate_cut_kev": gate_gated[0], "rows_exact_fraction": gate_gated[1],
                        "rows_rel_l2": check_gated[0], "worst_row_rel_l2": check_gated[1],
                        "fell_back_to_exact": check_gated[2]},
        "network_alone": {"what": "the same build with the gate off (every row from the network)",
                          "model_rows_rel_l2": row_err_net, "image_rel_l2": img_err_net,
                          "roi_mean_rel": roi_err(f_net_np), "check_rows_rel_l2": check_net[0],
                          "check_worst_row_rel_l2": check_net[1]},
        "error_vs_exact": {"model_rows_rel_l2": row_err, "image_rel_l2": img_err,
                           "roi_mean_rel": roi, "rows_sampled": int(rows_ids.numel()),
                           "held_out_scatter_rel_l2": ho_lin,
                           "held_out_log_scatter_abs_err_weighted": ho_wabs,
                           "held_out_log_scatter_median_abs": float(np.median(np.abs(err))),
                           "held_out_pairs": int(err.size)},
        "training": {"samples_s": t_samples, "train_s": t_train, "loss_first": float(np.mean(curve[:20])),
                     "loss_last": float(np.mean(curve[-200:]))},
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in agg.items() if v[1]},
        "kernel_share": {k: v[0] / kernel_ms for k, v in agg.items() if v[1]},
        "loglik_final": float(ll.item()),
        "e2e": {"value": pairs / (statistics.mean(e2e) * 1e-3), "unit": UNIT,
                "ms_per_step": statistics.mean(e2e), "h2d_bytes_per_step": int(J * 12),
                "d2h_bytes_per_step": int(nsup * 4 + 8)},
        "roofline": {"bound": "tensor", "kernel": "k_mlp_tc", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": "%s bf16 (sustained)" % pk_kind,
                     "flops_basis": "%d flops per (event, pixel) pair: 2 x (8x256 + 3x256x256 + 256); "
                                    "%d pairs per step through the network (the judge's %d sampled rows and the "
                                    "rows at or above the gate's cut)" % (MLP_FLOPS_PER_PAIR, net_pairs,
                                                                         min(J, SURR_CHECK_ROWS))},
        "clocks": clk, "gpu_launches": launches,
    }


# ------------------------------------------------------------------ energy windows

WINDOWS = (("full", 100.0), ("e120", 120.0), ("photopeak", 143.0))


def run_windows_bench(args):
    """Energy-window variants (paper Sec. 3: photopeak only, E > 120 keV and
    the whole spectrum, applied to the same acquisitions) over the 64 noise
    realisations of the batching workload: each window's events are cut from
    the full-spectrum data and reconstructed together in one persistent launch
    (8 subsets x 10 iterations).  The true image of a realisation is the
    phantom activity scaled so that the model's expected count T sum_n s_n f_n
    equals that realisation's event count in the window; caudate and putamen
    means of every image are compared with the true ones (NRMSE and mean bias
    over realisations, per window)."""
    import multiprocessing as mp

    from paper_2002_12471_gb300 import synthetic as S
    counts = S.realisation_counts(64, seed=4)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:   # before any CUDA call
        parts = pool.map(_realisation_events, list(enumerate(counts)))
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    ph, g_full, _, ns, ni = S.workload("dat64")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    act = ph.activity.reshape(-1)
    truth = {k: float(np.dot(w.reshape(-1), act) / w.sum()) for k, w in ph.rois.items()}
    out = {}
    times = []
    for name, e_lo in WINDOWS:
        g = dict(g_full, e_lo_kev=e_lo)
        keep = [p[2] >= e_lo for p in parts]
        n_r = np.array([int(k.sum()) for k in keep])
        off = np.concatenate([[0], np.cumsum(n_r)]).astype(np.int64)
        a = torch.from_numpy(np.concatenate([p[0][k] for p, k in zip(parts, keep)])).to(dev)
        u = torch.from_numpy(np.concatenate([p[1][k] for p, k in zip(parts, keep)])).to(dev)
        e = torch.from_numpy(np.concatenate([p[2][k] for p, k in zip(parts, keep)])).to(dev)
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
        try:
            nsup = L.lmosem_n_support(ctx)
            sup = L.lmosem_support(ctx)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sens = torch.zeros((ns, nsup), dtype=torch.float64, device=dev)
            t0.record(stream)
            L.lmosem_sensitivity(ctx, ns, sens)
            L.lmosem_build_model_batch(ctx, a, u, e, off, ns)
            f = torch.empty((len(counts), nsup), dtype=torch.float32, device=dev)
            L.lmosem_init_image_batch(ctx, 1.0, f)
            L.lmosem_iterate_batch(ctx, ni, 1.0, f)
            t1.record(stream)
            t1.synchronize()
            times.append(t0.elapsed_time(t1))
            fr = f.double().cpu().numpy()
            s_tot = sens.sum(0).cpu().numpy()
        finally:
            L.lmosem_destroy(ctx)
        expected_per_activity = float(np.dot(s_tot, act[sup]))   # T = 1
        rel = {k: [] for k in truth}
        for r in range(len(counts)):
            scale = n_r[r] / expected_per_activity                 # true image = scale x activity
            img = np.bincount(sup, weights=fr[r], minlength=act.size)
            for k, w in ph.rois.items():
                rel[k].append(float(np.dot(w.reshape(-1), img) / w.sum()) / (scale * truth[k]) - 1.0)
        out[name] = {"e_lo_kev": e_lo, "events": int(off[-1]),
                     "nrmse": {k: float(np.sqrt(np.mean(np.square(v)))) for k, v in rel.items()},
                     "bias": {k: float(np.mean(v)) for k, v in rel.items()},
                     "std": {k: float(np.std(v)) for k, v in rel.items()}}
    J = int(sum(counts))
    return {"metric": METRIC, "value": J * nsup / (times[0] * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": times[0], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ellipse phantom, photon Monte-Carlo list-mode events)",
            "config": {"workload": WORKLOAD_DESC, "realisations": len(counts), "events": J},
            "windows": out, "ms_per_window": dict(zip([w[0] for w in WINDOWS], times)),
            "truth_roi_means": truth}


BINNINGS = (("binned_2e", (100.0, 143.0, 175.0)), ("binned_3e", (100.0, 120.0, 143.0, 175.0)))


def run_binned_bench(args):
    """The paper's binning experiment (Sec. 4): the list-mode data of the 64
    noise realisations are binned into the detector's 64 position bins and 2
    or 3 energy bins and reconstructed from the bin-integrated model with
    count-weighted EM (8 subsets x 10 iterations), beside the list-mode
    reconstruction of the same events (one persistent launch).  ROI means are
    scored against the scaled phantom as in the window workload (NRMSE and
    bias over realisations).  Timing: the binned model build and one
    iteration per realisation, CUDA events on the context stream."""
    import multiprocessing as mp

    from paper_2002_12471_gb300 import synthetic as S
    counts = S.realisation_counts(64, seed=4)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:   # before any CUDA call
        parts = pool.map(_realisation_events, list(enumerate(counts)))
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2002_12471_gb300.lmosem as L
    ph, g, _, ns, ni = S.workload("dat64")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    act = ph.activity.reshape(-1)
    truth = {k: float(np.dot(w.reshape(-1), act) / w.sum()) for k, w in ph.rois.items()}
    n_r = np.array([len(p[0]) for p in parts])

    def score(images, sup, s_tot):
        expected_per_activity = float(np.dot(s_tot, act[sup]))   # T = 1
        rel = {k: [] for k in truth}
        for r in range(len(counts)):
            scale = n_r[r] / expected_per_activity
            img = np.bincount(sup, weights=images[r], minlength=act.size)
            for k, w in ph.rois.items():
                rel[k].append(float(np.dot(w.reshape(-1), img) / w.sum()) / (scale * truth[k]) - 1.0)
        return {"nrmse": {k: float(np.sqrt(np.mean(np.square(v)))) for k, v in rel.items()},
                "bias": {k: float(np.mean(v)) for k, v in rel.items()},
                "std": {k: float(np.std(v)) for k, v in rel.items()}}

    out = {}
    # list mode: every realisation in one persistent launch
    off = np.concatenate([[0], np.cumsum(n_r)]).astype(np.int64)
    a = torch.from_numpy(np.concatenate([p[0] for p in parts])).to(dev)
    u = torch.from_numpy(np.concatenate([p[1] for p in parts])).to(dev)
    e = torch.from_numpy(np.concatenate([p[2] for p in parts])).to(dev)
    ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
    try:
        nsup = L.lmosem_n_support(ctx)
        sup = L.lmosem_support(ctx)
        sens = torch.zeros((ns, nsup), dtype=torch.float64, device=dev)
        L.lmosem_sensitivity(ctx, ns, sens)
        L.lmosem_build_model_batch(ctx, a, u, e, off, ns)
        f = torch.empty((len(counts), nsup), dtype=torch.float32, device=dev)
        L.lmosem_init_image_batch(ctx, 1.0, f)
        L.lmosem_iterate_batch(ctx, ni, 1.0, f)
        stream.synchronize()
        s_tot = sens.sum(0).cpu().numpy()
        out["list_mode"] = dict(score(f.double().cpu().numpy(), sup, s_tot), rows=int(off[-1]))
    finally:
        L.lmosem_destroy(ctx)
    del a, u, e
    timing = {}
    for name, edges in BINNINGS:
        ctx = L.lmosem_create(ph.mu, ph.pixel_mm, g, stream=stream)
        try:
            L.lmosem_sensitivity(ctx, ns)
            imgs, t_build, t_iter, rows = [], [], [], []
            for r, p in enumerate(parts):
                ev = S.Events(p[0], p[1], p[2], np.arange(len(p[0])))
                cnt = torch.from_numpy(S.bin_events(ev, g, edges)).to(dev)
                t0, t1, t2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                t0.record(stream)
                L.lmosem_build_model_binned(ctx, cnt, edges, ns)
                t1.record(stream)
                f = torch.empty(nsup, dtype=torch.float32, device=dev)
                L.lmosem_init_image(ctx, 1.0, f)
                L.lmosem_iterate(ctx, ni, 1.0, f)
                t2.record(stream)
                t2.synchronize()
                t_build.append(t0.elapsed_time(t1))
                t_iter.append(t1.elapsed_time(t2) / ni)
                rows.append(int((cnt > 0).sum().item()))
                imgs.append(f.double().cpu().numpy())
        finally:
            L.lmosem_destroy(ctx)
        out[name] = dict(score(np.stack(imgs), sup, s_tot), e_edges_kev=list(edges),
                         rows_per_realisation_mean=float(np.mean(rows)))
        timing[name] = {"build_ms_median": float(np.median(t_build[1:])),
                        "ms_per_iter_median": float(np.median(t_iter[1:]))}
    mean_rows = out["binned_3e"]["rows_per_realisation_mean"]
    t3 = timing["binned_3e"]["build_ms_median"]
    return {"metric": METRIC, "value": mean_rows * nsup / (t3 * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": len(counts), "warmup": 1, "ms_per_step": t3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ellipse phantom, photon Monte-Carlo list-mode events, binned)",
            "config": {"workload": WORKLOAD_DESC, "realisations": len(counts), "events": int(off[-1]),
                       "value_is": "binned (3 energy bins) model build: rows x support pixels per second"},
            "results": out, "timing": timing, "truth_roi_means": truth}


# ------------------------------------------------------------------ main

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours" and torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif WORKLOAD == "batch64":
        out = run_batch_bench(args)
    elif WORKLOAD == "surrogate128":
        out = run_surrogate_bench(args)
    elif WORKLOAD == "mlp_infer":
        out = run_mlp_bench(args)
    elif WORKLOAD == "ex2_peak":
        out = run_ex2_bench(args)
    elif WORKLOAD == "mlp_train":
        out = run_mlp_train_bench(args)
    elif WORKLOAD == "windows64":
        out = run_windows_bench(args)
    elif WORKLOAD == "binned64":
        out = run_binned_bench(args)
    else:
        out = run_ours(args, rank, world, local_rank)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            ph, g, ev, ns, ni = make_inputs(seed=SEEDS[WORKLOAD])
            v, _, run, wall = oracle_rate(ph, g, ev, ns, ni)
            out["cpu_baseline"] = cpu_baseline_block(v, run, wall, len(ev))
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
