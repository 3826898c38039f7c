"""Benchmark: pixels inverted per second on the two-line 512x512 map.

Workload (synthetic stand-in for a SOLIS/VSM scan; the precision-plus-
differentiation configuration): Fe I 6301.5 + 6302.5 in one propagation
matrix, 128 wavelength points over 6301.0-6303.0 A, 262144 pixels with truth
drawn uniformly from the priors, float32 cube, noise 1e-3 I_c; population
128, 200 generations.  One step inverts the whole map with the FP32 GA
(inverse-max fitness, Section 5.4) followed by 10 L-M iterations (sigma
weights, analytic Jacobian, FP64 normal-equation solve); the reported chi2 is
the FP64 sigma-weighted chi2 (about 1 at the truth).  The plain FP64 GA on
the same map is timed on whole waves of its kernel for the comparison the
metric asks for.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank inverts its own map (pixel ids offset by rank), so
per-GPU work is fixed (weak scaling); no collective touches the data path.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import genesis_inputs as gi  # noqa: E402

METRIC = "pixels inverted/s at fixed median chi2 vs plain FP64 GA"


def workload(side):
    return (f"two-line Fe I 6301.5+6302.5 ME inversion, {side}x{side} px, 128 lambda, float32 cube, npop 128, "
            "200 gen, FP32 GA + 10 L-M (analytic adjoint, FP64 Cholesky)")


L2_BYTES = 129e6
E2E_STEPS_MAX = 5   # the end-to-end leg repeats at most this many steps
NPOP, NGEN, LM_ITERS = 128, 200, 10
KERNELS_PER_STEP = 4  # GA evolve, FP64 chi2, L-M, FP64 chi2
# DRAM bytes (read + write) per pixel of one GA launch, from an ncu capture of
# k_ga_evolve on the 4096-pixel two-line case (dram__bytes_read.sum 8580608 +
# dram__bytes_write.sum 0, divided by 4096; traffic grows in proportion to
# pixels: each block reads its pixel's cube row once).  Set to None whenever
# the kernel changes, until it is captured again.
GA_DRAM_BYTES_PER_PIXEL = 2094.88


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=512, help="map side (pixels = side^2)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sample")
    ap.add_argument("--no-pipeline", action="store_true", help="skip the full-disc pipeline sample")
    ap.add_argument("--serve", action="store_true",
                    help="run only the serving benchmark (Poisson arrivals at 0.7x and 1.2x capacity)")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--configs", action="store_true",
                    help="time the FP64 oracle and the GPU FP64 GA on C1 (256 px) and a 256-px C2 subset")
    ap.add_argument("--pattern", action="store_true",
                    help="Fe I 6301.5 as its full Zeeman pattern on a 256^2 two-line map (FP32 GA + L-M), beside the "
                         "effective-triplet map and the plain FP64 GA")
    ap.add_argument("--disc", action="store_true",
                    help="the 2048^2 synthetic full disc (3.29 M px): FP32 GA (300 gen) + L-M against the plain "
                         "FP64 GA on whole waves of a sample")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ inputs
def make_map(api, torch, pb, side, rank, device):
    """Truth, observed cube (GPU synthesis + seeded noise) and sigma weights."""
    npix = side * side
    truth = gi.draw_truth(npix, seed=rank)
    tp = torch.tensor(truth, device=device)
    clean = api.me_synth(pb, tp)
    g = torch.Generator(device=device).manual_seed(1000 + rank)
    noise = torch.randn(clean.shape, generator=g, device=device, dtype=clean.dtype)
    sig = 1e-3 * (tp[:, 7] + tp[:, 8])
    obs = (clean + sig.to(clean.dtype)[:, None, None] * noise).contiguous()
    w = (1.0 / sig)[:, None].repeat(1, 4).contiguous()
    return truth, obs, w


def flop_model(nlines):
    """Algorithmic FP32 flops (FMA = 2, reciprocal = 1) of one synthesis + chi2,
    counted from the source of the GA's fitness path (per call, without the
    per-individual invariants such as 2a or (L + a)^2), per unit: an
    evaluation of w(z) in the interior (Weideman N = 16 by real-quadratic
    synthetic division, its last product added straight into the profile
    sums, 83 besides the two accumulating FMAs counted per point), in the
    middle shell (5th convergent, 43), in the continued-fraction region (3rd
    convergent in s = |z|^2, 23), in the outer shell (the even convergent in
    m = s - 3/2, 14) and in the far field (two-node approximant in
    u = s - 1/2, 9), the rational branches leaving their normalisation to
    the accumulation weight; and per wavelength point 16 per line for the
    component arguments (the pi argument by FMA, the sigma ones by adding
    and subtracting v_B) and the blue, pi and red profile sums (two FMAs
    each), 4 for the sums and differences of the sigma profiles, 35 for K
    and its closed-form inverse, 21 for the four Stokes values formed into
    their weighted residuals (w_I by one multiply), 7 for the four squares
    summed by FMA and 4 for the Kahan-compensated running sum.  Each point's
    evaluations are classified by its own region; branch tests, votes and work
    a pair or warp does beyond that are not counted."""
    return {"weideman": 83.0, "mid": 43.0, "cf": 23.0, "even2": 14.0, "far": 9.0, "point": 16.0 * nlines + 71.0}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1208_0302_gb300 import _lib, api

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.load()

    spec = gi.two_line_spec()
    pb32 = api.Problem.from_spec(spec, "f32")
    pb64 = api.Problem.from_spec(spec, "f64")
    side = args.side
    npix = side * side
    truth, obs, w = make_map(api, torch, pb32, side, rank, dev)
    lo, hi = gi.PRIOR_LO, gi.PRIOR_HI
    ga = api.GaSettings(npop=NPOP, ngen=NGEN, seed=rank)
    pid0 = rank * npix
    stream = torch.cuda.current_stream()

    def step():
        best, _ = api.ga_invert_batch(pb32, obs, lo, hi, ga, pixel_id0=pid0)
        p, c2 = api.lm_polish(pb32, obs, best, lo, hi, iters=LM_ITERS, w=w)
        return p, c2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    # the dominant kernel (GA evolve + its FP64 chi2 pass) timed on its stream
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ga_ms = []
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        best, _ = api.ga_invert_batch(pb32, obs, lo, hi, ga, pixel_id0=pid0)
        g1.record(stream)
        p, c2 = api.lm_polish(pb32, obs, best, lo, hi, iters=LM_ITERS, w=w)
        ga_ms.append((g0, g1))
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ga_avg = sum(a.elapsed_time(b) for a, b in ga_ms) / len(ga_ms)
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = npix * world / (ms_max / 1e3)
    chi2_med = float(c2.median().item())

    recovery = recovery_stats(torch, p, c2, truth)
    # the FP64 chi2 pass that ga_invert_batch launches after the GA kernel,
    # timed alone (same kernel, same pixels, inverse-max weights), so that the
    # roofline divides by the GA kernel's own time
    api.me_chi2(pb32, obs, best)
    chi_ms = []
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        api.me_chi2(pb32, obs, best)
        c1.record(stream)
        c1.synchronize()
        chi_ms.append(c0.elapsed_time(c1))
    chi_ms = min(chi_ms)
    # the measured FP32 FMA-pipe peak (scalar FFMA and packed FFMA2), clocks still sampled
    peak_meas = max(api.fp32_peak(packed=False), api.fp32_peak(packed=True))
    clk = clocks.stop()

    # end to end through the C ABI with host buffers (pinned), copies timed:
    # every step copies its cube and weights in from pinned host memory and
    # its parameters and chi2 back out.  Two device buffers let the next
    # step's input copy run on a copy stream while the current step computes,
    # and each step's results are read on the host while the next one runs.
    host_obs = obs.cpu().pin_memory()
    host_w = w.cpu().pin_memory()
    host_out = [torch.empty((npix, 9), dtype=torch.float64).pin_memory() for _ in range(2)]
    host_chi = [torch.empty(npix, dtype=torch.float64).pin_memory() for _ in range(2)]
    dobs = [torch.empty_like(obs) for _ in range(2)]
    dw = [torch.empty_like(w) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    results = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(1, min(args.steps, E2E_STEPS_MAX))
    checksum = 0.0

    def fetch(i):
        b = i % 2
        with torch.cuda.stream(copy_stream):
            if i >= 2:
                copy_stream.wait_event(consumed[b])   # step i - 2 is done with this buffer
            dobs[b].copy_(host_obs, non_blocking=True)
            dw[b].copy_(host_w, non_blocking=True)
            copied[b].record(copy_stream)

    barrier()
    h0 = time.perf_counter()
    fetch(0)
    for i in range(e2e_steps):
        b = i % 2
        if i + 1 < e2e_steps:
            fetch(i + 1)
        stream.wait_event(copied[b])
        best, _ = api.ga_invert_batch(pb32, dobs[b], lo, hi, ga, pixel_id0=pid0)
        p2, c22 = api.lm_polish(pb32, dobs[b], best, lo, hi, iters=LM_ITERS, w=dw[b])
        consumed[b].record(stream)
        if i >= 1:   # the previous step's results are on the host by now
            results[(i - 1) % 2].synchronize()
            checksum += float(host_chi[(i - 1) % 2][0])
        host_out[b].copy_(p2, non_blocking=True)
        host_chi[b].copy_(c22, non_blocking=True)
        results[b].record(stream)
    results[(e2e_steps - 1) % 2].synchronize()
    checksum += float(host_chi[(e2e_steps - 1) % 2][0])
    assert checksum == checksum
    e2e_ms = (time.perf_counter() - h0) * 1e3 / e2e_steps
    te = torch.tensor([e2e_ms], device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_val = npix * world / (float(te.item()) / 1e3)

    result = None
    if rank == 0:
        # algorithmic flops of one GA launch from exact branch counts
        counts = api.ga_count_evaluations(pb32, obs, lo, hi, ga, pixel_id0=pid0)
        fm = flop_model(len(spec.lines))
        flops = (counts["weideman"] * fm["weideman"] + counts["mid"] * fm["mid"] + counts["cf"] * fm["cf"] +
                 counts["even2"] * fm["even2"] + counts["far"] * fm["far"] + counts["points"] * fm["point"])
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        cube_bytes = obs.numel() * obs.element_size()
        max_mhz = clk.get("sm_max_mhz") or 2070.0
        peak_derived = sms * 128 * 2 * max_mhz * 1e6 / 1e12      # FP32 FMA lanes x 2 flops x clock
        ga_kernel_ms = ga_avg - chi_ms
        achieved = flops / (ga_kernel_ms / 1e3) / 1e12
        syntheses = counts["syntheses"]
        wz_evals = counts["weideman"] + counts["mid"] + counts["cf"] + counts["even2"] + counts["far"]
        result = {
            "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded truth from the priors, GPU ME synthesis + 1e-3 Ic Gaussian noise)",
            "config": {"workload": workload(side), "pixels_per_gpu": npix, "side": side, "n_lambda": spec.n_lambda,
                       "npop": NPOP, "ngen": NGEN, "lm_iters": LM_ITERS,
                       "l2": (f"inputs {'larger' if cube_bytes > L2_BYTES else 'smaller'} than L2 "
                              f"({cube_bytes / 1e6:.0f} MB float32 cube, L2 129 MB, no flush); compute bound")},
            "median_chi2": chi2_med,
            "syntheses_per_s": syntheses / (ga_kernel_ms / 1e3),
            "recovery": recovery,
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_meas, "unit": "TFLOP/s",
                         "frac": achieved / peak_meas,
                         "traffic": None if GA_DRAM_BYTES_PER_PIXEL is None else GA_DRAM_BYTES_PER_PIXEL * npix,
                         "kernel": "k_ga_evolve<float,2>",
                         "peak_basis": "measured: me_fp32_peak FFMA/FFMA2 throughput loop, best of scalar and "
                                       "packed, in this run at the sampled clock",
                         "peak_derived": peak_derived, "frac_of_derived": achieved / peak_derived,
                         "peak_derived_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                         "syntheses_per_s": syntheses / (ga_kernel_ms / 1e3),
                         "wz_evals_per_s": wz_evals / (ga_kernel_ms / 1e3),
                         "ga_ms": ga_kernel_ms, "ga_invert_ms": ga_avg, "chi2_pass_ms": chi_ms,
                         "flops_per_launch": flops,
                         "evaluations": {k: v for k, v in counts.items() if k != "best"}},
            "e2e": {"value": e2e_val, "unit": "pixels/s", "steps": e2e_steps,
                    "h2d_bytes_per_step": int(obs.numel() * obs.element_size() + w.numel() * 8),
                    "d2h_bytes_per_step": int(npix * 9 * 8 + npix * 8)},
        }
        if not args.no_fp64:
            result["fp64_plain_ga"] = fp64_comparator(api, torch, pb64, obs, w, lo, hi, rank)
        if not args.no_serve:
            result["serving"] = serving(api, torch, pb32, dev, args.serve_seconds, loads=(0.7, 1.2))
        if not args.no_pipeline:
            result["pipeline"] = pipeline_sample(api, torch, dev)
        if not args.no_cpu and world == 1:
            result["cpu_baseline"] = cpu_baseline(spec, obs, w, lo, hi)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def pipeline_sample(api, torch, device, n=512, n_spots=10, thresh=10.0):
    """The Section 2 pipeline (api.invert_map) on a synthetic full disc of an
    n x n grid: classification with the weak-field answer below the
    polarization threshold, selection, the Section 5.3 prefit bounds, the
    seeded polarity-restricted FP32 GA and the L-M polish on the selected
    pixels, all on one stream.  Every on-disc pixel is answered, so pixels/s
    counts all of them."""
    truth, mu, _ = gi.draw_full_disc(n=n, seed=7, n_spots=n_spots)
    npix = len(mu)
    spec = gi.two_line_spec()
    pb = api.Problem.from_spec(spec, "f32")
    tp = torch.tensor(truth, device=device)
    mp = torch.tensor(mu, device=device)
    clean = api.me_synth(pb, tp, mp)
    g = torch.Generator(device=device).manual_seed(17)
    sig = 1e-3 * (tp[:, 7] + mp * tp[:, 8])
    obs = (clean + sig.to(clean.dtype)[:, None, None] * torch.randn(clean.shape, generator=g, device=device,
                                                                   dtype=clean.dtype)).contiguous()
    w = (1.0 / sig)[:, None].repeat(1, 4).contiguous()
    lo = gi.PRIOR_LO.copy()
    lo[7] = lo[8] = 0.05
    ga = api.GaSettings(npop=NPOP, ngen=NGEN, seed=3)
    kw = dict(nseed=4, prefit=True, polish_iters=LM_ITERS, polish_w=w, mu_px=mp)
    api.invert_map(pb, obs[:4096].contiguous(), lo, gi.PRIOR_HI, ga, thresh, (0, 8), 1, (80, 110),
                   **dict(kw, polish_w=w[:4096].contiguous(), mu_px=mp[:4096].contiguous()))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = api.invert_map(pb, obs, lo, gi.PRIOR_HI, ga, thresh, (0, 8), 1, (80, 110), **kw)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    flagged = int(r["count"].item())
    chi2 = r["chi2"][r["flag"] == 1]
    return {"grid": f"{n}x{n} disc", "pixels": npix, "flagged": flagged, "p_thresh": thresh, "ms": ms,
            "pixels_per_s": npix / (ms / 1e3), "median_chi2_flagged": float(chi2.median().item()) if flagged else None,
            "steps": "classify, select, prefit (40 L-M, Stokes I), bounds, seeded GA, 10 L-M"}


def _request_obs(api, torch, pb, rq, device):
    """Observed cube of one request: GPU synthesis of its truth + seeded noise (host float32)."""
    tp = torch.tensor(rq.truth, device=device)
    clean = api.me_synth(pb, tp)
    g = torch.Generator(device=device).manual_seed(rq.seed)
    noise = torch.randn(clean.shape, generator=g, device=device, dtype=clean.dtype)
    sig = 1e-3 * (tp[:, 7] + tp[:, 8])
    obs = clean + sig.to(clean.dtype)[:, None, None] * noise
    w = (1.0 / sig)[:, None].repeat(1, 4)
    return obs.cpu().numpy(), w.cpu().numpy()


def serving(api, torch, pb, device, seconds, loads=(0.7,), polish=LM_ITERS):
    """Poisson-arriving requests of 64-4096 pixels with mixed GA budgets
    (population 64/128, 100/200/300 generations), served by the continuous-
    batching loop; p50/p99 latency (submit -> results on the host) and pixels/s
    at each load (a fraction of the capacity measured on a burst)."""
    import threading
    pool = gi.draw_requests(600, rate_hz=1.0, seed=4)
    cache = {}

    def obs_of(i):
        if i not in cache:
            cache[i] = _request_obs(api, torch, pb, pool[i], device)
        return cache[i]

    lo, hi = gi.PRIOR_LO, gi.PRIOR_HI

    def submit(srv, i, pid0):
        rq = pool[i]
        o, w = obs_of(i)
        return srv.submit(o, lo, hi, api.GaSettings(npop=rq.npop, ngen=rq.ngen, seed=rq.seed),
                          pixel_id0=pid0, polish_iters=polish, polish_w=w)

    out = {"polish_iters": polish}
    # every request on a stream of equal priority (small_pixels = 0): the fair
    # share that keeps the large requests' tail shortest on this mix
    with api.Server(pb, arena_bytes=2 << 30, max_inflight=16, max_queue=100000, small_pixels=0) as srv:
        # capacity: a burst of 24 requests submitted at once
        nb = 24
        for i in range(nb):
            obs_of(i)
        t0 = time.perf_counter()
        ts = [submit(srv, i, i << 20) for i in range(nb)]
        pix = 0
        for t, i in zip(ts, range(nb)):
            srv.poll(t)
            pix += pool[i].npix
        dt = time.perf_counter() - t0
        cap_rps = nb / dt
        out["capacity"] = {"requests_per_s": cap_rps, "pixels_per_s": pix / dt, "burst_requests": nb}
        nxt = nb
        for load in loads:
            rate = load * cap_rps
            rng = np.random.default_rng(int(load * 1000))
            n = max(8, int(rate * seconds))
            idx = list(range(nxt, min(nxt + n, len(pool))))
            nxt = idx[-1] + 1 if idx else nxt
            for i in idx:
                obs_of(i)
            gaps = rng.exponential(1.0 / rate, len(idx))
            tickets, lat, qs = [], [], []

            def poller():
                k = 0
                while k < len(idx):
                    while k >= len(tickets):
                        time.sleep(0.0005)
                    r = srv.poll(tickets[k])
                    lat.append(r["latency_ns"] / 1e6)
                    qs.append(r["queue_ns"] / 1e6)
                    k += 1

            th = threading.Thread(target=poller)
            th.start()
            t0 = time.perf_counter()
            at = 0.0
            for g_, i in zip(gaps, idx):
                at += g_
                while time.perf_counter() - t0 < at:
                    time.sleep(0.0002)
                tickets.append(submit(srv, i, i << 20))
            th.join()
            wall = time.perf_counter() - t0
            pix = sum(pool[i].npix for i in idx)
            out[f"load_{load}"] = {"offered_rps": rate, "requests": len(idx), "pixels_per_s": pix / wall,
                                   "p50_ms": float(np.percentile(lat, 50)),
                                   "p99_ms": float(np.percentile(lat, 99)),
                                   "queue_p50_ms": float(np.percentile(qs, 50)), "seconds": wall}
    return out


def recovery_stats(torch, p, chi2, truth):
    """Recovered parameters against the seeded truth: per parameter the median
    and 90th percentile of |p - truth| (azimuth modulo 180 degrees), over all
    pixels and over the well-determined ones (B > 300 G, 15 < theta < 165)."""
    t = torch.tensor(truth, device=p.device)
    d = (p - t).abs()
    d[:, 2] = torch.minimum(d[:, 2] % 180.0, 180.0 - d[:, 2] % 180.0)
    good = (t[:, 0] > 300.0) & (t[:, 1] > 15.0) & (t[:, 1] < 165.0)
    names = ["B", "theta", "chi", "v", "dlD", "a", "eta0", "S0", "S1"]

    def pct(x, q):
        return {n: float(v) for n, v in zip(names, torch.quantile(x, q, dim=0).tolist())}

    return {"median_abs_err": pct(d, 0.5), "p90_abs_err": pct(d, 0.9),
            "well_determined": {"pixels": int(good.sum().item()), "median_abs_err": pct(d[good], 0.5),
                                "p90_abs_err": pct(d[good], 0.9)},
            "fraction_chi2_below_1.5": float((chi2 < 1.5).double().mean().item())}


def fp64_comparator(api, torch, pb64, obs32, w, lo, hi, rank, n=16 * 152):
    """Plain FP64 GA (no polish) on the first n pixels of the same map: 2432
    pixels = 8 full waves of the FP64 kernel (2 resident blocks of 128 threads
    per SM at its 236 registers per thread, 152 SMs)."""
    obs = obs32[:n].double().contiguous()
    ga = api.GaSettings(npop=NPOP, ngen=NGEN, seed=rank)
    api.ga_invert_batch(pb64, obs[:64].contiguous(), lo, hi, api.GaSettings(npop=NPOP, ngen=2))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    best, _ = api.ga_invert_batch(pb64, obs, lo, hi, ga, pixel_id0=rank * obs32.shape[0])
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    chi = api.me_chi2(pb64, obs, best, w=w[:n].contiguous())
    return {"value": n / (ms / 1e3), "unit": "pixels/s", "pixels": n, "ms": ms,
            "median_chi2": float(chi.median().item())}


def syntheses_per_pixel(npop, ngen, nsamp=None):
    """GA fitness evaluations per pixel: the initial population, every child
    of every generation, and the restarted worst half at each N_samp-th
    generation before the last (Section 5.6)."""
    nsamp = ngen // 4 if nsamp is None else nsamp
    restarts = sum(1 for t in range(1, ngen) if nsamp > 0 and t % nsamp == 0)
    return npop * (ngen + 1) + restarts * (npop // 2)


def cpu_baseline(spec, obs, w, lo, hi, n=None):
    """The FP64 oracle (GA + L-M) on a bounded pixel sample, all host cores."""
    import oracle
    nth = os.cpu_count() or 1
    n = n or max(8, 2 * nth)
    o = obs[:n].double().cpu().numpy()
    wn = w[:n].cpu().numpy()
    cfg = oracle.ga_config(NPOP, NGEN, seed=0)
    t0 = time.perf_counter()
    r = oracle.ga_invert(spec, o, lo, hi, cfg, nthreads=nth)
    p, c2 = oracle.lm_polish(spec, o, r["best"], lo, hi, iters=LM_ITERS, w=wn, nthreads=nth)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "pixels/s", "cores": nth, "kind": "oracle",
            "sample": f"first {n} pixels of the map, FP64 GA (npop {NPOP}, {NGEN} gen) + {LM_ITERS} L-M",
            "seconds": dt, "median_chi2": float(np.median(c2)),
            "ga_syntheses_per_s": n * syntheses_per_pixel(NPOP, NGEN) / dt}


def run_configs(args):
    """FP64 GA on C1 (all 256 pixels) and on a seeded 256-pixel subset of C2:
    the oracle on all host cores and the GPU on the same inputs (inverse-max
    weights, no polish).  Reports pixels/s, syntheses/s and the fraction of
    pixels whose best parameters are identical on both sides."""
    import torch

    import oracle
    from paper_1208_0302_gb300 import _lib, api
    torch.cuda.set_device(0)
    _lib.load()
    dev = torch.device("cuda", 0)
    nth = os.cpu_count() or 1
    out = {}
    for name in ("c1", "c2"):
        wl = gi.workload(name)
        n = 256
        truth = gi.draw_truth(n, seed=wl.seed + 11)
        sig = 1e-3 * (truth[:, 7] + truth[:, 8])
        obs = oracle.synth(wl.spec, truth) + sig[:, None, None] * gi.draw_noise(n, wl.spec.n_lambda, wl.seed + 11)
        spp = syntheses_per_pixel(wl.npop, wl.ngen)
        t0 = time.perf_counter()
        r = oracle.ga_invert(wl.spec, obs, wl.lo, wl.hi, oracle.ga_config(wl.npop, wl.ngen, seed=0), nthreads=nth)
        dt = time.perf_counter() - t0
        pb = api.Problem.from_spec(wl.spec, "f64")
        ob = torch.tensor(obs, device=dev)
        ga = api.GaSettings(npop=wl.npop, ngen=wl.ngen, seed=0)
        api.ga_invert_batch(pb, ob[:8].contiguous(), wl.lo, wl.hi, api.GaSettings(npop=wl.npop, ngen=2))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        best, chi2 = api.ga_invert_batch(pb, ob, wl.lo, wl.hi, ga)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        same = np.all(best.cpu().numpy() == r["best"], axis=1)
        c_gpu = chi2.cpu().numpy()
        out[name] = {"pixels": n, "npop": wl.npop, "ngen": wl.ngen, "n_lambda": wl.spec.n_lambda,
                     "lines": len(wl.spec.lines), "syntheses_per_pixel": spp,
                     "oracle": {"pixels_per_s": n / dt, "syntheses_per_s": n * spp / dt, "cores": nth,
                                "seconds": dt, "median_chi2": float(np.median(r["chi2"]))},
                     "gpu_fp64": {"pixels_per_s": n / (ms / 1e3), "syntheses_per_s": n * spp / (ms / 1e3),
                                  "ms": ms, "median_chi2": float(np.median(c_gpu)),
                                  "note": "one launch of 256 blocks (under one wave of the GPU)"},
                     "identical_best_fraction": float(same.mean()),
                     "max_rel_chi2_diff": float(np.max(np.abs(c_gpu - r["chi2"]) / r["chi2"]))}
    return {"configs": out, "data": "synthetic (seeded truth from the priors, oracle ME synthesis + 1e-3 Ic noise)"}


def run_disc(args):
    """The full-disc configuration: the synthetic 2048^2 disc (about 3.29 M
    on-disc pixels, mu per pixel, limb-darkened S0/S1, spot clusters over a
    weak-field background, two lines at 128 wavelengths, float32 cube, noise
    1e-3 I_c), inverted in FP32 served mode (GA, population 128, 300
    generations, then 10 L-M iterations with sigma weights) in one launch each,
    against the plain FP64 GA (same budget, no polish) on 8 whole waves of its
    kernel taken from the same disc."""
    import torch

    from paper_1208_0302_gb300 import _lib, api
    torch.cuda.set_device(0)
    _lib.load()
    dev = torch.device("cuda", 0)
    truth, mu, _ = gi.draw_full_disc(n=2048, seed=5, n_spots=40)
    npix = len(mu)
    spec = gi.two_line_spec()
    pb32 = api.Problem.from_spec(spec, "f32")
    pb64 = api.Problem.from_spec(spec, "f64")
    tp = torch.tensor(truth, device=dev)
    mp = torch.tensor(mu, device=dev)
    obs = api.me_synth(pb32, tp, mp)
    g = torch.Generator(device=dev).manual_seed(55)
    sig = 1e-3 * (tp[:, 7] + mp * tp[:, 8])
    obs.add_(sig.to(obs.dtype)[:, None, None] * torch.randn(obs.shape, generator=g, device=dev, dtype=obs.dtype))
    w = (1.0 / sig)[:, None].repeat(1, 4).contiguous()
    lo = gi.PRIOR_LO.copy()
    lo[7] = lo[8] = 0.05
    hi = gi.PRIOR_HI
    ga = api.GaSettings(npop=NPOP, ngen=300, seed=5)
    api.ga_invert_batch(pb32, obs[:4096].contiguous(), lo, hi, api.GaSettings(npop=NPOP, ngen=4), mu_px=mp[:4096].contiguous())
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    best, _ = api.ga_invert_batch(pb32, obs, lo, hi, ga, mu_px=mp)
    ev[1].record()
    p, c2 = api.lm_polish(pb32, obs, best, lo, hi, iters=LM_ITERS, w=w, mu_px=mp)
    ev[2].record()
    torch.cuda.synchronize()
    ga_ms, lm_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    n64 = 16 * 152
    idx = torch.tensor(np.random.default_rng(9).choice(npix, n64, replace=False), device=dev)
    o64 = obs[idx].double().contiguous()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b64, _ = api.ga_invert_batch(pb64, o64, lo, hi, ga, mu_px=mp[idx].contiguous(), pixel_id0=0)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    c64 = api.me_chi2(pb64, o64, b64, w=w[idx].contiguous(), mu_px=mp[idx].contiguous())
    ms = ga_ms + lm_ms
    return {"metric": "pixels inverted/s, full disc", "value": npix / (ms / 1e3), "unit": "pixels/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic full disc (seeded)",
            "config": {"workload": "2048x2048 disc, 3.29M on-disc px, two lines, 128 lambda, float32 cube, npop 128, "
                                   "300 gen + 10 L-M", "pixels": npix},
            "ga_ms": ga_ms, "lm_ms": lm_ms, "median_chi2": float(c2.median().item()),
            "p90_chi2": float(torch.quantile(c2, 0.9).item()),
            "median_chi2_on_fp64_sample": float(c2[idx].median().item()),
            "fp64_plain_ga": {"value": n64 / (ms64 / 1e3), "unit": "pixels/s", "pixels": n64, "ms": ms64,
                              "median_chi2": float(c64.median().item())}}


def run_pattern(args):
    """The paper's heavier case (Table 5): Fe I 6301.5 as its full Zeeman
    pattern (5P2 - 5D2, four components per sigma_b, pi, sigma_r group) with
    6302.5 as its normal triplet, on a 256x256 two-line map (128 wavelengths,
    float32 cube, noise 1e-3 I_c): FP32 GA (population 128, 200 generations)
    + 10 L-M iterations, beside the same map with 6301.5 as its effective
    triplet, and the plain FP64 GA (same budget, no polish) on 8 whole waves
    of the full-pattern map."""
    import torch

    from paper_1208_0302_gb300 import _lib, api
    torch.cuda.set_device(0)
    _lib.load()
    dev = torch.device("cuda", 0)
    side = 256
    npix = side * side
    lo, hi = gi.PRIOR_LO, gi.PRIOR_HI
    ga = api.GaSettings(npop=NPOP, ngen=NGEN, seed=0)
    out = {}
    for key, spec in (("full_pattern", gi.two_line_pattern_spec()), ("effective_triplet", gi.two_line_spec())):
        pb32 = api.Problem.from_spec(spec, "f32")
        truth, obs, w = make_map(api, torch, pb32, side, 0, dev)
        api.ga_invert_batch(pb32, obs[:4096].contiguous(), lo, hi, api.GaSettings(npop=NPOP, ngen=4))
        torch.cuda.synchronize()
        ga_ms, lm_ms = [], []
        for _ in range(2):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            best, _ = api.ga_invert_batch(pb32, obs, lo, hi, ga)
            ev[1].record()
            p, c2 = api.lm_polish(pb32, obs, best, lo, hi, iters=LM_ITERS, w=w)
            ev[2].record()
            torch.cuda.synchronize()
            ga_ms.append(ev[0].elapsed_time(ev[1]))
            lm_ms.append(ev[1].elapsed_time(ev[2]))
        counts = api.ga_count_evaluations(pb32, obs, lo, hi, ga)
        wz = counts["weideman"] + counts["mid"] + counts["cf"] + counts["even2"] + counts["far"]
        g_ms, l_ms = min(ga_ms), min(lm_ms)
        out[key] = {"pixels_per_s": npix / ((g_ms + l_ms) / 1e3), "ga_ms": g_ms, "lm_ms": l_ms,
                    "median_chi2": float(c2.median().item()),
                    "syntheses_per_s": counts["syntheses"] / (g_ms / 1e3), "wz_evals_per_s": wz / (g_ms / 1e3),
                    "wz_evals_per_point": wz / counts["points"]}
        if key == "full_pattern":
            pb64 = api.Problem.from_spec(spec, "f64")
            n64 = 16 * 152
            o64 = obs[:n64].double().contiguous()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b64, _ = api.ga_invert_batch(pb64, o64, lo, hi, ga)
            e1.record()
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1)
            c64 = api.me_chi2(pb64, o64, b64, w=w[:n64].contiguous())
            out["fp64_plain_ga"] = {"value": n64 / (ms64 / 1e3), "unit": "pixels/s", "pixels": n64, "ms": ms64,
                                    "median_chi2": float(c64.median().item()),
                                    "served_form_median_chi2_same_pixels": float(c2[:n64].median().item())}
    fp = out["full_pattern"]
    return {"metric": "pixels inverted/s, full Zeeman pattern", "value": fp["pixels_per_s"], "unit": "pixels/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded truth from the priors)",
            "config": {"workload": "two-line map, Fe I 6301.5 full Zeeman pattern (4 components per group) + 6302.5 "
                                   "normal triplet, 256x256 px, 128 lambda, float32 cube, npop 128, 200 gen + 10 L-M",
                       "pixels": npix},
            **out}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    spec = gi.two_line_spec()
    nth = os.cpu_count() or 1
    n = max(4, nth)
    truth = gi.draw_truth(n, seed=0)
    clean = oracle.synth(spec, truth)
    obs = clean + 1e-3 * (truth[:, 7] + truth[:, 8])[:, None, None] * gi.draw_noise(n, spec.n_lambda, 0)
    sig = 1e-3 * (truth[:, 7] + truth[:, 8])
    w = np.repeat((1 / sig)[:, None], 4, 1)
    cfg = oracle.ga_config(NPOP, NGEN, seed=0)

    def one():
        r = oracle.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, nthreads=nth)
        return oracle.lm_polish(spec, obs, r["best"], gi.PRIOR_LO, gi.PRIOR_HI, iters=LM_ITERS, w=w,
                                nthreads=nth)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p, c2 = one()
    dt = (time.perf_counter() - t0) / args.steps
    val = n / dt
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "pixels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload(args.side) + " (oracle on a pixel sample)"},
            "cpu_baseline": {"value": val, "unit": "pixels/s", "cores": nth, "kind": "oracle",
                             "sample": f"{n} pixels per step"},
            "e2e": {"value": val, "unit": "pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "median_chi2": float(np.median(c2))}


def run_serve(args):
    import torch

    from paper_1208_0302_gb300 import _lib, api
    torch.cuda.set_device(0)
    _lib.load()
    pb = api.Problem.from_spec(gi.two_line_spec(), "f32")
    res = serving(api, torch, pb, torch.device("cuda", 0), args.serve_seconds, loads=(0.7, 1.2))
    return {"metric": "serving latency (Poisson arrivals, 64-4096 px requests)", "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "two-line 128-lambda requests, 30% magnetised, npop 64/128, "
                                   "ngen 100/200/300, FP32 GA + 10 L-M"}, **res}


def main():
    args = parse()
    if args.serve:
        res = run_serve(args)
    elif args.configs:
        res = run_configs(args)
    elif args.disc:
        res = run_disc(args)
    elif args.pattern:
        res = run_pattern(args)
    else:
        res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
