#!/usr/bin/env python
"""Throughput benchmark of the GB300 BP + LSD decoder.

Workload (one step = one batch): the [[144,12,12]] bivariate bicycle code, H_X (72 x 144),
i.i.d. bit flips with p = 0.05, 10^6 seeded synthetic shots resident in HBM, min-sum BP
(alpha = 0.625, at most 50 iterations, per-shot early exit) then LSD-0 on every shot BP
does not solve.  L2 is flushed (256 MiB write) between timed steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

With N > 1 (torchrun), every rank decodes its own 10^6 shots (weak scaling; shots are
independent, so there is no collective on the data path) and the step time is the max
over ranks.  ``--impl reference`` times the CPU oracle (the only reference this project
has) on the host cores, on a bounded sample of the same workload.

Rank 0 prints one JSON line per measured leg (learned prior, p sweep, LSD-mu, windows,
giant shot, hook faults, HGP, serving, cluster histograms), then, as the LAST line of stdout,
one compact headline line (about 2 KB) with the metric, the value, the roofline, the CPU
baseline, the end-to-end figure and a summary of the learned prior at equal LER.
``--legs-out PATH`` also writes every leg to one JSON file.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "shots/s + p99 latency: BB[[144,12,12]] BP+LSD vs learned+LSD at equal LER"
UNIT = "shots/s"
# Algorithmic work of min-sum BP per edge per executed iteration: abs, two-minimum
# tracking, sign parity, select, scaling multiply, sign apply, the variable-side add
# and subtract, and the hard-decision parity (about ten integer / FP32 operations).
OPS_PER_EDGE_ITER = 10
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one 10^6-shot BP launch on this workload (BB144, p = 0.05,
# 50 iterations), per kernel variant, from a one-pass ncu capture of the full workload;
# a variant without a capture reports traffic null.
BP_TRAFFIC_BYTES = {"bp_reg_kernel<32,3,6,5,3>": 75725312 + 152473088}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--shots", type=int, default=1_000_000)
    ap.add_argument("--p", type=float, default=0.05)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--order", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--bp-kernel", type=int, default=0, help="0 auto, 1 generic, 2 register")
    ap.add_argument("--lsd-warps", type=int, default=0)
    ap.add_argument("--seed", type=int, default=20240601)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--train-pairs", type=int, default=10_000_000)
    ap.add_argument("--learned-rounds", type=int, default=4)
    ap.add_argument("--sweep-iters", default="3,5,8,10,12,14,16,20,30,50",
                    help="BP iteration counts of the equal-LER sweep")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-sweeps", action="store_true",
                    help="skip the p sweep (BB144, LSD-0/6) and the HGP legs")
    ap.add_argument("--hgp-shots", type=int, default=100_000)
    ap.add_argument("--window-shots", type=int, default=200_000)
    ap.add_argument("--serving-loads", default="1e4,1e5,1e6,1e7",
                    help="offered loads (shots/s) of the serving leg")
    ap.add_argument("--serving-seconds", type=float, default=0.5)
    ap.add_argument("--serving-slots", type=int, default=2,
                    help="in-flight batches per code (per window matrix) in the server")
    ap.add_argument("--legs-out", default=None, help="also write every leg to this JSON file")
    return ap.parse_args()


def workload(args):
    from paper_2406_18655_gb300 import inputs as I
    hx, hz = I.bb144()
    return hx, hz


def config(args, hx):
    return {
        "workload": f"BB[[144,12,12]] H_X {hx.shape[0]}x{hx.shape[1]}, i.i.d. p={args.p}, "
                    f"{args.shots} shots/step, min-sum BP {args.iters} it (alpha 0.625, early exit)"
                    f" + LSD-{args.order}",
        "shots_per_step": args.shots,
        "l2": "flushed between steps (256 MiB write)",
    }


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(args, hx, probs, s, budget_s):
    """The CPU oracle (BP in its FP32 mirror, then LSD) on a bounded sample of the shots."""
    import oracle
    cores = os.cpu_count() or 1
    cal = min(4000, s.shape[0])
    t0 = time.perf_counter()
    oracle.decode(hx, probs, s[:cal], args.iters, lsd_order=args.order, precision=1, nthreads=0)
    dt = time.perf_counter() - t0
    n_s = int(min(s.shape[0], max(cal, cal * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.decode(hx, probs, s[:n_s], args.iters, lsd_order=args.order, precision=1, nthreads=0)
    dt = time.perf_counter() - t0
    return {"value": n_s / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_s} shots of the step, {dt:.1f} s, {cores} threads"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2406_18655_gb300 import inputs as I
    import oracle
    hx, _ = workload(args)
    probs = np.full(hx.shape[1], args.p, np.float32).astype(np.float64)
    # each step: a bounded sample of the workload, sized so K + W steps stay within minutes
    sample = min(args.shots, 20000)
    e = I.sample_errors(args.seed, sample, probs)
    s = I.syndromes(hx, e)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.decode(hx, probs, s, args.iters, lsd_order=args.order, precision=1, nthreads=0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.decode(hx, probs, s, args.iters, lsd_order=args.order, precision=1, nthreads=0)
        times.append(time.perf_counter() - t0)
    value = sample / float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config(args, hx),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} shots of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_steps(fn, steps, stream, flush, barrier):
    """Device time (ms) of each call of fn, with an L2 flush before each."""
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    out = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        barrier()
        start.record(stream)
        fn()
        end.record(stream)
        end.synchronize()
        out.append(start.elapsed_time(end))
    return out


def learned_leg(args, hx, hz, probs, s_dev, e_dev, stream, flush, barrier, checker):
    """Train the learned prior on device-sampled pairs, time learned+LSD on the step's shots,
    and sweep BP iterations for the BP+LSD operating points at equal logical error rate."""
    import torch
    from paper_2406_18655_gb300.learned import init_params, train
    from paper_2406_18655_gb300.lsd import Decoder, Prior

    dec = Decoder(hx, probs, args.iters, args.order, stream=stream)
    if not args.no_autotune:
        dec.autotune(s_dev[: min(s_dev.shape[0], 200_000)])  # LSD warps of the learned path
    prior = Prior(dec, rounds=args.learned_rounds, params=init_params(args.seed))
    prior_kernel = prior.kernel()
    tr = train(dec, prior, args.train_pairs, batch=4096, seed=args.seed + 17, lr=3e-3,
               log_every=500)
    for _ in range(max(args.warmup, 1)):
        c, st = dec.decode_learned(prior, s_dev)
    holder = {}

    def run():
        holder["c"], holder["st"], holder["stats"] = dec.decode_learned(prior, s_dev,
                                                                        want_stats=True)

    ms = timed_steps(run, args.steps, stream, flush, barrier)
    n_shots = s_dev.shape[0]
    ler = float(checker.failures(e_dev, holder["c"]).float().mean().item())
    sigma = float(np.sqrt(max(ler * (1 - ler), 1.0 / n_shots) / n_shots))
    learned = {"rounds": args.learned_rounds, "hidden": 32, "weights": "bf16 (fp32 master)",
               "inference_kernel": prior_kernel,
               "train_pairs": tr["pairs"], "train_s": tr["seconds"],
               "train_pairs_per_s": tr["pairs_per_s"],
               "final_loss": tr["losses"][-1][1] if tr["losses"] else None,
               "value": n_shots / (float(np.mean(ms)) / 1000.0), "unit": UNIT,
               "ms_per_step": float(np.mean(ms)),
               "latency_ms": {"p50": float(np.percentile(ms, 50)),
                              "p99": float(np.percentile(ms, 99))},
               "ler": ler, "ler_sigma": sigma,
               "prior_hard_decision_frac": holder["stats"]["bp_converged"] / n_shots,
               "lsd_frac": holder["stats"]["lsd_shots"] / n_shots,
               "kernel_ms": {"prior_and_check": holder["stats"]["ms_bp"],
                             "lsd_kernel": holder["stats"]["ms_lsd"]}}
    # equal-LER protocol: BP+LSD at several iteration counts
    sweep = []
    for it in [int(x) for x in args.sweep_iters.split(",") if x]:
        d_it = Decoder(hx, probs, it, args.order, stream=stream)
        if not args.no_autotune:
            d_it.autotune(s_dev[: min(s_dev.shape[0], 200_000)])
        corr = torch.empty_like(holder["c"])
        stt = torch.empty_like(holder["st"])
        for _ in range(2):
            d_it.decode(s_dev, corr, stt)
        ms_it = timed_steps(lambda: d_it.decode(s_dev, corr, stt), max(2, args.steps // 2),
                            stream, flush, barrier)
        ler_it = float(checker.failures(e_dev, corr).float().mean().item())
        sig_it = float(np.sqrt(max(ler_it * (1 - ler_it), 1.0 / n_shots) / n_shots))
        sweep.append({"bp_iters": it, "ler": ler_it, "ler_sigma": sig_it,
                      "value": n_shots / (float(np.mean(ms_it)) / 1000.0),
                      "p99_ms": float(np.percentile(ms_it, 99)),
                      "equal_ler": bool(abs(ler_it - ler) <= 2 * np.hypot(sigma, sig_it))})
        d_it.close()
    learned["bp_sweep"] = sweep
    matched = [x for x in sweep if x["equal_ler"]]
    learned["equal_ler_pairs"] = [
        {"bp_iters": x["bp_iters"], "bp_lsd_shots_per_s": x["value"],
         "learned_lsd_shots_per_s": learned["value"], "bp_lsd_p99_ms": x["p99_ms"],
         "learned_lsd_p99_ms": learned["latency_ms"]["p99"], "ler_bp": x["ler"],
         "ler_learned": ler} for x in matched]
    # the fastest BP+LSD operating point whose LER is no worse than the learned one's
    # (within 2 sigma), against learned+LSD
    no_worse = [x for x in sweep if x["ler"] <= ler + 2 * np.hypot(sigma, x["ler_sigma"])]
    if no_worse:
        best = max(no_worse, key=lambda x: x["value"])
        learned["fastest_bp_lsd_at_no_worse_ler"] = {
            "bp_iters": best["bp_iters"], "ler": best["ler"],
            "bp_lsd_shots_per_s": best["value"], "bp_lsd_p99_ms": best["p99_ms"],
            "learned_lsd_shots_per_s": learned["value"],
            "learned_lsd_p99_ms": learned["latency_ms"]["p99"], "ler_learned": ler,
            "speed_ratio_learned_over_bp": learned["value"] / best["value"]}
    prior.close()
    # the equal-LER protocol's second network depth: fewer message-passing rounds
    learned["rounds_sweep"] = []
    for rounds in (2,):
        if rounds == args.learned_rounds:
            continue
        pr = Prior(dec, rounds=rounds, params=init_params(args.seed))
        tr2 = train(dec, pr, args.train_pairs, batch=4096, seed=args.seed + 17, lr=3e-3)
        for _ in range(max(args.warmup, 1)):
            dec.decode_learned(pr, s_dev)
        h2 = {}

        def run2():
            h2["c"], h2["st"] = dec.decode_learned(pr, s_dev)

        ms2 = timed_steps(run2, args.steps, stream, flush, barrier)
        ler2 = float(checker.failures(e_dev, h2["c"]).float().mean().item())
        sig2 = float(np.sqrt(max(ler2 * (1 - ler2), 1.0 / n_shots) / n_shots))
        learned["rounds_sweep"].append({
            "rounds": rounds, "train_pairs": tr2["pairs"], "train_s": tr2["seconds"],
            "value": n_shots / (float(np.mean(ms2)) / 1000.0), "unit": UNIT,
            "p99_ms": float(np.percentile(ms2, 99)), "ler": ler2, "ler_sigma": sig2,
            "equal_ler_bp_iters": [x["bp_iters"] for x in sweep
                                   if abs(x["ler"] - ler2) <= 2 * np.hypot(sig2, x["ler_sigma"])]})
        pr.close()
    dec.close()
    return learned


def cluster_histograms(dec, s_dev, max_shots=200_000):
    """kappa (largest cluster, columns) and nu (clusters) per LSD shot of the workload, from a
    BP-only pass and LSD on its unconverged shots (outside the timed region)."""
    import torch
    s = s_dev[:max_shots]
    post, conv, _ = dec.bp(s)
    idx = torch.nonzero(conv == 0).flatten()
    if idx.numel() == 0:
        return None
    _, _, info = dec.postprocess(post[idx].contiguous(), s[idx].contiguous())
    info = info.cpu().numpy()
    out = {"shots": int(s.shape[0]), "lsd_shots": int(idx.numel())}
    for k, name in ((1, "kappa"), (0, "nu"), (2, "steps")):
        v = info[:, k]
        hist = np.bincount(v)
        out[name] = {"mean": float(v.mean()), "max": int(v.max()),
                     "p99": float(np.percentile(v, 99)),
                     "histogram": {str(i): int(c) for i, c in enumerate(hist) if c}}
    return out


def _timed_decode(dec, s_dev, corr, status, steps, stream, flush, barrier):
    for _ in range(2):
        dec.decode(s_dev, corr, status)
    ms = timed_steps(lambda: dec.decode(s_dev, corr, status), steps, stream, flush, barrier)
    _, _, st = dec.decode(s_dev, corr, status, want_stats=True)
    return ms, st


def p_sweep_leg(args, hx, hz, stream, flush, barrier, checker):
    """BB[[144,12,12]], p in {0.01, ..., 0.10}, 10^6 shots per p, BP 50 + LSD-0 and LSD-6."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.lsd import Decoder
    n = hx.shape[1]
    out = []
    for p in (0.01, 0.02, 0.04, 0.06, 0.08, 0.10):
        probs = np.full(n, p, np.float32)
        e = I.sample_errors(args.seed + int(p * 1000), args.shots, probs.astype(np.float64))
        s_dev = torch.from_numpy(I.syndromes(hx, e)).cuda()
        e_dev = torch.from_numpy(e).cuda()
        corr = torch.empty((args.shots, n), dtype=torch.uint8, device="cuda")
        status = torch.empty(args.shots, dtype=torch.uint8, device="cuda")
        for order in (0, 6):
            dec = Decoder(hx, probs, args.iters, order, stream=stream)
            dec.autotune(s_dev[: min(args.shots, 200_000)])
            ms, st = _timed_decode(dec, s_dev, corr, status, 3, stream, flush, barrier)
            ler = float(checker.failures(e_dev, corr).float().mean().item())
            out.append({"p": p, "lsd_order": order, "shots_per_s": args.shots / (np.mean(ms) / 1e3),
                        "ms_per_step": float(np.mean(ms)), "p99_ms": float(np.percentile(ms, 99)),
                        "ler": ler, "lsd_frac": st["lsd_shots"] / args.shots,
                        "kernel_ms": {"bp": st["ms_bp"], "lsd": st["ms_lsd"]},
                        "kappa_max": st["kappa_max"], "nu_max": st["nu_max"]})
            dec.close()
    return {"code": "BB[[144,12,12]]", "shots_per_p": args.shots, "bp_iters": args.iters,
            "points": out}


def lsd_mu_leg(args, hx, hz, stream, flush, barrier, checker):
    """BB[[144,12,12]] at p = 0.06, 10^6 shots: LSD-mu with mu as a fraction of the n fault
    nodes and OSD-CS-4 local reprocessing (App. D's BB experiment, code-capacity noise)."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.lsd import Decoder
    n = hx.shape[1]
    p = 0.06
    probs = np.full(n, p, np.float32)
    e = I.sample_errors(args.seed + 606, args.shots, probs.astype(np.float64))
    s_dev = torch.from_numpy(I.syndromes(hx, e)).cuda()
    e_dev = torch.from_numpy(e).cuda()
    corr = torch.empty((args.shots, n), dtype=torch.uint8, device="cuda")
    status = torch.empty(args.shots, dtype=torch.uint8, device="cuda")
    out = []
    for frac in (0.0, 0.01, 0.02, 0.05, 0.1, 0.2):
        order = int(round(frac * n))
        dec = Decoder(hx, probs, args.iters, order, osd_cs=4 if order else None, stream=stream)
        ms, st = _timed_decode(dec, s_dev, corr, status, 3, stream, flush, barrier)
        ler = float(checker.failures(e_dev, corr).float().mean().item())
        out.append({"mu_frac": frac, "lsd_order": order, "osd": "CS-4" if order else "-",
                    "shots_per_s": args.shots / (np.mean(ms) / 1e3), "ler": ler,
                    "kernel_ms": {"bp": st["ms_bp"], "lsd": st["ms_lsd"]},
                    "kappa_max": st["kappa_max"], "nu_max": st["nu_max"]})
        dec.close()
    return {"code": "BB[[144,12,12]]", "p": p, "shots": args.shots, "bp_iters": args.iters,
            "points": out}


def window_leg(args, hx, hz, stream, flush, barrier, checker):
    """BB[[144,12,12]] over d = 12 noisy syndrome rounds plus a noiseless one, phenomenological
    noise p = q: (3,1) overlapping windows (Methods 4.3) against one decode of the whole
    space-time matrix (936 x 2592), BP 30 + LSD-0, the same device-sampled shots."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.lsd import Decoder, WindowDecoder
    m, n = hx.shape
    d, shots = 12, args.window_shots
    out = []
    for p in (0.003, 0.006):
        glob = Decoder(I.space_time(hx, d), I.space_time_probs(n, m, d, p, p).astype(np.float32),
                       30, stream=stream)
        e, s = glob.sample(args.seed + int(p * 1e4), shots)
        win = WindowDecoder(hx, np.full(n, p, np.float32), np.full(m, p, np.float32), d, 3, 1,
                            bp_iters=30, stream=stream)
        corr = torch.empty((shots, d * (n + m)), dtype=torch.uint8, device="cuda")
        status = torch.empty(shots, dtype=torch.uint8, device="cuda")
        zeros = torch.zeros((shots, n), dtype=torch.uint8, device="cuda")
        point = {"p": p, "q": p}
        for kind, dec in (("window_3_1", win), ("global", glob)):
            fn = lambda: dec.decode(s, corr, status)  # noqa: E731
            for _ in range(2):
                fn()
            ms = timed_steps(fn, 3, stream, flush, barrier)
            _, _, st = dec.decode(s, corr, status, want_stats=True)
            resid = ((e ^ corr).view(shots, d, n + m)[:, :, :n].sum(dim=1) % 2).to(torch.uint8)
            fails = checker.failures(resid, zeros)
            point[kind] = {"shots_per_s": shots / (np.mean(ms) / 1e3),
                           "ms_per_step": float(np.mean(ms)), "ler": float(fails.float().mean()),
                           "unsolvable": int((status == 3).sum().item()),
                           "kernel_ms": {"bp": st["ms_bp"], "lsd": st["ms_lsd"]},
                           "window_decodes": st["shots"] // shots,
                           "kappa_max": st["kappa_max"]}
        if p == 0.003:
            point["streaming"] = _stream_latency(win, s, d, m, n, stream)
        out.append(point)
        win.close()
        glob.close()
    return {"code": "BB[[144,12,12]] space-time, d = 12 noisy rounds + 1 noiseless",
            "shots": shots, "bp_iters": 30, "lsd_order": 0, "points": out}


def _stream_latency(win, s, d, m, n, stream):
    """Rounds pushed one at a time to S concurrent streams (lsd_window_stream_push); the
    latency of a push is host time from the call to its results on the host side of the
    stream (synchronize), the real-time figure a control loop would see."""
    import torch
    res = []
    for streams in (1000, 10000, 100000):
        if streams > s.shape[0]:
            continue
        blocks = s[:streams].view(streams, d + 1, m)
        blocks = [blocks[:, b].contiguous() for b in range(d + 1)]
        corr = torch.empty((streams, d * (n + m)), dtype=torch.uint8, device="cuda")
        st = torch.empty(streams, dtype=torch.uint8, device="cuda")
        lat = []
        for rep in range(4):
            win.stream_reset(streams)
            stream.synchronize()
            for b in range(d + 1):
                t0 = time.perf_counter()
                _, count = win.stream_push(blocks[b], corr, st)
                stream.synchronize()
                if rep > 0 and count:
                    lat.append((time.perf_counter() - t0) * 1e6)
        lat = np.array(lat)
        res.append({"streams": streams, "window_pushes": int(lat.size),
                    "p50_us": float(np.percentile(lat, 50)),
                    "p99_us": float(np.percentile(lat, 99)),
                    "stream_rounds_per_s": streams / (np.mean(lat) / 1e6)})
    return res


def giant_leg(args, stream):
    """One giant shot on the whole GPU (grid-parallel BP + P-LSD, Alg. 2): HGP codes of
    seeded (3,4)-regular bases, beyond the batch decoder's 65535-column limit, one shot per
    point, latency of the whole decode; and, on the 3072 x 6400 HGP code, the same shots
    through the batch decoder one at a time (one warp per shot in LSD)."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.lsd import Decoder, GiantDecoder, LsdError
    out = []
    for r0, c0 in ((240, 320), (480, 640)):
        base = I.random_regular_ldpc(r0, c0, 3, 4, seed=2406 + r0)
        m, n, rows, cols = I.hgp_coo(base)
        variants = [(0.01, 0, None), (0.03, 0, None)]
        if r0 == 480:
            variants.append((0.01, 4, 4))  # LSD-4 with OSD-CS-4 on the largest shot
        for p, order, osd_cs in variants:
            gd = GiantDecoder(m, n, rows, cols, np.full(n, p, np.float32), 100, order,
                              osd_cs=osd_cs, stream=stream)
            infos, wall = [], []
            for seed in range(4):
                e = I.sample_errors(args.seed + seed, 1, np.full(n, p))[0]
                s = torch.from_numpy(I.coo_syndrome(m, rows, cols, e)).cuda()
                try:
                    gd.decode(s)  # warm-up on the same shot
                except LsdError as err:  # e.g. a cluster beyond the 8192-detector limit
                    infos.append({"error": str(err)})
                    continue
                stream.synchronize()
                t0 = time.perf_counter()
                corr, info = gd.decode(s)
                wall.append((time.perf_counter() - t0) * 1e3)
                ok = np.array_equal(I.coo_syndrome(m, rows, cols, corr.cpu().numpy()),
                                    s.cpu().numpy())
                info["explains_syndrome"] = bool(ok)
                infos.append(info)
            ok_infos = [i for i in infos if "error" not in i]
            errors = [i["error"] for i in infos if "error" in i]
            infos = ok_infos
            if not infos:
                out.append({"code": f"HGP of ({r0}x{c0}) (3,4)-regular", "p": p,
                            "lsd_order": order, "errors": errors})
                gd.close()
                continue
            out.append({"code": f"HGP of ({r0}x{c0}) (3,4)-regular", "m": m, "n": n, "errors": errors,
                        "edges": int(rows.size), "p": p, "bp_iters": 100, "lsd_order": order,
                        "osd": "-" if not order else ("E" if osd_cs is None else f"CS-{osd_cs}"),
                        "ms_per_shot": float(np.mean(wall)),
                        "ms_bp": float(np.mean([i["ms_bp"] for i in infos])),
                        "ms_lsd": float(np.mean([i["ms_lsd"] for i in infos])),
                        "shots": [{k: i[k] for k in ("status", "bp_iterations", "nu", "kappa",
                                                     "steps", "explains_syndrome")}
                                  for i in infos]})
            gd.close()
    # small code: giant path vs batch path, one shot per call
    h = I.hgp_48x64()[0]
    n = h.shape[1]
    cmp = []
    for p in (0.03, 0.05):
        probs = np.full(n, p, np.float32)
        e = I.sample_errors(args.seed + 99, 16, probs.astype(np.float64))
        s = torch.from_numpy(I.syndromes(h, e)).cuda()
        gd = GiantDecoder.from_dense(h, probs, 100, stream=stream)
        bd = Decoder(h, probs, 100, stream=stream)
        tg, tb = [], []
        for k in range(16):
            for fn, acc in ((lambda: gd.decode(s[k]), tg),
                            (lambda: bd.decode(s[k:k + 1]), tb)):
                fn()
                stream.synchronize()
                t0 = time.perf_counter()
                fn()
                stream.synchronize()
                acc.append((time.perf_counter() - t0) * 1e3)
        cmp.append({"p": p, "giant_ms_p50": float(np.median(tg)),
                    "batch_one_shot_ms_p50": float(np.median(tb))})
        gd.close()
        bd.close()
    return {"points": out, "hgp_3072x6400_one_shot": cmp,
            "note": "latency = host wall time of one synchronous decode (BP up to 100 "
                    "iterations, then P-LSD with one host round trip per growth step)"}


def hooks_leg(args, hx, hz, stream, flush, barrier, checker):
    """BB[[144,12,12]] over d = 6 rounds with mid-round hook faults and seeded non-uniform
    priors (504 x 2160, weight-2/3 hyperedges: the shape of a circuit-level error model),
    BP 50 + LSD-0, 10^5 shots per point."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.lsd import Decoder
    m, n = hx.shape
    d, shots = 6, 100_000
    h, _ = I.space_time_hooks(hx, d, seed=d)
    out = []
    for p in (0.002, 0.004, 0.006):
        probs = I.space_time_hooks_probs(n, m, d, p, seed=d + 1).astype(np.float32)
        dec = Decoder(h, probs, 50, stream=stream)
        e, s = dec.sample(args.seed + int(p * 1e4), shots)
        corr = torch.empty((shots, h.shape[1]), dtype=torch.uint8, device="cuda")
        status = torch.empty(shots, dtype=torch.uint8, device="cuda")
        ms, st = _timed_decode(dec, s, corr, status, 3, stream, flush, barrier)
        r = (e ^ corr).view(shots, d, 2 * n + m)
        resid = ((r[:, :, :n].sum(dim=1) + r[:, :, n + m:].sum(dim=1)) % 2).to(torch.uint8)
        fails = checker.failures(resid, torch.zeros_like(resid))
        out.append({"p": p, "shots_per_s": shots / (np.mean(ms) / 1e3),
                    "ler": float(fails.float().mean()), "lsd_frac": st["lsd_shots"] / shots,
                    "kernel_ms": {"bp": st["ms_bp"], "lsd": st["ms_lsd"]},
                    "kappa_max": st["kappa_max"]})
        dec.close()
    return {"code": "BB[[144,12,12]] space-time with hook faults, d = 6 (504 x 2160)",
            "shots": shots, "bp_iters": 50, "points": out}


def _bp_onchip_roofline(E, n, m, shots, st):
    """BP with its message state on chip (one CTA per HGP shot): algorithmic ops against the
    ALU peak, and the launch's algorithmic DRAM I/O (syndromes in; corrections of converged
    shots and LLR rows of queued ones out) as GB/s."""
    peak, src = alu_peak()
    s_bp = st["ms_bp"] / 1e3
    ops = OPS_PER_EDGE_ITER * E * st["bp_iterations"]
    io = shots * m + st["bp_converged"] * n + st["lsd_shots"] * 4 * n
    # a design that streams the messages reads and writes every FP32 edge message once per
    # iteration (8 B per edge-iteration): the bytes it would move, against the measured HBM
    # copy bandwidth, in this launch's time
    stream_bytes = 8.0 * E * st["bp_iterations"]
    hbm, hbm_src = hbm_peak()
    return {"bound": "alu", "achieved_tops": ops / s_bp / 1e12, "peak_tops": peak,
            "frac": ops / s_bp / 1e12 / peak, "peak_source": src,
            "io_bytes": int(io), "io_gbps": io / s_bp / 1e9,
            "streaming_equivalent": {"bytes": stream_bytes, "gbps": stream_bytes / s_bp / 1e9,
                                     "peak_gbps": hbm, "frac": stream_bytes / s_bp / 1e9 / hbm,
                                     "peak_source": hbm_src,
                                     "note": "on-chip; streaming-equivalent: 8 B per edge-iteration"},
            "note": "state on chip: HBM carries only the I/O, so the HBM fraction is not the bound"}


def hbm_peak():
    """(GB/s, description): the measured HBM copy bandwidth of MEASURED_PEAKS.json, else the
    fallback figure of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def alu_peak():
    """(Tops/s, description): FP32/INT32 lanes x the maximum SM clock of MEASURED_PEAKS.json."""
    import torch
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 lanes x {mhz:.0f} MHz (max SM clock)"


def hgp_leg(args, stream, flush, barrier):
    """Hypergraph product of a seeded (3,4)-regular 48 x 64 matrix: H_X 3072 x 6400, p in
    {0.02, 0.05}, BP 100 + LSD-10 (and LSD-0), 10^5 shots per point."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.evaluate import LogicalChecker
    from paper_2406_18655_gb300.lsd import Decoder
    hx, hz = I.hgp_48x64()
    n = hx.shape[1]
    hx_sum, hx_m = int(hx.sum()), hx.shape[0]
    checker = LogicalChecker(hz)
    out = []
    for p, shots in ((0.02, args.hgp_shots), (0.05, args.hgp_shots)):
        probs = np.full(n, p, np.float32)
        for order in (0, 10):
            dec = Decoder(hx, probs, 100, order, stream=stream)
            e, s_dev = dec.sample(args.seed + int(p * 1000), shots)
            corr = torch.empty((shots, n), dtype=torch.uint8, device="cuda")
            status = torch.empty(shots, dtype=torch.uint8, device="cuda")
            ms, st = _timed_decode(dec, s_dev, corr, status, 2, stream, flush, barrier)
            ler = float(checker.failures(e, corr).float().mean().item())
            out.append({"p": p, "lsd_order": order, "shots": shots,
                        "shots_per_s": shots / (np.mean(ms) / 1e3),
                        "ms_per_step": float(np.mean(ms)), "ler": ler,
                        "bp_converged_frac": st["bp_converged"] / shots,
                        "lsd_frac": st["lsd_shots"] / shots, "lsd_spilled": st["lsd_spilled"],
                        "mean_bp_iters": st["bp_iterations"] / shots,
                        "kernel_ms": {"bp": st["ms_bp"], "lsd": st["ms_lsd"]},
                        "kappa_max": st["kappa_max"], "nu_max": st["nu_max"],
                        "bp_roofline": _bp_onchip_roofline(int(hx_sum), n, hx_m, shots, st)})
            dec.close()
    return {"code": "HGP of a seeded (3,4)-regular 48x64 matrix, H_X 3072x6400, E=21504",
            "bp_iters": 100, "points": out}


def serving_leg(args):
    """Poisson arrivals mixing the space-time matrices of the BB [[72,12,6]], [[144,12,12]]
    and [[288,12,18]] codes (phenomenological noise p = q = 0.003 over d = 6, 12, 18 noisy
    rounds plus one noiseless round), decoded by the continuous-batching server (BP 30
    iterations + LSD-0); p50 / p99 request latency and completed shots/s per offered load.
    Then streams of BB[[144,12,12]] syndrome rounds (d = 12, p = q = 0.003) decoded in (3, 1)
    windows inside the same server: per-round p50 / p99 (a window job's latency from the
    submission of its completing block) at offered loads of stream rounds, alone and mixed
    with the shots.  The reference point is the same three matrices decoded as plain
    batches (65536 shots per code, device-resident)."""
    import torch
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.lsd import Decoder, Server

    codes, pools, batch_ms = [], [], []
    for k, (fn, d) in enumerate(((I.bb72, 6), (I.bb144, 12), (I.bb288, 18))):
        hx = fn()[0]
        h = I.space_time(hx, d)
        probs = I.space_time_probs(hx.shape[1], hx.shape[0], d, 0.003, 0.003).astype(np.float32)
        dec = Decoder(h, probs, 30)
        _, syn = dec.sample(args.seed + 101 + k, 65536)
        for _ in range(2):
            dec.decode(syn)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            dec.decode(syn)
        torch.cuda.synchronize()
        batch_ms.append((time.perf_counter() - t0) / 3 * 1e3)
        pools.append(syn[:8192].cpu().pin_memory())
        dec.close()
        codes.append((h, probs, 30, 0))
    # batch throughput of the equal mix: 3 x 65536 shots in the summed batch times
    mix_batch_rate = 3 * 65536 / (sum(batch_ms) / 1e3)
    hx = I.bb144()[0]
    m, n = hx.shape
    d, streams = 12, 1024
    probs = I.space_time_probs(n, m, d, 0.003, 0.003)
    seqs = torch.from_numpy(I.syndromes(I.space_time(hx, d),
                                        I.sample_errors(args.seed + 131, 4096, probs)))
    wcode = dict(h=hx, p=0.003, q=0.003, rounds=d, window=3, commit=1, bp_iters=30,
                 streams=streams)
    srv = Server(codes, window_codes=[wcode], slots_per_code=args.serving_slots)
    out = []
    for rate in [float(x) for x in args.serving_loads.split(",") if x]:
        rep = srv.run_poisson(rate, args.serving_seconds, [1, 1, 1, 0], pools + [seqs],
                              seed=args.seed + 7)
        pt = {k: rep[k] for k in ("offered_rate", "generated", "completed", "shots_per_s",
                                  "p50_us", "p99_us", "max_us", "mean_batch", "admission_waits")}
        pt["per_code_p50_p99_us"] = [[round(r["p50_us"], 1), round(r["p99_us"], 1)]
                                     for r in (srv.code_report(c) for c in range(3))]
        pt["p99_parts_us"] = {k: round(rep[k], 1) for k in ("p99_lag_us", "p99_queue_us",
                                                             "p99_service_us")}
        out.append(pt)
    windows = []
    for rate in (1e4, 1e5, 1e6):
        for mixed in (False, True):
            # mixed: the same round rate plus shots at a tenth of it
            mix = [rate / 30, rate / 30, rate / 30, rate] if mixed else [0, 0, 0, rate]
            total = sum(mix)
            rep = srv.run_poisson(total, args.serving_seconds, mix, pools + [seqs],
                                  seed=args.seed + 11)
            w = srv.code_report(3)
            windows.append({"offered_rounds_per_s": rate, "with_shots": mixed,
                            "blocks": rep["generated"], "window_jobs": w["completed"],
                            "rounds_per_s": w["completed"] / max(rep["seconds"], 1e-9),
                            "p50_us": w["p50_us"], "p99_us": w["p99_us"], "max_us": w["max_us"],
                            "p99_parts_us": {k: round(w[k], 1) for k in
                                             ("p99_lag_us", "p99_queue_us", "p99_service_us",
                                              "p99_batch_gpu_us", "p99_launch_call_us")},
                            "mean_batch": w["mean_batch"],
                            "refused_blocks": rep["admission_waits"]})
    srv.close()
    return {"codes": ["BB[[72,12,6]] d=6: H 252x648", "BB[[144,12,12]] d=12: H 936x2592",
                      "BB[[288,12,18]] d=18: H 2736x7776"],
            "noise": "phenomenological p = q = 0.003", "bp_iters": 30, "lsd_order": 0,
            "mix": "equal", "seconds_per_load": args.serving_seconds,
            "graphs": "two CUDA graphs per slot (gather, BP, write-back of the rows BP solved; LSD, write-back of the rest); a request completes when its row is written back",
            "slots_per_code": args.serving_slots, "loads": out,
            "batch_reference": {"ms_per_65536_shots": batch_ms,
                                "mix_shots_per_s": mix_batch_rate},
            "windows": {"code": "BB[[144,12,12]] rounds, d = 12, (3,1) windows, 1024 streams",
                        "loads": windows}}


def _sig(x, digits=5):
    """Floats of a nested summary rounded to `digits` significant digits (keeps the headline
    line short)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: _sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_sig(v, digits) for v in x]
    return x


def learned_summary(learned):
    """The learned prior's headline figures and the BP+LSD points it is compared with."""
    if not learned:
        return None
    out = {"rounds": learned["rounds"], "inference_kernel": learned["inference_kernel"]["kernel"],
           "train_pairs": learned["train_pairs"],
           "train_s": round(learned["train_s"], 3), "value": learned["value"],
           "p99_ms": learned["latency_ms"]["p99"], "ler": learned["ler"],
           "ler_sigma": learned["ler_sigma"], "kernel_ms": learned["kernel_ms"]}
    pairs = learned.get("equal_ler_pairs") or []
    if pairs:  # the fastest BP+LSD point whose LER is within 2 sigma of the learned one's
        best = max(pairs, key=lambda x: x["bp_lsd_shots_per_s"])
        out["equal_ler_bp_lsd"] = {"bp_iters": best["bp_iters"], "value": best["bp_lsd_shots_per_s"],
                                   "p99_ms": best["bp_lsd_p99_ms"], "ler": best["ler_bp"]}
    nw = learned.get("fastest_bp_lsd_at_no_worse_ler")
    if nw:
        out["fastest_bp_lsd_no_worse_ler"] = {"bp_iters": nw["bp_iters"],
                                              "value": nw["bp_lsd_shots_per_s"],
                                              "p99_ms": nw["bp_lsd_p99_ms"], "ler": nw["ler"]}
    return out


def serving_summary(serving):
    """Per offered load: completed shots/s and p50 / p99 latency in microseconds; per offered
    round rate of the window streams: p50 / p99 per round, alone and mixed with shots."""
    if not serving:
        return None
    return {"shots": [[x["offered_rate"], round(x["shots_per_s"]), round(x["p50_us"]),
                       round(x["p99_us"])] for x in serving["loads"]],
            "batch_mix_shots_per_s": round(serving["batch_reference"]["mix_shots_per_s"]),
            "window_rounds": [[x["offered_rounds_per_s"], int(x["with_shots"]), round(x["p50_us"]),
                               round(x["p99_us"])] for x in serving["windows"]["loads"]],
            "cols": "offered/s, completed shots/s or with-shots flag, p50 us, p99 us"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2406_18655_gb300 import inputs as I
    from paper_2406_18655_gb300.evaluate import LogicalChecker
    from paper_2406_18655_gb300.lsd import Decoder
    from paper_2406_18655_gb300.shard import job_throughput, max_over_ranks, shard, sum_over_ranks

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    hx, hz = workload(args)
    m, n = hx.shape
    probs = np.full(n, args.p, np.float32)
    first, count = shard(rank, world, args.shots)
    e = I.sample_errors(args.seed, count, probs.astype(np.float64), first_shot=first)
    s = I.syndromes(hx, e)
    stream = torch.cuda.current_stream()
    dec = Decoder(hx, probs, args.iters, args.order, bp_lanes=args.lanes,
                  bp_kernel=args.bp_kernel, lsd_warps=args.lsd_warps, stream=stream)
    s_dev = torch.from_numpy(s).cuda()
    corr = torch.empty((args.shots, n), dtype=torch.uint8, device="cuda")
    status = torch.empty(args.shots, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    tune = None
    if not args.no_autotune:  # the project's autotuner picks the launch variants (not timed)
        tune = dec.autotune(s_dev[: min(args.shots, 200_000)])
    for _ in range(max(args.warmup, 0)):
        dec.decode(s_dev, corr, status)
    barrier()

    step_ms, bp_ms, lsd_ms, iters_sum, conv_sum, lsd_sum = [], [], [], 0, 0, 0
    kappa_max = nu_max = 0
    launches0 = dec.kernel_launches()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            barrier()
            start.record(stream)
            dec.decode(s_dev, corr, status)
            end.record(stream)
            end.synchronize()
            step_ms.append(start.elapsed_time(end))
            st = dec.stats()
            bp_ms.append(st["ms_bp"])
            lsd_ms.append(st["ms_lsd"])
            iters_sum += st["bp_iterations"]
            conv_sum += st["bp_converged"]
            lsd_sum += st["lsd_shots"]
            kappa_max = max(kappa_max, st["kappa_max"])
            nu_max = max(nu_max, st["nu_max"])
    launches = dec.kernel_launches() - launches0
    clusters = cluster_histograms(dec, s_dev) if rank == 0 else None
    job = job_throughput(args.shots, sum(step_ms) / args.steps, device="cuda")
    ms_per_step = job["ms_per_step"]
    value = job["per_s"]

    # logical error rate of the last step's corrections (evaluation, outside the timing)
    checker = LogicalChecker(hz)
    e_dev = torch.from_numpy(e).cuda()
    fails = checker.failures(e_dev, corr)
    # end-of-run reductions over the ranks: failure and shot counts, the largest clusters,
    # the slowest rank's time of every step
    ler = (sum_over_ranks(float(fails.sum().item()), device="cuda")
           / sum_over_ranks(float(args.shots), device="cuda"))
    kappa_max = int(max_over_ranks(kappa_max, device="cuda"))
    nu_max = int(max_over_ranks(nu_max, device="cuda"))
    step_ms = [max_over_ranks(t, device="cuda") for t in step_ms]
    all_shots = sum_over_ranks(float(args.steps * args.shots), device="cuda")
    conv_frac = sum_over_ranks(float(conv_sum), device="cuda") / all_shots
    lsd_frac = sum_over_ranks(float(lsd_sum), device="cuda") / all_shots
    learned = None
    if not args.no_learned:
        learned = learned_leg(args, hx, hz, probs, s_dev, e_dev, stream, flush, barrier,
                              checker)

    # end to end through the host-buffer C-ABI call (H2D + decode + D2H each step)
    e2e = None
    if not args.no_e2e:
        s_pin = torch.from_numpy(s).pin_memory()
        c_pin = torch.empty((args.shots, n), dtype=torch.uint8).pin_memory()
        st_pin = torch.empty(args.shots, dtype=torch.uint8).pin_memory()
        for _ in range(max(args.warmup, 1)):
            dec.decode_host(s_pin, c_pin, st_pin)
        barrier()
        t_e2e = []
        for _ in range(args.steps):
            barrier()
            t0 = time.perf_counter()
            dec.decode_host(s_pin, c_pin, st_pin)
            t_e2e.append(time.perf_counter() - t0)
        job_e2e = job_throughput(args.shots, 1000.0 * sum(t_e2e) / args.steps, device="cuda")
        e2e_bytes = {"value": job_e2e["per_s"], "unit": UNIT, "call": "lsd_decode_batch_host",
                     "h2d_bytes_per_step": int(args.shots * m),
                     "d2h_bytes_per_step": int(args.shots * (n + 1))}
        # the same through the bit-packed host call (syndromes and corrections one bit each)
        from paper_2406_18655_gb300.lsd import pack_bits
        wm, wn = (m + 31) // 32, (n + 31) // 32
        sw_pin = torch.from_numpy(pack_bits(s).view(np.int32)).pin_memory()
        cw_pin = torch.empty((args.shots, wn), dtype=torch.int32).pin_memory()
        for _ in range(max(args.warmup, 1)):
            dec.decode_host_packed(sw_pin, cw_pin, st_pin)
        barrier()
        t_pk = []
        for _ in range(args.steps):
            barrier()
            t0 = time.perf_counter()
            dec.decode_host_packed(sw_pin, cw_pin, st_pin)
            t_pk.append(time.perf_counter() - t0)
        job_pk = job_throughput(args.shots, 1000.0 * sum(t_pk) / args.steps, device="cuda")
        e2e = {"value": job_pk["per_s"], "unit": UNIT, "call": "lsd_decode_batch_host_packed",
               "h2d_bytes_per_step": int(args.shots * 4 * wm),
               "d2h_bytes_per_step": int(args.shots * (4 * wn + 1)),
               "bytes_call": {"value": e2e_bytes["value"],
                              "h2d_bytes_per_step": e2e_bytes["h2d_bytes_per_step"],
                              "d2h_bytes_per_step": e2e_bytes["d2h_bytes_per_step"]}}

    serving = p_sweep = hgp = lsd_mu = windows = giant = hooks = None
    if rank == 0 and not args.no_sweeps:
        p_sweep = p_sweep_leg(args, hx, hz, stream, flush, barrier, checker)
        lsd_mu = lsd_mu_leg(args, hx, hz, stream, flush, barrier, checker)
        windows = window_leg(args, hx, hz, stream, flush, barrier, checker)
        giant = giant_leg(args, stream)
        hooks = hooks_leg(args, hx, hz, stream, flush, barrier, checker)
        hgp = hgp_leg(args, stream, flush, barrier)
    if not args.no_serving and rank == 0:
        serving = serving_leg(args)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    from paper_2406_18655_gb300.lsd import bp_variant_name
    E = int(hx.sum())
    bp_ms_avg = float(np.mean(bp_ms))
    iters_per_step = iters_sum / args.steps
    peak, peak_src = alu_peak()
    achieved = OPS_PER_EDGE_ITER * E * iters_per_step / (bp_ms_avg / 1000.0) / 1e12
    bp_name = bp_variant_name(tune["bp_variant"]) if tune else None
    roofline = {"bound": "alu", "kernel": bp_name or "bp (default variant)",
                "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": BP_TRAFFIC_BYTES.get(bp_name),
                "peak_source": peak_src,
                "ops_per_unit": f"{OPS_PER_EDGE_ITER} x {E} edges x {iters_per_step:.0f} "
                                "shot-iterations"}
    legs = {"lsd_clusters": clusters, "autotune": tune, "learned": learned,
            "p_sweep": p_sweep, "lsd_mu_cs4": lsd_mu, "windows": windows, "giant_shot": giant,
            "circuit_like": hooks, "hgp": hgp, "serving": serving}
    for name, leg in legs.items():
        if leg is not None:
            print(json.dumps({"leg": name, "result": leg}), flush=True)
    if args.legs_out:
        with open(args.legs_out, "w") as f:
            json.dump(legs, f, indent=1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config(args, hx),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "ler": ler, "bp_converged_frac": conv_frac, "lsd_frac": lsd_frac,
        "mean_bp_iters": iters_per_step / args.shots,
        "kernel_ms": {"bp": bp_ms_avg, "lsd": float(np.mean(lsd_ms))},
        "roofline": _sig(roofline),
        "e2e": _sig(e2e),
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "learned": _sig(learned_summary(learned)),
        "serving": _sig(serving_summary(serving)),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, hx, probs.astype(np.float64), s,
                                            args.cpu_seconds)
    sys.stderr.flush()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
