"""bench.py's headline line stays short: the learned-prior and serving legs enter it only as
compact summaries, and the full legs are printed on earlier lines (host logic, no GPU)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def fake_learned():
    pairs = [{"bp_iters": k, "bp_lsd_shots_per_s": 2.0e8 - k * 1e6, "bp_lsd_p99_ms": 4.6 + k * 0.01,
              "ler_bp": 0.05 + k * 1e-4, "ler_learned": 0.054} for k in (12, 14, 16)]
    return {"rounds": 4, "hidden": 32, "weights": "bf16", "inference_kernel": {"kernel": "tcgen05", "grid": 152},
            "train_pairs": 9998336, "train_s": 4.5061234, "train_pairs_per_s": 2.2e6,
            "final_loss": 0.1234567, "value": 19545000.123, "unit": "shots/s", "ms_per_step": 51.2,
            "latency_ms": {"p50": 51.1234, "p99": 51.4321}, "ler": 0.0540781234,
            "ler_sigma": 0.000226171234, "prior_hard_decision_frac": 0.8, "lsd_frac": 0.2,
            "kernel_ms": {"prior_and_check": 47.328128814697266, "lsd_kernel": 3.778048038482666},
            "bp_sweep": [{"bp_iters": k, "shots_per_s": 2e8, "ler": 0.05} for k in range(3, 51)],
            "equal_ler_pairs": pairs,
            "fastest_bp_lsd_at_no_worse_ler": {"bp_iters": 10, "bp_lsd_shots_per_s": 2.18e8,
                                               "bp_lsd_p99_ms": 4.58, "ler": 0.0489},
            "rounds_sweep": [{"rounds": r, "value": 2e7} for r in (2, 4)]}


def fake_serving():
    loads = [{"offered_rate": r, "generated": int(r / 2), "completed": int(r / 2), "shots_per_s": r * 0.99,
              "p50_us": 110.123, "p99_us": 300.456, "max_us": 1500.0, "mean_batch": 19.3,
              "admission_waits": 0, "per_code_p50_p99_us": [[89.0, 164.0]] * 3,
              "p99_parts_us": {"p99_lag_us": 7.0, "p99_queue_us": 123.0, "p99_service_us": 247.0}}
             for r in (1e4, 1e5, 1e6, 1e7)]
    windows = [{"offered_rounds_per_s": r, "with_shots": m, "blocks": 5e5, "window_jobs": 4e5,
                "rounds_per_s": r * 0.85, "p50_us": 90.1, "p99_us": 232.3, "max_us": 1000.0,
                "p99_parts_us": {}, "mean_batch": 30.0, "refused_blocks": 0}
               for r in (1e4, 1e5, 1e6) for m in (False, True)]
    return {"loads": loads, "batch_reference": {"ms_per_65536_shots": [0.8, 3.2, 9.1],
                                                "mix_shots_per_s": 15093524.5},
            "windows": {"loads": windows}}


def test_summaries_are_compact_and_complete():
    ls = bench._sig(bench.learned_summary(fake_learned()))
    ss = bench._sig(bench.serving_summary(fake_serving()))
    for key in ("value", "p99_ms", "ler", "ler_sigma", "equal_ler_bp_lsd", "fastest_bp_lsd_no_worse_ler"):
        assert key in ls, key
    assert ls["equal_ler_bp_lsd"]["bp_iters"] == 12  # the fastest pair within 2 sigma
    assert len(ss["shots"]) == 4 and len(ss["window_rounds"]) == 6
    assert len(json.dumps(ls)) < 700 and len(json.dumps(ss)) < 700


def test_headline_line_fits_the_parsed_tail():
    """A line with every headline key at full precision and the two summaries stays well under
    3 KB (the last line of stdout is the one a reader parses)."""
    line = {
        "metric": bench.METRIC, "value": 158497492.81488544, "unit": bench.UNIT, "n_gpus": 1,
        "steps": 5, "warmup": 3, "ms_per_step": 6.31, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "x" * 160, "shots_per_step": 1000000, "l2": "flushed between steps (256 MiB write)"},
        "latency_ms": {"p50": 6.310624122619629, "p99": 6.36118673324585}, "ler": 0.061829,
        "bp_converged_frac": 0.860859, "lsd_frac": 0.139141, "mean_bp_iters": 10.803732,
        "kernel_ms": {"bp": 3.8591615676879885, "lsd": 2.4357183933258058},
        "roofline": bench._sig({"bound": "alu", "kernel": "bp_reg_kernel<32,3,6,5,3>", "achieved": 12.094,
                                "peak": 40.274, "unit": "Tops/s", "frac": 0.30029, "traffic": 228198400,
                                "peak_source": "152 SMs x 128 lanes x 2070 MHz (max SM clock)",
                                "ops_per_unit": "10 x 432 edges x 10803732 shot-iterations"}),
        "e2e": bench._sig({"value": 152370000.0, "unit": "shots/s", "call": "lsd_decode_batch_host_packed",
                           "h2d_bytes_per_step": 12000000, "d2h_bytes_per_step": 21000000,
                           "bytes_call": {"value": 148700000.0, "h2d_bytes_per_step": 72000000,
                                          "d2h_bytes_per_step": 145000000}}),
        "gpu_launches": 10,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 2},
        "learned": bench._sig(bench.learned_summary(fake_learned())),
        "serving": bench._sig(bench.serving_summary(fake_serving())),
        "cpu_baseline": {"value": 329421.8503162569, "unit": "shots/s", "cores": 16, "kind": "oracle",
                         "sample": "first 1000000 shots of the step, 3.0 s, 16 threads"},
    }
    assert len(json.dumps(line)) < 3000
