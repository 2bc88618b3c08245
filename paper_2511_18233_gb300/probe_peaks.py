"""Measure the arithmetic-pipe peaks that bound the engine's kernels and write
them as JSON: FP64 and FP32 FMA, FP64 mma.sync, tcgen05 kind::tf32 and
kind::f16 (ris_debug_peak_probe), each the best of several CUDA-event timed
runs, with the SM clocks nvidia-smi reported while they ran.

    python -m paper_2511_18233_gb300.probe_peaks --out profiles/peaks_probe_gb300.json
"""
from __future__ import annotations

import argparse
import json
import subprocess
import sys
import threading
import time


def _clock_sampler(samples, stop):
    q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", "0", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                              "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return
    while not stop.is_set():
        line = p.stdout.readline()
        if not line:
            break
        samples.append([x.strip() for x in line.split(",")])
    p.terminate()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    import torch
    from paper_2511_18233_gb300 import build, ris
    build.build()
    torch.cuda.set_device(0)
    props = torch.cuda.get_device_properties(0)
    res = {}
    for kind in ris.PROBE_KINDS:
        samples, stop = [], threading.Event()
        th = threading.Thread(target=_clock_sampler, args=(samples, stop), daemon=True)
        th.start()
        time.sleep(0.3)
        rate, ms = ris.debug_peak_probe(kind, args.reps)
        stop.set()
        th.join(timeout=5)
        sm = [float(s[0]) for s in samples if s and s[0].replace(".", "").isdigit()]
        res[kind] = {"tflops": round(rate, 3), "best_run_ms": round(ms, 3),
                     "sm_mhz_max_seen": max(sm) if sm else None}
    line = {"gpu": props.name, "sms": props.multi_processor_count,
            "how": "ris_debug_peak_probe: independent FMA chains (8 per thread, 8 blocks of 256 per SM) "
                   "or back-to-back MMAs (mma.sync: 4 accumulators per warp; tcgen05: one CTA per SM, "
                   "M128 N256, operands fixed in shared memory); best of reps after one warm-up; "
                   "an FMA / multiply-add counts 2 flops",
            "command": "python -m paper_2511_18233_gb300.probe_peaks --out " + args.out,
            "rates": res}
    with open(args.out, "w") as f:
        json.dump(line, f, indent=1)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
