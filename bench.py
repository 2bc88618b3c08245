#!/usr/bin/env python
"""Throughput benchmark of the sm_103a TDDFT-ris engine.

One step = one evaluation at one geometry of the C20H22 chain workload
(42 atoms, 512 AOs, nocc 71, 102 J / 42 K auxiliary functions): screened
three-centre integrals and metric Cholesky, B tensors, Davidson for the 10
lowest TDA-ris states, gradients of all 10 states and the 9 couplings
between adjacent states.  Metric: evaluations per second.

* value: the mixed-precision form (the throughput form; the FP64 form is
  timed the same way and reported beside it under "fp64"); device-resident
  inputs (coordinates, MO coefficients, orbital energies as CUDA tensors),
  outputs into CUDA tensors, each step timed with CUDA events on the
  library's stream; L2 flushed (512 MB write) between steps, outside the
  timed events.
* e2e: the same evaluation through host (numpy) buffers, host<->device copies
  inside the timed region, wall clock.
* roofline: the kernel class with the largest share of the timed region
  (per-class CUDA events inside the library).
* cpu_baseline / --impl reference: the FP64 oracle on the host cores on a
  bounded sample of the same workload (setup, Davidson, the derivative of
  two pair energies w.r.t. one atom), extrapolated to the full evaluation.

Multi-GPU: replicas only (each rank evaluates its own copy; no collective
in the data path); value = evaluations of all ranks / max time over ranks.
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
sys.path.insert(0, ROOT)

METRIC = "ris grad+NAC evals/s"
CONFIG = {"workload": None, "precision": "mixed", "l2": "flushed (512 MB write) between steps",
          "parallelism": "replicas"}
WORKLOAD = "C20H22 chain, 42 atoms, nao 512, TDA-ris 10 states, 10 gradients + 9 adjacent NACs"
NSTATES = 10


def replica_throughput(seconds: float, steps: int, world: int, dist=None, device="cpu") -> float:
    """Whole-job evaluations/s of `world` replicas that each ran `steps`
    evaluations: world * steps / the slowest rank's time (an all-reduce MAX
    over the process group when there is one; every rank gets the value)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
        dist.barrier()
    return world * steps / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(s[0]) for s in self.samples])
        util = np.array([num(s[3]) for s in self.samples])
        load = sm[util > 0] if np.any(util > 0) else sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for k, n in enumerate(names) if any(s[4 + k].lower() == "active" for s in self.samples)]
        return {"sm_mhz": float(np.nanmedian(load)), "sm_max_mhz": float(np.nanmax([num(s[1]) for s in self.samples])),
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ oracle leg
def oracle_sample(mol, reps=1):
    """Time the oracle on a bounded sample; returns (evals/s, seconds used,
    sample description, omega, sample derivative)."""
    from oracle import ris_oracle
    ris_oracle.build()
    t0 = time.perf_counter()
    orc = ris_oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                               mol.nocc)
    t1 = time.perf_counter()
    w, X, _ = orc.tda_davidson(NSTATES, tol=1e-10)
    t2 = time.perf_counter()
    pairs = [(0, 0), (0, 1)]
    d = orc.pair_energy_derivs(pairs, X, atoms=[0])
    t3 = time.perf_counter()
    npair_full = NSTATES + (NSTATES - 1)
    t_full = (t1 - t0) + (t2 - t1) + (t3 - t2) / len(pairs) * npair_full * mol.natm
    sample = (f"oracle setup + Davidson({NSTATES}) + d/dR of {len(pairs)} pair energies for 1 of "
              f"{mol.natm} atoms; derivative time extrapolated to {npair_full} pairs x {mol.natm} atoms")
    return 1.0 / t_full, t3 - t0, sample, w, X, d


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2511_18233_gb300 import synth
    mol = synth.workload(1)
    vals, used = [], 0.0
    for it in range(args.warmup + args.steps):
        v, t, sample, *_ = oracle_sample(mol)
        used += t
        if it >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, workload=WORKLOAD, subspace_eig="fp32" if args.eig_fp32 else "fp64"),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU leg
def run_serving(args):
    """Serving stream of surface-hopping requests (energies + active-state
    gradient + NACs to the neighbouring states) from a closed pool of
    trajectories with Poisson arrivals; mixed precision with continuous
    batching over several slots, then the same stream replayed on the plain
    FP64 path one request at a time (cold Davidson, one slot)."""
    import torch
    from paper_2511_18233_gb300 import build, serve
    build.build()
    torch.cuda.set_device(0)
    specs = serve.make_trajectories(args.serve_trajectories, seed=2025)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    out = {}
    for mode in ("mixed", "fp64_plain"):
        mixed = mode == "mixed"
        nreq = args.serve_requests if mixed else args.serve_fp64_requests
        nwarm = args.serve_warmup if mixed else max(2, args.serve_warmup // 20)
        with Clocks(0) as clk:
            res = serve.serve(specs, n_requests=nreq, n_warmup=nwarm, rate=args.serve_rate,
                              nslots=args.serve_slots if mixed else 1, budget_bytes=budget,
                              precision="mixed" if mixed else "fp64", use_guess=args.serve_guess and mixed, seed=7,
                              **({"eig_fp32": 1} if mixed and args.eig_fp32 else {}))
        done = res.pop("done")
        res.pop("trajectories")
        iters = [r.result["n_iter"] for r in done if r.result]
        res["mean_davidson_iterations"] = float(np.mean(iters)) if iters else None
        res["clocks"] = clk.summary()
        out[mode] = res
    m, f = out["mixed"], out["fp64_plain"]
    line = {"metric": "serving grad+NAC evals/s; p50/p99 latency", "value": m["throughput_per_s"],
            "unit": "evals/s", "higher_is_better": True, "n_gpus": 1,
            "p50_ms": m["p50_ms"], "p99_ms": m["p99_ms"],
            "vs_fp64_plain": m["throughput_per_s"] / f["throughput_per_s"],
            "dtype": "f32/tf32x3+f64", "data": "synthetic",
            "config": {"workload": f"{args.serve_trajectories} trajectories, chains C4..C40 and flakes "
                                   f"4-7 A, 5-10 states, Poisson {args.serve_rate}/s, closed pool",
                       "slots": args.serve_slots, "budget_bytes": budget,
                       "davidson_seed": "previous step" if args.serve_guess else "cold",
                       "subspace_eig": "fp32" if args.eig_fp32 else "fp64"},
            "mixed": m, "fp64_plain": f}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: mixed is the headline value, FP64 reported beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true", help="run the serving stream instead")
    ap.add_argument("--eig-fp32", action="store_true",
                    help="mixed form: Davidson subspace eigenproblem in FP32 (option eig_fp32)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-fp64-requests", type=int, default=100)
    ap.add_argument("--serve-trajectories", type=int, default=64)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-guess", action="store_true",
                    help="seed each step's Davidson with the trajectory's resident amplitudes")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serving(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2511_18233_gb300 import build, synth
    build.build()
    mol = synth.workload(1)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_sample(mol)  # before any CUDA work of the library
    precs = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    res = {p: measure(p, mol, args, world, local, dist) for p in precs}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    head = res[precs[0]]
    line = {"metric": METRIC, "value": head["value"], "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": head["dtype"], "data": "synthetic",
            "config": dict(CONFIG, workload=WORKLOAD, precision=precs[0],
                           subspace_eig="fp32" if args.eig_fp32 and precs[0] == "mixed" else "fp64"),
            "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
            "stages_last_step": head["stages"], "roofline": head["roofline"],
            "roofline_classes": head["classes"], "clocks": head["clocks"]}
    for p in precs[1:]:
        r = res[p]
        line[p] = {k: r[k] for k in ("value", "ms_per_step", "dtype", "e2e", "gpu_launches",
                                    "stages", "roofline", "classes", "clocks")}
    if len(precs) > 1:
        line["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    if cpu is not None:
        v, used, sample, w_ref, X_ref, d_ref = cpu
        line["cpu_baseline"] = {"value": v, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": sample, "seconds": round(used, 2)}
        line["error_vs_oracle"] = {p: {"omega_max_abs": float(np.max(np.abs(res[p]["omega"] - w_ref)))}
                                   for p in precs}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def measure(precision, mol, args, world, local, dist):
    """Time one precision form on the device-resident workload (CUDA events on
    the library's stream, L2 flushed between steps) and end to end through
    host buffers; per-class kernel timings from the library's profile."""
    import torch
    from paper_2511_18233_gb300 import ris
    stream = torch.cuda.Stream()
    prec = ris.FP64 if precision == "fp64" else ris.MIXED
    extra = {"eig_fp32": 1} if precision == "mixed" and args.eig_fp32 else {}
    ctx = ris.Context(device=local, precision=prec, cuda_stream=stream.cuda_stream, profile=1, **extra)
    dev = f"cuda:{local}"
    coords_d = torch.as_tensor(mol.coords, device=dev)
    C_d = torch.as_tensor(mol.C, device=dev)
    eps_d = torch.as_tensor(mol.mo_energy, device=dev)
    nov = mol.nocc * mol.nvir
    om_d = torch.zeros(NSTATES, dtype=torch.float64, device=dev)
    X_d = torch.zeros((NSTATES, mol.nocc, mol.nvir), dtype=torch.float64, device=dev)
    g_d = torch.zeros((NSTATES, mol.natm, 3), dtype=torch.float64, device=dev)
    pairs = [(s, s + 1) for s in range(NSTATES - 1)]
    n_d = torch.zeros((len(pairs), mol.natm, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step_dev():
        ctx.build_aux(coords_d, mol.shells, mol.aux_j, mol.aux_k)
        ctx.build_B(C_d, eps_d, mol.nocc)
        ctx.excite(NSTATES, out=(om_d, X_d, None))
        ctx.gradient(range(NSTATES), out=g_d)
        ctx.nac(pairs, out=n_d)

    for _ in range(args.warmup):
        step_dev()
    torch.cuda.synchronize()
    ctx.stats()  # reset the per-class profile
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    l0 = ctx.stats()["launches"]
    with Clocks(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step_dev()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    st = ctx.stats()
    launches = int(st["launches"] - l0)
    stages = {k: round(st[k], 3) for k in ("aux_ms", "B_ms", "excite_ms", "deriv_ms")}
    stages.update({"davidson_products": int(st["n_products"]), "davidson_iterations": int(st["n_iter"])})
    torch.cuda.synchronize()
    tot = sum(times) / 1000.0
    value = replica_throughput(tot, args.steps, world, dist, dev)
    tot = world * args.steps / value  # the slowest rank's time

    # end to end through host buffers
    h2d = mol.coords.nbytes + mol.C.nbytes + mol.mo_energy.nbytes
    d2h = 8 * (NSTATES + NSTATES * nov + NSTATES * mol.natm * 3 + len(pairs) * mol.natm * 3)
    e2e_t = []
    for it in range(max(2, args.steps // 2) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
        ctx.build_B(mol.C, mol.mo_energy, mol.nocc)
        om, X = ctx.excite(NSTATES)
        g = ctx.gradient(range(NSTATES))
        n = ctx.nac(pairs)
        t1 = time.perf_counter()
        if it > 0:
            e2e_t.append(t1 - t0)
    e2e = world / float(np.mean(e2e_t))

    peaks, src = _peaks()
    fp64_peak = peaks["bf16_tflops"] * 1.25 / 2250.0  # measured bf16 x nominal FP64/BF16 ratio
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25     # measured bf16 x nominal TF32/BF16 ratio
    classes = {
        "tc_gemm_3xtf32": (st["tc_gemm_ms"], 3 * st["tc_gemm_flops"] / 1e12, "tensor", "TFLOP/s", tf32_peak,
                           f"of {src} bf16 x nominal TF32/BF16 (1.1/2.25); achieved counts the 3 TF32 passes"),
        "dgemm_fp64": (st["gemm_ms"], st["gemm_flops"] / 1e12, "tensor", "TFLOP/s", fp64_peak,
                       f"of {src} bf16 x nominal FP64/BF16 (1.25/2250)"),
        # FP64-accurate products on the FP16 tensor cores: 55 digit-slice
        # products per FP64 product, counted as FP16 tensor work
        "emu_gemm_f64": (st["emu_gemm_ms"], 55 * st["emu_gemm_flops"] / 1e12, "tensor", "TFLOP/s",
                         peaks["bf16_tflops"], f"of {src} bf16 (FP16 runs at the same rate); "
                         "achieved counts the 55 slice products"),
        "int3c_deriv": (st["int3c_deriv_ms"], None, "alu", None, None,
                        "side stream: runs under the B build and Davidson, time not additive"),
        "int3c": (st["int3c_ms"], None, "alu", None, None, ""),
        "contract": (st["contract_ms"], st["contract_bytes"] / 1e9, "hbm", "GB/s", peaks["hbm_gbs"],
                     f"of {src} HBM copy"),
        "subspace_eig": (st["eig_ms"], None, "alu", None, None, ""),
    }
    table = {}
    for k, (ms, work, bound, unit, peak, note) in classes.items():
        row = {"ms_per_step": round(ms / args.steps, 3), "share_of_step": ms / (sum(times) or 1.0),
               "bound": bound}
        if work is not None and ms > 0:
            ach = work / (ms / 1000.0)
            row.update({"achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak})
        elif note:
            row["note"] = note
        table[k] = row
    dom = max((k for k in classes if k != "int3c_deriv"), key=lambda k: classes[k][0])
    ms, work, bound, unit, peak, note = classes[dom]
    roof = {"kernel": dom, "bound": bound, "share_of_step": ms / (sum(times) or 1.0)}
    if work is not None:
        ach = work / (ms / 1000.0)
        roof.update({"achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak, "peak_source": note,
                     "traffic": None})
    ctx.close()
    return {"value": value, "ms_per_step": 1000.0 * tot / args.steps,
            "dtype": "f64" if precision == "fp64" else "f32/tf32x3+f64",
            "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches, "stages": stages, "roofline": roof, "classes": table,
            "clocks": clk.summary(), "omega": om_d.cpu().numpy()}


if __name__ == "__main__":
    sys.exit(main())
