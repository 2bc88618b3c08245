#!/usr/bin/env python
"""Throughput benchmark of the sm_103a TDDFT-ris engine.

Headline: one step = one evaluation at one geometry of the C20H22 chain
workload (42 atoms, 512 AOs, nocc 71, 102 J / 42 K auxiliary functions):
screened three-centre integrals and metric Cholesky, B tensors, Davidson for
the 10 lowest TDA-ris states, gradients of all 10 states and the 9 couplings
between adjacent states.  Metric: evaluations per second.

* value: the mixed-precision form (the throughput form; the FP64 form is
  timed the same way and reported beside it under "fp64"); device-resident
  inputs (coordinates, MO coefficients, orbital energies as CUDA tensors),
  outputs into CUDA tensors, each step timed with CUDA events on the
  library's stream; L2 flushed (512 MB write) between steps, outside the
  timed events.
* e2e: the same evaluation through host (numpy) buffers, host<->device copies
  inside the timed region, wall clock.
* roofline: the kernel class with the largest share of the timed region;
  `achieved` counts the method's algorithmic work of that class (the
  per-unit figures of the scope table: B build, A X per product, Gamma per
  pair) over its CUDA-event time; peaks are the measured pipe rates
  (profiles/peaks_probe_gb300.json, MEASURED_PEAKS.json).
* error_vs_oracle: per result (energies, sampled gradients and couplings of
  the timed evaluation) against the FP64 oracle.
* configs: the other workloads as extra keys (C4H6 absolute time; the
  C54H18 flake RPA-ris with the autograd state-1 gradient; the packed
  12 x C20H22 workload in the streamed mixed form).
* serving: the surface-hopping stream (64 trajectories, 2000 requests after
  200, Poisson 200/s, Davidson seeded with the trajectory's resident
  amplitudes) against a shorter cold-Davidson stream and plain FP64 replay.
* cpu_baseline / --impl reference: the FP64 oracle on the host cores: the
  C20H22 sample (setup, Davidson, derivatives of two pair energies w.r.t.
  one atom, extrapolated to the full evaluation) and the C4H6 evaluation in
  full, on all cores and on one.

Multi-GPU: replicas only (each rank evaluates its own copy; no collective
in the data path); value = evaluations of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
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


def peaks():
    """Roofline denominators: HBM copy and bf16 from MEASURED_PEAKS.json, the
    FP64 FMA, TF32 and FP16 tensor pipes from the committed probe run."""
    out = {"src": {}}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        out["hbm_gbs"], out["bf16_tflops"] = p["hbm_gbs"], p["bf16_tflops"]
        out["src"]["hbm"] = "measured (MEASURED_PEAKS.json, copy)"
    except Exception:
        out["hbm_gbs"], out["bf16_tflops"] = 6800.0, 1900.0
        out["src"]["hbm"] = "fallback"
    try:
        with open(os.path.join(ROOT, "profiles", "peaks_probe_gb300.json")) as f:
            r = json.load(f)["rates"]
        out["fp64_tflops"] = r["fp64_fma"]["tflops"]
        out["tf32_tflops"] = r["tf32_tcgen05"]["tflops"]
        out["f16_tflops"] = r["f16_tcgen05"]["tflops"]
        out["fp32_tflops"] = r["fp32_fma"]["tflops"]
        out["src"]["pipes"] = "measured (profiles/peaks_probe_gb300.json)"
    except Exception:
        out["fp64_tflops"] = out["bf16_tflops"] * 1.25 / 2250.0
        out["tf32_tflops"] = out["bf16_tflops"] * 1.1 / 2.25
        out["f16_tflops"] = out["bf16_tflops"]
        out["fp32_tflops"] = out["bf16_tflops"] * 80.0 / 2250.0
        out["src"]["pipes"] = "fallback (bf16 x nominal ratios)"
    return out


# DRAM traffic of each GEMM class per C20H22 mixed evaluation: the sum of
# dram__bytes_read.sum + dram__bytes_write.sum over the class's launches of
# one evaluation, from one ncu capture of `bench.py --no-extra
# --no-cpu-baseline --precision mixed --steps 1 --warmup 1` (five
# evaluations, divided by five; ncu runs each launch with a cold L2).  Valid
# while the kernel's source file is unchanged (sha256 prefix); the summary is
# in profiles/launches_mixed_c20h22.md.
TRAFFIC = {
    "dgemm_fp64": {"bytes_per_eval": 0.4933e9, "source": "paper_2511_18233_gb300/csrc/la.cu",
                   "sha": "5d8e96e3ff2bf3cb"},
    "tc_gemm_3xtf32": {"bytes_per_eval": 5.1348e9, "source": "paper_2511_18233_gb300/csrc/gemm_tc.cu",
                       "sha": "80f44d6f789f2b89"},
    "emu_gemm_f64": {"bytes_per_eval": 0.9350e9, "source": "paper_2511_18233_gb300/csrc/gemm_emu.cu",
                     "sha": "6eca5b2a53ba7b71"},
    "ff_gemm_f64x": {"bytes_per_eval": 0.5702e9, "source": "paper_2511_18233_gb300/csrc/gemm_ff.cu",
                     "sha": "66a9f1945925d817"},
}


def _src_sha(rel):
    try:
        with open(os.path.join(ROOT, rel), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def traffic_for(cls):
    t = TRAFFIC.get(cls)
    if not t or _src_sha(t["source"]) != t["sha"]:
        return None
    return t["bytes_per_eval"]


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


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for key in ("Model name", "BIOS Model name"):
            for line in out.splitlines():
                if line.strip().startswith(key + ":"):
                    v = line.split(":", 1)[1].strip()
                    if v and v != "-":
                        return v
    except Exception:
        pass
    return os.uname().machine


# ------------------------------------------------------------------ oracle leg
def oracle_sample(mol):
    """Time the oracle on a bounded sample of the C20H22 evaluation; returns
    (evals/s, seconds used, sample description, reference values)."""
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
    # reference values of the per-result errors (not timed): gradients of
    # states 0 and 9 and the (0,1) coupling on atoms 0 and 20
    atoms = [0, 20]
    g = orc.gradients([0, NSTATES - 1], X, atoms=atoms)
    nac = orc.nacs([(0, 1)], w, X, atoms=atoms)
    ref = {"omega": w, "atoms": atoms, "grad": g[:, atoms], "nac01": nac[0, atoms]}
    return 1.0 / t_full, t3 - t0, sample, ref


_CFG1_ORACLE = r"""
import sys, time, json
sys.path.insert(0, %r)
import numpy as np
from paper_2511_18233_gb300 import synth
from oracle import ris_oracle
ris_oracle.build()
mol = synth.workload(0)
ts = []
for rep in range(3):
    t0 = time.perf_counter()
    orc = ris_oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc)
    w, X, _ = orc.tda_davidson(5, tol=1e-10)
    g = orc.gradients(range(5), X)
    n = orc.nacs([(0, 1)], w, X)
    ts.append(time.perf_counter() - t0)
print(json.dumps({"seconds": sorted(ts)[1]}))
"""


def oracle_cfg1_full(threads):
    """The C4H6 evaluation (5 states, 5 gradients, NAC(S1,S2)) by the oracle in
    full, in a child process with `threads` OpenMP/BLAS threads (None: all
    cores); median of 3."""
    env = dict(os.environ)
    if threads:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", _CFG1_ORACLE % ROOT], capture_output=True, text=True,
                       env=env, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    s = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    return {"evals_per_s": 1.0 / s, "ms_per_eval": 1e3 * s,
            "threads": threads or os.cpu_count()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2511_18233_gb300 import synth
    mol = synth.workload(1)
    vals, walls = [], []
    for it in range(args.warmup + args.steps):
        v, t, sample, _ = oracle_sample(mol)
        if it >= args.warmup:
            vals.append(v)
            walls.append(t)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, workload=WORKLOAD, subspace_eig="fp32" if args.eig_fp32 else "fp64"),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": os.cpu_count(),
                             "cpu": cpu_model(), "kind": "oracle (extrapolated)", "sample": sample,
                             "sample_wall_ms_per_step": 1000.0 * float(np.mean(walls)),
                             "note": "ms_per_step is one full evaluation extrapolated from the "
                                     "timed sample; each step runs the sample only"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU legs
def run_serving(args, quick=False):
    """Serving stream of surface-hopping requests (energies + active-state
    gradient + NACs to the neighbouring states) from a closed pool of
    trajectories with Poisson arrivals; mixed precision with continuous
    batching over several slots (Davidson seeded with the trajectory's
    resident amplitudes unless --serve-cold), then the same stream replayed
    on the plain FP64 path one request at a time (cold Davidson, one slot)."""
    import torch
    from paper_2511_18233_gb300 import build, serve
    build.build()
    torch.cuda.set_device(0)
    specs = serve.make_trajectories(args.serve_trajectories, seed=2025)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    warm = not args.serve_cold
    out = {}
    modes = ["mixed", "fp64_plain"]
    if warm and args.serve_cold_requests > 0:
        modes.insert(1, "mixed_cold")  # the same stream with every Davidson started cold
    for mode in modes:
        mixed = mode.startswith("mixed")
        nreq = {"mixed": args.serve_requests, "mixed_cold": args.serve_cold_requests,
                "fp64_plain": args.serve_fp64_requests}[mode]
        nwarm = {"mixed": args.serve_warmup, "mixed_cold": max(2, args.serve_warmup // 5),
                 "fp64_plain": max(2, args.serve_warmup // 20)}[mode]
        seeded = warm and mode == "mixed"
        with Clocks(0) as clk:
            res = serve.serve(specs, n_requests=nreq, n_warmup=nwarm, rate=args.serve_rate,
                              nslots=args.serve_slots if mixed else 1, budget_bytes=budget,
                              precision="mixed" if mixed else "fp64", use_guess=seeded, seed=7,
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
                       "requests": args.serve_requests, "warmup_requests": args.serve_warmup,
                       "slots": args.serve_slots, "budget_bytes": budget,
                       "davidson_seed": "previous step" if warm else "cold",
                       "subspace_eig": "fp32" if args.eig_fp32 else "fp64"},
            "mixed": m, "fp64_plain": f}
    if "mixed_cold" in out:
        line["mixed_cold"] = out["mixed_cold"]
        line["warm_over_cold"] = m["throughput_per_s"] / out["mixed_cold"]["throughput_per_s"]
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both: mixed is the headline value, FP64 reported beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads and serving")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-packed", action="store_true", help="skip the 12 x C20H22 streamed workload")
    ap.add_argument("--serve", action="store_true", help="run only the serving stream")
    ap.add_argument("--eig-fp32", action="store_true",
                    help="mixed form: Davidson subspace eigenproblem in FP32 (option eig_fp32)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-fp64-requests", type=int, default=30)
    ap.add_argument("--serve-cold-requests", type=int, default=400,
                    help="requests of the cold-Davidson comparison stream (0: skip)")
    ap.add_argument("--serve-trajectories", type=int, default=64)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-cold", action="store_true",
                    help="start every step's Davidson cold instead of from the resident amplitudes")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        print(json.dumps(run_serving(args)))
        return 0

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
    cpu = cfg1_cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_sample(mol)  # before any CUDA work of the library
        cfg1_cpu = {"all_cores": oracle_cfg1_full(None), "one_thread": oracle_cfg1_full(1)}
    precs = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    res = {p: measure(p, mol, args, world, local, dist) for p in precs}
    extra = {}
    if not args.no_extra and world == 1:
        extra["c4h6"] = {p: measure_small(p, args) for p in precs}
        extra["c54h18_flake_rpa"] = {"fp64": measure_flake("fp64", args),
                                     "mixed": {"measured": False,
                                               "reason": "the RPA Davidson with 3xTF32 exchange products "
                                                         "does not reach the 1e-6 residual tolerance on "
                                                         "this system (exchange product error ~3e-6 "
                                                         "relative); the flake runs in FP64"}}
        if not args.no_packed:
            extra["packed_12x_c20h22"] = measure_packed(args)
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
        v, used, sample, ref = cpu
        line["cpu_baseline"] = {"value": v, "unit": "evals/s", "cores": os.cpu_count(), "cpu": cpu_model(),
                                "kind": "oracle (extrapolated)", "sample": sample, "seconds": round(used, 2),
                                "c4h6_full_evaluation": cfg1_cpu}
        errs = {}
        for p in precs:
            r = res[p]
            a = ref["atoms"]
            errs[p] = {"omega_max_abs_ha": float(np.max(np.abs(r["omega"] - ref["omega"][:NSTATES]))),
                       "grad_max_abs_ha_bohr": float(np.max(np.abs(r["grad"][[0, NSTATES - 1]][:, a] - ref["grad"]))),
                       "nac01_max_abs_per_bohr": float(np.max(np.abs(r["nac"][0, a] - ref["nac01"]))),
                       "nac01_numerator_max_abs_ha_bohr": float(np.max(np.abs(
                           r["nac"][0, a] * (r["omega"][1] - r["omega"][0])
                           - ref["nac01"] * (ref["omega"][1] - ref["omega"][0])))),
                       "sample": f"all {NSTATES} energies; gradients of states 0 and {NSTATES - 1} and the "
                                 f"(0,1) coupling on atoms {a}, oracle amplitudes vs the library's"}
        line["error_vs_oracle"] = errs
    if extra:
        line["configs"] = extra
    if not args.no_extra and not args.no_serve and world == 1:
        line["serving"] = run_serving(args)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def algorithmic_work(precision, d, nprod, npair, rpa=False, ff=True):
    """The method's own work per evaluation and kernel class (scope-table
    counts, dense, no screening credit): flops for the GEMM classes (a
    3xTF32 or double-FP32 product counts once), bytes are reported by the
    library.  In the mixed form the Coulomb part of A.X runs as double-FP32
    products (option subspace_ff, on by default)."""
    n, o, v, nJ, nK = d["nao"], d["nocc"], d["nvir"], d["nJ"], d["nK"]
    nov = o * v
    coul_ax = 4.0 * nov * nJ * nprod * (2 if rpa else 1)
    exch_ax = (2.0 * v * v * o * nK + 2.0 * o * o * v * nK) * nprod * (2 if rpa else 1)
    b_coul = 2.0 * o * n * n * nJ + 2.0 * o * v * n * nJ
    b_k = 2.0 * o * n * n * nK + 2.0 * o * o * n * nK + 2.0 * v * n * n * nK + 2.0 * v * v * n * nK
    gam = (2.0 * o * v * v * nK + 4.0 * n * n * o * nK) * npair
    if precision == "fp64":
        return {"dgemm_fp64": coul_ax + exch_ax + b_coul + b_k + gam}
    return {"dgemm_fp64": (0.0 if ff else coul_ax) + 2.0 * o * o * n * nK,
            "ff_gemm_f64x": coul_ax if ff else 0.0,
            "tc_gemm_3xtf32": exch_ax + 2.0 * v * n * n * nK + 2.0 * v * v * n * nK + gam,
            "emu_gemm_f64": b_coul}


def classify(st, steps, step_ms_total, precision, dims, nprod, npair, workload="c20h22"):
    """Per kernel class: time share, executed and algorithmic work against
    the pipe's measured peak."""
    pk = peaks()
    alg = algorithmic_work(precision, dims, nprod, npair)
    tf32x3 = pk["tf32_tflops"] / 3.0           # three TF32 passes per product
    emu = pk["f16_tflops"] / 55.0               # 55 FP16 slice products per FP64 product
    ffx = pk["fp32_tflops"] / 12.0              # 12 FP32 instructions per double-FP32 multiply-add
    classes = {
        "tc_gemm_3xtf32": (st["tc_gemm_ms"], st["tc_gemm_flops"], "tensor (tf32)", tf32x3,
                           "TF32 tcgen05 probe / 3 passes"),
        "dgemm_fp64": (st["gemm_ms"], st["gemm_flops"], "fp64 fma", pk["fp64_tflops"], "FP64 FMA probe"),
        "emu_gemm_f64": (st["emu_gemm_ms"], st["emu_gemm_flops"], "tensor (f16)", emu,
                         "FP16 tcgen05 probe / 55 slice products (FP64-equivalent)"),
        "ff_gemm_f64x": (st.get("ff_gemm_ms", 0.0), st.get("ff_gemm_flops", 0.0), "fp32 fma (double-FP32)",
                         ffx, "FP32 FMA probe / 12 instructions per multiply-add"),
        "contract": (st["contract_ms"], None, "hbm", None, "HBM copy"),
        "subspace_eig": (st["eig_ms"], None, "latency (fp64, one CTA per eigenvalue)", None, ""),
        "int3c": (st["int3c_ms"], None, "fp64 alu", None,
                  "McMurchie-Davidson recursion on the FP64 pipe; executed FP64 operations not counted, no achieved/peak"),
        "int3c_deriv": (st["int3c_deriv_ms"], None, "fp64 alu", None,
                        "side stream under the B build and Davidson, time not additive"),
    }
    table = {}
    for k, (ms, exe, bound, peak, note) in classes.items():
        row = {"ms_per_step": round(ms / steps, 3), "share_of_step": ms / (step_ms_total or 1.0), "bound": bound}
        if k == "contract" and ms > 0:
            ach = st["contract_bytes"] / 1e9 / (ms / 1000.0)
            row.update({"achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                        "peak_source": pk["src"]["hbm"], "work": "algorithmic bytes"})
        elif peak is not None and ms > 0:
            a = alg.get(k, 0.0) * steps / 1e12 / (ms / 1000.0)
            e = exe / 1e12 / (ms / 1000.0)
            row.update({"achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                        "executed_tflops": e, "executed_frac": e / peak,
                        "peak_source": note + ", " + pk["src"]["pipes"],
                        "work": "algorithmic flops (scope-table counts)"})
        elif note:
            row["note"] = note
        table[k] = row
    dom = max((k for k in classes if k != "int3c_deriv"), key=lambda k: classes[k][0])
    # the contract's vocabulary (hbm | tensor | alu), the pipe itself under "pipe"
    kind = {"tensor (tf32)": "tensor", "tensor (f16)": "tensor", "fp64 fma": "alu",
            "fp32 fma (double-FP32)": "alu", "hbm": "hbm", "fp64 alu": "alu"}
    pipe = table[dom]["bound"]
    roof = {"kernel": dom, "bound": kind.get(pipe, pipe), "pipe": pipe,
            "share_of_step": table[dom]["share_of_step"]}
    for key in ("achieved", "peak", "unit", "frac", "peak_source", "executed_frac"):
        if key in table[dom]:
            roof[key] = table[dom][key]
    roof["traffic"] = traffic_for(dom) if workload == "c20h22" and precision == "mixed" else None
    if roof["traffic"] is not None:
        roof["traffic_unit"] = "bytes per evaluation (all launches of the class, ncu, cold L2)"
    return roof, table


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
    nprod = 0
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
    nprod = int(st["n_products"])
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
    dm = ctx.dims()
    dims = {"nao": dm["nao"], "nocc": mol.nocc, "nvir": mol.nvir, "nJ": dm["nauxJ"], "nK": dm["nauxK"]}
    roof, table = classify(st, args.steps, sum(times), precision, dims, nprod, NSTATES + len(pairs))
    ctx.close()
    return {"value": value, "ms_per_step": 1000.0 * tot / args.steps,
            "dtype": "f64" if precision == "fp64" else "f32/tf32x3+f64",
            "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches, "stages": stages, "roofline": roof, "classes": table,
            "clocks": clk.summary(), "omega": om_d.cpu().numpy(), "grad": g_d.cpu().numpy(),
            "nac": n_d.cpu().numpy()}


def _timed(fn, steps, warmup, stream, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def measure_small(precision, args):
    """C4H6 chain (10 atoms, 112 AOs): 5 states, 5 gradients, NAC(S1,S2); it
    fits in L2, so it is reported as absolute time per evaluation."""
    import torch
    from paper_2511_18233_gb300 import ris, synth
    mol = synth.workload(0)
    stream = torch.cuda.Stream()
    ctx = ris.Context(precision=ris.FP64 if precision == "fp64" else ris.MIXED,
                      cuda_stream=stream.cuda_stream)
    dev = "cuda:0"
    c, C, e = (torch.as_tensor(a, device=dev) for a in (mol.coords, mol.C, mol.mo_energy))
    om = torch.zeros(5, dtype=torch.float64, device=dev)
    X = torch.zeros((5, mol.nocc, mol.nvir), dtype=torch.float64, device=dev)
    g = torch.zeros((5, mol.natm, 3), dtype=torch.float64, device=dev)
    n = torch.zeros((1, mol.natm, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        ctx.build_aux(c, mol.shells, mol.aux_j, mol.aux_k)
        ctx.build_B(C, e, mol.nocc)
        ctx.excite(5, out=(om, X, None))
        ctx.gradient(range(5), out=g)
        ctx.nac([(0, 1)], out=n)

    ts = _timed(step, max(args.steps, 5), args.warmup, stream, flush)
    ctx.close()
    ms = float(np.median(ts))
    return {"workload": "C4H6 chain, 10 atoms, nao 112, TDA-ris 5 states, 5 gradients + NAC(S1,S2)",
            "ms_per_eval_median": ms, "evals_per_s": 1000.0 / ms, "steps": len(ts)}


def measure_packed(args):
    """12 x C20H22 packed in a 40 A cube (504 atoms, 6144 AOs, nocc 852,
    1224 J / 504 K auxiliary functions): 8 states, 8 gradients, 7 adjacent
    NACs in the streamed mixed form (the dense AO three-index tensors would
    need about a terabyte).  One warm-up and one timed evaluation (each over
    a minute, working set far larger than L2)."""
    import torch
    from paper_2511_18233_gb300 import ris, synth
    t0 = time.perf_counter()
    mol = synth.workload(3)
    t_host = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    ctx = ris.Context(precision=ris.MIXED, cuda_stream=stream.cuda_stream, profile=1)
    dev = "cuda:0"
    c, C, e = (torch.as_tensor(a, device=dev) for a in (mol.coords, mol.C, mol.mo_energy))
    ns = 8
    pairs = [(k, k + 1) for k in range(ns - 1)]
    om = torch.zeros(ns, dtype=torch.float64, device=dev)
    X = torch.zeros((ns, mol.nocc, mol.nvir), dtype=torch.float64, device=dev)
    g = torch.zeros((ns, mol.natm, 3), dtype=torch.float64, device=dev)
    n = torch.zeros((len(pairs), mol.natm, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(16, dtype=torch.float32, device=dev)  # inputs are far larger than L2

    def step():
        ctx.build_aux(c, mol.shells, mol.aux_j, mol.aux_k)
        ctx.build_B(C, e, mol.nocc)
        ctx.excite(ns, out=(om, X, None))
        ctx.gradient(range(ns), out=g)
        ctx.nac(pairs, out=n)

    step()
    torch.cuda.synchronize()
    ctx.stats()
    with Clocks(0) as clk:
        ts = _timed(step, 1, 0, stream, flush)
    st = ctx.stats()
    dm = ctx.dims()
    dims = {"nao": dm["nao"], "nocc": mol.nocc, "nvir": mol.nvir, "nJ": dm["nauxJ"], "nK": dm["nauxK"]}
    roof, table = classify(st, len(ts), sum(ts), "mixed", dims, int(st["n_products"]), ns + len(pairs),
                           workload="packed")
    ga = g.cpu().numpy()
    ctx.close()
    ms = float(np.mean(ts))
    pk = peaks()
    # the FP64 form of this workload: counted algorithmic flops at the
    # measured FP64 FMA rate (not run: about an hour per evaluation)
    fp64_flops = algorithmic_work("fp64", dims, int(st["n_products"]), ns + len(pairs))["dgemm_fp64"]
    return {"workload": "12 x C20H22 packed (40 A cube), 504 atoms, nao 6144, TDA-ris 8 states, "
                        "8 gradients + 7 adjacent NACs, streamed form",
            "precision": "mixed", "ms_per_eval": ms, "evals_per_s": 1000.0 / ms, "steps": len(ts),
            "warmup": 1, "stages_last_step": {k: round(st[k], 1) for k in ("aux_ms", "B_ms", "excite_ms",
                                                                            "deriv_ms")},
            "davidson_products": int(st["n_products"]), "residual_max": st["residual_max"],
            "peak_device_bytes": int(st["bytes_peak"]), "host_setup_s": round(t_host, 1),
            "translation_sum_rule_max_rel": float(np.max(np.abs(ga.sum(axis=1))) / np.max(np.abs(ga))),
            "roofline": roof, "roofline_classes": table, "clocks": clk.summary(),
            "fp64": {"measured": False,
                     "projected_s_per_eval": fp64_flops / (pk["fp64_tflops"] * 1e12),
                     "basis": "scope-table algorithmic flops of this evaluation at the measured FP64 "
                              "FMA rate; not run (about an hour per evaluation on GB300's FP64 pipe)"}}


def measure_flake(precision, args):
    """C54H18 flake (72 atoms, 1134 AOs), full RPA-ris, 20 states; one
    evaluation = the autograd forward (integrals, B, RPA Davidson) and the
    backward of the state-1 energy (analytic gradient kernel)."""
    import torch
    from paper_2511_18233_gb300 import ris, synth
    from paper_2511_18233_gb300.autograd import RisModel
    mol = synth.workload(2)
    stream = torch.cuda.Stream()
    model = RisModel(mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc, 20, rpa=True,
                     precision=ris.FP64 if precision == "fp64" else ris.MIXED,
                     cuda_stream=stream.cuda_stream)
    R0 = torch.as_tensor(mol.coords, device="cuda:0")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda:0")

    def step():
        R = R0.clone().requires_grad_(True)
        with torch.cuda.stream(stream):
            w = model.energy(R, 0)
            w.backward()

    # the FP64 RPA evaluation takes about a minute: one timed evaluation (the
    # library is already warm from the other workloads)
    steps = 1 if precision == "fp64" else max(args.steps, 3)
    ts = _timed(step, steps, 0 if precision == "fp64" else args.warmup, stream, flush)
    st = model.ctx.stats()
    model.ctx.close()
    ms = float(np.median(ts))
    return {"workload": "C54H18 flake, 72 atoms, nao 1134, RPA-ris 20 states, autograd state-1 gradient",
            "ms_per_eval_median": ms, "evals_per_s": 1000.0 / ms, "steps": len(ts),
            "davidson_iterations_last": int(st["n_iter"])}


if __name__ == "__main__":
    sys.exit(main())
