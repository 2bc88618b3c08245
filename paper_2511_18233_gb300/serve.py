"""Serving form of the ris gradient/NAC path for surface-hopping dynamics.

Trajectory surface hopping (Sec. 1; the NAC of Eq. (fo-nacme) between
neighbouring states and the gradient of the active state at every step)
needs many independent trajectories, each stepping sequentially.  This
module serves such a stream on one GPU:

* continuous batching: a fixed set of slots, each a library context with
  its own CUDA stream driven by its own host thread (the ctypes calls
  release the GIL), so requests of different molecules run concurrently
  on the device; a queued request starts as soon as a slot and enough HBM
  are free;
* residency: per trajectory, the MO coefficients and orbital energies
  stay on the device (they are fixed along a trajectory) together with the
  last step's amplitudes, which seed the next step's Davidson search;
* admission by HBM footprint: a request is admitted only while the bytes
  of all running requests plus all resident trajectory state fit the
  budget; a request's footprint is estimated from its dimensions on a
  trajectory's first step and measured by the library afterwards;
* phases: from its second step on, each state's sign follows the previous
  step (overlap over the five most dominant determinants, ris_phase_align),
  so the couplings keep a consistent sign along the trajectory, and the
  time-derivative coupling T_IJ = d_IJ . v (v: the step's nuclear
  velocities) is returned with them;
* latency is arrival -> results on the host; p50/p99 and throughput are
  reported.

The host logic (stream generation, admission, scheduling) is plain Python
and is exercised on the CPU with a stand-in executor; `RisExecutor` is the
GPU executor on top of the C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import synth

ANGSTROM = synth.ANGSTROM


def _ld8(k: int) -> int:
    return (k + 7) & ~7


def _ld4(n: int) -> int:
    return (n + 3) // 4 * 4


# ---------------------------------------------------------------- footprint

def footprint_bytes(nao: int, nocc: int, nJ: int, nK: int, nU: int, nstates: int,
                    nstate_deriv: int, mixed: bool) -> int:
    """Upper estimate of the device bytes one request holds at its peak.

    Persistent per-request buffers (3c integrals of both fitting sets, the
    metric and its inverse factors, the transformed B tensors and, in mixed
    precision, their FP32 hi/lo splits and the tensor-core operands of the
    (ab|P)_K transform) plus the larger of the Davidson work space and the
    derivative stage (the derivative integrals d(mu nu|P)/dR, the exchange
    parts of a batch of pair densities and per-state densities).  The
    derivative integrals d(mu nu|P)/dR (FP32 in mixed precision) are computed
    on a side stream from the auxiliary build on, so they count as persistent.
    """
    n, o = nao, nocc
    v = n - o
    nov = o * v
    M = max(nJ, nK)
    d, f = 8, 4
    aux = d * (n * n * (nJ + nK) + 4 * nU * nU + nJ * nJ + nK * nK + M * M)
    B = d * (n * n + 3 * n + nov + o * n * M + o * n * nK + max(v * n * nK, o * n * M)
             + max(max(nov, o * o) * M, v * v * nK) + nov * nJ + 2 * o * o * nK
             + 3 * v * v * nK)
    if mixed:
        B += f * (2 * o * nK * _ld4(o) + 4 * nK * v * _ld4(v) + 2 * nK * o * _ld4(o)
                  + 2 * n * (_ld4(o) + _ld4(v))) + d * o * o * nK
        # (ab|P)_K on tensor cores: T^K and H splits, C_v^T split, FP64 G
        B += f * 2 * _ld4(n) * (nK * n + v * nK + v) + d * v * nK * v
        # Coulomb transforms on the tensor cores: ten FP16 digit slices of T^J
        # and of C, row exponents
        B += 2 * 10 * (n * nJ + max(o, v)) * _ld8(n) + 4 * (n * nJ + max(o, v))
        # and of the metric products B^J = W L_J^-T, c^K_vv = B^K_vv L_K^-1
        B += 2 * 10 * (max(nov, v * v) + M) * _ld8(M) + 4 * (max(nov, v * v) + M)
    ns = nstates
    nb0 = min(nov, ns + min(ns, 8))
    maxsp = min(max(nb0 + 2 * ns, 8 * ns), 256, nov)
    dav = d * ((2 * maxsp + 8 * ns) * nov + 2 * nb0 * nov * nK + maxsp * maxsp)
    if mixed:
        dav += f * 2 * nb0 * v * _ld4(o)
    s = nstate_deriv
    nbp = min(s, 8)  # pairs sharing one pass over the derivative integrals
    dint = (f if mixed else d) * 3 * n * n * nU
    deriv = d * (nbp * (n * n * nK + 3 * n * nK + nU * nU) + s * n * n
                 + 3 * s * n * nU + 4 * s * o * n + n * v + 2 * o * v * nK + 2 * n * o * nK)
    if mixed:
        deriv += f * 4 * s * (o * _ld4(v) + n * _ld4(2 * o))
    total = aux + B + dint + d * 2 * ns * nov + max(dav, deriv)
    return int(1.25 * total) + (32 << 20)


def molecule_dims(mol) -> Dict[str, int]:
    """nao, nocc and the fitting-set sizes (J, K and their union) of a molecule."""
    nJ = mol.naux("J")
    nK = mol.naux("K")
    kset = {(int(a), int(l), float(e)) for a, l, e in mol.aux_k}
    extra = sum(synth.ncart(int(l)) for a, l, e in mol.aux_j
                if (int(a), int(l), float(e)) not in kset)
    return dict(nao=mol.nao, nocc=mol.nocc, nJ=nJ, nK=nK, nU=nK + extra)


# ------------------------------------------------------------------ stream

@dataclasses.dataclass
class TrajectorySpec:
    """One surface-hopping trajectory: molecule, number of states, active state."""

    tid: int
    kind: str          # "chain" or "flake"
    size: float        # chain length n or flake radius in Angstrom
    nstates: int
    active: int        # 0-based index of the active excited state (S_{active+1})
    seed: int

    @property
    def pairs(self) -> List[Tuple[int, int]]:
        """NACs to the neighbouring excited states (the ground state excluded)."""
        p = []
        if self.active >= 1:
            p.append((self.active - 1, self.active))
        if self.active + 1 < self.nstates:
            p.append((self.active, self.active + 1))
        return p


def valid_flake_radius(r: float) -> float:
    """The radius itself, or, where the honeycomb cut at r leaves a carbon with
    a single neighbour, the largest radius below r (in 0.01 A steps) that
    does not."""
    while r > 0:
        try:
            synth.flake_geometry(r)
            return r
        except ValueError:
            r = round(r - 0.01, 2)
    raise ValueError("no valid flake radius")


def make_trajectories(ntraj: int, seed: int, chain_sizes: Sequence[int] = tuple(range(4, 41, 4)),
                      flake_radius: Tuple[float, float] = (4.0, 7.0),
                      nstates: Tuple[int, int] = (5, 10)) -> List[TrajectorySpec]:
    """A pool of trajectories: molecule kind chain/flake with equal odds, the
    chain length uniform over chain_sizes, the flake radius uniform in
    flake_radius, nstates uniform in the closed range, and the active state
    uniform over S_1 .. S_{nstates-1} (so that the upper neighbour exists)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(ntraj):
        if rng.random() < 0.5:
            kind, size = "chain", float(rng.choice(np.asarray(chain_sizes)))
        else:
            kind, size = "flake", valid_flake_radius(float(rng.uniform(*flake_radius)))
        ns = int(rng.integers(nstates[0], nstates[1] + 1))
        active = int(rng.integers(0, ns - 1))
        out.append(TrajectorySpec(t, kind, size, ns, active, seed * 1000 + t))
    return out


def step_coords(ref: np.ndarray, spec: TrajectorySpec, step: int,
                sigma_ang: float = 0.05) -> np.ndarray:
    """Geometry of a trajectory's step: the reference geometry plus independent
    Gaussian displacements (sigma per Cartesian component), seeded per
    (trajectory, step)."""
    rng = np.random.default_rng([spec.seed, step])
    return synth.perturb(ref, sigma_ang, rng)


# atomic masses (electron masses) and k_B T at 300 K (Hartree)
_MASS = {"H": 1.00794 * 1822.888486, "C": 12.0107 * 1822.888486}
_KT300 = 300.0 * 3.166811563e-6


def step_velocities(elements: Sequence[str], spec: TrajectorySpec, step: int) -> np.ndarray:
    """Nuclear velocities of a step (bohr per atomic time unit): Maxwell-Boltzmann
    at 300 K per Cartesian component, seeded per (trajectory, step); they enter
    only T_IJ = d_IJ . v, the quantity surface hopping uses."""
    rng = np.random.default_rng([spec.seed, step, 1])
    m = np.array([_MASS[e] for e in elements])
    return rng.normal(size=(len(elements), 3)) * np.sqrt(_KT300 / m)[:, None]


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """n arrival instants (seconds from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


# --------------------------------------------------------------- admission

class Admission:
    """HBM budget: bytes resident (trajectory state) plus bytes of running requests."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.resident = 0
        self.running = 0
        self.peak = 0

    def fits(self, nbytes: int) -> bool:
        return self.resident + self.running + nbytes <= self.budget

    def take(self, nbytes: int):
        self.running += nbytes
        self.peak = max(self.peak, self.resident + self.running)

    def give(self, nbytes: int):
        self.running -= nbytes

    def reside(self, nbytes: int):
        self.resident += nbytes
        self.peak = max(self.peak, self.resident + self.running)


@dataclasses.dataclass
class Request:
    traj: "Trajectory"
    step: int
    coords: np.ndarray
    t_arrive: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    footprint: int = 0
    slot: int = -1
    result: Optional[dict] = None
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


class Trajectory:
    """Per-trajectory host record; `state` holds what the executor keeps resident."""

    def __init__(self, spec: TrajectorySpec, mol, ref_coords: np.ndarray):
        self.spec = spec
        self.mol = mol
        self.ref = ref_coords
        self.dims = molecule_dims(mol)
        self.next_step = 0
        self.busy = False
        self.state = None          # executor-owned resident state
        self.resident_bytes = 0
        self.measured = 0          # footprint measured on an earlier step

    def footprint(self, mixed: bool) -> int:
        if self.measured:
            return int(self.measured * 1.05) + (8 << 20)
        dm = self.dims
        return footprint_bytes(dm["nao"], dm["nocc"], dm["nJ"], dm["nK"], dm["nU"],
                               self.spec.nstates, 1 + len(self.spec.pairs), mixed)


class Scheduler:
    """Continuous batching over `nslots` slots with HBM admission.

    `executor(slot, request) -> (result dict, measured peak bytes)` runs one
    request on a slot (its thread); it may raise.  Queued requests are
    taken first-come first-served, except that a request which does not fit
    the budget may be overtaken by later ones that fit, within a window of
    `window` queued requests, for at most `max_bypass` times."""

    def __init__(self, nslots: int, admission: Admission,
                 executor: Callable[[int, Request], Tuple[dict, int]],
                 window: int = 8, max_bypass: int = 16):
        self.nslots = nslots
        self.adm = admission
        self.executor = executor
        self.window = window
        self.max_bypass = max_bypass
        self.queue: collections.deque = collections.deque()
        self.cv = threading.Condition()
        self.free_slots = list(range(nslots))[::-1]
        self.inflight = 0
        self.max_inflight = 0
        self.done: List[Request] = []
        self.on_done: Optional[Callable[[Request], None]] = None
        self.closed = False
        self.bypassed = 0
        self.threads = [threading.Thread(target=self._worker, args=(s,), daemon=True)
                        for s in range(nslots)]
        self.slot_work: List[Optional[Request]] = [None] * nslots
        for t in self.threads:
            t.start()

    # queue side ------------------------------------------------------
    def submit(self, req: Request):
        with self.cv:
            req.t_arrive = time.perf_counter() if not req.t_arrive else req.t_arrive
            self.queue.append(req)
            self._dispatch()

    def _pick(self) -> Optional[int]:
        for k, r in enumerate(self.queue):
            if k >= self.window:
                return None
            if self.adm.fits(r.footprint):
                if k > 0:
                    self.bypassed += 1
                return k
            if k == 0 and self.bypassed >= self.max_bypass:
                return None   # the head has waited long enough: hold the rest back
        return None

    def _dispatch(self):
        # caller holds self.cv
        while self.free_slots and self.queue:
            k = self._pick()
            if k is None:
                if self.inflight == 0 and self.queue:
                    # nothing running and the head still does not fit: run it alone
                    k = 0
                else:
                    return
            r = self.queue[k]
            del self.queue[k]
            if k == 0:
                self.bypassed = 0
            slot = self.free_slots.pop()
            self.adm.take(r.footprint)
            r.slot = slot
            self.inflight += 1
            self.max_inflight = max(self.max_inflight, self.inflight)
            self.slot_work[slot] = r
            self.cv.notify_all()

    # slot side -------------------------------------------------------
    def _worker(self, slot: int):
        while True:
            with self.cv:
                while self.slot_work[slot] is None and not self.closed:
                    self.cv.wait()
                if self.slot_work[slot] is None and self.closed:
                    return
                r = self.slot_work[slot]
            r.t_start = time.perf_counter()
            peak = 0
            try:
                r.result, peak = self.executor(slot, r)
            except Exception as e:  # reported per request, the server keeps going
                r.error = f"{type(e).__name__}: {e}"
            r.t_done = time.perf_counter()
            with self.cv:
                self.slot_work[slot] = None
                self.adm.give(r.footprint)
                if peak:
                    r.traj.measured = max(r.traj.measured, int(peak))
                self.inflight -= 1
                self.free_slots.append(slot)
                self.done.append(r)
                cb = self.on_done
                self._dispatch()
                self.cv.notify_all()
            if cb is not None:
                cb(r)

    def wait_idle(self, timeout: Optional[float] = None) -> bool:
        end = None if timeout is None else time.perf_counter() + timeout
        with self.cv:
            while self.queue or self.inflight:
                rem = None if end is None else end - time.perf_counter()
                if rem is not None and rem <= 0:
                    return False
                self.cv.wait(rem)
        return True

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()


# ---------------------------------------------------------------- drivers

def percentile(x: Sequence[float], q: float) -> float:
    """Nearest-rank percentile (q in [0, 100])."""
    xs = sorted(x)
    if not xs:
        return float("nan")
    k = max(0, min(len(xs) - 1, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


def run_stream(trajs: List[Trajectory], scheduler: Scheduler, n_requests: int, n_warmup: int,
               rate: float, seed: int, mixed: bool, max_steps: Optional[int] = None,
               timeout: float = 3600.0) -> dict:
    """Drive a closed pool of trajectories with Poisson arrivals.

    Arrival instants come from a Poisson process of the given rate; at each
    instant one idle trajectory (chosen uniformly among the idle ones)
    issues its next step.  When every trajectory is busy, the arrival waits
    for the next one to finish (a trajectory's steps are sequential) and its
    latency is counted from that moment.  The first n_warmup completed
    requests are excluded from the statistics."""
    total = n_requests + n_warmup
    arrivals = poisson_arrivals(total, rate, seed)
    rng = np.random.default_rng(seed + 1)
    idle = threading.Condition()
    done_list: List[Request] = []

    def on_done(r: Request):
        with idle:
            r.traj.busy = False
            done_list.append(r)
            idle.notify_all()

    scheduler.on_done = on_done
    t0 = time.perf_counter()
    issued = 0
    while issued < total:
        target = t0 + arrivals[issued]
        now = time.perf_counter()
        if target > now:
            time.sleep(target - now)
        with idle:
            while True:
                cand = [t for t in trajs if not t.busy
                        and (max_steps is None or t.next_step < max_steps)]
                if cand:
                    break
                if not idle.wait(timeout):
                    raise TimeoutError("no trajectory became idle")
            tr = cand[int(rng.integers(len(cand)))]
            tr.busy = True
        step = tr.next_step
        tr.next_step += 1
        req = Request(tr, step, step_coords(tr.ref, tr.spec, step))
        req.footprint = tr.footprint(mixed)
        req.t_arrive = time.perf_counter()
        scheduler.submit(req)
        issued += 1
    if not scheduler.wait_idle(timeout):
        raise TimeoutError("stream did not drain")
    with idle:
        while len(done_list) < total:
            idle.wait(1.0)
    done_sorted = sorted(done_list, key=lambda r: r.t_done)
    timed = done_sorted[n_warmup:]
    errors = [r.error for r in done_list if r.error]
    lat = [r.latency for r in timed if not r.error]
    span = (timed[-1].t_done - done_sorted[n_warmup - 1].t_done) if n_warmup > 0 and timed \
        else (timed[-1].t_done - t0 if timed else float("nan"))
    return {
        "requests": len(timed),
        "errors": len(errors),
        "first_error": errors[0] if errors else None,
        "throughput_per_s": len(timed) / span if span > 0 else float("nan"),
        "p50_ms": 1e3 * percentile(lat, 50),
        "p99_ms": 1e3 * percentile(lat, 99),
        "mean_ms": 1e3 * float(np.mean(lat)) if lat else float("nan"),
        "max_inflight": scheduler.max_inflight,
        "peak_admitted_bytes": scheduler.adm.peak,
        "done": done_list,
    }


# ------------------------------------------------------------- GPU executor

class RisExecutor:
    """Runs requests on the library: one context (own stream) per slot.

    Per trajectory it keeps on the device: C [nao][nmo], the orbital
    energies, and a pair of amplitude buffers [nstates][nocc][nvir] (the
    last step's X, which seeds the next Davidson search, and the one the
    current step writes).  `evict` drops that state (the next step starts
    cold from the MO data on the host)."""

    def __init__(self, nslots: int, precision: str = "mixed", device: int = 0,
                 use_guess: bool = True, **opts):
        import torch

        from . import ris
        self.torch = torch
        self.ris = ris
        self.device = device
        self.mixed = precision == "mixed"
        self.use_guess = use_guess
        o = dict(opts)
        o.setdefault("precision", ris.MIXED if self.mixed else ris.FP64)
        o.setdefault("device", device)
        self.ctx = [ris.Context(**o) for _ in range(nslots)]
        self.shell_cache: Dict[int, tuple] = {}
        self.lock = threading.Lock()

    def close(self):
        for c in self.ctx:
            c.close()

    def resident_bytes(self, tr: Trajectory) -> int:
        dm = tr.dims
        nmo = tr.mol.C.shape[1]
        return 8 * (dm["nao"] * nmo + nmo + 2 * tr.spec.nstates * dm["nocc"] * (nmo - dm["nocc"]))

    def make_resident(self, tr: Trajectory):
        torch = self.torch
        dev = f"cuda:{self.device}"
        nocc = tr.mol.nocc
        nvir = tr.mol.C.shape[1] - nocc
        ns = tr.spec.nstates
        tr.state = {
            "C": torch.as_tensor(tr.mol.C, dtype=torch.float64).to(dev).contiguous(),
            "eps": torch.as_tensor(tr.mol.mo_energy, dtype=torch.float64).to(dev).contiguous(),
            "X": [torch.zeros((ns, nocc, nvir), dtype=torch.float64, device=dev) for _ in range(2)],
            "om": torch.zeros(ns, dtype=torch.float64, device=dev),
            "have_X": False,
            "cur": 0,
        }
        torch.cuda.synchronize(self.device)

    def evict(self, tr: Trajectory):
        tr.state = None

    def _shells(self, tr: Trajectory):
        with self.lock:
            c = self.shell_cache.get(tr.spec.tid)
            if c is None:
                c = tuple(self.ris._shells(a) for a in (tr.mol.shells, tr.mol.aux_j, tr.mol.aux_k))
                self.shell_cache[tr.spec.tid] = c
            return c

    def __call__(self, slot: int, req: Request) -> Tuple[dict, int]:
        tr = req.traj
        ctx = self.ctx[slot]
        if tr.state is None:
            self.make_resident(tr)
        s = tr.state
        spec = tr.spec
        ns = spec.nstates
        sh, aj, ak = self._shells(tr)
        try:
            ctx.build_aux(req.coords, sh, aj, ak)
            ctx.build_B(s["C"], s["eps"], tr.mol.nocc)
            out = s["X"][1 - s["cur"]]
            if self.use_guess and s["have_X"]:
                ctx.excite_guess(ns, s["X"][s["cur"]], out=(s["om"], out, None))
            else:
                ctx.excite(ns, out=(s["om"], out, None))
            signs = np.ones(ns, dtype=np.int32)
            if s["have_X"]:  # phases consistent with the previous step
                signs = ctx.phase_align(s["X"][s["cur"]], X_out=out)
            s["cur"] = 1 - s["cur"]
            s["have_X"] = True
            grad = ctx.gradient([spec.active])[0]
            nac = ctx.nac(spec.pairs) if spec.pairs else np.zeros((0, ctx.natm, 3))
            v = step_velocities(tr.mol.elements, spec, req.step)
            T = ctx.time_coupling(nac, v) if len(spec.pairs) else np.zeros(0)
            omega = s["om"].cpu().numpy()
            st = ctx.stats()
        finally:
            ctx.trim()
        return ({"omega": omega, "grad": grad, "nac": nac, "T": T, "signs": signs,
                 "n_iter": int(st["n_iter"]), "n_products": int(st["n_products"])},
                int(st["bytes_peak"]))


def build_trajectories(specs: Sequence[TrajectorySpec]) -> List[Trajectory]:
    """Molecules (geometry, basis, MOs at the reference geometry) for each spec;
    trajectories with the same molecule and seed share nothing but are
    built independently."""
    out = []
    for sp in specs:
        mol = synth.serving_molecule(sp.kind, sp.size, sp.seed)
        out.append(Trajectory(sp, mol, mol.coords.copy()))
    return out


def serve(specs: Sequence[TrajectorySpec], n_requests: int, n_warmup: int, rate: float,
          nslots: int, budget_bytes: int, precision: str = "mixed", use_guess: bool = True,
          seed: int = 7, device: int = 0, max_steps: Optional[int] = None, **opts) -> dict:
    """Serve a stream end to end on one GPU; returns statistics and the requests."""
    trajs = build_trajectories(specs)
    ex = RisExecutor(nslots, precision, device, use_guess, **opts)
    adm = Admission(budget_bytes)
    for tr in trajs:
        tr.resident_bytes = ex.resident_bytes(tr)
        adm.reside(tr.resident_bytes)
        ex.make_resident(tr)
    sch = Scheduler(nslots, adm, ex)
    try:
        res = run_stream(trajs, sch, n_requests, n_warmup, rate, seed, precision == "mixed",
                         max_steps=max_steps)
    finally:
        sch.close()
        ex.close()
    res["trajectories"] = trajs
    return res
