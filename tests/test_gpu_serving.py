"""Serving form on the GPU: every result is the same alone and in the mix.

A few trajectories of different molecules are served concurrently (one
library context and CUDA stream per slot, requests overlapping on the
device, Davidson seeded from each trajectory's resident amplitudes).  Each
trajectory is then replayed alone on one slot.  Tolerances are those of the
mixed-precision path: 1e-6 Ha for energies, 1e-5 Ha/bohr for gradients and
for the coupling numerators dE_IJ/dR = g_IJ (omega_J - omega_I), so 1e-5/gap
for the couplings themselves; one request is also checked against the FP64
oracle with the same tolerances.
"""
import numpy as np
import pytest

from paper_2511_18233_gb300 import serve, synth

gpu = pytest.mark.gpu

E_TOL, G_TOL = 1e-6, 1e-5


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


def _specs():
    return [serve.TrajectorySpec(0, "chain", 4, 5, 1, 11),
            serve.TrajectorySpec(1, "chain", 12, 6, 2, 12),
            serve.TrajectorySpec(2, "chain", 20, 8, 0, 13),
            serve.TrajectorySpec(3, "flake", 4.5, 5, 3, 14)]


NSTEP = 3


def _run(specs, nslots, rate, use_guess=True, evict_at=None):
    trajs = serve.build_trajectories(specs)
    ex = serve.RisExecutor(nslots, "mixed", 0, use_guess)
    adm = serve.Admission(200 << 30)
    for tr in trajs:
        ex.make_resident(tr)
    if evict_at is not None:
        base = ex.__call__

        def call(slot, req):
            if req.step == evict_at:
                ex.evict(req.traj)
            return base(slot, req)
        executor = call
    else:
        executor = ex
    sch = serve.Scheduler(nslots, adm, executor)
    try:
        res = serve.run_stream(trajs, sch, n_requests=len(trajs) * NSTEP, n_warmup=0,
                               rate=rate, seed=5, mixed=True, max_steps=NSTEP, timeout=600)
    finally:
        sch.close()
        ex.close()
    assert res["errors"] == 0, res["first_error"]
    return {(r.traj.spec.tid, r.step): r for r in res["done"]}, res


@pytest.fixture(scope="module")
def mixed_run(ris_mod):
    return _run(_specs(), nslots=4, rate=1000.0)


def _nac_close(nac, ref, omega, pairs, signs=None, ref_signs=None):
    """Couplings compared with the phases factored out: a state's sign is
    set by the previous step (phase tracking), the reference's by its own
    convention or history."""
    for k, (i, j) in enumerate(pairs):
        gap = abs(omega[j] - omega[i])
        f = 1.0 if signs is None else float(signs[i] * signs[j])
        fr = 1.0 if ref_signs is None else float(ref_signs[i] * ref_signs[j])
        assert np.max(np.abs(f * nac[k] - fr * ref[k])) * gap <= G_TOL


def _same(a, b):
    ra, rb = a.result, b.result
    assert np.max(np.abs(ra["omega"] - rb["omega"])) <= E_TOL
    assert np.max(np.abs(ra["grad"] - rb["grad"])) <= G_TOL
    _nac_close(ra["nac"], rb["nac"], rb["omega"], a.traj.spec.pairs, ra["signs"], rb["signs"])


@gpu
def test_mix_overlaps_requests(mixed_run):
    got, res = mixed_run
    assert len(got) == len(_specs()) * NSTEP
    assert res["max_inflight"] >= 2
    # requests of different trajectories were on the device at the same time
    reqs = list(got.values())
    overlap = any(a.t_start < b.t_done and b.t_start < a.t_done
                  for i, a in enumerate(reqs) for b in reqs[i + 1:] if a.traj is not b.traj)
    assert overlap


@gpu
def test_each_result_same_alone_and_in_mix(mixed_run):
    got, _ = mixed_run
    for sp in _specs():
        alone, _ = _run([sp], nslots=1, rate=1000.0)
        for s in range(NSTEP):
            _same(got[(sp.tid, s)], alone[(sp.tid, s)])


@gpu
def test_cold_start_after_eviction_matches(mixed_run):
    got, _ = mixed_run
    cold, _ = _run(_specs(), nslots=4, rate=1000.0, evict_at=1)
    for k, r in cold.items():
        _same(r, got[k])


@gpu
def test_request_matches_fp64_oracle(mixed_run, oracle):
    got, _ = mixed_run
    sp = _specs()[0]
    tr = serve.build_trajectories([sp])[0]
    r = got[(sp.tid, 1)]
    xyz = serve.step_coords(tr.ref, sp, 1)
    mol = tr.mol
    orc = oracle.RisOracle(xyz, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc)
    w, X = orc.tda_dense(sp.nstates)
    assert np.max(np.abs(r.result["omega"] - w)) <= E_TOL
    g = orc.gradients([sp.active], X)[0]
    assert np.max(np.abs(r.result["grad"] - g)) <= G_TOL
    nac = orc.nacs(sp.pairs, w, X)
    _nac_close(r.result["nac"], nac, w, sp.pairs, r.result["signs"])


@gpu
def test_footprint_estimate_bounds_measured_peak(mixed_run):
    got, _ = mixed_run
    for sp in _specs():
        tr = got[(sp.tid, 0)].traj
        dm = tr.dims
        est = serve.footprint_bytes(dm["nao"], dm["nocc"], dm["nJ"], dm["nK"], dm["nU"],
                                    sp.nstates, 1 + len(sp.pairs), True)
        assert tr.measured > 0
        assert tr.measured <= est <= 4 * tr.measured + (64 << 20)
