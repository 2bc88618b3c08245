"""The profile option times kernel classes per context: a context collects
only the records of its own streams, so concurrent contexts (the serving
loop's slots) neither see nor disturb each other's timings."""
import threading

import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


def _run(c, mol, ns=3):
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    c.excite(ns)


@gpu
def test_profile_is_per_context(ris_mod):
    mol = synth.workload(0)
    a = ris_mod.Context(profile=1)
    b = ris_mod.Context()
    _run(a, mol)
    _run(b, mol)
    sa, sb = a.stats(), b.stats()
    assert sa["gemm_ms"] > 0 and sa["int3c_ms"] > 0
    assert sb["gemm_ms"] == 0 and sb["int3c_ms"] == 0
    assert a.stats()["gemm_ms"] == 0  # collected
    a.close()
    b.close()


@gpu
def test_concurrent_profiled_contexts(ris_mod):
    """Several profiled and unprofiled contexts on host threads, each reading
    its statistics after every call: no error, and each profiled context's
    timings cover its own work only."""
    mol = synth.workload(0)
    errors, gemm = [], {}

    def worker(i):
        try:
            c = ris_mod.Context(profile=i % 2)
            tot = 0.0
            for _ in range(4):
                _run(c, mol)
                tot += c.stats()["gemm_ms"]
            gemm[i] = tot
            c.close()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(repr(e))

    th = [threading.Thread(target=worker, args=(i,)) for i in range(6)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert all(gemm[i] > 0 for i in (1, 3, 5))
    assert all(gemm[i] == 0 for i in (0, 2, 4))
    assert np.isfinite(list(gemm.values())).all()
