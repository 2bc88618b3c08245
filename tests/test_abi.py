"""CPU checks of the C ABI: the library builds, loads and exports every
function include/ris.h declares; host-side argument validation."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ris.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ris_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris.load()


def test_header_declares_the_boundary():
    names = _declared()
    for f in ["ris_build_aux", "ris_build_B", "ris_excite", "ris_gradient", "ris_nac",
              "ris_create", "ris_destroy", "ris_last_error", "ris_options_default"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for f in _declared():
        assert hasattr(lib, f), f


def test_binding_lists_the_same_symbols():
    from paper_2511_18233_gb300 import ris
    assert sorted(ris.EXPORTS) == _declared()


def test_options_defaults(lib):
    from paper_2511_18233_gb300 import ris
    o = ris.options()
    assert o.cx == 0.25 and o.conv_tol == 1e-10 and o.max_iter == 100
    assert o.precision == ris.FP64 and o.rpa == 0 and o.screen_thr == 1e-14
    assert o.mixed_tol == 1e-6 and o.refine == 0 and o.profile == 0
    assert o.precond == 0 and o.mo_window == 0.0 and o.deriv_prefetch == 1
    assert o.emu_f64 == 1 and o.eig_fp32 == 0
    assert o.stream == 0 and o.stream_block == 0 and o.occ_block == 0
    assert o.subspace_ff == 1


def test_create_rejects_bad_options(lib):
    import ctypes
    from paper_2511_18233_gb300 import ris
    h = ctypes.c_void_p()
    o = ris.options(precision=7)
    assert lib.ris_create(ctypes.byref(h), ctypes.byref(o)) == -1
    o = ris.options(conv_tol=-1.0)
    assert lib.ris_create(ctypes.byref(h), ctypes.byref(o)) == -1
    o = ris.options(deriv_prefetch=2)
    assert lib.ris_create(ctypes.byref(h), ctypes.byref(o)) == -1
    o = ris.options(precond=3)
    assert lib.ris_create(ctypes.byref(h), ctypes.byref(o)) == -1
    o = ris.options(eig_fp32=2)
    assert lib.ris_create(ctypes.byref(h), ctypes.byref(o)) == -1
    assert lib.ris_create(None, None) == -1
    assert lib.ris_get_stats(None, None, 1) == -1
    lib.ris_destroy(None)  # ignored


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2511_18233_gb300 import ris
    saved = ris._lib
    try:
        ris._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            ris.load(str(tmp_path / "missing.so"))
    finally:
        ris._lib = saved
