"""The C-ABI library builds, loads and exports every symbol include/ttn.h declares.

No CUDA call is made (this runs on machines without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ttn_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native
    return native.load()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("ttn_create", "ttn_set_hamiltonian", "ttn_apply_pulse", "ttn_tdvp_step",
                     "ttn_fidelity", "ttn_measure", "ttn_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2210_03763_gb300 import native
    bound = {n for n, _, _ in native.SIGNATURES}
    assert set(_declared_symbols()) <= bound


def test_invalid_create_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    assert lib.ttn_create(2, 2, 2, 16, ctypes.byref(h)) == 1      # levels != 3
    assert lib.ttn_create(2, 2, 3, 0, ctypes.byref(h)) == 1       # chi < 1
    assert lib.ttn_create(64, 64, 3, 8, ctypes.byref(h)) == 1     # > 1024 atoms
    assert lib.ttn_create(0, 2, 3, 8, ctypes.byref(h)) == 1
    assert not h.value


def test_pulse_struct_matches_header():
    from paper_2210_03763_gb300.workloads import PULSE_DTYPE
    text = open(os.path.join(ROOT, "include", "ttn.h")).read()
    assert "Layout: 64 bytes" in text and PULSE_DTYPE.itemsize == 64
    assert PULSE_DTYPE.fields["t0"][1] == 8


def test_missing_library_fails_loudly(monkeypatch):
    # the product path has no CPU fallback: without libttn.so the binding
    # refuses to load
    from paper_2210_03763_gb300 import native
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(ImportError):
        native.load(os.path.join(ROOT, "no_such_dir", "libttn.so"))


def test_selftest_qr_rejects_bad_arguments_without_gpu(lib):
    # size and candidate checks run before any CUDA call
    D = ctypes.POINTER(ctypes.c_double)
    a = (ctypes.c_double * 64)()
    q = (ctypes.c_double * 64)()
    r = (ctypes.c_double * 64)()
    ap, qp, rp = (ctypes.cast(x, D) for x in (a, q, r))
    assert lib.ttn_selftest_qr(ap, 3, 5, None, 0, qp, rp, None, None) == 1      # M < D
    assert lib.ttn_selftest_qr(ap, 4, 0, None, 0, qp, rp, None, None) == 1      # D < 1
    assert lib.ttn_selftest_qr(ap, 8, 300, None, 0, qp, rp, None, None) == 1    # D > 256
    bad = (ctypes.c_int * 2)(0, 9)
    assert lib.ttn_selftest_qr(ap, 8, 2, bad, 2, qp, rp, None, None) == 1       # row 9 of 8
    assert lib.ttn_selftest_qr(None, 8, 2, None, 0, qp, rp, None, None) == 1    # no input
