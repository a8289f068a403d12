"""CPU checks of the C-ABI library: it builds, loads, and exports every entry
point include/tred.h declares (no compute call: there may be no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tred_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_12052_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["tred_drift", "tred_effq", "tred_blockbin", "tred_convolve",
                     "tred_gather_pixels", "tred_readout", "tred_create", "tred_destroy",
                     "tred_set_response", "tred_sync_status"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2602_12052_b300 import abi
    assert sorted(abi.EXPORTS) == sorted(n for n in _declared())


def test_create_rejects_bad_geometry_without_gpu(lib):
    """Argument validation runs before any device call."""
    from paper_2602_12052_b300 import abi
    abi.load()
    g = abi.Geometry(pitch_cm=0.44, n_sub=10, tick_us=0.05, npx_x=32, npx_y=32, nt=1024, bp=6,
                     bt=256, kp=9, nr=200, lt=512)
    p = abi.Params(v_cm_per_us=0.16, DL_cm2_per_s=4, DT_cm2_per_s=8.8, lifetime_us=2200,
                   sigma0_cells_xy=0.5, sigma0_ticks=0.5, nsigma=4, max_drift_cm=50, gl_order=2)
    h = ctypes.c_void_p()
    rc = abi.load().tred_create(ctypes.byref(g), ctypes.byref(p), 10, 10, 10, ctypes.byref(h))
    assert rc == abi.TRED_ERR_INVALID_ARG and not h.value


def test_noalloc_blockbin_rejects_bad_arguments_without_gpu(lib):
    """The allocation-free binning checks its arguments as the handle path does, before
    any device call: a deposit set with one null array, a negative event count, a
    geometry tred_create rejects and a missing output all give TRED_ERR_INVALID_ARG."""
    from paper_2602_12052_b300 import abi
    L = abi.load()

    def geom(**kw):
        base = dict(pitch_cm=0.44, n_sub=10, tick_us=0.05, npx_x=32, npx_y=32, nt=1024, bp=8, bt=256,
                    kp=9, nr=200, lt=512, n_events=0)
        base.update(kw)
        return abi.Geometry(**base)

    fake = ctypes.c_void_p(256)                       # never dereferenced: the checks come first
    full = abi.Deposits(**{f: 256 for f in abi.DEPOSIT_FIELDS})
    one_null = abi.Deposits(**{f: (None if f == "hi_x" else 256) for f in abi.DEPOSIT_FIELDS})

    def call(g, n, deps, out=fake):
        return L.tred_blockbin_noalloc(ctypes.byref(g), n, ctypes.byref(deps) if deps is not None else None,
                                       out, fake, fake, fake, 64, 512, fake, fake, None)

    assert call(geom(), 10, one_null) == abi.TRED_ERR_INVALID_ARG
    assert call(geom(), 10, None) == abi.TRED_ERR_INVALID_ARG
    assert call(geom(n_events=-1), 10, full) == abi.TRED_ERR_INVALID_ARG
    assert call(geom(n_events=2), 10, full) == abi.TRED_ERR_INVALID_ARG
    assert call(geom(n_sub=1 << 20), 10, full) == abi.TRED_ERR_INVALID_ARG     # n_sub * npx overflow
    assert call(geom(bp=6), 10, full) == abi.TRED_ERR_INVALID_ARG
    assert call(geom(), 10, full, out=None) == abi.TRED_ERR_INVALID_ARG
    assert call(geom(), -1, full) == abi.TRED_ERR_INVALID_ARG


def test_fp32_peak_rejects_bad_arguments_without_gpu(lib):
    """The FMA-peak measurement checks its arguments before any device call."""
    from paper_2602_12052_b300 import abi
    L = abi.load()
    tf = ctypes.c_double()
    assert L.tred_fp32_peak(None, 1 << 20, 16, None, ctypes.byref(tf), None) == abi.TRED_ERR_INVALID_ARG
    assert L.tred_fp32_peak(ctypes.c_void_p(256), 1 << 20, 0, None, ctypes.byref(tf), None) == abi.TRED_ERR_INVALID_ARG
    assert L.tred_fp32_peak(ctypes.c_void_p(256), 1 << 20, 16, None, None, None) == abi.TRED_ERR_INVALID_ARG
