"""FP64 CPU oracle for the TRED hot path (arXiv 2602.12052) -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference
leg may import this package.  The CUDA product path never imports, loads or calls
it, and shares no code with it; the two meet only through the seeded inputs of
``synth``.

The arithmetic lives in ``tred_oracle.c`` (plain loops, binary64); this module is
argument marshalling and composition of those steps in the paper's order
(Fig. flowchart: transport -> raster [Q] -> bin -> convolve [I] -> electrode gather ->
readout).  Each function names the passage it follows.

Parity status: every function is pinned by tests/test_oracle_*.py (see the header of
``tred_oracle.c`` for the list of pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tred_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
               "-fopenmp", "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", _LIB, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _setup(_lib)
    return _lib


class Params(ctypes.Structure):
    _fields_ = [
        ("pitch_cm", ctypes.c_float), ("n_sub", ctypes.c_int32),
        ("tick_us", ctypes.c_float),
        ("npx_x", ctypes.c_int32), ("npx_y", ctypes.c_int32), ("nt", ctypes.c_int32),
        ("bp", ctypes.c_int32), ("bt", ctypes.c_int32),
        ("v_cm_per_us", ctypes.c_float), ("DL_cm2_per_s", ctypes.c_float),
        ("DT_cm2_per_s", ctypes.c_float), ("lifetime_us", ctypes.c_float),
        ("sigma0_cells_xy", ctypes.c_float), ("sigma0_ticks", ctypes.c_float),
        ("nsigma", ctypes.c_float), ("gl_order", ctypes.c_int32),
        ("effq_mode", ctypes.c_int32),
    ]


DEP_DTYPE = np.dtype([
    ("mu", "<f8", 3), ("sig", "<f8", 3), ("q", "<f8"),
    ("lo", "<i4", 3), ("hi", "<i4", 3), ("valid", "<i4"),
], align=True)

_P = ctypes.c_void_p


def _setup(L):
    L.orc_gl_rule.argtypes = [ctypes.c_int, _P, _P]
    L.orc_gl_rule.restype = ctypes.c_int
    L.orc_drift.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]
    L.orc_drift.restype = None
    L.orc_weights_gl.argtypes = [ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, _P]
    L.orc_weights_tent.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, _P]
    L.orc_block_counts.argtypes = [_P, ctypes.c_int, _P, _P]
    L.orc_block_counts.restype = ctypes.c_long
    L.orc_block_deposits.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int32, _P, ctypes.c_int]
    L.orc_block_deposits.restype = ctypes.c_int
    L.orc_qeff_blocks.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int, _P, _P]
    L.orc_pixel_currents.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _P, _P]
    L.orc_active_pixels.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int, _P]
    L.orc_active_pixels.restype = ctypes.c_int
    L.orc_readout.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_double,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_double, _P, _P, _P, ctypes.c_long, _P]
    L.orc_readout.restype = ctypes.c_long
    L.orc_num_threads.restype = ctypes.c_int
    L.orc_weights_gl_grad.argtypes = [ctypes.c_int, _P, _P, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, _P, _P, _P]
    L.orc_adjoint.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              _P, _P, _P]
    L.orc_param_grads.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]
    L.orc_drift_lines.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.orc_drift_lines.restype = None
    L.orc_line_density.argtypes = [_P, _P, _P, ctypes.c_double, _P]
    L.orc_line_density.restype = ctypes.c_double
    L.orc_qeff_line_blocks.argtypes = [_P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int, _P, _P]
    L.orc_currents_from_qeff.argtypes = [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _P, _P]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def params(cfg, effq_mode: int = 0, **over) -> Params:
    """Oracle parameters from a ``synth.Config`` (binary32 constants)."""
    p = Params(
        pitch_cm=cfg.pitch_cm, n_sub=cfg.n_sub, tick_us=cfg.tick_us,
        npx_x=cfg.npx, npx_y=cfg.npx, nt=cfg.nt, bp=cfg.bp, bt=cfg.bt,
        v_cm_per_us=cfg.v_cm_per_us, DL_cm2_per_s=cfg.DL_cm2_per_s,
        DT_cm2_per_s=cfg.DT_cm2_per_s, lifetime_us=cfg.lifetime_us,
        sigma0_cells_xy=cfg.sigma0_cells_xy, sigma0_ticks=cfg.sigma0_ticks,
        nsigma=cfg.nsigma, gl_order=cfg.gl_order, effq_mode=effq_mode)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def num_threads() -> int:
    return lib().orc_num_threads()


def gl_rule(n: int):
    """N-point Gauss-Legendre nodes (ascending) and weights on [-1, 1] (Sec. II-C)."""
    xi = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gl_rule(n, _ptr(xi), _ptr(w)) != 0:
        raise ValueError("gl order out of range")
    return xi, w


def drift(p: Params, dep: dict) -> np.ndarray:
    """Transport [A;D] per deposit (Sec. II-A): mean, width, charge, window."""
    n = len(dep["x"])
    out = np.zeros(n, dtype=DEP_DTYPE)
    arrs = [np.ascontiguousarray(dep[k], dtype=np.float32) for k in ("x", "y", "z", "t0", "ne")]
    lib().orc_drift(ctypes.byref(p), n, *[_ptr(a) for a in arrs], _ptr(out))
    return out


def axis_weights(p: Params, d, axis: int) -> np.ndarray:
    """Effective-charge weights of one drifted deposit on one axis, g = lo-1..hi+1."""
    lo, hi = int(d["lo"][axis]), int(d["hi"][axis])
    e = np.zeros(hi - lo + 3)
    if p.effq_mode == 1:
        lib().orc_weights_tent(float(d["mu"][axis]), float(d["sig"][axis]), lo, hi, _ptr(e))
    else:
        xi, w = gl_rule(p.gl_order)
        lib().orc_weights_gl(p.gl_order, _ptr(xi), _ptr(w), float(d["mu"][axis]),
                             float(d["sig"][axis]), lo, hi, _ptr(e))
    return e


def weights_gl(nl: int, mu: float, sig: float, lo: int, hi: int) -> np.ndarray:
    xi, w = gl_rule(nl)
    e = np.zeros(hi - lo + 3)
    lib().orc_weights_gl(nl, _ptr(xi), _ptr(w), mu, sig, lo, hi, _ptr(e))
    return e


def weights_tent(mu: float, sig: float, lo: int, hi: int) -> np.ndarray:
    e = np.zeros(hi - lo + 3)
    lib().orc_weights_tent(mu, sig, lo, hi, _ptr(e))
    return e


def block_counts(p: Params, d: np.ndarray):
    """Occupancy of every block of the plane (Sec. III-B-1); returns (counts, pairs)."""
    nb = (p.npx_x // p.bp) * (p.npx_y // p.bp) * (p.nt // p.bt)
    counts = np.zeros(nb, dtype=np.int32)
    pairs = lib().orc_block_counts(ctypes.byref(p), len(d), _ptr(d), _ptr(counts))
    return counts, int(pairs)


def active_blocks(p: Params, d: np.ndarray):
    """Sorted active block ids and their occupancy."""
    counts, _ = block_counts(p, d)
    ids = np.nonzero(counts)[0].astype(np.int32)
    return ids, counts[ids]


def block_deposits(p: Params, d: np.ndarray, block: int) -> np.ndarray:
    cap = len(d)
    idx = np.zeros(max(cap, 1), dtype=np.int32)
    m = lib().orc_block_deposits(ctypes.byref(p), len(d), _ptr(d), int(block), _ptr(idx), cap)
    return idx[:m].copy()


def qeff_blocks(p: Params, d: np.ndarray, blocks) -> np.ndarray:
    """Effective charge of the listed blocks, [nb][ns][ns][bp][bp][bt] (Eq. eff_q)."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    q = np.zeros((len(blocks), p.n_sub, p.n_sub, p.bp, p.bp, p.bt))
    lib().orc_qeff_blocks(ctypes.byref(p), len(d), _ptr(d), len(blocks), _ptr(blocks), _ptr(q))
    return q


def pixel_currents(p: Params, d: np.ndarray, resp: np.ndarray, pixel_ids) -> np.ndarray:
    """Induced current [npix][nt] on the listed pixels (Sec. II-D)."""
    resp = np.ascontiguousarray(resp, dtype=np.float32)
    kp, nr = resp.shape[0], resp.shape[-1]
    pixel_ids = np.ascontiguousarray(pixel_ids, dtype=np.int32)
    w = np.zeros((len(pixel_ids), p.nt))
    lib().orc_pixel_currents(ctypes.byref(p), len(d), _ptr(d), _ptr(resp), kp, nr,
                             len(pixel_ids), _ptr(pixel_ids), _ptr(w))
    return w


def active_pixels(p: Params, blocks, kp: int) -> np.ndarray:
    """Sorted ids (py * npx_x + px) of the pixels in active blocks' output footprint."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    flags = np.zeros(p.npx_x * p.npx_y, dtype=np.uint8)
    lib().orc_active_pixels(ctypes.byref(p), len(blocks), _ptr(blocks), kp, _ptr(flags))
    return np.nonzero(flags)[0].astype(np.int32)


def readout(pixel_ids, wave: np.ndarray, threshold: float, clock: int, hold: int,
            reset: int, tol: float | None = None, mode: int = 0, n_samples: int = 1):
    """Pixel readout (Sec. II-E): mode 0 trigger-reset, mode 1 ``n_samples`` successive
    digitisations per trigger without intervening resets, mode 2 fixed-charge
    integration (quanta of ``threshold``).  Returns (pixel, tick, charge) arrays sorted
    by (pixel, tick) and, per pixel, the first tested edge whose charge is within
    ``tol`` (default 1e-4 * threshold) of the threshold, or -1."""
    pixel_ids = np.ascontiguousarray(pixel_ids, dtype=np.int32)
    wave = np.ascontiguousarray(wave, dtype=np.float64)
    npix, nt = wave.shape
    tol = 1e-4 * threshold if tol is None else tol
    if mode == 2:
        cap = max(1, npix * (nt // max(1, clock) + 1))
    else:
        cap = max(1, npix * n_samples * (nt // max(1, hold + reset + 1) + 1))
    hp = np.zeros(cap, np.int32)
    ht = np.zeros(cap, np.int32)
    hc = np.zeros(cap, np.float64)
    amb = np.zeros(npix, np.int32)
    m = lib().orc_readout(npix, nt, _ptr(pixel_ids), _ptr(wave), float(threshold), clock,
                          hold, reset, int(mode), int(n_samples), float(tol), _ptr(hp), _ptr(ht),
                          _ptr(hc), cap, _ptr(amb))
    assert m <= cap
    return hp[:m].copy(), ht[:m].copy(), hc[:m].copy(), amb


def simulate(cfg, dep: dict, resp: np.ndarray, effq_mode: int = 0, pixels=None):
    """The whole path in the paper's order (Fig. flowchart).  With ``pixels`` given, only
    those pixels' currents are computed (sampled parity at full size)."""
    p = params(cfg, effq_mode=effq_mode)
    d = drift(p, dep)
    ids, counts = active_blocks(p, d)
    pix = active_pixels(p, ids, resp.shape[0]) if pixels is None else np.asarray(pixels, np.int32)
    wave = pixel_currents(p, d, resp, pix)
    return {"params": p, "deps": d, "block_ids": ids, "block_counts": counts,
            "pixel_ids": pix, "waveforms": wave}


# ----------------------------------------------------------------- differentiation
def weights_gl_grad(nl: int, mu: float, sig: float, lo: int, hi: int):
    """GL weights and their derivatives in mu and sigma (window held fixed)."""
    xi, w = gl_rule(nl)
    e, dm, ds = (np.zeros(hi - lo + 3) for _ in range(3))
    lib().orc_weights_gl_grad(nl, _ptr(xi), _ptr(w), mu, sig, lo, hi, _ptr(e), _ptr(dm), _ptr(ds))
    return e, dm, ds


def adjoint(p: Params, d: np.ndarray, resp: np.ndarray, pixel_ids, resid: np.ndarray) -> np.ndarray:
    """dL/d(q, mu_x, mu_y, mu_t, sig_x, sig_y, sig_t) per deposit for L = 1/2 sum r^2,
    given r = dL/dI on the listed pixels (Sec. V-C; windows held fixed)."""
    resp = np.ascontiguousarray(resp, dtype=np.float32)
    kp, nr = resp.shape[0], resp.shape[-1]
    pixel_ids = np.ascontiguousarray(pixel_ids, dtype=np.int32)
    resid = np.ascontiguousarray(resid, dtype=np.float64)
    g = np.zeros((len(d), 7))
    lib().orc_adjoint(ctypes.byref(p), len(d), _ptr(d), _ptr(resp), kp, nr, len(pixel_ids),
                      _ptr(pixel_ids), _ptr(resid), _ptr(g))
    return g


def param_grads(p: Params, dep: dict, d: np.ndarray, grad7: np.ndarray):
    """Per deposit dL/d(x, y, t0, ne) and global dL/d(DL, DT, tau) from grad7."""
    z = np.ascontiguousarray(dep["z"], dtype=np.float32)
    ne = np.ascontiguousarray(dep["ne"], dtype=np.float32)
    out = np.zeros((len(d), 4))
    glob = np.zeros(3)
    lib().orc_param_grads(ctypes.byref(p), len(d), _ptr(z), _ptr(ne), _ptr(d),
                          _ptr(np.ascontiguousarray(grad7)), _ptr(out), _ptr(glob))
    return out, glob


def currents_frozen(p: Params, dep: dict, frozen: np.ndarray, resp, pixel_ids):
    """Pixel currents with the windows of `frozen` (the unperturbed drift) kept: the
    loss is then smooth in the inputs, as the adjoint assumes."""
    d = drift(p, dep)
    d["lo"] = frozen["lo"]
    d["hi"] = frozen["hi"]
    return pixel_currents(p, d, resp, pixel_ids)


# ----------------------------------------------------------------- line segments
LINE_DTYPE = np.dtype([("d", DEP_DTYPE), ("p0", "<f8", 3), ("p1", "<f8", 3)], align=True)
SHORT_FRAC = 0.1          # segments shorter than this many sigma on every axis are points


def drift_lines(p: Params, seg: dict) -> np.ndarray:
    """Transport of line segments (Sec. II-A, II-C): both endpoints in grid units, one
    width per axis at the midpoint's drift time, window over both endpoints."""
    n = len(seg["x0"])
    out = np.zeros(n, dtype=LINE_DTYPE)
    f = {k: np.ascontiguousarray(seg[k], dtype=np.float32) for k in ("x0", "y0", "z0", "x1", "y1", "z1", "t0", "ne")}
    lib().orc_drift_lines(ctypes.byref(p), n, _ptr(f["x0"]), _ptr(f["y0"]), _ptr(f["z0"]), _ptr(f["x1"]),
                          _ptr(f["y1"]), _ptr(f["z1"]), _ptr(f["t0"]), _ptr(f["ne"]), _ptr(out))
    return out


def line_density(p0, p1, sig, x, frac: float = SHORT_FRAC) -> float:
    """Normalised Eq. qline (grid units) at x; the point Gaussian for short segments."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (p0, p1, sig, x)]
    return lib().orc_line_density(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), float(frac), _ptr(a[3]))


def line_windows(lines: np.ndarray) -> np.ndarray:
    """The per-segment window records (DEP_DTYPE) that drive the block functions."""
    return np.ascontiguousarray(lines["d"])


def qeff_line_blocks(p: Params, lines: np.ndarray, blocks, frac: float = SHORT_FRAC) -> np.ndarray:
    """Effective charge of the listed blocks from line segments, [nb][ns][ns][bp][bp][bt]."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    q = np.zeros((len(blocks), p.n_sub, p.n_sub, p.bp, p.bp, p.bt))
    lib().orc_qeff_line_blocks(ctypes.byref(p), len(lines), _ptr(lines), float(frac), len(blocks),
                               _ptr(blocks), _ptr(q))
    return q


def currents_from_qeff(p: Params, blocks, qeff: np.ndarray, resp: np.ndarray, pixel_ids) -> np.ndarray:
    """Eq. interlaced from block-stored effective charge on the listed pixels."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    qeff = np.ascontiguousarray(qeff, dtype=np.float64)
    resp = np.ascontiguousarray(resp, dtype=np.float32)
    kp, nr = resp.shape[0], resp.shape[-1]
    pixel_ids = np.ascontiguousarray(pixel_ids, dtype=np.int32)
    w = np.zeros((len(pixel_ids), p.nt))
    lib().orc_currents_from_qeff(ctypes.byref(p), len(blocks), _ptr(blocks), _ptr(qeff), _ptr(resp), kp, nr,
                                 len(pixel_ids), _ptr(pixel_ids), _ptr(w))
    return w


def simulate_lines(cfg, seg: dict, resp: np.ndarray, pixels=None, frac: float = SHORT_FRAC):
    """The path for line segments: transport, blocks, effective charge, currents."""
    p = params(cfg)
    L = drift_lines(p, seg)
    w = line_windows(L)
    ids, counts = active_blocks(p, w)
    q = qeff_line_blocks(p, L, ids, frac)
    pix = active_pixels(p, ids, resp.shape[0]) if pixels is None else np.asarray(pixels, np.int32)
    wave = currents_from_qeff(p, ids, q, resp, pix)
    return {"params": p, "lines": L, "block_ids": ids, "block_counts": counts, "qeff": q,
            "pixel_ids": pix, "waveforms": wave}
