"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the FP64 oracle.

This module holds no arithmetic of the simulation method itself (no drift, no
effective charge, no convolution).  It only draws the inputs the method consumes:

* point ionisation deposits (x, y, z, t0, n_e) at the midpoints of 0.1 mm steps
  along straight tracks, with Poisson-distributed electron counts, standing in for
  the GEANT4/edep-sim segments of the paper's test sample (Sec. IV-A), which are
  not available here;
* a synthetic field response i[Ky][Kx][jy][jx][tau] on a K_p x K_p pixel
  neighbourhood x n_sub x n_sub impact positions x N_r ticks (Sec. II-B, Fig. frillu:
  impacts at the centres of the n_sub x n_sub sub-cells of a pixel), standing in
  for the COMSOL/pochoir response of the paper.

Everything is drawn with numpy's PCG64 (``np.random.default_rng``) from fixed seeds
and returned as float32 arrays, the precision of the inputs both sides consume.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Config", "CONFIGS", "get_config", "make_deposits", "make_event",
    "make_response", "make_events",
]


@dataclasses.dataclass(frozen=True)
class Config:
    """Geometry, physics and generator settings of one workload."""

    name: str
    # geometry
    pitch_cm: float = 0.44          # pixel pitch a (4.4 mm)
    n_sub: int = 10                 # impact positions per pixel axis
    tick_us: float = 0.05           # sampling tick (50 ns)
    npx: int = 32                   # plane is npx x npx pixels
    nt: int = 1024                  # readout window in ticks
    bp: int = 8                     # block: bp x bp pixels
    bt: int = 256                   # block: bt ticks
    lt: int = 512                   # FFT length along time (>= bt + nr - 1)
    kp: int = 9                     # response neighbourhood (pixels per axis, odd)
    nr: int = 200                   # response length in ticks
    # physics
    v_cm_per_us: float = 0.16       # drift velocity 1.6 mm/us
    DL_cm2_per_s: float = 4.0
    DT_cm2_per_s: float = 8.8
    lifetime_us: float = 2200.0
    sigma0_cells_xy: float = 0.5    # diffusion floor, added in quadrature (cells)
    sigma0_ticks: float = 0.5       # diffusion floor, added in quadrature (ticks)
    nsigma: float = 4.0             # raster half-width in units of sigma
    gl_order: int = 2
    max_drift_cm: float = 50.0      # largest drift distance the capacities cover
    # generator
    kind: str = "single_track"      # single_track | tracks
    n_tracks: int = 1
    min_deposits: int = 0           # keep drawing tracks until N >= this
    track_len_cm: tuple = (5.0, 5.0)
    z_range_cm: tuple = (0.0, 20.0)
    ne_mean: float = 600.0
    step_cm: float = 0.01
    seed: int = 1001
    response_seed: int = 7
    # readout: 0 trigger-reset, 1 successive digitisations, 2 fixed-charge quanta
    threshold_e: float = 5000.0
    clock_ticks: int = 2
    hold_ticks: int = 32
    reset_ticks: int = 2
    readout_mode: int = 0
    n_samples: int = 1

    @property
    def n_blocks(self) -> int:
        return (self.npx // self.bp) ** 2 * (self.nt // self.bt)

    def with_(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


CONFIGS = {
    # One straight 5 cm track in a 32 x 32 pixel plane, 1,024 ticks, GL-2.
    "tiny": Config(name="tiny"),
    # One module plane: 512 x 512 pixels x 6,400 ticks; 200 tracks of log-uniform
    # length in [1, 100] cm, 60 e- per 0.1 mm.
    "module200": Config(
        name="module200", npx=512, nt=6400, kind="tracks", n_tracks=200,
        track_len_cm=(1.0, 100.0), z_range_cm=(0.0, 50.0), ne_mean=60.0, seed=1002),
    # The same generator drawing tracks until at least 1e6 deposits exist.
    "module1M": Config(
        name="module1M", npx=512, nt=6400, kind="tracks", n_tracks=0,
        min_deposits=1_000_000, track_len_cm=(1.0, 100.0), z_range_cm=(0.0, 50.0),
        ne_mean=60.0, seed=1002),
    # A 20-track module plane (a few hundred active blocks): profiling captures.
    "module20": Config(
        name="module20", npx=512, nt=6400, kind="tracks", n_tracks=20,
        track_len_cm=(1.0, 100.0), z_range_cm=(0.0, 50.0), ne_mean=60.0, seed=1020),
    # Spill-scale plane: GL-3, 13 x 13 pixel x 400 tick response, 4 x 4 pixel blocks
    # (so the padded spatial extent stays 16), FFT length 768 = 3 x 256 along time (the
    # smallest 2^a 3^b at or above bt + nr - 1 = 655).
    # Line segments (Sec. II-C, Eq. qline): the tiny track and a 200-track module plane
    # cut into 0.25 cm and 0.3 cm segments (make_segments).
    "tiny_lines": Config(name="tiny_lines"),
    "module_lines": Config(
        name="module_lines", npx=512, nt=6400, kind="tracks", n_tracks=200,
        track_len_cm=(1.0, 100.0), z_range_cm=(0.0, 50.0), ne_mean=60.0, seed=1002),
    "spill_plane": Config(
        name="spill_plane", npx=512, nt=6400, kind="tracks", n_tracks=0,
        min_deposits=290_000, track_len_cm=(1.0, 100.0), z_range_cm=(0.0, 50.0),
        ne_mean=60.0, seed=1005, gl_order=3, kp=13, nr=400, bp=4, bt=256, lt=768),
}


SEG_CM = {"tiny_lines": 0.25, "module_lines": 0.3}


def get_config(name: str, **overrides) -> Config:
    cfg = CONFIGS[name]
    return cfg.with_(**overrides) if overrides else cfg


def _isotropic(rng, n):
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _track_points(start, direction, length, step):
    n = int(math.floor(length / step))
    s = (np.arange(n, dtype=np.float64) + 0.5) * step
    return start[None, :] + s[:, None] * direction[None, :]


def make_deposits(cfg: Config, seed: int | None = None) -> dict:
    """Return float32 SoA deposits {x, y, z, t0, ne} (cm, cm, cm, us, electrons).

    x, y are positions on the anode plane measured from its lower corner; z is the
    distance to the response reference plane (the drift distance).
    """
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    width = cfg.npx * cfg.pitch_cm
    pts = []
    t0s = []
    if cfg.kind == "single_track":
        # Reject until the whole track, widened by 4 pixels, lies in the plane and
        # its z range lies inside z_range_cm.
        margin = 4 * cfg.pitch_cm
        L = cfg.track_len_cm[0]
        while True:
            start = np.array([rng.uniform(0.0, width), rng.uniform(0.0, width),
                              rng.uniform(*cfg.z_range_cm)])
            d = _isotropic(rng, 1)[0]
            end = start + L * d
            lo = np.minimum(start, end)
            hi = np.maximum(start, end)
            if (lo[0] >= margin and hi[0] <= width - margin and lo[1] >= margin
                    and hi[1] <= width - margin and lo[2] >= cfg.z_range_cm[0]
                    and hi[2] <= cfg.z_range_cm[1]):
                break
        p = _track_points(start, d, L, cfg.step_cm)
        pts.append(p)
        # Common start time: the nearest deposit arrives at tick 32, so that the
        # whole event (track, diffusion and response) fits the readout window.
        zmin = float(p[:, 2].min())
        t0 = 32.0 * cfg.tick_us - zmin / cfg.v_cm_per_us
        t0s.append(np.full(len(p), t0))
    else:
        n_total = 0
        k = 0
        while True:
            if cfg.n_tracks and k >= cfg.n_tracks:
                break
            if not cfg.n_tracks and n_total >= cfg.min_deposits:
                break
            lo_len, hi_len = cfg.track_len_cm
            L = math.exp(rng.uniform(math.log(lo_len), math.log(hi_len)))
            start = np.array([rng.uniform(0.0, width), rng.uniform(0.0, width),
                              rng.uniform(*cfg.z_range_cm)])
            d = _isotropic(rng, 1)[0]
            p = _track_points(start, d, L, cfg.step_cm)
            inside = ((p[:, 0] >= 0.0) & (p[:, 0] < width) & (p[:, 1] >= 0.0)
                      & (p[:, 1] < width) & (p[:, 2] >= cfg.z_range_cm[0])
                      & (p[:, 2] <= cfg.z_range_cm[1]))
            p = p[inside]
            pts.append(p)
            t0s.append(np.zeros(len(p)))
            n_total += len(p)
            k += 1
    p = np.concatenate(pts, axis=0) if pts else np.zeros((0, 3))
    t0 = np.concatenate(t0s) if t0s else np.zeros(0)
    ne = rng.poisson(cfg.ne_mean, size=len(p)).astype(np.float64)
    return {
        "x": p[:, 0].astype(np.float32), "y": p[:, 1].astype(np.float32),
        "z": p[:, 2].astype(np.float32), "t0": t0.astype(np.float32),
        "ne": ne.astype(np.float32),
    }


def make_segments(cfg: Config, seg_cm: float, seed: int | None = None) -> dict:
    """Line-segment deposits {x0, y0, z0, x1, y1, z1, t0, ne}: the tracks of
    ``make_deposits`` cut into consecutive segments of ``seg_cm`` (the last piece of a
    track may be shorter), n_e ~ Poisson(ne_mean * length / step_cm).  Segments with
    an endpoint outside the volume are dropped."""
    rng = np.random.default_rng((cfg.seed if seed is None else seed) + 7777)
    width = cfg.npx * cfg.pitch_cm
    a_all, b_all, t_all = [], [], []

    def cut(start, d, L):
        k = np.arange(int(math.ceil(L / seg_cm)))
        s0 = k * seg_cm
        s1 = np.minimum((k + 1) * seg_cm, L)
        return start[None, :] + s0[:, None] * d[None, :], start[None, :] + s1[:, None] * d[None, :]

    def inside(p):
        return ((p[:, 0] >= 0.0) & (p[:, 0] < width) & (p[:, 1] >= 0.0) & (p[:, 1] < width)
                & (p[:, 2] >= cfg.z_range_cm[0]) & (p[:, 2] <= cfg.z_range_cm[1]))
    if cfg.kind == "single_track":
        margin = 4 * cfg.pitch_cm
        L = cfg.track_len_cm[0]
        while True:
            start = np.array([rng.uniform(0.0, width), rng.uniform(0.0, width), rng.uniform(*cfg.z_range_cm)])
            d = _isotropic(rng, 1)[0]
            end = start + L * d
            lo, hi = np.minimum(start, end), np.maximum(start, end)
            if (lo[0] >= margin and hi[0] <= width - margin and lo[1] >= margin and hi[1] <= width - margin
                    and lo[2] >= cfg.z_range_cm[0] and hi[2] <= cfg.z_range_cm[1]):
                break
        a, b = cut(start, d, L)
        t0 = 32.0 * cfg.tick_us - float(min(a[:, 2].min(), b[:, 2].min())) / cfg.v_cm_per_us
        a_all.append(a); b_all.append(b); t_all.append(np.full(len(a), t0))
    else:
        for _ in range(cfg.n_tracks):
            L = math.exp(rng.uniform(math.log(cfg.track_len_cm[0]), math.log(cfg.track_len_cm[1])))
            start = np.array([rng.uniform(0.0, width), rng.uniform(0.0, width), rng.uniform(*cfg.z_range_cm)])
            d = _isotropic(rng, 1)[0]
            a, b = cut(start, d, L)
            keep = inside(a) & inside(b)
            a_all.append(a[keep]); b_all.append(b[keep]); t_all.append(np.zeros(int(keep.sum())))
    a = np.concatenate(a_all) if a_all else np.zeros((0, 3))
    b = np.concatenate(b_all) if b_all else np.zeros((0, 3))
    t0 = np.concatenate(t_all) if t_all else np.zeros(0)
    length = np.linalg.norm(b - a, axis=1)
    ne = rng.poisson(cfg.ne_mean * length / cfg.step_cm).astype(np.float32)
    f = lambda v: np.ascontiguousarray(v, dtype=np.float32)
    return {"x0": f(a[:, 0]), "y0": f(a[:, 1]), "z0": f(a[:, 2]), "x1": f(b[:, 0]), "y1": f(b[:, 1]),
            "z1": f(b[:, 2]), "t0": f(t0), "ne": ne}


def make_event(cfg: Config, seed: int | None = None):
    """Deposits and the matching field response for one workload."""
    return make_deposits(cfg, seed), make_response(cfg)


def make_events(cfg: Config, n_events: int, lo: int, hi: int, seed: int):
    """Uneven events: deposit counts log-uniform in [lo, hi] drawn from ``cfg``'s
    track generator (each event keeps drawing tracks until it reaches its count,
    then is cut to exactly that count)."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(lo), math.log(hi), n_events)).astype(np.int64)
    events = []
    for e, n in enumerate(counts):
        c = cfg.with_(n_tracks=0, min_deposits=int(n))
        dep = make_deposits(c, seed=seed * 1000 + e)
        events.append({k: v[: int(n)] for k, v in dep.items()})
    return events


def make_response(cfg: Config, symmetric: bool = True, seed: int | None = None):
    """Synthetic field response i[Ky][Kx][jy][jx][tau], float32.

    The charge sits at the impact position (jx+1/2)h - a/2 (and likewise in y) of
    pixel K relative to the electrode centre, Delta = K a + lambda_j, and

        i = A exp(-|Delta|^2 / 2 s^2) [exp(-tau dt / tau1(|Delta|)) - beta exp(-tau dt / tau2)]
        tau1(r) = tau1_0 (1 + kappa r / a)

    which is not separable in space x time but depends on |Delta| only, so it has
    the point-mirror symmetry i[-j, -K] = i[j, K].  A makes the mean, over the
    central pixel's impacts, of the time-summed response equal to one (unit
    collected charge).  ``symmetric=False`` adds an x-odd term that breaks the
    mirror symmetry (used only to pin orientation in tests).
    """
    rng = np.random.default_rng(cfg.response_seed if seed is None else seed)
    a = cfg.pitch_cm
    h = a / cfg.n_sub
    s = rng.uniform(0.4, 0.6) * a
    tau1_0 = rng.uniform(0.3, 0.6)
    kappa = rng.uniform(0.2, 0.5)
    tau2 = rng.uniform(1.0, 2.0)
    beta = rng.uniform(0.05, 0.1)
    R = (cfg.kp - 1) // 2
    K = np.arange(cfg.kp) - R
    lam = (np.arange(cfg.n_sub) + 0.5) * h - a / 2
    dx = K[None, :, None, None] * a + lam[None, None, None, :]      # [1,Kx,1,jx]
    dy = K[:, None, None, None] * a + lam[None, None, :, None]      # [Ky,1,jy,1]
    dx, dy = np.broadcast_arrays(dx, dy)
    r = np.sqrt(dx * dx + dy * dy)
    tau = np.arange(cfg.nr) * cfg.tick_us
    tau1 = tau1_0 * (1.0 + kappa * r / a)
    g = np.exp(-(r * r) / (2 * s * s))
    resp = g[..., None] * (np.exp(-tau / tau1[..., None]) - beta * np.exp(-tau / tau2))
    if not symmetric:
        resp = resp + 0.3 * (dx / a)[..., None] * g[..., None] * np.exp(-tau / 0.5)
    central = resp[R, R].sum(axis=-1).mean()
    resp = resp / central
    return resp.astype(np.float32)
