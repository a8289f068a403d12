"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: textbook
values, library routines (numpy/scipy), closed forms, invariants or brute force.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _normal_pdf(x, mu, sig):
    return np.exp(-0.5 * ((x - mu) / sig) ** 2) / (sig * math.sqrt(2 * math.pi))


def _window_mass(mu, sig, lo, hi):
    a, b = lo - 0.5, hi + 0.5
    return 0.5 * (special.erf((b - mu) / (sig * math.sqrt(2))) - special.erf((a - mu) / (sig * math.sqrt(2))))


# --------------------------------------------------------------- Gauss-Legendre rule
def test_gl_textbook_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "gauss_legendre.txt"))
    for n in range(1, 5):
        xi, w = oracle.gl_rule(n)
        ref = rows[rows[:, 0] == n]
        np.testing.assert_allclose(xi, ref[:, 1], atol=1e-14)
        np.testing.assert_allclose(w, ref[:, 2], atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 32])
def test_gl_matches_numpy_and_polynomial_exactness(n):
    xi, w = oracle.gl_rule(n)
    rx, rw = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(xi, rx, atol=1e-13)
    np.testing.assert_allclose(w, rw, atol=1e-13)
    for k in range(2 * n):                         # exact up to degree 2N-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * xi ** k) - exact) < 1e-13
    if n <= 4:                                     # and not beyond
        k = 2 * n
        assert abs(np.sum(w * xi ** k) - 2.0 / (k + 1)) > 1e-3


# --------------------------------------------------------------- effective charge, 1-D
def _window(mu, sig, ns=4.0):
    return int(math.floor(mu - ns * sig)), int(math.ceil(mu + ns * sig))


@pytest.mark.parametrize("mu,sig", [(10.3, 1.0), (7.77, 2.5), (3.05, 0.6), (50.5, 6.3)])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gl_weights_conserve_quadrature_total(mu, sig, n):
    """The interpolation coefficients form a partition of unity (Eq. trilinear), so
    the effective charge keeps the quadrature total sum_C sum_l (w_l/2) phi(C+s_l)."""
    lo, hi = _window(mu, sig)
    e = oracle.weights_gl(n, mu, sig, lo, hi)
    xi, w = np.polynomial.legendre.leggauss(n)
    C = np.arange(lo, hi + 1)[:, None]
    total = np.sum(0.5 * w[None, :] * _normal_pdf(C + 0.5 * xi[None, :], mu, sig))
    assert abs(e.sum() - total) < 1e-14
    if sig >= 1.0 and n >= 2:                      # composite GL error ~ exp(-2 pi^2 sig^2)
        assert abs(e.sum() - _window_mass(mu, sig, lo, hi)) < 1e-6


@pytest.mark.parametrize("mu,sig", [(10.3, 1.0), (3.05, 0.7)])
def test_gl1_is_grid_point_sampling(mu, sig):
    """N = 1 puts one node at the cell centre: 'sampling at grid points' (Sec. IV-B)."""
    lo, hi = _window(mu, sig)
    e = oracle.weights_gl(1, mu, sig, lo, hi)
    g = np.arange(lo - 1, hi + 2)
    ref = _normal_pdf(g.astype(float), mu, sig)
    ref[0] = ref[-1] = 0.0                         # g = lo-1, hi+1 get no node
    np.testing.assert_allclose(e, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mu,sig", [(10.3, 1.0), (7.77, 2.5), (3.05, 0.5), (12.0, 0.3)])
def test_tent_weights_match_numerical_integral(mu, sig):
    """Exact-tent weights = integral of N(x) Lambda(x-g) over the window (closed form
    with erf) -- checked against adaptive numerical quadrature."""
    lo, hi = _window(mu, sig)
    e = oracle.weights_tent(mu, sig, lo, hi)
    A, B = lo - 0.5, hi + 0.5
    for k, g in enumerate(range(lo - 1, hi + 2)):
        f = lambda x: _normal_pdf(x, mu, sig) * max(0.0, 1.0 - abs(x - g))
        a, b = max(g - 1.0, A), min(g + 1.0, B)
        ref = 0.0
        if b > a:
            pts = [g] if a < g < b else None
            ref = integrate.quad(f, a, b, points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
        assert abs(e[k] - ref) < 1e-12, (g, e[k], ref)
    assert abs(e.sum() - _window_mass(mu, sig, lo, hi)) < 1e-14


@pytest.mark.parametrize("mu,sig", [(10.3, 1.0), (7.77, 2.5), (3.05, 0.6)])
def test_gl_converges_to_exact_tent(mu, sig):
    """GL-N on each cell -> the exact cell integral as N grows (Eq. cub).  The
    interpolation coefficient u has a kink at the cell centre (s = 0), so the rule
    converges at second order: the error falls ~4x per doubling of N."""
    lo, hi = _window(mu, sig)
    tent = oracle.weights_tent(mu, sig, lo, hi)
    errs = [np.abs(oracle.weights_gl(n, mu, sig, lo, hi) - tent).max() for n in (4, 8, 16, 32, 64)]
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < r < 4.6 for r in ratios), ratios
    assert errs[-1] < 1e-4 * tent.max()


def test_tent_sigma_to_zero_is_linear_interpolation():
    """sigma -> 0: the effective charge becomes the hat function at the deposit,
    i.e. linear interpolation of the response to the deposit position."""
    mu, sig = 10.3, 1e-4
    lo, hi = _window(mu, sig)
    e = oracle.weights_tent(mu, sig, lo, hi)
    g = np.arange(lo - 1, hi + 2)
    np.testing.assert_allclose(e, np.maximum(0.0, 1.0 - np.abs(mu - g)), atol=1e-12)


def test_separable_form_equals_eq_effq_3d():
    """Eq. (eff_q) literally in 3-D (tensor nodes, tensor weights, trilinear
    coefficients over the 27 neighbours) equals the separable product the oracle
    uses for a point deposit."""
    cfg = synth.get_config("tiny", npx=8, nt=256, bt=256)
    p = oracle.params(cfg)
    dep = {"x": np.array([1.0101], np.float32), "y": np.array([1.2345], np.float32),
           "z": np.array([3.0], np.float32), "t0": np.array([2.0], np.float32),
           "ne": np.array([1000.0], np.float32)}
    d = oracle.drift(p, dep)[0]
    ex, ey, et = (oracle.axis_weights(p, d, a) for a in range(3))
    xi, w = np.polynomial.legendre.leggauss(2)
    s = 0.5 * xi
    lo, hi, mu, sig = d["lo"], d["hi"], d["mu"], d["sig"]
    shape = tuple(int(hi[a] - lo[a] + 3) for a in range(3))
    Q = np.zeros(shape)

    def u1(sl, r):  # linear interpolation coefficient toward neighbour r in {-1,0,1}
        if r == 0:
            return 1.0 - abs(sl)
        return abs(sl) if np.sign(sl) == r else 0.0

    for cx in range(lo[0], hi[0] + 1):
        for cy in range(lo[1], hi[1] + 1):
            for ct in range(lo[2], hi[2] + 1):
                for l in range(2):
                    for m in range(2):
                        for nn in range(2):
                            wlmn = w[l] * w[m] * w[nn] / 8.0
                            q = d["q"] * (_normal_pdf(cx + s[l], mu[0], sig[0])
                                          * _normal_pdf(cy + s[m], mu[1], sig[1])
                                          * _normal_pdf(ct + s[nn], mu[2], sig[2]))
                            for r in (-1, 0, 1):
                                for s_ in (-1, 0, 1):
                                    for t in (-1, 0, 1):
                                        c = u1(s[l], r) * u1(s[m], s_) * u1(s[nn], t)
                                        if c:
                                            Q[cx + r - lo[0] + 1, cy + s_ - lo[1] + 1,
                                              ct + t - lo[2] + 1] += wlmn * q * c
    sep = d["q"] * ex[:, None, None] * ey[None, :, None] * et[None, None, :]
    np.testing.assert_allclose(sep, Q, rtol=1e-12, atol=1e-12 * np.abs(Q).max())


# --------------------------------------------------------------- transport
def test_drift_closed_form():
    cfg = synth.get_config("tiny")
    p = oracle.params(cfg)
    dep = {"x": np.array([1.0, 14.07, -0.1, 3.0], np.float32),
           "y": np.array([2.0, 0.2, 1.0, 3.0], np.float32),
           "z": np.array([10.0, 0.0, 1.0, 20.0], np.float32),
           "t0": np.array([-50.0, 3.0, 0.0, 0.0], np.float32),
           "ne": np.array([600.0, 100.0, 10.0, 0.0], np.float32)}
    d = oracle.drift(p, dep)
    assert list(d["valid"]) == [1, 1, 0, 1]       # x < 0 is off the plane
    h = np.float32(0.44) / 10.0
    # deposit 0: 10 cm at 1.6 mm/us -> 62.5 us; arrival 12.5 us = 250 ticks
    td = 10.0 / np.float64(np.float32(0.16))
    assert abs(d["mu"][0, 2] - (-50.0 + td) / np.float64(np.float32(0.05))) < 1e-9
    assert abs(d["mu"][0, 0] - (1.0 / np.float64(h) - 0.5)) < 1e-12
    sT_cm = math.sqrt(2 * np.float64(np.float32(8.8)) * 1e-6 * td)   # sqrt(2 D_T t)
    sx = math.sqrt((sT_cm / np.float64(h)) ** 2 + 0.25)
    assert abs(d["sig"][0, 0] - sx) < 1e-12
    sL_ticks = math.sqrt(2 * 4e-6 * td) / np.float64(np.float32(0.16)) / np.float64(np.float32(0.05))
    assert abs(d["sig"][0, 2] - math.sqrt(sL_ticks ** 2 + 0.25)) < 1e-12
    assert abs(d["q"][0] - 600.0 * math.exp(-td / 2200.0)) < 1e-9
    assert d["lo"][0, 0] == math.floor(d["mu"][0, 0] - 4 * d["sig"][0, 0])
    assert d["hi"][0, 2] == math.ceil(d["mu"][0, 2] + 4 * d["sig"][0, 2])
    # worked by hand for deposit 0 (62.5 us of drift): transverse spread
    # sqrt(2 * 8.8 cm^2/s * 62.5 us) = 0.3317 mm = 0.7538 sub-cells of 0.44 mm, 0.9045 with
    # the 0.5-cell floor added in quadrature; longitudinal sqrt(2 * 4 cm^2/s * 62.5 us) =
    # 0.2236 mm = 2.795 ticks at 1.6 mm/us and 50 ns, 2.839 with the floor; charge after
    # attachment 600 exp(-62.5 / 2200) = 583.19 electrons; x = 1 cm is 22.727 sub-cell
    # widths, grid coordinate 22.227 (grid points at sub-cell centres), y = 2 cm 44.955
    assert abs(d["sig"][0, 0] - 0.9045) < 1e-4 and abs(d["sig"][0, 1] - 0.9045) < 1e-4
    assert abs(d["sig"][0, 2] - 2.8395) < 1e-4
    assert abs(d["q"][0] - 583.19) < 1e-2
    assert abs(d["mu"][0, 0] - 22.227) < 1e-3 and abs(d["mu"][0, 1] - 44.955) < 1e-3
    # zero drift: widths at the floor
    assert abs(d["sig"][1, 0] - 0.5) < 1e-15 and abs(d["sig"][1, 2] - 0.5) < 1e-15
    assert d["q"][3] == 0.0


# --------------------------------------------------------------- block-sparse binning
def test_blocks_match_brute_force_enumeration():
    cfg = synth.get_config("tiny")
    dep = synth.make_deposits(cfg)
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    counts, pairs = oracle.block_counts(p, d)
    nbx = cfg.npx // cfg.bp
    nbt = cfg.nt // cfg.bt
    ref = np.zeros_like(counts)
    ngx = cfg.npx * cfg.n_sub
    for blk in range(len(counts)):
        bt, bxy = blk % nbt, blk // nbt
        bx, by = bxy % nbx, bxy // nbx
        x0, y0, t0 = bx * cfg.bp * 10, by * cfg.bp * 10, bt * cfg.bt
        # box of sub-cells / ticks covered by the block
        lo_x = np.maximum(d["lo"][:, 0] - 1, 0)
        hi_x = np.minimum(d["hi"][:, 0] + 1, ngx - 1)
        lo_y = np.maximum(d["lo"][:, 1] - 1, 0)
        hi_y = np.minimum(d["hi"][:, 1] + 1, ngx - 1)
        lo_t = np.maximum(d["lo"][:, 2] - 1, 0)
        hi_t = np.minimum(d["hi"][:, 2] + 1, cfg.nt - 1)
        hit = ((hi_x >= x0) & (lo_x <= x0 + cfg.bp * 10 - 1) & (hi_y >= y0)
               & (lo_y <= y0 + cfg.bp * 10 - 1) & (hi_t >= t0) & (lo_t <= t0 + cfg.bt - 1)
               & (d["valid"] == 1) & (lo_x <= hi_x) & (lo_y <= hi_y) & (lo_t <= hi_t))
        ref[blk] = hit.sum()
        if ref[blk]:
            np.testing.assert_array_equal(oracle.block_deposits(p, d, blk), np.nonzero(hit)[0])
    np.testing.assert_array_equal(counts, ref)
    assert pairs == ref.sum()


# --------------------------------------------------------------- induced current
def _small_cfg(**kw):
    base = dict(npx=16, nt=512, bp=8, bt=256)
    base.update(kw)
    return synth.get_config("tiny", **base)


def _few_deposits(cfg, n=6, seed=3, z=(1.0, 6.0)):
    rng = np.random.default_rng(seed)
    w = cfg.npx * cfg.pitch_cm
    return {"x": rng.uniform(0.3 * w, 0.7 * w, n).astype(np.float32),
            "y": rng.uniform(0.3 * w, 0.7 * w, n).astype(np.float32),
            "z": rng.uniform(*z, n).astype(np.float32),
            "t0": np.full(n, 2.0, np.float32),
            "ne": rng.uniform(100, 1000, n).astype(np.float32)}


def _all_pixels(cfg):
    return np.arange(cfg.npx * cfg.npx, dtype=np.int32)


def test_current_equals_fine_grid_correlation():
    """Interlaced convolution (Eq. interlaced) == a dense correlation on the fine
    sub-pixel grid sampled at pixel stride, computed with scipy's FFT convolution."""
    from scipy import signal
    cfg = _small_cfg()
    resp = synth.make_response(cfg, symmetric=False)   # orientation-sensitive
    dep = _few_deposits(cfg)
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    ids, _ = oracle.active_blocks(p, d)
    q = oracle.qeff_blocks(p, d, ids)                   # [nb][jy][jx][py][px][t]
    ns, bp = cfg.n_sub, cfg.bp
    nbx, nbt = cfg.npx // bp, cfg.nt // cfg.bt
    G = np.zeros((cfg.npx * ns, cfg.npx * ns, cfg.nt))
    for b, blk in enumerate(ids):
        bt, bxy = blk % nbt, blk // nbt
        bx, by = bxy % nbx, bxy // nbx
        blkq = q[b].transpose(2, 0, 3, 1, 4).reshape(bp * ns, bp * ns, cfg.bt)  # [py jy][px jx][t]
        G[by * bp * ns:(by + 1) * bp * ns, bx * bp * ns:(bx + 1) * bp * ns,
          bt * cfg.bt:(bt + 1) * cfg.bt] += blkq
    R = (cfg.kp - 1) // 2
    # fine kernel F[dy, dx, tau] = i[K, j, tau] with d = 10 K + j, K in [-R, R]
    F = resp.astype(np.float64).transpose(0, 2, 1, 3, 4).reshape(cfg.kp * ns, cfg.kp * ns, cfg.nr)
    # I[P, t] = sum_d sum_tau G[10 P + d, t - tau] F[d, tau]   (d offset from 10(P-R))
    full = signal.fftconvolve(G, F[::-1, ::-1, :], mode="full")
    # full[y, x, t] = sum G[y - a, ...] Frev[a] = sum_d G[y - (Kp ns - 1) + d] F[d]
    off = cfg.kp * ns - 1 - R * ns
    P = np.arange(cfg.npx)
    ref = full[(P * ns + off)[:, None], (P * ns + off)[None, :], :cfg.nt]
    wave = oracle.pixel_currents(p, d, resp, _all_pixels(cfg)).reshape(cfg.npx, cfg.npx, cfg.nt)
    scale = np.abs(ref).max()
    assert scale > 0
    np.testing.assert_allclose(wave, ref, atol=1e-10 * scale)


def test_sigma_zero_reproduces_response_at_impact_position():
    """Exact-tent effective charge with sigma -> 0 gives Q times the response
    interpolated (bilinearly in the plane, linearly in time) at the deposit."""
    cfg = _small_cfg(DL_cm2_per_s=0.0, DT_cm2_per_s=0.0, sigma0_cells_xy=1e-6, sigma0_ticks=1e-6)
    resp = synth.make_response(cfg)
    p = oracle.params(cfg, effq_mode=1)
    x, y = 3.4567, 3.1111
    dep = {"x": np.array([x], np.float32), "y": np.array([y], np.float32),
           "z": np.array([0.0], np.float32), "t0": np.array([10.31 * 0.05], np.float32),
           "ne": np.array([1000.0], np.float32)}
    d = oracle.drift(p, dep)
    wave = oracle.pixel_currents(p, d, resp, _all_pixels(cfg)).reshape(cfg.npx, cfg.npx, cfg.nt)
    h = np.float64(np.float32(0.44)) / 10
    mux, muy = np.float64(np.float32(x)) / h - 0.5, np.float64(np.float32(y)) / h - 0.5
    mut = np.float64(np.float32(10.31 * 0.05)) / np.float64(np.float32(0.05))
    R = (cfg.kp - 1) // 2
    ref = np.zeros_like(wave)
    for gy in (int(np.floor(muy)), int(np.floor(muy)) + 1):
        for gx in (int(np.floor(mux)), int(np.floor(mux)) + 1):
            wxy = (1 - abs(mux - gx)) * (1 - abs(muy - gy))
            for gt in (int(np.floor(mut)), int(np.floor(mut)) + 1):
                wt = 1 - abs(mut - gt)
                for Py in range(cfg.npx):
                    for Px in range(cfg.npx):
                        Ky, Kx = gy // 10 - Py, gx // 10 - Px
                        if abs(Ky) <= R and abs(Kx) <= R:
                            r = resp[Ky + R, Kx + R, gy % 10, gx % 10].astype(np.float64)
                            n = min(cfg.nr, cfg.nt - gt)
                            ref[Py, Px, gt:gt + n] += 1000.0 * wxy * wt * r[:n]
    np.testing.assert_allclose(wave, ref, atol=1e-6 * np.abs(ref).max())


def test_translation_and_mirror_symmetry_and_linearity():
    cfg = _small_cfg()
    resp = synth.make_response(cfg)
    dep = _few_deposits(cfg, n=8)
    p = oracle.params(cfg)
    pix = _all_pixels(cfg)

    def run(dp):
        return oracle.pixel_currents(p, oracle.drift(p, dp), resp, pix).reshape(cfg.npx, cfg.npx, cfg.nt)

    base = run(dep)
    scale = np.abs(base).max()
    # translation by one pixel in x and by 7 ticks in time (Sec. II-B symmetry)
    sh = dict(dep)
    sh["x"] = (dep["x"].astype(np.float64) + 0.44).astype(np.float32)
    sh["t0"] = (dep["t0"].astype(np.float64) + 7 * 0.05).astype(np.float32)
    moved = run(sh)
    np.testing.assert_allclose(moved[:, 1:, 7:], base[:, :-1, :-7], atol=2e-5 * scale)
    # point mirror through the plane centre (symmetric response, Sec. III-A-2)
    w = cfg.npx * 0.44
    mi = dict(dep)
    mi["x"] = (w - dep["x"].astype(np.float64)).astype(np.float32)
    mi["y"] = (w - dep["y"].astype(np.float64)).astype(np.float32)
    mirrored = run(mi)
    np.testing.assert_allclose(mirrored, base[::-1, ::-1, :], atol=2e-5 * scale)
    # linearity: two halves sum to the whole (batching order is irrelevant)
    a = {k: v[:4] for k, v in dep.items()}
    b = {k: v[4:] for k, v in dep.items()}
    np.testing.assert_allclose(run(a) + run(b), base, atol=1e-11 * scale)


# --------------------------------------------------------------- readout
def test_readout_hand_computed_step():
    ref = np.loadtxt(os.path.join(GOLDEN, "readout_step.txt"))
    wave = np.zeros((1, 400))
    wave[0, 10:] = 100.0
    hp, ht, hc, amb = oracle.readout(np.array([7], np.int32), wave, 5000.0, 2, 32, 2)
    assert list(hp) == [7] * len(ref)
    np.testing.assert_array_equal(ht, ref[:, 0].astype(int))
    np.testing.assert_allclose(hc, ref[:, 1], rtol=0, atol=1e-9)
    # the edge at 144 has C == threshold exactly: flagged as ambiguous
    assert amb[0] == 144


def test_readout_below_threshold_and_bipolar():
    wave = np.zeros((2, 300))
    wave[0, 50:60] = 400.0                       # 4000 e-: never triggers
    wave[1, 20:40] = 300.0                       # 6000 e- then a negative lobe
    wave[1, 40:60] = -100.0
    hp, ht, hc, _ = oracle.readout(np.array([0, 1], np.int32), wave, 5000.0, 2, 32, 2)
    assert list(hp) == [1]
    # C(k)=300(k-19) >= 5000 at k=36 (5100); sample at 68: 6000 - 2000 = 4000
    assert ht[0] == 68 and abs(hc[0] - 4000.0) < 1e-9


# --------------------------------------------------------------- readout variants
def test_readout_variants_hand_computed():
    """Successive digitisations (3 per trigger) and fixed-charge quanta on the
    hand-worked step waveform (tests/golden/readout_modes.txt, Sec. II-E)."""
    ref = np.loadtxt(os.path.join(GOLDEN, "readout_modes.txt"))
    wave = np.zeros((1, 400))
    wave[0, 10:] = 100.0
    for mode, ns in ((1, 3), (2, 1)):
        hp, ht, hc, amb = oracle.readout(np.array([7], np.int32), wave, 5000.0, 2, 32, 2, mode=mode, n_samples=ns)
        r = ref[ref[:, 0] == mode]
        assert list(hp) == [7] * len(r)
        np.testing.assert_array_equal(ht, r[:, 1].astype(int))
        np.testing.assert_allclose(hc, r[:, 2], rtol=0, atol=1e-9)
    # fixed charge: hits x quantum + what is left on the front end = all the charge
    assert 7 * 5000.0 + 4000.0 == wave.sum()


def test_readout_single_digitisation_is_trigger_reset():
    rng = np.random.default_rng(5)
    wave = rng.normal(0.0, 60.0, (6, 900)) + np.where(rng.random((6, 900)) < 0.05, 900.0, 0.0)
    pix = np.arange(6, dtype=np.int32)
    a = oracle.readout(pix, wave, 5000.0, 2, 32, 2, mode=0)
    b = oracle.readout(pix, wave, 5000.0, 2, 32, 2, mode=1, n_samples=1)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_readout_fixed_charge_cumulative_thresholds():
    """For non-negative currents below one quantum per clock period, the k-th quantum
    is recorded at the first clock edge whose cumulative charge reaches k quanta."""
    rng = np.random.default_rng(6)
    clock, thr, nt = 4, 5000.0, 2000
    wave = rng.uniform(0.0, thr / clock * 0.9, (5, nt)) * (rng.random((5, nt)) < 0.3)
    hp, ht, hc, _ = oracle.readout(np.arange(5, dtype=np.int32), wave, thr, clock, 32, 2, mode=2)
    edges = np.arange(0, nt, clock)
    for p in range(5):
        Q = np.cumsum(wave[p])[edges]
        n = int(np.floor(Q[-1] / thr))
        want = edges[np.searchsorted(Q, thr * np.arange(1, n + 1), side="left")]
        np.testing.assert_array_equal(ht[hp == p], want)
        assert np.all(hc[hp == p] == thr)


def test_readout_successive_digitisations_follow_the_running_sum():
    """Each trigger gives n samples hold apart with the integrator not reset between
    them: sample m minus sample 1 is the charge collected in between; the first group
    is the trigger-reset hit."""
    rng = np.random.default_rng(7)
    nt, hold, ns = 1500, 24, 4
    wave = np.where(rng.random((4, nt)) < 0.08, rng.uniform(0, 900, (4, nt)), 0.0)
    pix = np.arange(4, dtype=np.int32)
    hp, ht, hc, _ = oracle.readout(pix, wave, 5000.0, 2, hold, 3, mode=1, n_samples=ns)
    h0p, h0t, h0c, _ = oracle.readout(pix, wave, 5000.0, 2, hold, 3, mode=0)
    for p in range(4):
        t, q = ht[hp == p], hc[hp == p]
        assert len(t) > ns
        full = len(t) - len(t) % ns
        g = t[:full].reshape(-1, ns)
        assert np.all(np.diff(g, axis=1) == hold)
        cq = q[:full].reshape(-1, ns)
        cs = np.cumsum(wave[p])
        np.testing.assert_allclose(cq[:, 1:] - cq[:, :1], cs[g[:, 1:]] - cs[g[:, :1]], rtol=0, atol=1e-6)
        assert t[0] == h0t[h0p == p][0] and abs(q[0] - h0c[h0p == p][0]) < 1e-9


# --------------------------------------------------------------- active pixel set
def _footprint_brute_force(cfg, blocks):
    """Pixels of each block's output footprint written out per pixel: block bx covers
    pixels [bx bp, bx bp + bp - 1]; the response reaches R pixels further each way, so
    the footprint is [bx bp - R, bx bp + bp - 1 + R] per axis, clipped to the plane."""
    R = (cfg.kp - 1) // 2
    nbx, nbt = cfg.npx // cfg.bp, cfg.nt // cfg.bt
    out = set()
    for blk in blocks:
        bxy = int(blk) // nbt
        bx, by = bxy % nbx, bxy // nbx
        for py in range(cfg.npx):
            for px in range(cfg.npx):
                if (by * cfg.bp - R <= py <= by * cfg.bp + cfg.bp - 1 + R
                        and bx * cfg.bp - R <= px <= bx * cfg.bp + cfg.bp - 1 + R):
                    out.add(py * cfg.npx + px)
    return np.array(sorted(out), np.int32)


def test_active_pixels_cover_every_pixel_with_current():
    """The electrode set the gather accumulates on (Fig. flowchart: unique electrodes)
    is every pixel some active block's output reaches.  Pinned two ways on the 32 x 32
    plane with an x-odd response: it equals a per-pixel brute-force footprint of the
    active blocks (including blocks on the plane's edges, where it is clipped), and every
    pixel whose current (computed on the whole plane) is nonzero belongs to it.  The
    nonzero set needs the full R-pixel halo (a footprint one pixel narrower misses
    pixels with current), so a footprint too small or too large fails."""
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg, symmetric=False)
    w = cfg.npx * cfg.pitch_cm
    rng = np.random.default_rng(17)
    # deposits in corner, edge and interior blocks, some on block boundaries; two sit in
    # the last pixel column / row of a block, clear of its neighbours, so that their
    # current reaches R pixels past the block into a footprint no other block covers
    a = cfg.pitch_cm
    xs = [0.05, w - 0.05, 0.05, w - 0.05, 8 * a, 8 * a - 0.01, 0.5 * w, 7.5 * a, 20.5 * a]
    ys = [0.05, 0.05, w - 0.05, w - 0.05, 8 * a, 24 * a - 0.01, 0.5 * w, 12.5 * a, 23.5 * a]
    n = len(xs)
    dep = {"x": np.asarray(xs, np.float32), "y": np.asarray(ys, np.float32),
           "z": rng.uniform(0.5, 6.0, n).astype(np.float32), "t0": np.full(n, 2.0, np.float32),
           "ne": np.full(n, 2000.0, np.float32)}
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    assert np.all(d["valid"] == 1)
    ids, _ = oracle.active_blocks(p, d)
    act = oracle.active_pixels(p, ids, cfg.kp)
    np.testing.assert_array_equal(act, _footprint_brute_force(cfg, ids))
    nbx, nbt = cfg.npx // cfg.bp, cfg.nt // cfg.bt
    bxy = ids // nbt
    assert {0, nbx - 1} <= set((bxy % nbx).tolist()) and {0, nbx - 1} <= set((bxy // nbx).tolist())
    wave = oracle.pixel_currents(p, d, resp, _all_pixels(cfg))
    live = np.nonzero(np.any(wave != 0.0, axis=1))[0].astype(np.int32)
    assert len(live) > 0
    assert np.all(np.isin(live, act)), np.setdiff1d(live, act)[:10]
    narrow = _footprint_brute_force(synth.get_config("tiny", kp=cfg.kp - 2), ids)
    assert not np.all(np.isin(live, narrow))
