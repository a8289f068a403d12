"""Pins of the line-segment oracle (Sec. II-C, Eq. qline and the short-segment limit)
against things other than its own formula: brute-force integration of point
Gaussians along the segment, unit mass, the point path of the oracle for a
zero-length segment, charge conservation and translation."""
import numpy as np
import pytest

import oracle
import synth


def _brute_density(p0, p1, sig, x, m=20000):
    """Mean of the normalised 3-D Gaussian over m midpoints along the segment."""
    p0, p1, sig, x = (np.asarray(v, float) for v in (p0, p1, sig, x))
    lam = (np.arange(m) + 0.5) / m
    pts = p0[None, :] + lam[:, None] * (p1 - p0)[None, :]
    u = (x[None, :] - pts) / sig[None, :]
    g = np.exp(-0.5 * (u * u).sum(1)) / ((2 * np.pi) ** 1.5 * sig.prod())
    return g.mean()


@pytest.mark.parametrize("p0,p1,sig,x", [
    ([10.0, 10.0, 10.0], [13.0, 11.0, 15.0], [1.2, 1.2, 2.0], [11.0, 10.5, 12.0]),
    ([0.0, 0.0, 0.0], [5.0, 0.0, 0.0], [1.0, 1.0, 1.0], [2.5, 1.5, 0.0]),       # isotropic, off axis
    ([2.0, 3.0, 4.0], [2.5, 7.0, 4.2], [0.7, 0.9, 3.0], [2.9, 8.1, 3.0]),       # beyond an end
    ([1.0, 1.0, 1.0], [1.0, 1.0, 9.0], [0.5, 0.5, 1.5], [1.2, 0.8, 5.0]),       # along one axis
])
def test_line_density_equals_integrated_point_gaussians(p0, p1, sig, x):
    # Eq. qline read with the factor 1/2 in the exponent: the integral of a Gaussian
    # over the segment, which brute force approximates to ~1e-8 with 20000 midpoints
    got = oracle.line_density(p0, p1, sig, x)
    ref = _brute_density(p0, p1, sig, x)
    assert abs(got - ref) <= 2e-7 * max(ref, 1e-12) + 1e-15, (got, ref)


def test_line_density_isotropic_perpendicular_closed_form():
    # x at perpendicular distance r from the middle of a segment of length L along x:
    # rho = exp(-r^2 / 2 s^2) / (2 pi s^2) * erf(L / (2 sqrt2 s)) / L
    s, L, r = 1.3, 4.0, 0.9
    from math import erf, exp, pi, sqrt
    ref = exp(-r * r / (2 * s * s)) / (2 * pi * s * s) * erf(L / (2 * sqrt(2) * s)) / L
    got = oracle.line_density([0, 0, 0], [L, 0, 0], [s, s, s], [L / 2, r, 0.0])
    assert abs(got - ref) <= 1e-12 * ref


def test_line_density_has_unit_mass():
    p0, p1, sig = [0.0, 0.0, 0.0], [3.0, -2.0, 4.0], [1.0, 0.8, 1.5]
    h = 0.25
    xs = np.arange(-6, 9 + h, h)
    ys = np.arange(-8, 6 + h, h)
    zs = np.arange(-9, 13 + h, h)
    tot = 0.0
    for x in xs:
        for y in ys:
            for z in zs:
                tot += oracle.line_density(p0, p1, sig, [x, y, z])
    assert abs(tot * h ** 3 - 1.0) < 1e-6


def test_short_segment_switch_is_continuous():
    sig = [1.0, 1.0, 2.0]
    x = [0.4, -0.3, 0.5]
    just_point = oracle.line_density([0, 0, 0], [0.0999, 0, 0], sig, x)
    just_line = oracle.line_density([0, 0, 0], [0.1001, 0, 0], sig, x)
    assert abs(just_point - just_line) < 1e-3 * just_point


def _segments_from_points(dep, dx=0.0, dy=0.0, dz=0.0):
    return {"x0": dep["x"], "y0": dep["y"], "z0": dep["z"], "x1": dep["x"] + dx, "y1": dep["y"] + dy,
            "z1": dep["z"] + dz, "t0": dep["t0"], "ne": dep["ne"]}


def test_zero_length_segments_reproduce_the_point_path():
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sub = {k: v[100:160] for k, v in dep.items()}
    p = oracle.params(cfg)
    d = oracle.drift(p, sub)
    L = oracle.drift_lines(p, _segments_from_points(sub))
    w = oracle.line_windows(L)
    for f in ("mu", "sig", "q", "lo", "hi", "valid"):
        np.testing.assert_array_equal(w[f], d[f])
    ids, _ = oracle.active_blocks(p, d)
    qp = oracle.qeff_blocks(p, d, ids)
    ql = oracle.qeff_line_blocks(p, L, ids)
    np.testing.assert_allclose(ql, qp, rtol=0, atol=1e-12 * np.abs(qp).max())
    pix = oracle.active_pixels(p, ids, cfg.kp)[::7]
    np.testing.assert_allclose(oracle.currents_from_qeff(p, ids, qp, resp, pix),
                               oracle.pixel_currents(p, d, resp, pix), rtol=0, atol=1e-12 * np.abs(qp).max())


def test_line_effective_charge_conserves_charge_and_translates():
    cfg = synth.get_config("tiny")
    p = oracle.params(cfg)
    seg = {"x0": np.array([4.0], np.float32), "y0": np.array([5.0], np.float32),
           "z0": np.array([1.0], np.float32), "x1": np.array([4.6], np.float32),
           "y1": np.array([5.3], np.float32), "z1": np.array([1.4], np.float32),
           "t0": np.array([2.0], np.float32), "ne": np.array([10000.0], np.float32)}
    L = oracle.drift_lines(p, seg)
    ids, _ = oracle.active_blocks(p, oracle.line_windows(L))
    q = oracle.qeff_line_blocks(p, L, ids)
    assert abs(q.sum() / L["d"]["q"][0] - 1.0) < 1e-3
    h = cfg.pitch_cm / cfg.n_sub
    shifted = dict(seg, x0=seg["x0"] + np.float32(3 * h), x1=seg["x1"] + np.float32(3 * h))
    L2 = oracle.drift_lines(p, shifted)
    ids2, _ = oracle.active_blocks(p, oracle.line_windows(L2))
    q2 = oracle.qeff_line_blocks(p, L2, ids2)
    # same total, and the (y, t) marginal is unchanged by a shift along x
    assert abs(q2.sum() - q.sum()) < 1e-9 * q.sum()

    def yt_marginal(qb, blocks):
        nbx, nbt = cfg.npx // cfg.bp, cfg.nt // cfg.bt
        ny = cfg.npx * cfg.n_sub
        m = np.zeros((ny, cfg.nt))
        for k, blk in enumerate(blocks):
            bt, bxy = blk % nbt, blk // nbt
            by = bxy // nbx
            a = qb[k].sum(axis=(1, 3))                  # [jy][py][t]
            for py in range(cfg.bp):
                for jy in range(cfg.n_sub):
                    m[(by * cfg.bp + py) * cfg.n_sub + jy, bt * cfg.bt:(bt + 1) * cfg.bt] += a[jy, py]
        return m
    np.testing.assert_allclose(yt_marginal(q2, ids2), yt_marginal(q, ids), rtol=0, atol=1e-9 * q.sum())
