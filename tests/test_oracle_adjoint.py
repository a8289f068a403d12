"""Pins of the oracle's gradient (Sec. V-C, differentiable simulation) against central
finite differences of the oracle's own forward pass, with the raster windows frozen
(they are piecewise constant in the inputs)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("mu,sig", [(10.3, 1.0), (3.05, 0.6), (20.7, 2.3)])
@pytest.mark.parametrize("nl", [1, 2, 3])
def test_weight_derivatives_match_finite_differences(mu, sig, nl):
    lo, hi = int(np.floor(mu - 4 * sig)), int(np.ceil(mu + 4 * sig))
    e, dm, ds = oracle.weights_gl_grad(nl, mu, sig, lo, hi)
    np.testing.assert_allclose(e, oracle.weights_gl(nl, mu, sig, lo, hi), rtol=0, atol=1e-15)
    h = 1e-6
    fm = (oracle.weights_gl(nl, mu + h, sig, lo, hi) - oracle.weights_gl(nl, mu - h, sig, lo, hi)) / (2 * h)
    fs = (oracle.weights_gl(nl, mu, sig + h, lo, hi) - oracle.weights_gl(nl, mu, sig - h, lo, hi)) / (2 * h)
    np.testing.assert_allclose(dm, fm, atol=1e-8)
    np.testing.assert_allclose(ds, fs, atol=1e-8)


def _setup(n=80):
    cfg = synth.get_config("tiny")
    dep_all, resp = synth.make_event(cfg)
    dep = {k: v[200:200 + n].copy() for k, v in dep_all.items()}
    p = oracle.params(cfg)
    d0 = oracle.drift(p, dep)
    ids, _ = oracle.active_blocks(p, d0)
    pix = oracle.active_pixels(p, ids, cfg.kp)
    # targets: the same deposits simulated with other transport constants
    pt = oracle.params(cfg, DL_cm2_per_s=cfg.DL_cm2_per_s * 1.3, DT_cm2_per_s=cfg.DT_cm2_per_s * 0.75,
                       lifetime_us=cfg.lifetime_us * 0.5)
    target = oracle.currents_frozen(pt, dep, oracle.drift(pt, dep), resp, pix)
    return cfg, p, dep, d0, resp, pix, target


def _loss(p, dep, d0, resp, pix, target):
    w = oracle.currents_frozen(p, dep, d0, resp, pix)
    return 0.5 * np.sum((w - target) ** 2), w


def test_adjoint_matches_central_differences():
    cfg, p, dep, d0, resp, pix, target = _setup()
    L0, w0 = _loss(p, dep, d0, resp, pix, target)
    g7 = oracle.adjoint(p, d0, resp, pix, w0 - target)
    gdep, gglob = oracle.param_grads(p, dep, d0, g7)
    rel = 1e-4
    # per-deposit inputs
    for k in (3, 40, 77):
        for col, name in enumerate(["x", "y", "t0", "ne"]):
            dp, dm = ({kk: v.copy() for kk, v in dep.items()} for _ in range(2))
            v = float(dep[name][k])
            dp[name][k] = np.float32(v * (1 + rel))
            dm[name][k] = np.float32(v * (1 - rel))
            step = float(dp[name][k]) - float(dm[name][k])
            fd = (_loss(p, dp, d0, resp, pix, target)[0] - _loss(p, dm, d0, resp, pix, target)[0]) / step
            ana = gdep[k, col]
            scale = np.abs(gdep[:, col]).max()
            assert abs(fd - ana) <= 2e-3 * scale + 1e-9, (name, k, fd, ana, scale)
    # global transport constants
    for j, name in enumerate(["DL_cm2_per_s", "DT_cm2_per_s", "lifetime_us"]):
        base = getattr(p, name)
        pp, pm = oracle.params(cfg), oracle.params(cfg)
        setattr(pp, name, base * (1 + rel))
        setattr(pm, name, base * (1 - rel))
        step = float(np.float32(getattr(pp, name))) - float(np.float32(getattr(pm, name)))
        fd = (_loss(pp, dep, d0, resp, pix, target)[0] - _loss(pm, dep, d0, resp, pix, target)[0]) / step
        assert abs(fd - gglob[j]) <= 2e-3 * abs(fd) + 1e-9, (name, fd, gglob[j])


def test_adjoint_is_linear_in_the_residual():
    cfg, p, dep, d0, resp, pix, target = _setup(n=40)
    rng = np.random.default_rng(5)
    r1 = rng.normal(size=(len(pix), cfg.nt))
    r2 = rng.normal(size=(len(pix), cfg.nt))
    g1 = oracle.adjoint(p, d0, resp, pix, r1)
    g2 = oracle.adjoint(p, d0, resp, pix, r2)
    g12 = oracle.adjoint(p, d0, resp, pix, 2.0 * r1 - r2)
    np.testing.assert_allclose(g12, 2.0 * g1 - g2, atol=1e-9 * np.abs(g12).max())
