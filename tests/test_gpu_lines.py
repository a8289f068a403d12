"""GPU parity of the line-segment form (Sec. II-C, Eq. qline and the short-segment
limit) against the FP64 oracle: bit-exact windows, blocks and pixels; effective
charge per block and pixel waveforms within 1e-5 relative L2; hit lists."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import (WAVE_TOL, check_blocks, check_drift, check_hits, check_qeff, pixel_rel_errors)

pytestmark = pytest.mark.gpu


def _run(cfg, seg, resp, max_blocks=None, max_pixels=None, skip_empty=0, conv_mode=0, fuse=False):
    import torch
    from paper_2602_12052_b300 import build, tred
    build.build()
    n = len(seg["x0"])
    sim = tred.LineSimulator(cfg, torch.from_numpy(np.ascontiguousarray(resp)), max_segments=max(n, 1),
                             max_blocks=max_blocks or min(cfg.n_blocks, 20000),
                             max_pixels=max_pixels or min(cfg.npx * cfg.npx, 400000), effq_skip_empty=skip_empty,
                             conv_mode=conv_mode, fuse_gather=fuse)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in seg.items()}
    sim.step_lines(n, t["x0"], t["y0"], t["z0"], t["x1"], t["y1"], t["z1"], t["t0"], t["ne"])
    res = sim.results()
    res["status"] = sim.status()
    from parity_util import DEP_FIELDS
    res["deps"] = {f: sim.deps[f][:n].cpu().numpy() for f in DEP_FIELDS}
    nb = res["n_blocks"]
    res["dep_offsets"] = sim.dep_offsets[:nb + 1].cpu().numpy()
    res["qeff"] = sim.qeff[:nb].cpu().numpy()
    res["waveforms"] = sim.waveforms[:res["n_pixels"]].cpu().numpy()
    return sim, res


def _full(cfg, seg, resp, check_readout=True, conv_mode=0, fuse=False):
    sim, res = _run(cfg, seg, resp, conv_mode=conv_mode, fuse=fuse)
    assert res["status"][0] == 0, res["status"]
    ref = oracle.simulate_lines(cfg, seg, resp)
    p = ref["params"]
    w = oracle.line_windows(ref["lines"])
    check_drift(res, w)
    ids, _ = check_blocks(res, p, w)
    check_qeff(res["qeff"], ref["qeff"])
    np.testing.assert_array_equal(res["pixel_ids"], ref["pixel_ids"])
    err = pixel_rel_errors(res["waveforms"], ref["waveforms"])
    assert err.max() <= WAVE_TOL, (err.max(), int(err.argmax()))
    if check_readout:
        hp, ht, hc, _ = oracle.readout(ref["pixel_ids"], ref["waveforms"], cfg.threshold_e, cfg.clock_ticks,
                                       cfg.hold_ticks, cfg.reset_ticks)
        check_hits((res["hit_pixel"], res["hit_tick"], res["hit_charge"]), (hp, ht, hc), ref["waveforms"],
                   ref["pixel_ids"], cfg.threshold_e, cfg.hold_ticks, cfg.reset_ticks)
    return res, ref, err


@pytest.mark.parametrize("conv_mode,fuse", [(0, False), (4, False), (4, True)])
def test_tiny_track_in_segments(conv_mode, fuse):
    """The tiny 5 cm track as twenty 2.5 mm segments, full path against the oracle, with
    the FFT form and the direct spatial form of the convolution (with the per-block inverse
    and the gather, or the inverse fused with the gather per pixel tile)."""
    cfg = synth.get_config("tiny_lines")
    seg = synth.make_segments(cfg, synth.SEG_CM["tiny_lines"])
    resp = synth.make_response(cfg)
    res, ref, err = _full(cfg, seg, resp, conv_mode=conv_mode, fuse=fuse)
    assert res["n_hits"] > 0 and res["n_blocks"] >= 2


@pytest.mark.parametrize("gl", [1, 3])
def test_segments_gl_orders(gl):
    cfg = synth.get_config("tiny_lines", gl_order=gl)
    seg = synth.make_segments(cfg, synth.SEG_CM["tiny_lines"])
    _full(cfg, seg, synth.make_response(cfg), check_readout=False)


def test_short_and_axis_aligned_segments():
    """Segments shorter than 0.1 sigma on every axis (point form), segments along one
    axis, a zero-length one, and one with an endpoint off the plane (dropped)."""
    cfg = synth.get_config("tiny_lines")
    resp = synth.make_response(cfg)
    h = cfg.pitch_cm / cfg.n_sub
    x0 = np.array([5.0, 5.0, 6.0, 7.0, 4.0, 13.9], np.float32)
    y0 = np.array([5.0, 6.0, 6.0, 7.0, 4.0, 5.0], np.float32)
    z0 = np.array([2.0, 2.0, 3.0, 1.0, 1.5, 1.0], np.float32)
    x1 = x0 + np.array([0.01 * h, 0.5, 0.0, 0.0, 0.0, 0.5], np.float32)
    y1 = y0 + np.array([0.0, 0.0, 0.4, 0.0, 0.0, 0.0], np.float32)
    z1 = z0 + np.array([0.0, 0.0, 0.0, 0.3, 0.0, 0.0], np.float32)
    n = len(x0)
    seg = {"x0": x0, "y0": y0, "z0": z0, "x1": x1, "y1": y1, "z1": z1, "t0": np.full(n, 2.0, np.float32),
           "ne": np.full(n, 20000.0, np.float32)}
    res, ref, err = _full(cfg, seg, resp, check_readout=False)
    assert res["status"][1] == 1          # the segment leaving the plane is dropped


def test_module_plane_segments_sampled():
    """A 200-track module plane in 3 mm segments: bit-exact blocks and pixels, sampled
    effective-charge blocks and pixel waveforms against the oracle."""
    cfg = synth.get_config("module_lines")
    seg = synth.make_segments(cfg, synth.SEG_CM["module_lines"])
    resp = synth.make_response(cfg)
    sim, res = _run(cfg, seg, resp, max_blocks=9000, max_pixels=300000)
    assert res["status"][0] == 0, res["status"]
    p = oracle.params(cfg)
    L = oracle.drift_lines(p, seg)
    w = oracle.line_windows(L)
    check_drift(res, w)
    ids, _ = check_blocks(res, p, w)
    np.testing.assert_array_equal(res["pixel_ids"], oracle.active_pixels(p, ids, cfg.kp))
    rng = np.random.default_rng(2)
    qsel = np.sort(rng.choice(len(ids), 5, replace=False))
    check_qeff(res["qeff"][qsel], oracle.qeff_line_blocks(p, L, ids[qsel]))
    # sampled pixels: their currents from the oracle's effective charge of the blocks
    # that reach them (every block within the response half-width)
    e = np.linalg.norm(res["waveforms"], axis=1)
    rows = np.unique(np.concatenate([np.argsort(e)[-12:], rng.choice(len(e), 12, replace=False)]))
    pix = res["pixel_ids"][rows]
    nbx, nbt = cfg.npx // cfg.bp, cfg.nt // cfg.bt
    R = (cfg.kp - 1) // 2
    bx = (ids // nbt) % nbx
    by = (ids // nbt) // nbx
    near = np.zeros(len(ids), bool)
    for q in pix:
        px, py = q % cfg.npx, q // cfg.npx
        near |= ((bx * cfg.bp <= px + R) & (bx * cfg.bp + cfg.bp - 1 >= px - R) &
                 (by * cfg.bp <= py + R) & (by * cfg.bp + cfg.bp - 1 >= py - R))
    sel = ids[near]
    ref = oracle.currents_from_qeff(p, sel, oracle.qeff_line_blocks(p, L, sel), resp, pix)
    err = pixel_rel_errors(res["waveforms"][rows], ref)
    assert err.max() <= WAVE_TOL, (err.max(), int(pix[err.argmax()]))


def test_tiny_track_segments_covered_columns_only():
    """The same tiny track with the effective charge written only for the sub-cell
    columns some segment's support covers (the bench's setting): pixel waveforms
    within tolerance of the oracle, and the same pixels and hits as the dense run."""
    cfg = synth.get_config("tiny_lines")
    seg = synth.make_segments(cfg, synth.SEG_CM["tiny_lines"])
    resp = synth.make_response(cfg)
    _, dense = _run(cfg, seg, resp)
    sim, res = _run(cfg, seg, resp, skip_empty=1)
    assert res["status"][0] == 0, res["status"]
    ref = oracle.simulate_lines(cfg, seg, resp)
    np.testing.assert_array_equal(res["pixel_ids"], ref["pixel_ids"])
    err = pixel_rel_errors(res["waveforms"], ref["waveforms"])
    assert err.max() <= WAVE_TOL, (err.max(), int(err.argmax()))
    np.testing.assert_array_equal(res["pixel_ids"], dense["pixel_ids"])
    np.testing.assert_array_equal(res["hit_pixel"], dense["hit_pixel"])
    np.testing.assert_array_equal(res["hit_tick"], dense["hit_tick"])

