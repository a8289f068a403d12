"""GPU parity of the direct spatial form of the convolution (conv_mode 4): the time axis
by FFT, then for every time-frequency bin the sum over impacts and response taps of the
block pixels that hold charge as a split-BF16 tcgen05 GEMM (Sec. II-D, Eq. interlaced;
Sec. III-A-2).  The oracle is the FP64 direct convolution; the bar is the FP32 one,
relative L2 1e-5 per pixel waveform."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import (WAVE_TOL, check_blocks, check_drift, check_hits, make_sim, pixel_rel_errors, run)
from test_gpu_parity import _error_report, _full_check, _contributing_blocks, _targeted_pixels

pytestmark = pytest.mark.gpu


def _report(capsys, label, err):
    with capsys.disabled():
        print(f"\n{label}: max per-pixel rel L2 {err.max():.3e}, median {np.median(err):.3e}")


@pytest.mark.parametrize("skip", [0, 1])
def test_direct_tiny_full_path(skip, capsys):
    """One 5 cm track, 32 x 32 pixels x 1024 ticks, GL-2: waveforms and hit lists."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    res, ref, err = _full_check(cfg, dep, resp, conv_mode=4, skip_empty=skip)
    _report(capsys, f"direct form, tiny, skip_empty {skip}", err)


def test_direct_asymmetric_response():
    """An x-odd response (no mirror symmetry): pins the orientation of the tap index
    K = p' - P on both axes and the sign of the time axis."""
    cfg = synth.get_config("tiny")
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    _full_check(cfg, dep, resp, mpcp=0, conv_mode=4, check_readout=False)


@pytest.mark.parametrize("bt,lt,bp,kp,nr,gl", [(128, 384, 8, 9, 200, 2), (64, 384, 8, 9, 200, 2),
                                              (256, 512, 4, 9, 200, 2), (128, 384, 4, 7, 150, 1)])
def test_direct_shapes(bt, lt, bp, kp, nr, gl):
    """FFT length 384 (radix-3 stage) and 512; 8 x 8 and 4 x 4 pixel blocks; 9 x 9 and
    7 x 7 responses."""
    cfg = synth.get_config("tiny", bt=bt, lt=lt, bp=bp, kp=kp, nr=nr, gl_order=gl)
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    _full_check(cfg, dep, resp, mpcp=0, conv_mode=4, check_readout=False)


@pytest.mark.parametrize("n_sub", [8, 6, 4])
def test_direct_impact_counts(n_sub):
    """64, 36 and 16 impacts per pixel: the forward transform cuts a row's impacts into
    3, 2 and 1 items at multiples of 4 (groups of 16 partly filled)."""
    cfg = synth.get_config("tiny", n_sub=n_sub)
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    _full_check(cfg, dep, resp, mpcp=0, conv_mode=4, skip_empty=1, check_readout=False)


def test_direct_row_chunks_are_bitwise_the_same():
    """Rows in launch pairs of 128 (blocks whose rows cross a tile or a launch boundary
    get two partial sums added onto zero) give the same bits as one launch pair, and a
    second run gives the same bits again."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    one = run(make_sim(cfg, resp, n, conv_mode=4, effq_skip_empty=1), dep, readout=False)
    sim = make_sim(cfg, resp, n, conv_mode=4, effq_skip_empty=1, conv_rows_cap=128)
    a = run(sim, dep, readout=False)
    b = run(sim, dep, readout=False)
    assert a["status"][0] == 0 and one["status"][0] == 0
    np.testing.assert_array_equal(a["pixel_ids"], one["pixel_ids"])
    np.testing.assert_array_equal(a["waveforms"], one["waveforms"])
    np.testing.assert_array_equal(a["waveforms"], b["waveforms"])


def test_direct_dense_block_all_pixels():
    """Every pixel of a block holds charge (64 rows: a block fills half a tile) and
    neighbouring blocks overlap: a wide diffuse cloud of deposits."""
    cfg = synth.get_config("tiny")
    rng = np.random.default_rng(7)
    m = 3000
    dep = {"x": rng.uniform(0.3, 5.0, m).astype(np.float32), "y": rng.uniform(0.3, 5.0, m).astype(np.float32),
           "z": rng.uniform(1.0, 3.0, m).astype(np.float32), "t0": rng.uniform(0.0, 20.0, m).astype(np.float32),
           "ne": rng.uniform(200.0, 2000.0, m).astype(np.float32)}
    resp = synth.make_response(cfg)
    res, _, _ = _full_check(cfg, dep, resp, conv_mode=4, skip_empty=1, check_readout=False)
    assert res["n_blocks"] >= 4


@pytest.mark.parametrize("name", ["module200", "module1M"])
def test_direct_module_plane_sampled(name, capsys):
    """512 x 512 pixels x 6400 ticks at full size in the bench's launch configuration
    (effq_skip_empty): blocks and pixels bit-exact, targeted pixel waveforms (on module1M
    every pixel of four overlapping blocks' footprints and the 100 weakest above 1e-3 of
    the largest norm) and their hit lists against the oracle."""
    cfg = synth.get_config(name)
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    sim = make_sim(cfg, resp, n, max_blocks=9000, max_pixels=300000, effq_skip_empty=1, conv_mode=4)
    res = run(sim, dep, keep_qeff=False)
    assert res["status"][0] == 0, res["status"]
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    check_drift(res, d)
    ids, _ = check_blocks(res, p, d)
    np.testing.assert_array_equal(res["pixel_ids"], oracle.active_pixels(p, ids, cfg.kp))
    rows, weak = _targeted_pixels(res, cfg, ids)
    mult = _contributing_blocks(cfg, ids, res["pixel_ids"][rows])
    assert {2, 3, 4} <= set(mult.tolist()), np.bincount(mult)
    pix = res["pixel_ids"][rows]
    ref = oracle.pixel_currents(p, d, resp, pix)
    with capsys.disabled():
        err, unf = _error_report(f"direct form, {name} targeted pixels", res["waveforms"][rows], ref)
    assert err.max() <= WAVE_TOL, (err.max(), int(pix[err.argmax()]))
    hp, ht, hc, _ = oracle.readout(pix, ref, cfg.threshold_e, cfg.clock_ticks, cfg.hold_ticks, cfg.reset_ticks)
    sel = np.isin(res["hit_pixel"], pix)
    check_hits((res["hit_pixel"][sel], res["hit_tick"][sel], res["hit_charge"][sel]), (hp, ht, hc),
               ref, pix, cfg.threshold_e, cfg.hold_ticks, cfg.reset_ticks)


def test_direct_matches_fft_form_on_module200():
    """The direct form and the FFT form (conv_mode 0) of the same event agree to the FP32
    bar on every active pixel."""
    cfg = synth.get_config("module200")
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    a = run(make_sim(cfg, resp, n, max_blocks=9000, max_pixels=300000, effq_skip_empty=1), dep, readout=False)
    b = run(make_sim(cfg, resp, n, max_blocks=9000, max_pixels=300000, effq_skip_empty=1, conv_mode=4), dep,
            readout=False)
    np.testing.assert_array_equal(a["pixel_ids"], b["pixel_ids"])
    err = pixel_rel_errors(b["waveforms"], a["waveforms"])
    assert err.max() <= 2 * WAVE_TOL, err.max()


# ---- the inverse time DFT fused with the electrode gather (tred_convolve_gather_readout)
def _fused_sim(cfg, resp, n, **kw):
    kw.setdefault("effq_skip_empty", 1)
    return make_sim(cfg, resp, n, conv_mode=4, fuse_gather=True, **kw)


@pytest.mark.parametrize("skip", [0, 1])
def test_fused_gather_tiny_full_path(skip, capsys):
    """Per 8 x 8 pixel tile, the summed block spectra inverted straight into the pixel
    waveforms, time blocks chained through their overlapping tails: waveforms, pixel list
    and hit list of the tiny event against the oracle."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sim = _fused_sim(cfg, resp, len(dep["x"]), effq_skip_empty=skip)
    assert sim.fuse_gather
    res, ref, err = _full_check(cfg, dep, resp, conv_mode=4, skip_empty=skip, sim=sim)
    _report(capsys, f"direct form + fused gather, tiny, skip_empty {skip}", err)


@pytest.mark.parametrize("bt,lt,nr,nt", [(128, 384, 129, 1024), (64, 384, 60, 1024), (256, 384, 100, 1280),
                                         (320, 512, 150, 1280), (128, 512, 100, 1152)])
def test_fused_gather_shapes(bt, lt, nr, nt):
    """FFT length 384 and 512; the tail exactly one time block long (nr - 1 = bt); short
    time blocks (20 per window); nt / bt odd."""
    cfg = synth.get_config("tiny", bt=bt, lt=lt, nr=nr, nt=nt)
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    sim = _fused_sim(cfg, resp, len(dep["x"]))
    _full_check(cfg, dep, resp, mpcp=0, conv_mode=4, skip_empty=1, check_readout=False, sim=sim)


def test_fused_gather_is_deterministic_and_matches_the_block_path():
    """Two runs give the same bits; against the per-block inverse + gather of the same
    spectra the waveforms agree to FP32 rounding (the spatial sum is taken on the spectra)
    and the pixel lists are identical."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    sim = _fused_sim(cfg, resp, n)
    a = run(sim, dep)
    b = run(sim, dep)
    ref = run(make_sim(cfg, resp, n, conv_mode=4, effq_skip_empty=1), dep)
    for r in (a, b, ref):
        assert r["status"][0] == 0, r["status"]
    for k in ("pixel_ids", "waveforms", "hit_pixel", "hit_tick", "hit_charge"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(a["pixel_ids"], ref["pixel_ids"])
    assert pixel_rel_errors(a["waveforms"], ref["waveforms"]).max() <= 1e-6


def test_fused_gather_edge_events():
    """An empty event (no blocks, no pixels), a single deposit, and a single deposit that
    carries no charge (its blocks are active, their pixels' waveforms are all zero)."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sim = _fused_sim(cfg, resp, len(dep["x"]))
    empty = {k: v[:0].copy() for k, v in dep.items()}
    r0 = run(sim, empty)
    assert r0["status"][0] == 0 and r0["n_blocks"] == 0 and r0["n_pixels"] == 0 and r0["n_hits"] == 0
    one = {k: v[:1].copy() for k, v in dep.items()}
    _full_check(cfg, one, resp, conv_mode=4, skip_empty=1, check_readout=False, sim=sim)
    dead = dict(one)
    dead["ne"] = np.zeros(1, np.float32)
    r2 = run(sim, dead)
    assert r2["status"][0] == 0 and r2["n_pixels"] > 0
    ref = oracle.simulate(cfg, dead, resp)
    np.testing.assert_array_equal(r2["pixel_ids"], ref["pixel_ids"])
    assert not np.any(r2["waveforms"]) and r2["n_hits"] == 0


def test_fused_gather_dense_blocks():
    """A wide diffuse cloud: every pixel of the blocks holds charge and tiles sum four
    active blocks."""
    cfg = synth.get_config("tiny")
    rng = np.random.default_rng(7)
    m = 3000
    dep = {"x": rng.uniform(0.3, 5.0, m).astype(np.float32), "y": rng.uniform(0.3, 5.0, m).astype(np.float32),
           "z": rng.uniform(1.0, 3.0, m).astype(np.float32), "t0": rng.uniform(0.0, 20.0, m).astype(np.float32),
           "ne": rng.uniform(200.0, 2000.0, m).astype(np.float32)}
    resp = synth.make_response(cfg)
    sim = _fused_sim(cfg, resp, m)
    _full_check(cfg, dep, resp, conv_mode=4, skip_empty=1, check_readout=False, sim=sim)


@pytest.mark.parametrize("name", ["module200", "module1M"])
def test_fused_gather_module_plane_sampled(name, capsys):
    """512 x 512 pixels x 6400 ticks at full size in the bench's launch configuration:
    pixel list bit-exact, targeted pixel waveforms (every pixel of four overlapping
    blocks' footprints, the weakest above 1e-3 of the largest norm) and their hit lists
    against the oracle, and every pixel against the per-block inverse + gather."""
    cfg = synth.get_config(name)
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    sim = _fused_sim(cfg, resp, n, max_blocks=9000, max_pixels=300000)
    res = run(sim, dep, keep_qeff=False)
    assert res["status"][0] == 0, res["status"]
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    ids, _ = check_blocks(res, p, d)
    np.testing.assert_array_equal(res["pixel_ids"], oracle.active_pixels(p, ids, cfg.kp))
    rows, weak = _targeted_pixels(res, cfg, ids)
    pix = res["pixel_ids"][rows]
    ref = oracle.pixel_currents(p, d, resp, pix)
    with capsys.disabled():
        err, unf = _error_report(f"direct form + fused gather, {name} targeted pixels", res["waveforms"][rows], ref)
    assert err.max() <= WAVE_TOL, (err.max(), int(pix[err.argmax()]))
    hp, ht, hc, _ = oracle.readout(pix, ref, cfg.threshold_e, cfg.clock_ticks, cfg.hold_ticks, cfg.reset_ticks)
    sel = np.isin(res["hit_pixel"], pix)
    check_hits((res["hit_pixel"][sel], res["hit_tick"][sel], res["hit_charge"][sel]), (hp, ht, hc),
               ref, pix, cfg.threshold_e, cfg.hold_ticks, cfg.reset_ticks)
    del sim
    other = run(make_sim(cfg, resp, n, max_blocks=9000, max_pixels=300000, effq_skip_empty=1, conv_mode=4), dep,
                keep_qeff=False)
    np.testing.assert_array_equal(res["pixel_ids"], other["pixel_ids"])
    assert pixel_rel_errors(res["waveforms"], other["waveforms"]).max() <= WAVE_TOL


def test_fused_gather_refuses_other_shapes():
    """4 x 4 pixel blocks, a tail longer than a time block and the FFT form have no fused
    gather: tred_convolve_gather_supported says so and the Simulator refuses it."""
    from paper_2602_12052_b300 import tred
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    assert tred.tred_convolve_gather_supported(make_sim(cfg, resp, n, conv_mode=4).h)
    for c2, mode in ((cfg.with_(bp=4, bt=256, lt=512), 4), (cfg.with_(bt=128, lt=384, nr=200), 4), (cfg, 0)):
        r2 = synth.make_response(c2)
        assert not tred.tred_convolve_gather_supported(make_sim(c2, r2, n, conv_mode=mode).h)
        with pytest.raises(ValueError):
            make_sim(c2, r2, n, conv_mode=mode, fuse_gather=True)


def test_fused_entry_points_reject_bad_calls():
    """The fused calls return TRED_ERR_INVALID_ARG (and the handle stays usable) on a
    handle whose shape has no fused gather, and for a slot range past slot 0 on a handle
    that does not keep every slot's spectra."""
    import torch
    from paper_2602_12052_b300 import abi, tred
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    fft = make_sim(cfg, resp, n, conv_mode=0)
    with pytest.raises(abi.TredError) as e:
        tred.tred_convolve_gather_readout(fft.h, fft.block_ids, fft.n_blocks_dev, fft.qeff, fft.pixel_ids,
                                          fft.waveforms, fft.n_pixels_dev)
    assert e.value.code == abi.TRED_ERR_INVALID_ARG
    direct = make_sim(cfg, resp, n, conv_mode=4, effq_skip_empty=1)   # spectra of one pass only
    with pytest.raises(abi.TredError) as e:
        tred.tred_convolve_spectra_range(direct.h, direct.block_ids, direct.n_blocks_dev, 8, 8, direct.qeff)
    assert e.value.code == abi.TRED_ERR_INVALID_ARG
    res = run(direct, dep, keep_qeff=False)   # the handle still runs an event
    assert res["status"][0] == 0 and res["n_pixels"] > 0
    torch.cuda.synchronize()
