"""Batches of events through one pass of each kernel (event dimension, sub-batched
effective charge and convolution, CUDA graph), against the oracle per event and
against the single-event path."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import WAVE_TOL, check_hits, make_sim, pixel_rel_errors, run

pytestmark = pytest.mark.gpu


def _tiny_events(k, cfg):
    return [synth.make_deposits(cfg, seed=cfg.seed + 1000 * i) for i in range(k)]


def _batch(cfg, events, resp, chunk, persistent=False, conv_mode=0, fuse_gather=None):
    import torch
    from paper_2602_12052_b300 import autotune
    sim = autotune.make_batch(cfg, events, torch.from_numpy(resp), chunk_blocks=chunk, persistent=persistent,
                              conv_mode=conv_mode, fuse_gather=fuse_gather)
    sim.step()
    torch.cuda.synchronize()
    return sim


def _uneven_tiny_events(cfg, k=8):
    """k events of the 32 x 32 pixel plane with uneven deposit counts (from one deposit
    to the whole 5 cm track, one of them empty), each from its own seeded track."""
    sizes = [500, 1, 37, 0, 260, 5, 499, 120, 333, 64][:k]
    out = []
    for i, m in enumerate(sizes):
        dep = synth.make_deposits(cfg, seed=cfg.seed + 1000 * i)
        out.append({kk: v[:m].copy() for kk, v in dep.items()})
    return out


def _results(sim):
    import torch
    torch.cuda.synchronize()
    nb, npix, nh = (int(v) for v in sim.counts[:3].cpu())
    return {"block_ids": sim.block_ids[:nb].cpu().numpy(), "block_counts": sim.block_counts[:nb].cpu().numpy(),
            "pixel_ids": sim.pixel_ids[:npix].cpu().numpy(), "waveforms": sim.waveforms[:npix].cpu().numpy(),
            "hit_pixel": sim.hit_pixel[:nh].cpu().numpy(), "hit_tick": sim.hit_tick[:nh].cpu().numpy(),
            "hit_charge": sim.hit_charge[:nh].cpu().numpy()}


@pytest.mark.parametrize("chunk,persistent,conv_mode,fuse", [(3, False, 0, None), (64, False, 0, None),
                                                            (0, True, 0, None), (3, False, 4, True),
                                                            (64, False, 4, True), (3, False, 4, False)])
def test_batch_matches_oracle_per_event(chunk, persistent, conv_mode, fuse):
    """Eight events of uneven size (one empty, one with a single deposit) through the
    batched path, against the oracle run on each event alone: sub-batches of 3 or 64
    slots, or the one persistent launch over the batch's active-block queue; the FFT form
    and the direct spatial form (conv_mode 4) of the convolution, the latter with every
    chunk stopping at the output spectra and one fused inverse + gather over the batch
    (fuse) or with the per-chunk inverse and the gather."""
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    events = _uneven_tiny_events(cfg)
    sim = _batch(cfg, events, resp, chunk or 64, persistent, conv_mode, fuse)
    assert sim.persistent == persistent
    assert sim.fuse_gather == bool(fuse)
    assert sim.status()[0] == 0
    res = _results(sim)
    nblk, npx2 = cfg.n_blocks, cfg.npx * cfg.npx
    for e, dep in enumerate(events):
        ref = oracle.simulate(cfg, dep, resp)
        sel_b = (res["block_ids"] // nblk) == e
        np.testing.assert_array_equal(res["block_ids"][sel_b] - e * nblk, ref["block_ids"])
        np.testing.assert_array_equal(res["block_counts"][sel_b], ref["block_counts"])
        sel_p = (res["pixel_ids"] // npx2) == e
        np.testing.assert_array_equal(res["pixel_ids"][sel_p] - e * npx2, ref["pixel_ids"])
        if len(dep["x"]) == 0:
            assert not sel_b.any() and not sel_p.any()
            continue
        err = pixel_rel_errors(res["waveforms"][sel_p], ref["waveforms"])
        assert err.max() <= WAVE_TOL, (e, err.max())
        hp, ht, hc, _ = oracle.readout(ref["pixel_ids"], ref["waveforms"], cfg.threshold_e, cfg.clock_ticks,
                                       cfg.hold_ticks, cfg.reset_ticks)
        sel_h = (res["hit_pixel"] // npx2) == e
        check_hits((res["hit_pixel"][sel_h] - e * npx2, res["hit_tick"][sel_h], res["hit_charge"][sel_h]),
                   (hp, ht, hc), ref["waveforms"], ref["pixel_ids"], cfg.threshold_e, cfg.hold_ticks,
                   cfg.reset_ticks)


@pytest.mark.parametrize("persistent,conv_mode", [(False, 0), (True, 0), (False, 4)])
def test_batch_graph_replay_matches_eager(persistent, conv_mode):
    """The batched step recorded in a CUDA graph and replayed gives the eager step's
    outputs bit for bit: every sum of the effective charge and the convolution runs in
    a fixed order (sorted deposit lists, no atomics on data), whichever CTA takes a block
    (the direct form: chunks up to the spectra, then the fused inverse + gather)."""
    import torch
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    sim = _batch(cfg, _tiny_events(4, cfg), resp, 8, persistent, conv_mode)
    eager = _results(sim)
    sim.capture()
    for _ in range(2):
        sim.waveforms.zero_()
        sim.out_blocks.zero_()
        sim.replay()
        torch.cuda.synchronize()
        got = _results(sim)
        for k in ("block_ids", "block_counts", "pixel_ids", "hit_pixel", "hit_tick", "hit_charge", "waveforms"):
            np.testing.assert_array_equal(got[k], eager[k])


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_of_uneven_events_equals_single_event_runs(persistent):
    """Config-3 style events (uneven deposit counts) batched vs one at a time, and each
    event's brightest and random pixels against the oracle directly."""
    cfg = synth.get_config("module200")
    resp = synth.make_response(cfg)
    events = synth.make_events(cfg, 4, 1000, 30000, seed=33)
    sim = _batch(cfg, events, resp, 256, persistent)
    assert sim.status()[0] == 0
    res = _results(sim)
    nblk, npx2 = cfg.n_blocks, cfg.npx * cfg.npx
    p = oracle.params(cfg)
    rng = np.random.default_rng(9)
    for e, dep in enumerate(events):
        sel_p = (res["pixel_ids"] // npx2) == e
        pix_e, wav_e = res["pixel_ids"][sel_p] - e * npx2, res["waveforms"][sel_p]
        nrm = np.linalg.norm(wav_e, axis=1)
        rows = np.unique(np.concatenate([np.argsort(nrm)[-8:], rng.choice(len(nrm), 8, replace=False)]))
        ref = oracle.pixel_currents(p, oracle.drift(p, dep), resp, pix_e[rows])
        assert pixel_rel_errors(wav_e[rows], ref).max() <= WAVE_TOL, e
    for e, dep in enumerate(events):
        one = make_sim(cfg, resp, len(dep["x"]), max_blocks=4000, max_pixels=200000)
        r1 = run(one, dep, keep_qeff=False)
        sel_b = (res["block_ids"] // nblk) == e
        np.testing.assert_array_equal(res["block_ids"][sel_b] - e * nblk, r1["block_ids"])
        sel_p = (res["pixel_ids"] // npx2) == e
        np.testing.assert_array_equal(res["pixel_ids"][sel_p] - e * npx2, r1["pixel_ids"])
        assert pixel_rel_errors(res["waveforms"][sel_p], r1["waveforms"]).max() <= WAVE_TOL
        sel_h = (res["hit_pixel"] // npx2) == e
        np.testing.assert_array_equal(res["hit_pixel"][sel_h] - e * npx2, r1["hit_pixel"])
        np.testing.assert_array_equal(res["hit_tick"][sel_h], r1["hit_tick"])


@pytest.mark.parametrize("bp,bt,lt", [(8, 64, 384), (8, 128, 384), (8, 128, 512), (4, 256, 512), (8, 320, 768),
                                      (8, 320, 1024), (8, 512, 768), (8, 640, 1024)])
def test_autotuner_shapes_match_oracle(bp, bt, lt):
    """Every block shape / FFT length the autotuner may pick is parity-checked."""
    from test_gpu_parity import _full_check
    cfg = synth.get_config("tiny", nt=1280 if 1280 % bt == 0 else 1536, bp=bp, bt=bt, lt=lt)
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, check_readout=False)


@pytest.mark.parametrize("bp,bt,lt", [(8, 64, 384), (8, 128, 384), (8, 128, 512), (4, 256, 512), (8, 256, 512)])
def test_persistent_shapes_match_oracle(bp, bt, lt):
    """Every block shape the autotuner runs in the persistent form (lt = 384 or 512;
    4-pixel blocks with their half-zero spatial stages), two uneven events against the
    oracle per event."""
    cfg = synth.get_config("tiny", nt=1280, bp=bp, bt=bt, lt=lt)
    resp = synth.make_response(cfg)
    events = _uneven_tiny_events(cfg, 3)[::2]          # 500 and 37 deposits
    sim = _batch(cfg, events, resp, 64, True)
    assert sim.status()[0] == 0
    res = _results(sim)
    nblk, npx2 = cfg.n_blocks, cfg.npx * cfg.npx
    for e, dep in enumerate(events):
        ref = oracle.simulate(cfg, dep, resp)
        sel_b = (res["block_ids"] // nblk) == e
        np.testing.assert_array_equal(res["block_ids"][sel_b] - e * nblk, ref["block_ids"])
        sel_p = (res["pixel_ids"] // npx2) == e
        np.testing.assert_array_equal(res["pixel_ids"][sel_p] - e * npx2, ref["pixel_ids"])
        assert pixel_rel_errors(res["waveforms"][sel_p], ref["waveforms"]).max() <= WAVE_TOL


def test_batch_direct_fused_equals_single_event_runs():
    """Module-plane events of uneven size (config-3 style) batched through the direct form
    with the fused inverse + gather (spectra of every slot kept, chunks of 1024 slots),
    against each event alone through the single-event fused step: identical block and
    pixel lists, waveforms within FP32 rounding (the GEMM's row tiles differ)."""
    cfg = synth.get_config("module200")
    resp = synth.make_response(cfg)
    events = synth.make_events(cfg, 3, 1000, 30000, seed=41)
    sim = _batch(cfg, events, resp, 1024, False, 4, True)
    assert sim.fuse_gather and sim.status()[0] == 0
    res = _results(sim)
    nblk, npx2 = cfg.n_blocks, cfg.npx * cfg.npx
    for e, dep in enumerate(events):
        one = make_sim(cfg, resp, len(dep["x"]), max_blocks=4000, max_pixels=200000, conv_mode=4,
                       effq_skip_empty=1, fuse_gather=True)
        r1 = run(one, dep, keep_qeff=False)
        assert r1["status"][0] == 0
        sel_b = (res["block_ids"] // nblk) == e
        np.testing.assert_array_equal(res["block_ids"][sel_b] - e * nblk, r1["block_ids"])
        sel_p = (res["pixel_ids"] // npx2) == e
        np.testing.assert_array_equal(res["pixel_ids"][sel_p] - e * npx2, r1["pixel_ids"])
        assert pixel_rel_errors(res["waveforms"][sel_p], r1["waveforms"]).max() <= 1e-6
