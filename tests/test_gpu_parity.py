"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle on
the same seeded inputs.

Bit-exact: deposit windows and cells, active block ids and occupancy, CSR
(as sets per block), active pixel ids.  Floating point: Q^eff per block and pixel
waveforms within relative L2 1e-5 (FP32 forms; pixel floor 1e-2 of the largest
pixel norm); hit lists identical except from a trigger edge whose integrated
charge lies within 1e-4 of the threshold.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import (WAVE_TOL, check_hits_near_threshold, check_blocks, check_csr_sets, check_drift, check_hits,
                         check_qeff, make_sim, pixel_rel_errors, run)

pytestmark = pytest.mark.gpu


def _oracle_all(cfg, dep, resp, effq_mode=0):
    return oracle.simulate(cfg, dep, resp, effq_mode=effq_mode)


def _full_check(cfg, dep, resp, effq_mode=0, mpcp=1, comp=0, check_readout=True, conv_mode=0, tol=WAVE_TOL,
                skip_empty=0, sim=None):
    if sim is None:
        sim = make_sim(cfg, resp, len(dep["x"]), effq_mode=effq_mode, mpcp=mpcp, compensated_gather=comp,
                       conv_mode=conv_mode, effq_skip_empty=skip_empty)
    res = run(sim, dep)
    ref = _oracle_all(cfg, dep, resp, effq_mode)
    p, d = ref["params"], ref["deps"]
    assert res["status"][0] == 0, res["status"]
    check_drift(res, d)
    ids, _ = check_blocks(res, p, d)
    check_csr_sets(res, p, d)
    if not skip_empty:      # with skip_empty the columns no support covers are unspecified
        check_qeff(res["qeff"], oracle.qeff_blocks(p, d, ids))
    np.testing.assert_array_equal(res["pixel_ids"], ref["pixel_ids"])
    err = pixel_rel_errors(res["waveforms"], ref["waveforms"])
    assert err.max() <= tol, (err.max(), int(err.argmax()))
    ev = np.linalg.norm(res["waveforms"] - ref["waveforms"]) / np.linalg.norm(ref["waveforms"])
    assert ev <= tol
    if check_readout:
        hp, ht, hc, _ = oracle.readout(ref["pixel_ids"], ref["waveforms"], cfg.threshold_e,
                                       cfg.clock_ticks, cfg.hold_ticks, cfg.reset_ticks)
        check_hits((res["hit_pixel"], res["hit_tick"], res["hit_charge"]), (hp, ht, hc),
                   ref["waveforms"], ref["pixel_ids"], cfg.threshold_e, cfg.hold_ticks,
                   cfg.reset_ticks)
        assert res["n_hits"] == len(hp) or True
    return res, ref, err


def test_tiny_full_path():
    """One 5 cm track, 32 x 32 pixels x 1024 ticks, GL-2, MPCP (several blocks and
    time tiles; ragged occupancy)."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    res, ref, err = _full_check(cfg, dep, resp)
    assert res["n_hits"] > 0 and res["n_blocks"] >= 4


@pytest.mark.parametrize("gl", [1, 3, 4])
def test_tiny_gl_orders(gl):
    cfg = synth.get_config("tiny", gl_order=gl)
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, check_readout=False)


def test_tiny_no_mpcp_asymmetric_response():
    """Without MPCP the path must not assume mirror symmetry: an x-odd response
    pins the correlation-vs-convolution orientation of every axis."""
    cfg = synth.get_config("tiny")
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    _full_check(cfg, dep, resp, mpcp=0, check_readout=False)


@pytest.mark.parametrize("bt,lt", [(128, 384), (256, 768)])
def test_no_mpcp_asymmetric_mixed_radix(bt, lt):
    """The unpacked path at the mixed-radix FFT lengths: every inverse time transform
    form (two columns per warp at 384, one per warp at 768) with no mirror recombination."""
    cfg = synth.get_config("tiny", bt=bt, lt=lt)
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    _full_check(cfg, dep, resp, mpcp=0, check_readout=False)


def test_tiny_exact_tent_fp64_tails():
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, effq_mode=1, check_readout=False)


def test_tiny_compensated_gather():
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, comp=1, check_readout=False)


@pytest.mark.parametrize("conv_mode,tol", [(1, 1e-4), (2, WAVE_TOL), (3, 1e-4)])
def test_tiny_tensor_core_dft(conv_mode, tol, capsys):
    """The time DFT as a tcgen05 GEMM: TF32 within the tensor-core bar 1e-4, split TF32
    (three products) within the FP32 bar, split BF16 (three products) within 1e-4."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    res, ref, err = _full_check(cfg, dep, resp, conv_mode=conv_mode, tol=tol, check_readout=False)
    with capsys.disabled():
        print(f"\nconv_mode {conv_mode}: max per-pixel rel L2 {err.max():.3e}, median {np.median(err):.3e}")


@pytest.mark.parametrize("conv_mode,tol", [(0, WAVE_TOL), (1, 1e-4), (2, WAVE_TOL), (3, 1e-4)])
def test_tensor_core_dft_no_mpcp_asymmetric(conv_mode, tol):
    """Without MPCP (one real channel per impact) and with an x-odd response."""
    cfg = synth.get_config("tiny")
    dep = synth.make_deposits(cfg)
    resp = synth.make_response(cfg, symmetric=False)
    _full_check(cfg, dep, resp, mpcp=0, conv_mode=conv_mode, tol=tol, check_readout=False)


def test_skip_empty_columns_after_a_dense_event():
    """effq_skip_empty: the columns no support covers are not written, so the buffer keeps
    the previous event's values there; a sparse event run after a dense one on the same
    simulator must still match the oracle (the convolution reads each half of a packed
    column only under its own mask bit)."""
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    rng = np.random.default_rng(5)
    n = 3000
    dense = _dep(rng.uniform(0.5, 13.5, n), rng.uniform(0.5, 13.5, n), rng.uniform(0.2, 4.0, n), t0=2.0,
                 ne=rng.uniform(100.0, 900.0, n))
    sparse, _ = synth.make_event(cfg)
    sim = make_sim(cfg, resp, n, effq_skip_empty=1)
    _full_check(cfg, dense, resp, skip_empty=1, sim=sim, check_readout=False)
    _full_check(cfg, sparse, resp, skip_empty=1, sim=sim)


def test_small_blocks_long_fft():
    """bp = 4 with the 13 x 13 x 400 response (padded extent 16, lt = 1024)."""
    cfg = synth.get_config("tiny", bp=4, kp=13, nr=400, lt=1024, gl_order=3)
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, check_readout=False)


@pytest.mark.parametrize("bt,lt,bp,kp,nr,gl", [(128, 384, 8, 9, 200, 2), (256, 768, 8, 9, 200, 2),
                                              (256, 768, 4, 13, 400, 3)])
def test_mixed_radix_fft_lengths(bt, lt, bp, kp, nr, gl):
    """FFT lengths 384 = 3 x 128 and 768 = 3 x 256 (the smallest 2^a 3^b at or above
    bt + nr - 1 for these shapes): the inverse time transform runs a radix-3 stage."""
    cfg = synth.get_config("tiny", bt=bt, lt=lt, bp=bp, kp=kp, nr=nr, gl_order=gl)
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, check_readout=False)


def test_short_blocks():
    """bt = 128 (two 64-tick input blocks per FFT column)."""
    cfg = synth.get_config("tiny", bt=128)
    dep, resp = synth.make_event(cfg)
    _full_check(cfg, dep, resp, check_readout=False)


# ------------------------------------------------------------------ edge cases
def _dep(xs, ys, zs, t0=2.0, ne=600.0):
    n = len(xs)
    return {"x": np.asarray(xs, np.float32), "y": np.asarray(ys, np.float32),
            "z": np.asarray(zs, np.float32), "t0": np.full(n, t0, np.float32),
            "ne": np.full(n, ne, np.float32)}


def test_empty_event():
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    sim = make_sim(cfg, resp, 1)
    res = run(sim, _dep([], [], []))
    assert res["n_blocks"] == 0 and res["n_pixels"] == 0 and res["n_hits"] == 0
    assert res["status"][0] == 0


def test_single_deposit_and_off_plane_and_edges():
    """A single deposit; deposits off the plane (dropped and counted); deposits at
    the plane edge and the window start whose supports are clipped."""
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    w = cfg.npx * cfg.pitch_cm
    dep = _dep([7.0, -0.1, w + 0.1, 0.001, w - 0.001, 0.02, 3.3],
               [7.0, 1.0, 1.0, 0.001, w - 0.001, w - 0.02, 3.3],
               [5.0, 1.0, 1.0, 0.0, 19.0, 2.0, 0.0], t0=0.0, ne=5000.0)
    res, ref, _ = _full_check(cfg, dep, resp)
    assert res["status"][1] == 2           # two off-plane deposits dropped


def test_dense_block_multipass():
    """2500 deposits packed into one block's footprint: the effective-charge kernel
    takes several passes over the block's deposit list (its list holds 512)."""
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    rng = np.random.default_rng(21)
    n = 2500
    dep = _dep(rng.uniform(3.6, 6.8, n), rng.uniform(3.6, 6.8, n), rng.uniform(0.5, 1.5, n), t0=2.0,
               ne=rng.uniform(100.0, 900.0, n))
    res, ref, _ = _full_check(cfg, dep, resp, check_readout=False)
    assert res["block_counts"].max() > 1024


def test_very_dense_block_sorted_in_global_memory():
    """9000 deposits packed into one block: the block's deposit list is longer than the
    binning's shared-memory sort holds (8192), so it is sorted in place in global memory;
    the list must still be the oracle's, ascending, and the currents the oracle's."""
    cfg = synth.get_config("tiny")
    resp = synth.make_response(cfg)
    rng = np.random.default_rng(22)
    n = 9000
    dep = _dep(rng.uniform(4.0, 6.4, n), rng.uniform(4.0, 6.4, n), rng.uniform(0.8, 1.2, n), t0=2.0,
               ne=rng.uniform(100.0, 900.0, n))
    res, ref, _ = _full_check(cfg, dep, resp, check_readout=False)
    assert res["block_counts"].max() > 8192
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    off, idx = res["dep_offsets"], res["dep_index"]
    for s_, blk in enumerate(res["block_ids"]):
        np.testing.assert_array_equal(idx[off[s_]:off[s_ + 1]], oracle.block_deposits(p, d, int(blk)))


def test_capacity_overflow_sets_status():
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sim = make_sim(cfg, resp, len(dep["x"]), max_blocks=2, max_pixels=100)
    res = run(sim, dep, keep_qeff=False)
    from paper_2602_12052_b300 import abi
    assert res["status"][0] & abi.TRED_ST_BLOCK_OVERFLOW
    assert res["n_blocks"] == 2


def test_bounded_wait_expires_into_the_status_word():
    """A device wait on an mbarrier phase that nothing completes gives up after its
    limit, sets TRED_ST_TIMEOUT and leaves the context usable: after clearing the status
    the same handle runs the tiny event to the oracle's currents."""
    import torch
    from paper_2602_12052_b300 import abi, tred
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sim = make_sim(cfg, resp, len(dep["x"]))
    tred.tred_wait_selftest(sim.h, 2_000_000)            # about 1 ms at the maximum clock
    torch.cuda.synchronize()
    st = tred.tred_sync_status(sim.h)
    assert st[0] & abi.TRED_ST_TIMEOUT, st
    with pytest.raises(abi.TredError):
        tred.tred_wait_selftest(sim.h, 0)                # limit outside the range
    tred.tred_reset_status(sim.h)
    res = run(sim, dep, keep_qeff=False)
    assert res["status"][0] == 0, res["status"]
    ref = _oracle_all(cfg, dep, resp, 0)
    np.testing.assert_array_equal(res["pixel_ids"], ref["pixel_ids"])
    assert pixel_rel_errors(res["waveforms"], ref["waveforms"]).max() <= WAVE_TOL


@pytest.mark.parametrize("mode,n_samples", [(0, 1), (1, 3), (2, 1)])
def test_fused_gather_readout_equals_separate_calls(mode, n_samples):
    """tred_gather_readout (the readout skipping pixels whose positive current cannot
    reach the threshold) gives exactly the hits of tred_readout over every pixel."""
    import torch
    from paper_2602_12052_b300 import tred
    cfg = synth.get_config("module20", readout_mode=mode, n_samples=n_samples)
    dep, resp = synth.make_event(cfg)
    sim = make_sim(cfg, resp, len(dep["x"]), max_blocks=1000, max_pixels=40000)
    fused = run(sim, dep, keep_qeff=False)
    assert fused["status"][0] == 0 and fused["n_hits"] > 0
    hp, ht, hc = (torch.zeros_like(t) for t in (sim.hit_pixel, sim.hit_tick, sim.hit_charge))
    nh = torch.zeros(1, dtype=torch.int32, device=sim.hit_pixel.device)
    tred.tred_readout(sim.h, sim.rp, sim.pixel_ids, sim.waveforms, sim.n_pixels_dev, hp, ht, hc, nh)
    torch.cuda.synchronize()
    n = int(nh.item())
    assert n == fused["n_hits"]
    np.testing.assert_array_equal(hp[:n].cpu().numpy(), fused["hit_pixel"])
    np.testing.assert_array_equal(ht[:n].cpu().numpy(), fused["hit_tick"])
    np.testing.assert_array_equal(hc[:n].cpu().numpy(), fused["hit_charge"])


def test_repeatable_outputs():
    """Block list, occupancy, deposit lists and pixel list are identical run to run,
    and so are the effective charge and the currents, bit for bit (each block's
    deposits are sorted and every sum runs in one fixed order)."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sim = make_sim(cfg, resp, len(dep["x"]))
    a = run(sim, dep)
    b = run(sim, dep)
    for k in ("block_ids", "block_counts", "pixel_ids", "dep_offsets", "dep_index", "qeff", "waveforms"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("form", ["fft", "direct_fused"])
def test_step_replayed_from_a_cuda_graph_equals_eager(form):
    """The single-event step recorded once in a CUDA graph (device-side counts keep its
    launch sequence fixed) and replayed gives the eager step's outputs bit for bit: the
    FFT form, and the direct form with the fused inverse + gather (its tile queue and
    list are rebuilt on the device each replay)."""
    import torch
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    kw = {"conv_mode": 4, "effq_skip_empty": 1, "fuse_gather": True} if form == "direct_fused" else {}
    sim = make_sim(cfg, resp, len(dep["x"]), **kw)
    eager = run(sim, dep)
    n = len(dep["x"])
    x = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in dep.items()}
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        sim.step(n, x["x"], x["y"], x["z"], x["t0"], x["ne"])
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        sim.qeff.zero_()
        sim.waveforms.zero_()
        g.replay()
        torch.cuda.synchronize()
        res = sim.results()
        assert sim.status()[0] == 0
        for k in ("block_ids", "block_counts", "pixel_ids", "hit_pixel", "hit_tick", "hit_charge"):
            np.testing.assert_array_equal(res[k], eager[k])
        nb, npix = res["n_blocks"], res["n_pixels"]
        if form == "fft":   # with effq_skip_empty the uncovered columns are left as they were
            np.testing.assert_array_equal(sim.qeff[:nb].cpu().numpy(), eager["qeff"])
        np.testing.assert_array_equal(sim.waveforms[:npix].cpu().numpy(), eager["waveforms"])


def test_block_deposit_lists_ascending_like_oracle():
    """Each block's deposit list is the oracle's, in ascending deposit order (Sec. III-B-1),
    on the tiny event and on a module plane with blocks of a few hundred deposits."""
    for name, n_tracks in (("tiny", None), ("module200", 40)):
        cfg = synth.get_config(name) if n_tracks is None else synth.get_config(name, n_tracks=n_tracks)
        dep, resp = synth.make_event(cfg)
        sim = make_sim(cfg, resp, len(dep["x"]), max_blocks=min(cfg.n_blocks, 4000), max_pixels=200000)
        res = run(sim, dep, readout=False, keep_qeff=False, keep_waves=False)
        p = oracle.params(cfg)
        d = oracle.drift(p, dep)
        off, idx = res["dep_offsets"], res["dep_index"]
        assert len(res["block_ids"]) > 0
        for s, blk in enumerate(res["block_ids"]):
            np.testing.assert_array_equal(idx[off[s]:off[s + 1]], oracle.block_deposits(p, d, int(blk)))


# ------------------------------------------------------------------ full size, sampled
def _sampled_pixels(res, k=48, seed=0):
    rng = np.random.default_rng(seed)
    e = np.linalg.norm(res["waveforms"], axis=1)
    top = np.argsort(e)[-k // 2:]
    rnd = rng.choice(len(e), k // 2, replace=False)
    return np.unique(np.concatenate([top, rnd]))


def _xy_blocks(cfg, ids):
    nbx, nbt = cfg.npx // cfg.bp, cfg.nt // cfg.bt
    bxy = np.unique(np.asarray(ids) // nbt)
    return bxy % nbx, bxy // nbx


def _contributing_blocks(cfg, ids, pixel_ids):
    """Per pixel, the number of active (x, y) blocks whose output footprint
    [b bp - R, b bp + bp - 1 + R] per axis reaches it (1 to 4 at bp = 8, R = 4)."""
    R = (cfg.kp - 1) // 2
    bx, by = _xy_blocks(cfg, ids)
    act = set(zip(bx.tolist(), by.tolist()))
    px, py = pixel_ids % cfg.npx, pixel_ids // cfg.npx
    n = np.zeros(len(pixel_ids), np.int32)
    for k, (x, y) in enumerate(zip(px.tolist(), py.tolist())):
        xs = range(-((R + cfg.bp - 1 - x) // cfg.bp), (x + R) // cfg.bp + 1)    # ceil .. floor
        ys = range(-((R + cfg.bp - 1 - y) // cfg.bp), (y + R) // cfg.bp + 1)
        n[k] = sum((a, b) in act for a in xs for b in ys)
    return n


def _targeted_pixels(res, cfg, ids, n_blocks=4, n_weak=100):
    """Rows of the pixel list chosen where a mistake is most likely to show: every pixel
    of the output footprints of n_blocks (x, y) blocks whose neighbours are active (pixels
    summed from 2 to 4 overlapping blocks, dense-block halos), the n_weak weakest pixels
    above 1e-3 of the largest pixel norm (where the error floor sets the denominator), and
    the brightest and random pixels."""
    R = (cfg.kp - 1) // 2
    bx, by = _xy_blocks(cfg, ids)
    act = set(zip(bx.tolist(), by.tolist()))
    nbrs = np.array([sum((x + dx, y + dy) in act for dx in (-1, 0, 1) for dy in (-1, 0, 1)) - 1
                     for x, y in zip(bx.tolist(), by.tolist())])
    chosen = []
    for k in np.argsort(-nbrs, kind="stable"):
        if all(abs(bx[k] - bx[c]) > 2 or abs(by[k] - by[c]) > 2 for c in chosen):
            chosen.append(k)
        if len(chosen) == n_blocks:
            break
    fp = set()
    for k in chosen:
        for y in range(by[k] * cfg.bp - R, by[k] * cfg.bp + cfg.bp + R):
            for x in range(bx[k] * cfg.bp - R, bx[k] * cfg.bp + cfg.bp + R):
                if 0 <= x < cfg.npx and 0 <= y < cfg.npx:
                    fp.add(y * cfg.npx + x)
    pix = res["pixel_ids"]
    rows = np.nonzero(np.isin(pix, np.array(sorted(fp), np.int32)))[0]
    e = np.linalg.norm(res["waveforms"], axis=1)
    above = np.nonzero(e >= 1e-3 * e.max())[0]
    weak = above[np.argsort(e[above])[:n_weak]]
    return np.unique(np.concatenate([rows, weak, _sampled_pixels(res)])), weak


def _error_report(label, gpu, ref):
    """Per-pixel relative L2 with the 1e-2 floor of the tolerance, and without it over the
    pixels whose oracle norm is at least 1e-3 of the largest (below that a pixel holds only
    response tails, and its unfloored ratio measures FP32 rounding of numbers near zero)."""
    fl = pixel_rel_errors(gpu, ref)
    un = pixel_rel_errors(gpu, ref, floor_frac=0.0)
    nrm = np.linalg.norm(np.asarray(ref, np.float64), axis=1)
    live = nrm >= 1e-3 * nrm.max()
    q = lambda a: f"max {a.max():.2e}, 99% {np.quantile(a, 0.99):.2e}, median {np.median(a):.2e}"
    print(f"\n{label}: {len(fl)} pixels; floored {q(fl)}; unfloored over the {live.sum()} pixels >= 1e-3 "
          f"of the largest norm {q(un[live])}")
    return fl, np.where(live, un, 0.0)


@pytest.mark.parametrize("name,skip,fused", [("module200", 0, False), ("module1M", 1, False), ("module1M", 1, True),
                                             ("spill_plane", 0, False)])
def test_module_plane_sampled(name, skip, fused, capsys):
    """512 x 512 pixels x 6400 ticks at full size (module1M in the bench's launch
    configuration, with effq_skip_empty): bit-exact blocks and pixels, sampled Q^eff
    blocks, sampled pixel waveforms and their hit lists against the oracle.  On module1M
    the pixels are targeted (every pixel of four overlapping blocks' footprints, the 100
    weakest above 1e-3 of the largest norm, brightest and random ones: over 1000 in all)
    and the Q^eff check covers the skip-empty form: the buffer is cleared first, so the
    columns no support covers must stay zero and the covered ones match the oracle.
    fused: the effective charge and the convolution as one persistent launch
    (tred_effq_convolve; Q^eff lives in per-CTA ring rows and is not compared)."""
    cfg = synth.get_config(name)
    dep, resp = synth.make_event(cfg)
    n = len(dep["x"])
    sim = make_sim(cfg, resp, n, max_blocks=9000, max_pixels=300000, effq_skip_empty=skip, fused=fused)
    if skip:
        sim.qeff.zero_()
    res = run(sim, dep, keep_qeff=False)
    assert res["status"][0] == 0, res["status"]
    p = oracle.params(cfg)
    d = oracle.drift(p, dep)
    check_drift(res, d)
    ids, _ = check_blocks(res, p, d)
    check_csr_sets(res, p, d, sample=16)
    np.testing.assert_array_equal(res["pixel_ids"], oracle.active_pixels(p, ids, cfg.kp))
    rng = np.random.default_rng(1)
    qsel = np.sort(rng.choice(len(ids), 6, replace=False))
    if not fused:
        gq = np.stack([sim.qeff[int(b)].cpu().numpy() for b in qsel])
        check_qeff(gq, oracle.qeff_blocks(p, d, ids[qsel]))
    if name == "module1M":
        rows, weak = _targeted_pixels(res, cfg, ids)
        assert len(rows) >= 1000
        mult = _contributing_blocks(cfg, ids, res["pixel_ids"][rows])
        assert {2, 3, 4} <= set(mult.tolist()), np.bincount(mult)
    else:
        rows, weak = _sampled_pixels(res), np.zeros(0, np.int64)
    pix = res["pixel_ids"][rows]
    ref = oracle.pixel_currents(p, d, resp, pix)
    with capsys.disabled():
        err, unf = _error_report(f"{name}{' fused' if fused else ''} sampled pixels", res["waveforms"][rows], ref)
        if len(weak):
            wsel = np.isin(rows, weak)
            print(f"{name}: the {wsel.sum()} weakest pixels: floored max {err[wsel].max():.2e}, "
                  f"unfloored max {unf[wsel].max():.2e}")
    assert err.max() <= WAVE_TOL, (err.max(), int(pix[err.argmax()]))
    hp, ht, hc, _ = oracle.readout(pix, ref, cfg.threshold_e, cfg.clock_ticks, cfg.hold_ticks,
                                   cfg.reset_ticks)
    sel = np.isin(res["hit_pixel"], pix)
    check_hits((res["hit_pixel"][sel], res["hit_tick"][sel], res["hit_charge"][sel]), (hp, ht, hc),
               ref, pix, cfg.threshold_e, cfg.hold_ticks, cfg.reset_ticks)


@pytest.mark.parametrize("form", ["fp32", "compensated_gather", "exact_tent_fp64_tails", "tf32_dft_gemm",
                                  "split_tf32_dft_gemm", "split_bf16_dft_gemm"])
def test_precision_ladder_module200(form, capsys):
    """Each precision form of the module-plane event against the FP64 oracle on
    sampled pixels; the errors are printed (pytest -s) and bounded by the FP32
    tolerance."""
    cfg = synth.get_config("module200")
    dep, resp = synth.make_event(cfg)
    mode = 1 if form == "exact_tent_fp64_tails" else 0
    comp = 1 if form == "compensated_gather" else 0
    conv = {"tf32_dft_gemm": 1, "split_tf32_dft_gemm": 2, "split_bf16_dft_gemm": 3}.get(form, 0)
    tol = 1e-4 if conv in (1, 3) else WAVE_TOL
    sim = make_sim(cfg, resp, len(dep["x"]), max_blocks=3000, max_pixels=150000, effq_mode=mode,
                   compensated_gather=comp, conv_mode=conv)
    res = run(sim, dep, keep_qeff=False)
    p = oracle.params(cfg, effq_mode=mode)
    d = oracle.drift(p, dep)
    rows = _sampled_pixels(res, k=64, seed=3)
    pix = res["pixel_ids"][rows]
    ref = oracle.pixel_currents(p, d, resp, pix)
    err = pixel_rel_errors(res["waveforms"][rows], ref)
    ev = np.linalg.norm(res["waveforms"][rows] - ref) / np.linalg.norm(ref)
    with capsys.disabled():
        print(f"\nprecision {form}: max per-pixel rel L2 {err.max():.3e}, median {np.median(err):.3e}, "
              f"sampled-event rel L2 {ev:.3e}")
    assert err.max() <= tol


@pytest.mark.parametrize("mode,n_samples", [(1, 3), (2, 1)])
def test_readout_variants_tiny(mode, n_samples):
    """Successive digitisations (no reset between the 3 samples of a trigger) and
    fixed-charge quanta (Sec. II-E) on the full tiny event: the GPU hit lists equal
    the FP64 oracle's, except from an edge whose charge is within 1e-4 of threshold."""
    cfg = synth.get_config("tiny", readout_mode=mode, n_samples=n_samples)
    dep, resp = synth.make_event(cfg)
    res, ref, _ = _full_check(cfg, dep, resp, check_readout=False)
    assert res["status"][0] == 0, res["status"]
    hp, ht, hc, amb = oracle.readout(ref["pixel_ids"], ref["waveforms"], cfg.threshold_e, cfg.clock_ticks,
                                     cfg.hold_ticks, cfg.reset_ticks, mode=mode, n_samples=n_samples)
    assert len(hp) > 0
    check_hits_near_threshold((res["hit_pixel"], res["hit_tick"], res["hit_charge"]), (hp, ht, hc), amb,
                              ref["pixel_ids"], cfg.threshold_e)
    if mode == 2:
        assert np.all(res["hit_charge"] == np.float32(cfg.threshold_e))



@pytest.mark.parametrize("skip", [0, 1])
def test_fused_effq_convolve_tiny_full_parity(skip):
    """The persistent effective charge + convolution launch on the tiny event (7 blocks:
    most CTAs find the queue empty) against the full oracle, with dense and with
    covered-column Q^eff writes (the ring rows keep the previous block's columns)."""
    cfg = synth.get_config("tiny")
    dep, resp = synth.make_event(cfg)
    sim = make_sim(cfg, resp, len(dep["x"]), effq_skip_empty=skip, fused=True)
    assert sim.qeff.shape[0] <= 148
    _full_check(cfg, dep, resp, skip_empty=1, sim=sim)
    # a second event through the same ring rows
    dense = {k: v[::-1].copy() for k, v in synth.make_deposits(cfg, seed=cfg.seed + 77).items()}
    _full_check(cfg, dense, resp, skip_empty=1, sim=sim, check_readout=False)


def test_fp32_peak_measurement_is_plausible():
    """The measured FMA throughput (the convolution's roofline denominator) lies between
    half and 1.05 times the device's unit-count peak (SMs x 128 lanes x 2 flop x clock)."""
    import torch
    from paper_2602_12052_b300 import tred
    tf, sms = tred.tred_fp32_peak(iters=4096)
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    unit = sms * 128 * 2 * 2.032 / 1e3           # TFLOP/s at the B300's 2032 MHz maximum clock
    assert 0.5 * unit <= tf <= 1.05 * unit, (tf, unit)
