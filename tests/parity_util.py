"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI on
seeded inputs and compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np

DEP_FIELDS = ["cell_x", "cell_y", "cell_t", "frac_x", "frac_y", "frac_t", "sigma_x", "sigma_y",
              "sigma_t", "lo_x", "lo_y", "lo_t", "hi_x", "hi_y", "hi_t", "q"]

# Tolerances (the metric's own: 1e-5 per pixel for FP32 forms, floor 1e-2 of the
# largest pixel norm; Q^eff per block in relative L2).
WAVE_TOL = 1e-5
WAVE_FLOOR = 1e-2
QEFF_TOL = 1e-5


def make_sim(cfg, resp, n, max_blocks=None, max_pixels=None, **kw):
    import torch
    from paper_2602_12052_b300 import build, tred
    build.build()
    return tred.Simulator(cfg, torch.from_numpy(np.ascontiguousarray(resp)),
                          max_deposits=max(n, 1),
                          max_blocks=max_blocks or min(cfg.n_blocks, 20000),
                          max_pixels=max_pixels or min(cfg.npx * cfg.npx, 400000), **kw)


def to_dev(dep):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in dep.items()}


def run(sim, dep, readout=True, keep_qeff=True, keep_waves=True):
    import torch
    n = len(dep["x"])
    t = to_dev(dep)
    sim.step(n, t["x"], t["y"], t["z"], t["t0"], t["ne"], readout=readout)
    res = sim.results()
    res["status"] = sim.status()
    res["deps"] = {f: sim.deps[f][:n].cpu().numpy() for f in DEP_FIELDS} if n else {}
    nb, npix = res["n_blocks"], res["n_pixels"]
    res["dep_offsets"] = sim.dep_offsets[:nb + 1].cpu().numpy()
    res["dep_index"] = sim.dep_index[:max(int(res["dep_offsets"][-1]) if nb else 0, 0)].cpu().numpy()
    if keep_qeff:
        res["qeff"] = sim.qeff[:nb].cpu().numpy()
    if keep_waves:
        res["waveforms"] = sim.waveforms[:npix].cpu().numpy()
    torch.cuda.synchronize()
    return res


def pixel_rel_errors(gpu, ref, floor_frac=WAVE_FLOOR):
    """Per-pixel ||gpu - ref|| / max(||ref||, floor_frac * max_q ||ref_q||)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    nrm = np.linalg.norm(ref, axis=1)
    floor = floor_frac * nrm.max() if nrm.size else 0.0
    den = np.maximum(nrm, floor)
    den[den == 0] = 1.0
    return np.linalg.norm(gpu - ref, axis=1) / den


def check_drift(res, d_oracle):
    """Windows bit-exact; cells consistent with the oracle's binary64 mean."""
    g = res["deps"]
    valid = d_oracle["valid"] == 1
    for ax, s in enumerate("xyt"):
        np.testing.assert_array_equal(g["lo_" + s][valid], d_oracle["lo"][valid, ax])
        np.testing.assert_array_equal(g["hi_" + s][valid], d_oracle["hi"][valid, ax])
        mu = d_oracle["mu"][valid, ax]
        np.testing.assert_array_equal(g["cell_" + s][valid], np.floor(mu).astype(np.int32))
        np.testing.assert_allclose(g["frac_" + s][valid], mu - np.floor(mu), rtol=0, atol=1e-6)
        np.testing.assert_allclose(g["sigma_" + s][valid], d_oracle["sig"][valid, ax], rtol=2e-7)
    np.testing.assert_allclose(g["q"][valid], d_oracle["q"][valid], rtol=1e-6)
    assert np.all(g["q"][~valid] == 0)
    assert np.all(g["lo_x"][~valid] > g["hi_x"][~valid])


def check_blocks(res, p, d_oracle):
    import oracle
    ids, counts = oracle.active_blocks(p, d_oracle)
    np.testing.assert_array_equal(res["block_ids"], ids)
    np.testing.assert_array_equal(res["block_counts"], counts)
    off = res["dep_offsets"]
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
    return ids, counts


def check_csr_sets(res, p, d_oracle, sample=None, seed=0):
    import oracle
    ids = res["block_ids"]
    off = res["dep_offsets"]
    idx = res["dep_index"]
    rng = np.random.default_rng(seed)
    sel = range(len(ids)) if sample is None else rng.choice(len(ids), min(sample, len(ids)), replace=False)
    for b in sel:
        # the binning sorts each block's list: same ids, same (ascending) order
        np.testing.assert_array_equal(idx[off[b]:off[b + 1]], oracle.block_deposits(p, d_oracle, int(ids[b])))


def check_qeff(gpu_q, ref_q, tol=QEFF_TOL):
    g = gpu_q.reshape(len(gpu_q), -1).astype(np.float64)
    r = ref_q.reshape(len(ref_q), -1)
    err = np.linalg.norm(g - r, axis=1) / np.maximum(np.linalg.norm(r, axis=1), 1e-300)
    assert err.max() <= tol, (err.max(), int(err.argmax()))
    return err


def hits_by_pixel(hp, ht, hc):
    out = {}
    for p_, t_, c_ in zip(hp, ht, hc):
        out.setdefault(int(p_), []).append((int(t_), float(c_)))
    return out


def check_hits(gpu_hits, ref_hits, ref_waves, pixel_ids, thr, hold, reset, charge_rtol=1e-4,
               amb_rtol=1e-4):
    """Hit lists identical per pixel, except from a first differing hit whose
    trigger edge has the oracle's integrated charge within amb_rtol * thr of the
    threshold.  ref_waves: oracle FP64 waveforms, rows aligned with pixel_ids.
    Returns the exempted pixels."""
    g = hits_by_pixel(*gpu_hits)
    r = hits_by_pixel(*ref_hits)
    exempt = []
    for row, pid in enumerate(pixel_ids):
        pid = int(pid)
        gl, rl = g.get(pid, []), r.get(pid, [])
        k = 0
        while k < min(len(gl), len(rl)) and gl[k][0] == rl[k][0]:
            assert abs(gl[k][1] - rl[k][1]) <= charge_rtol * max(abs(rl[k][1]), thr), (pid, gl[k], rl[k])
            k += 1
        if k == len(gl) == len(rl):
            continue
        start = 0 if k == 0 else rl[k - 1][0] + reset + 1
        edge = min(h[0] - hold for h in (gl[k:k + 1] + rl[k:k + 1]))
        C = float(np.sum(ref_waves[row][start:edge + 1]))
        assert abs(C - thr) <= amb_rtol * thr, (pid, gl[k:k + 2], rl[k:k + 2], C)
        exempt.append(pid)
    return exempt


def check_hits_near_threshold(gpu_hits, ref_hits, amb, pixel_ids, thr, charge_rtol=1e-4):
    """Hit lists identical per pixel (ticks equal, charges within charge_rtol of
    max(|charge|, thr)), except from a first differing hit at or after the oracle's
    first tested edge whose integrated charge lies within 1e-4 * thr of the threshold
    (``amb``, per row of pixel_ids).  Valid for every readout mode."""
    g = hits_by_pixel(*gpu_hits)
    r = hits_by_pixel(*ref_hits)
    exempt = []
    for row, pid in enumerate(pixel_ids):
        pid = int(pid)
        gl, rl = g.get(pid, []), r.get(pid, [])
        k = 0
        while k < min(len(gl), len(rl)) and gl[k][0] == rl[k][0]:
            assert abs(gl[k][1] - rl[k][1]) <= charge_rtol * max(abs(rl[k][1]), thr), (pid, gl[k], rl[k])
            k += 1
        if k == len(gl) == len(rl):
            continue
        first = min(h[0] for h in (gl[k:k + 1] + rl[k:k + 1]))
        assert 0 <= amb[row] <= first, (pid, gl[k:k + 2], rl[k:k + 2], int(amb[row]))
        exempt.append(pid)
    return exempt
