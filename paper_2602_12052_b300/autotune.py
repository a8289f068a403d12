"""Block-shape and FFT-length autotuner for batched runs.

Block shape trades binning against convolution (Sec. IV-B: small time bins keep the
block-sparse tensor sparse, but bins much smaller than the response multiply the
convolutions).  The tuner times one warm step of the batched path on a sample of
the events for each valid (bp, bt, lt) and keeps the fastest per deposit.  Every
candidate is a shape the parity tests cover."""
from __future__ import annotations

import time

import torch

from . import tred

# (bp, bt, lt): pixels per block side, ticks per block, FFT length along time
CANDIDATES = [(8, 64, 384), (8, 128, 384), (8, 128, 512), (8, 256, 512), (4, 256, 512), (8, 320, 768),
              (8, 320, 1024), (8, 512, 768), (8, 640, 1024)]


def valid(cfg, bp, bt, lt) -> bool:
    return (bp + cfg.kp - 1 <= 16 and bt % 64 == 0 and bt + cfg.nr - 1 <= lt and cfg.nt % bt == 0
            and cfg.npx % bp == 0 and cfg.n_sub ** 2 * bp ** 2 <= 6400)


def probe_blocks(cfg, events, resp, device=None):
    """Active blocks and an upper bound on active pixels of a batch (drift + binning only)."""
    import numpy as np
    dev = torch.device(device or "cuda")
    n = int(sum(len(e["x"]) for e in events))
    x = {k: torch.from_numpy(np.concatenate([e[k] for e in events]).astype(np.float32)).to(dev)
         for k in ("x", "y", "z", "t0", "ne")}
    ev = torch.from_numpy(np.concatenate([np.full(len(e["x"]), i, np.int32)
                                          for i, e in enumerate(events)])).to(dev)
    nblk = cfg.n_blocks * len(events)
    h = tred.Handle(tred.geometry(cfg, len(events)), tred.params(cfg), max(n, 1), nblk, 1)
    deps = tred.DepositBuffers(max(n, 1), dev)
    nb_dev = torch.zeros(1, dtype=torch.int32, device=dev)
    ids = torch.zeros(nblk, dtype=torch.int32, device=dev)
    cnt = torch.zeros_like(ids)
    off = torch.zeros(nblk + 1, dtype=torch.int32, device=dev)
    idx = torch.zeros(8 * max(n, 1), dtype=torch.int32, device=dev)
    tred.tred_drift_events(h, n, x["x"], x["y"], x["z"], x["t0"], x["ne"], ev, deps)
    tred.tred_blockbin(h, n, deps, ids, cnt, off, idx, nb_dev)
    nb = int(nb_dev.item())
    blocks = ids[:nb].cpu().numpy()
    h.close()
    return nb, count_pixels(cfg, len(events), blocks)


def count_pixels(cfg, n_events, block_ids):
    """Number of active pixels of an active-block list (union of the output
    footprints, clipped to each event's plane), computed on the host to size buffers."""
    import numpy as np
    R = (cfg.kp - 1) // 2
    nbx, nbt, nby_e = cfg.npx // cfg.bp, cfg.nt // cfg.bt, cfg.npx // cfg.bp
    cols = np.unique(np.asarray(block_ids) // nbt)
    bx, by = cols % nbx, cols // nbx
    ev = by // nby_e
    flags = np.zeros((n_events, cfg.npx, cfg.npx), dtype=bool)
    for dy in range(-R, cfg.bp + R):
        for dx in range(-R, cfg.bp + R):
            y = (by % nby_e) * cfg.bp + dy
            x = bx * cfg.bp + dx
            ok = (x >= 0) & (x < cfg.npx) & (y >= 0) & (y < cfg.npx)
            flags[ev[ok], y[ok], x[ok]] = True
    return int(flags.sum())


def make_batch(cfg, events, resp, chunk_blocks=2048, device=None, persistent=None, conv_mode=0, fuse_gather=None):
    """A BatchSimulator sized to the batch; in the FFT form (conv_mode 0) persistent
    (default: whenever the FFT length allows it, lt = 384 or 512) runs the effective charge
    and the convolution as one persistent launch over the batch's active-block queue; the
    direct form (conv_mode 4) runs chunks of chunk_blocks slots, by default (fuse_gather
    None) up to the output spectra and then the inverse time DFT fused with the gather
    where the block shape allows it (bp 8, kp 9, nr - 1 <= bt)."""
    nb, npix = probe_blocks(cfg, events, resp, device)
    if persistent is None:
        persistent = cfg.lt in (384, 512) and conv_mode == 0

    def make(fg):
        return tred.BatchSimulator(cfg, resp, events, max_blocks=nb + 8, max_pixels=npix,
                                   chunk_blocks=chunk_blocks, device=device, persistent=persistent,
                                   conv_mode=conv_mode, fuse_gather=fg)
    if conv_mode == 4 and fuse_gather is None:
        try:
            return make(True)
        except ValueError:
            return make(False)
    return make(bool(fuse_gather))


def autotune(cfg, events, resp, candidates=CANDIDATES, sample=8, device=None, conv_mode=0):
    """Return ((bp, bt, lt), {shape: ms per deposit}) measured on the first `sample` events
    (each shape in the form make_batch gives it: persistent at lt = 384 and 512)."""
    evs = events[:sample]
    n = sum(len(e["x"]) for e in evs)
    timings = {}
    for bp, bt, lt in candidates:
        if not valid(cfg, bp, bt, lt) or (conv_mode == 4 and lt not in (384, 512)):
            continue
        c = cfg.with_(bp=bp, bt=bt, lt=lt)
        sim = make_batch(c, evs, resp, device=device, conv_mode=conv_mode)
        sim.step()
        torch.cuda.synchronize()
        t = time.perf_counter()
        sim.step()
        torch.cuda.synchronize()
        timings[(bp, bt, lt)] = 1e3 * (time.perf_counter() - t) / n
        del sim
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    return best, timings
