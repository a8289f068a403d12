"""Python face of libtred: torch tensors in, device pointers out.

Functions carry the C ABI's names and only marshal arguments (tensor -> pointer,
stream -> handle).  ``Simulator`` strings the calls together for one step of the
hot path on one CUDA stream with no host synchronisation inside.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import abi
from .abi import DEPOSIT_FIELDS, Deposits, Geometry, Params, ReadoutParams, TredError


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("libtred takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libtred takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def geometry(cfg, n_events: int = 1) -> Geometry:
    """Geometry struct from any object with the config's attribute names."""
    return Geometry(pitch_cm=cfg.pitch_cm, n_sub=cfg.n_sub, tick_us=cfg.tick_us, npx_x=cfg.npx,
                    npx_y=cfg.npx, nt=cfg.nt, bp=cfg.bp, bt=cfg.bt, kp=cfg.kp, nr=cfg.nr, lt=cfg.lt,
                    n_events=n_events)


def params(cfg, effq_mode=0, mpcp=1, compensated_gather=0, conv_mode=0, effq_skip_empty=0, conv_rows_cap=0,
           conv_keep_spectra=0) -> Params:
    return Params(v_cm_per_us=cfg.v_cm_per_us, DL_cm2_per_s=cfg.DL_cm2_per_s,
                  DT_cm2_per_s=cfg.DT_cm2_per_s, lifetime_us=cfg.lifetime_us,
                  sigma0_cells_xy=cfg.sigma0_cells_xy, sigma0_ticks=cfg.sigma0_ticks,
                  nsigma=cfg.nsigma, max_drift_cm=cfg.max_drift_cm, gl_order=cfg.gl_order,
                  effq_mode=effq_mode, conv_mode=conv_mode, mpcp=mpcp,
                  compensated_gather=compensated_gather, effq_skip_empty=effq_skip_empty,
                  conv_rows_cap=conv_rows_cap, conv_keep_spectra=conv_keep_spectra)


def fused_gather_shape_ok(cfg, conv_mode: int) -> bool:
    """The block shapes the direct form's fused inverse + gather covers (the library
    checks the same rules in tred_convolve_gather_supported): conv_mode 4, lt 384 or 512,
    8 x 8-pixel blocks with a 9 x 9 response (kp = bp + 1), a response no longer than a
    time block plus one tick, at most 128 time blocks."""
    return (conv_mode == 4 and cfg.lt in (384, 512) and cfg.bp == 8 and cfg.kp == cfg.bp + 1
            and cfg.nr - 1 <= cfg.bt and cfg.nt // cfg.bt <= 128)


def readout_params(cfg) -> ReadoutParams:
    return ReadoutParams(threshold_e=cfg.threshold_e, clock_ticks=cfg.clock_ticks,
                         hold_ticks=cfg.hold_ticks, reset_ticks=cfg.reset_ticks,
                         mode=getattr(cfg, "readout_mode", 0), n_samples=getattr(cfg, "n_samples", 1))


class DepositBuffers:
    """Caller-owned device arrays of ``tred_deposits`` (SoA, capacity n)."""

    INT_FIELDS = {"cell_x", "cell_y", "cell_t", "lo_x", "lo_y", "lo_t", "hi_x", "hi_y", "hi_t"}

    def __init__(self, n: int, device):
        self.n = n
        self.t = {}
        for f in DEPOSIT_FIELDS:
            dt = torch.int32 if f in self.INT_FIELDS else torch.float32
            self.t[f] = torch.empty(max(n, 1), dtype=dt, device=device)
        self.struct = Deposits(**{f: self.t[f].data_ptr() for f in DEPOSIT_FIELDS})

    def __getitem__(self, k):
        return self.t[k]


class Handle:
    """Owns a ``tred_handle*``; destroyed with the object."""

    def __init__(self, geom: Geometry, prm: Params, max_deposits: int, max_blocks: int,
                 max_pixels: int):
        self.lib = abi.load()
        self.geom, self.prm = geom, prm
        self.max_deposits, self.max_blocks, self.max_pixels = max_deposits, max_blocks, max_pixels
        h = ctypes.c_void_p()
        rc = self.lib.tred_create(ctypes.byref(geom), ctypes.byref(prm), max_deposits, max_blocks,
                                  max_pixels, ctypes.byref(h))
        if rc != abi.TRED_OK:
            raise TredError(rc, "tred_create failed (see stderr)")
        self.h = h

    def check(self, rc: int):
        if rc != abi.TRED_OK:
            raise TredError(rc, self.lib.tred_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tred_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- the ABI, by name
def tred_set_response(h: Handle, resp: torch.Tensor, stream=None):
    h.check(h.lib.tred_set_response(h.h, _ptr(resp), _stream(stream)))


def tred_drift(h: Handle, n: int, x, y, z, t0, ne, out: DepositBuffers, stream=None):
    h.check(h.lib.tred_drift(h.h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(t0), _ptr(ne),
                             ctypes.byref(out.struct), _stream(stream)))


def tred_drift_events(h: Handle, n: int, x, y, z, t0, ne, event, out: DepositBuffers, stream=None):
    h.check(h.lib.tred_drift_events(h.h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(t0), _ptr(ne), _ptr(event),
                                    ctypes.byref(out.struct), _stream(stream)))


def tred_drift_lines(h: Handle, n: int, x0, y0, z0, x1, y1, z1, t0, ne, out: DepositBuffers, half, stream=None):
    h.check(h.lib.tred_drift_lines(h.h, n, _ptr(x0), _ptr(y0), _ptr(z0), _ptr(x1), _ptr(y1), _ptr(z1), _ptr(t0),
                                   _ptr(ne), ctypes.byref(out.struct), _ptr(half), _stream(stream)))


def tred_effq_lines(h: Handle, n: int, deps: DepositBuffers, half, block_ids, dep_offsets, dep_index,
                    n_blocks_dev, qeff, stream=None):
    h.check(h.lib.tred_effq_lines(h.h, n, ctypes.byref(deps.struct), _ptr(half), _ptr(block_ids),
                                  _ptr(dep_offsets), _ptr(dep_index), _ptr(n_blocks_dev), _ptr(qeff),
                                  _stream(stream)))


def tred_effq_range(h: Handle, n: int, deps: DepositBuffers, block_ids, dep_offsets, dep_index,
                    n_blocks_dev, slot_base: int, slot_count: int, qeff, stream=None):
    h.check(h.lib.tred_effq_range(h.h, n, ctypes.byref(deps.struct), _ptr(block_ids), _ptr(dep_offsets),
                                  _ptr(dep_index), _ptr(n_blocks_dev), slot_base, slot_count, _ptr(qeff),
                                  _stream(stream)))


def tred_convolve_range(h: Handle, block_ids, n_blocks_dev, slot_base: int, slot_count: int, qeff,
                        out_blocks, stream=None):
    h.check(h.lib.tred_convolve_range(h.h, _ptr(block_ids), _ptr(n_blocks_dev), slot_base, slot_count,
                                      _ptr(qeff), _ptr(out_blocks), _stream(stream)))


def tred_blockbin(h: Handle, n: int, deps: DepositBuffers, block_ids, block_counts, dep_offsets,
                  dep_index, n_blocks_dev, stream=None):
    h.check(h.lib.tred_blockbin(h.h, n, ctypes.byref(deps.struct), _ptr(block_ids),
                                _ptr(block_counts), _ptr(dep_offsets), _ptr(dep_index),
                                dep_index.numel(), _ptr(n_blocks_dev), _stream(stream)))


def tred_effq(h: Handle, n: int, deps: DepositBuffers, block_ids, dep_offsets, dep_index,
              n_blocks_dev, qeff, stream=None):
    h.check(h.lib.tred_effq(h.h, n, ctypes.byref(deps.struct), _ptr(block_ids), _ptr(dep_offsets),
                            _ptr(dep_index), _ptr(n_blocks_dev), _ptr(qeff), _stream(stream)))


def tred_effq_convolve(h: Handle, n: int, deps: DepositBuffers, block_ids, dep_offsets, dep_index, n_blocks_dev,
                       qeff_ring, out_blocks, stream=None):
    h.check(h.lib.tred_effq_convolve(h.h, n, ctypes.byref(deps.struct), _ptr(block_ids), _ptr(dep_offsets),
                                     _ptr(dep_index), _ptr(n_blocks_dev), _ptr(qeff_ring), qeff_ring.shape[0],
                                     _ptr(out_blocks), _stream(stream)))


def tred_convolve(h: Handle, block_ids, n_blocks_dev, qeff, out_blocks, stream=None):
    h.check(h.lib.tred_convolve(h.h, _ptr(block_ids), _ptr(n_blocks_dev), _ptr(qeff),
                                _ptr(out_blocks), _stream(stream)))


def tred_gather_pixels(h: Handle, block_ids, n_blocks_dev, out_blocks, pixel_ids, waveforms,
                       n_pixels_dev, stream=None):
    h.check(h.lib.tred_gather_pixels(h.h, _ptr(block_ids), _ptr(n_blocks_dev), _ptr(out_blocks),
                                     _ptr(pixel_ids), _ptr(waveforms), _ptr(n_pixels_dev),
                                     _stream(stream)))


def tred_gather_readout(h: Handle, block_ids, n_blocks_dev, out_blocks, pixel_ids, waveforms, n_pixels_dev,
                        rp: ReadoutParams, hit_pixel, hit_tick, hit_charge, n_hits_dev, stream=None):
    h.check(h.lib.tred_gather_readout(h.h, _ptr(block_ids), _ptr(n_blocks_dev), _ptr(out_blocks), _ptr(pixel_ids),
                                      _ptr(waveforms), _ptr(n_pixels_dev), ctypes.byref(rp), _ptr(hit_pixel),
                                      _ptr(hit_tick), _ptr(hit_charge), _ptr(n_hits_dev), hit_pixel.numel(),
                                      _stream(stream)))


def tred_convolve_gather_supported(h: Handle) -> bool:
    """Whether the handle's shape allows tred_convolve_gather_readout."""
    return h.lib.tred_convolve_gather_supported(h.h) == 1


def tred_convolve_gather_readout(h: Handle, block_ids, n_blocks_dev, qeff, pixel_ids, waveforms, n_pixels_dev,
                                 rp: ReadoutParams | None = None, hit_pixel=None, hit_tick=None, hit_charge=None,
                                 n_hits_dev=None, stream=None):
    """Convolution (direct form) + gather (+ readout when rp is given) without the
    per-block output buffer: the inverse time DFT runs per pixel tile into the waves."""
    h.check(h.lib.tred_convolve_gather_readout(
        h.h, _ptr(block_ids), _ptr(n_blocks_dev), _ptr(qeff), _ptr(pixel_ids), _ptr(waveforms), _ptr(n_pixels_dev),
        ctypes.byref(rp) if rp is not None else None, _ptr(hit_pixel) if hit_pixel is not None else None,
        _ptr(hit_tick) if hit_tick is not None else None, _ptr(hit_charge) if hit_charge is not None else None,
        _ptr(n_hits_dev) if n_hits_dev is not None else None, hit_pixel.numel() if hit_pixel is not None else 0,
        _stream(stream)))


def tred_convolve_spectra_range(h: Handle, block_ids, n_blocks_dev, slot_base: int, slot_count: int, qeff,
                                stream=None):
    """The direct form's convolution of a slot range up to the output spectra (kept in the
    handle for tred_wave_gather_readout)."""
    h.check(h.lib.tred_convolve_spectra_range(h.h, _ptr(block_ids), _ptr(n_blocks_dev), int(slot_base),
                                              int(slot_count), _ptr(qeff), _stream(stream)))


def tred_wave_gather_readout(h: Handle, block_ids, n_blocks_dev, pixel_ids, waveforms, n_pixels_dev,
                             rp: ReadoutParams | None = None, hit_pixel=None, hit_tick=None, hit_charge=None,
                             n_hits_dev=None, stream=None):
    """Pixel list, the inverse time DFT per pixel tile into the waveforms (from the kept
    spectra of every active slot) and, with rp, the readout."""
    h.check(h.lib.tred_wave_gather_readout(
        h.h, _ptr(block_ids), _ptr(n_blocks_dev), _ptr(pixel_ids), _ptr(waveforms), _ptr(n_pixels_dev),
        ctypes.byref(rp) if rp is not None else None, _ptr(hit_pixel) if hit_pixel is not None else None,
        _ptr(hit_tick) if hit_tick is not None else None, _ptr(hit_charge) if hit_charge is not None else None,
        _ptr(n_hits_dev) if n_hits_dev is not None else None, hit_pixel.numel() if hit_pixel is not None else 0,
        _stream(stream)))


def tred_readout(h: Handle, rp: ReadoutParams, pixel_ids, waveforms, n_pixels_dev, hit_pixel,
                 hit_tick, hit_charge, n_hits_dev, stream=None):
    h.check(h.lib.tred_readout(h.h, ctypes.byref(rp), _ptr(pixel_ids), _ptr(waveforms),
                               _ptr(n_pixels_dev), _ptr(hit_pixel), _ptr(hit_tick),
                               _ptr(hit_charge), _ptr(n_hits_dev), hit_pixel.numel(),
                               _stream(stream)))


def tred_wait_selftest(h: Handle, limit_cycles: int, stream=None):
    h.check(h.lib.tred_wait_selftest(h.h, int(limit_cycles), _stream(stream)))


def tred_sync_status(h: Handle, stream=None):
    buf = (ctypes.c_int32 * abi.TRED_STATUS_WORDS)()
    h.check(h.lib.tred_sync_status(h.h, _stream(stream), ctypes.cast(buf, ctypes.c_void_p)))
    return list(buf)


KT_EFFQ, KT_DX_FWD, KT_DX_GEMM, KT_DX_INV, KT_DX_WAVE = 0, 1, 2, 3, 4
KT_NAMES = {KT_EFFQ: "k_effq_blocks", KT_DX_FWD: "k_dx_fwd", KT_DX_GEMM: "k_dx_gemm", KT_DX_INV: "k_dx_inv",
            KT_DX_WAVE: "k_dx_wave"}


def tred_set_kernel_timing(h: Handle, enable: bool) -> None:
    h.check(h.lib.tred_set_kernel_timing(h.h, 1 if enable else 0))


def tred_kernel_time(h: Handle, which: int):
    """(milliseconds, launches) of one kernel class since the previous query."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int32(0)
    h.check(h.lib.tred_kernel_time(h.h, which, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def tred_direct_counts(h: Handle):
    """(non-empty rows, non-empty columns) of the last conv_mode 4 pass."""
    r = ctypes.c_int64(0)
    c = ctypes.c_int64(0)
    h.check(h.lib.tred_direct_counts(h.h, ctypes.byref(r), ctypes.byref(c)))
    return r.value, c.value


def tred_launch_count(h: Handle) -> int:
    c = ctypes.c_int64()
    h.check(h.lib.tred_launch_count(h.h, ctypes.byref(c)))
    return int(c.value)


def tred_set_transport(h: Handle, prm: Params):
    h.check(h.lib.tred_set_transport(h.h, ctypes.byref(prm)))
    h.prm = prm


def tred_residual(h: Handle, pixel_ids, n_pixels_dev, waveforms, target_ids, target_waves, resid,
                  loss_dev, stream=None):
    h.check(h.lib.tred_residual(h.h, _ptr(pixel_ids), _ptr(n_pixels_dev), _ptr(waveforms),
                                _ptr(target_ids), target_ids.numel(), _ptr(target_waves),
                                _ptr(resid), _ptr(loss_dev), _stream(stream)))


def tred_adjoint(h: Handle, n: int, deps: DepositBuffers, block_ids, dep_offsets, dep_index,
                 n_blocks_dev, pixel_ids, n_pixels_dev, resid, dqeff, grad7, stream=None):
    h.check(h.lib.tred_adjoint(h.h, n, ctypes.byref(deps.struct), _ptr(block_ids), _ptr(dep_offsets),
                               _ptr(dep_index), _ptr(n_blocks_dev), _ptr(pixel_ids),
                               _ptr(n_pixels_dev), _ptr(resid), _ptr(dqeff), _ptr(grad7),
                               _stream(stream)))


def tred_param_grads(h: Handle, n: int, z, deps: DepositBuffers, grad7, grad_inputs, grad_global,
                     stream=None):
    h.check(h.lib.tred_param_grads(h.h, n, _ptr(z), ctypes.byref(deps.struct), _ptr(grad7),
                                   _ptr(grad_inputs), _ptr(grad_global), _stream(stream)))


def tred_fp32_peak(iters: int = 4096, stream=None):
    """Measured FP32 FMA throughput of the current device in TFLOP/s and its SM count
    (the convolution's roofline denominator)."""
    lib = abi.load()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sink = torch.empty(props.multi_processor_count * 2048, dtype=torch.float32, device="cuda")
    tf = ctypes.c_double()
    sms = ctypes.c_int32()
    rc = lib.tred_fp32_peak(_ptr(sink), sink.numel(), int(iters), _stream(stream), ctypes.byref(tf), ctypes.byref(sms))
    if rc != abi.TRED_OK:
        raise abi.TredError(rc, "tred_fp32_peak")
    return float(tf.value), int(sms.value)


def tred_reset_status(h: Handle, stream=None):
    h.check(h.lib.tred_reset_status(h.h, _stream(stream)))


# ----------------------------------------------------------------- one step of the path
class Simulator:
    """All device buffers for one configuration and the ordered ABI calls of a step:
    drift -> blockbin -> effq -> convolve -> gather -> readout (Fig. flowchart)."""

    def __init__(self, cfg, resp: torch.Tensor, max_deposits: int, max_blocks: int,
                 max_pixels: int, max_pairs: int | None = None, max_hits: int | None = None,
                 effq_mode=0, mpcp=1, compensated_gather=0, conv_mode=0, effq_skip_empty=0, device=None,
                 fused=False, conv_rows_cap=0, fuse_gather=False):
        self.cfg = cfg
        self.mpcp = mpcp
        self.fused = bool(fused)
        # fuse_gather: conv_mode 4's inverse time DFT per pixel tile straight into the waves
        # (tred_convolve_gather_readout); out_blocks is then not written
        self.fuse_gather = bool(fuse_gather)
        self.conv_mode = conv_mode
        if self.fuse_gather and not fused_gather_shape_ok(cfg, conv_mode):
            raise ValueError("fuse_gather needs conv_mode 4, lt 384 or 512, bp 8, kp 9, nr - 1 <= bt, nt / bt <= 128")
        self.device = torch.device(device or "cuda")
        self.h = Handle(geometry(cfg), params(cfg, effq_mode, mpcp, compensated_gather, conv_mode, effq_skip_empty,
                                              conv_rows_cap, 1 if self.fuse_gather and conv_mode == 4 else 0),
                        max_deposits, max_blocks, max_pixels)
        self.rp = readout_params(cfg)
        d = self.device
        ns, bp, bt, lt = cfg.n_sub, cfg.bp, cfg.bt, cfg.lt
        self.deps = DepositBuffers(max_deposits, d)
        self.block_ids = torch.zeros(max_blocks, dtype=torch.int32, device=d)
        self.block_counts = torch.zeros(max_blocks, dtype=torch.int32, device=d)
        self.dep_offsets = torch.zeros(max_blocks + 1, dtype=torch.int32, device=d)
        self.dep_index = torch.zeros(max_pairs or 8 * max_deposits, dtype=torch.int32, device=d)
        self.counts = torch.zeros(4, dtype=torch.int32, device=d)    # nb, npix, nhits, spare
        # fused: the effective charge and the convolution in one persistent launch
        # (tred_effq_convolve), Q^eff staged in one ring row per resident CTA
        qrows = min(torch.cuda.get_device_properties(d).multi_processor_count, max_blocks, 8192) if self.fused \
            else max_blocks
        self.qeff = torch.empty((qrows, ns, ns, bp, bp, bt), dtype=torch.float32, device=d)
        if self.fuse_gather and not tred_convolve_gather_supported(self.h):
            raise ValueError("fuse_gather needs conv_mode 4, bp 8, kp 9, nr - 1 <= bt, nt / bt <= 128 and "
                             "max_blocks within one pass of the direct form")
        self.out_blocks = torch.empty((1 if self.fuse_gather else max_blocks, 16, 16, lt), dtype=torch.float32,
                                      device=d)
        self.pixel_ids = torch.zeros(max_pixels, dtype=torch.int32, device=d)
        self.waveforms = torch.empty((max_pixels, cfg.nt), dtype=torch.float32, device=d)
        mh = max_hits or 4 * max_pixels
        self.hit_pixel = torch.zeros(mh, dtype=torch.int32, device=d)
        self.hit_tick = torch.zeros(mh, dtype=torch.int32, device=d)
        self.hit_charge = torch.zeros(mh, dtype=torch.float32, device=d)
        self.resp = resp.to(d, torch.float32).contiguous()
        tred_set_response(self.h, self.resp)

    @property
    def n_blocks_dev(self):
        return self.counts[0:1]

    @property
    def n_pixels_dev(self):
        return self.counts[1:2]

    @property
    def n_hits_dev(self):
        return self.counts[2:3]

    def step(self, n, x, y, z, t0, ne, stream=None, readout=True):
        """Enqueue one pass of the hot path for n deposits already on the device."""
        tred_drift(self.h, n, x, y, z, t0, ne, self.deps, stream)
        tred_blockbin(self.h, n, self.deps, self.block_ids, self.block_counts, self.dep_offsets,
                      self.dep_index, self.n_blocks_dev, stream)
        if self.fused:
            tred_effq_convolve(self.h, n, self.deps, self.block_ids, self.dep_offsets, self.dep_index,
                               self.n_blocks_dev, self.qeff, self.out_blocks, stream)
        else:
            tred_effq(self.h, n, self.deps, self.block_ids, self.dep_offsets, self.dep_index,
                      self.n_blocks_dev, self.qeff, stream)
        self._convolve_gather(stream, readout)

    def _convolve_gather(self, stream, readout):
        if self.fuse_gather:
            hits = (self.rp, self.hit_pixel, self.hit_tick, self.hit_charge, self.n_hits_dev) if readout else ()
            tred_convolve_gather_readout(self.h, self.block_ids, self.n_blocks_dev, self.qeff, self.pixel_ids,
                                         self.waveforms, self.n_pixels_dev, *hits, stream=stream)
            return
        if not self.fused:
            tred_convolve(self.h, self.block_ids, self.n_blocks_dev, self.qeff, self.out_blocks, stream)
        if readout:      # gather and readout in one call (readout skips pixels that cannot trigger)
            tred_gather_readout(self.h, self.block_ids, self.n_blocks_dev, self.out_blocks, self.pixel_ids,
                                self.waveforms, self.n_pixels_dev, self.rp, self.hit_pixel, self.hit_tick,
                                self.hit_charge, self.n_hits_dev, stream)
        else:
            tred_gather_pixels(self.h, self.block_ids, self.n_blocks_dev, self.out_blocks,
                               self.pixel_ids, self.waveforms, self.n_pixels_dev, stream)

    def status(self, stream=None):
        return tred_sync_status(self.h, stream)

    def results(self):
        """Host copies of the step's results (synchronising)."""
        torch.cuda.synchronize()
        nb, npix, nh = (int(v) for v in self.counts[:3].cpu())
        return {
            "n_blocks": nb, "n_pixels": npix, "n_hits": nh,
            "block_ids": self.block_ids[:nb].cpu().numpy(),
            "block_counts": self.block_counts[:nb].cpu().numpy(),
            "pixel_ids": self.pixel_ids[:npix].cpu().numpy(),
            "hit_pixel": self.hit_pixel[:nh].cpu().numpy(),
            "hit_tick": self.hit_tick[:nh].cpu().numpy(),
            "hit_charge": self.hit_charge[:nh].cpu().numpy(),
        }


class StreamRunner:
    """A stream of host-resident events through one Simulator with the host copies
    overlapped with the computation.  Event k's deposits are copied (from pinned host
    memory, on an input stream) into one of two device input sets while event k - 1
    computes; at the end of its step the device counts and the capacity-sized hit list
    are copied on the device into one of two staging sets, and read back to pinned host
    memory on an output stream while event k + 1 computes.  Results come back in event
    order, two events behind the submissions (queue depth two).  Every wait is a CUDA
    event: the host blocks only when it takes a result."""

    FIELDS = ("x", "y", "z", "t0", "ne")

    def __init__(self, sim: Simulator, max_deposits: int, readout: bool = True, timing: bool = False):
        self.sim = sim
        self.readout = readout
        # timing: CUDA events around each step on the compute stream; take() then adds
        # the step's device milliseconds to its result ("step_ms")
        self.timing = timing
        self.ev_t = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        d = sim.device
        self.compute = torch.cuda.current_stream(d)
        self.s_in = torch.cuda.Stream(d)
        self.s_out = torch.cuda.Stream(d)
        self.inputs = [{f: torch.empty(max(max_deposits, 1), dtype=torch.float32, device=d) for f in self.FIELDS}
                       for _ in range(2)]
        self.stage = [{"counts": torch.empty_like(sim.counts), "hit_pixel": torch.empty_like(sim.hit_pixel),
                       "hit_tick": torch.empty_like(sim.hit_tick), "hit_charge": torch.empty_like(sim.hit_charge)}
                      for _ in range(2)]
        self.host = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in st.items()}
                     for st in self.stage]
        self.ev_in_ready = [torch.cuda.Event() for _ in range(2)]
        self.ev_step_done = [torch.cuda.Event() for _ in range(2)]
        self.ev_d2h_done = [torch.cuda.Event() for _ in range(2)]
        self.pending = []          # (slot, tag) of the submitted events not yet taken, oldest first
        self.count = 0
        self.h2d_bytes = 0
        self.d2h_bytes = sum(v.numel() * v.element_size() for v in self.stage[0].values())

    def submit(self, host: dict, n: int, tag=None):
        """Enqueue one event: host[f] pinned float32 tensors of at least n deposits.
        Returns the (tag, result) of the event submitted two calls earlier, or None."""
        out = self.take() if len(self.pending) == 2 else None
        b = self.count % 2
        inp, st = self.inputs[b], self.stage[b]
        with torch.cuda.stream(self.s_in):
            if self.count >= 2:
                self.s_in.wait_event(self.ev_step_done[b])   # event k - 2 has read this input set
            for f in self.FIELDS:
                if n:
                    inp[f][:n].copy_(host[f][:n], non_blocking=True)
            self.ev_in_ready[b].record(self.s_in)
        self.h2d_bytes = 4 * n * len(self.FIELDS)
        self.compute.wait_event(self.ev_in_ready[b])
        if self.timing:
            self.ev_t[b][0].record(self.compute)
        self.sim.step(n, inp["x"], inp["y"], inp["z"], inp["t0"], inp["ne"], stream=self.compute,
                      readout=self.readout)
        if self.timing:
            self.ev_t[b][1].record(self.compute)
        if self.count >= 2:
            self.compute.wait_event(self.ev_d2h_done[b])   # event k - 2's staging has been read back
        with torch.cuda.stream(self.compute):
            st["counts"].copy_(self.sim.counts, non_blocking=True)
            st["hit_pixel"].copy_(self.sim.hit_pixel, non_blocking=True)
            st["hit_tick"].copy_(self.sim.hit_tick, non_blocking=True)
            st["hit_charge"].copy_(self.sim.hit_charge, non_blocking=True)
        self.ev_step_done[b].record(self.compute)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(self.ev_step_done[b])
            for k, v in st.items():
                self.host[b][k].copy_(v, non_blocking=True)
            self.ev_d2h_done[b].record(self.s_out)
        self.pending.append((b, tag))
        self.count += 1
        return out

    def take(self):
        """Wait for the oldest submitted event and return (tag, result): counts (n_blocks,
        n_pixels, n_hits) and host copies of its hit list."""
        b, tag = self.pending.pop(0)
        self.ev_d2h_done[b].synchronize()
        h = self.host[b]
        nb, npix, nh = (int(v) for v in h["counts"][:3])
        nh_k = min(nh, h["hit_pixel"].numel())
        res = {"n_blocks": nb, "n_pixels": npix, "n_hits": nh,
               "hit_pixel": h["hit_pixel"][:nh_k].numpy().copy(), "hit_tick": h["hit_tick"][:nh_k].numpy().copy(),
               "hit_charge": h["hit_charge"][:nh_k].numpy().copy()}
        if self.timing:
            res["step_ms"] = self.ev_t[b][0].elapsed_time(self.ev_t[b][1])
        return tag, res

    def drain(self):
        """Every result still pending, oldest first."""
        out = []
        while self.pending:
            out.append(self.take())
        return out


# ----------------------------------------------------------------- differentiation
class LineSimulator(Simulator):
    """The hot path for line-shape track segments (Sec. II-C, Eq. qline): segment
    transport, the same binning, the segments' effective charge, then the same
    convolution, gather and readout."""

    def __init__(self, cfg, resp: torch.Tensor, max_segments: int, max_blocks: int, max_pixels: int, **kw):
        super().__init__(cfg, resp, max_deposits=max_segments, max_blocks=max_blocks, max_pixels=max_pixels, **kw)
        self.half = torch.zeros(3 * max(max_segments, 1), dtype=torch.float32, device=self.device)

    def step_lines(self, n, x0, y0, z0, x1, y1, z1, t0, ne, stream=None, readout=True):
        """Enqueue one pass for n segments already on the device."""
        tred_drift_lines(self.h, n, x0, y0, z0, x1, y1, z1, t0, ne, self.deps, self.half[:3 * max(n, 1)], stream)
        tred_blockbin(self.h, n, self.deps, self.block_ids, self.block_counts, self.dep_offsets,
                      self.dep_index, self.n_blocks_dev, stream)
        tred_effq_lines(self.h, n, self.deps, self.half[:3 * max(n, 1)], self.block_ids, self.dep_offsets,
                        self.dep_index, self.n_blocks_dev, self.qeff, stream)
        self._convolve_gather(stream, readout)


class DiffState:
    """Buffers of the backward pass bound to a Simulator."""

    def __init__(self, sim: "Simulator"):
        if sim.fused:
            raise ValueError("the adjoint needs a Simulator with fused=False (dL/dQeff uses the full Q^eff buffer)")
        d = sim.device
        self.sim = sim
        self.resid = torch.zeros((sim.h.max_pixels, sim.cfg.nt), dtype=torch.float32, device=d)
        self.loss = torch.zeros(1, dtype=torch.float64, device=d)
        self.grad7 = torch.zeros((sim.h.max_deposits, 7), dtype=torch.float32, device=d)
        self.gin = torch.zeros((sim.h.max_deposits, 4), dtype=torch.float32, device=d)
        self.gglob = torch.zeros(3, dtype=torch.float64, device=d)


class TredLoss(torch.autograd.Function):
    """L = 1/2 sum over pixels and ticks of (I - I*)^2 for one event, differentiable in
    the deposits' x, y, t0, n_e and in the transport constants DL, DT and lifetime
    (Sec. V-C).  Forward: the CUDA hot path (drift -> blockbin -> effq -> convolve ->
    gather) and the residual against the target rows; backward: tred_adjoint and
    tred_param_grads (windows held fixed, quadrature recomputed)."""

    @staticmethod
    def forward(ctx, state: DiffState, target_ids, target_waves, x, y, z, t0, ne, DL, DT, tau):
        sim = state.sim
        prm = params(sim.cfg, mpcp=sim.mpcp, conv_mode=sim.conv_mode)   # the transport constants are taken
        prm.DL_cm2_per_s, prm.DT_cm2_per_s, prm.lifetime_us = float(DL), float(DT), float(tau)
        tred_set_transport(sim.h, prm)
        n = x.numel()
        sim.step(n, x, y, z, t0, ne, readout=False)
        tred_residual(sim.h, sim.pixel_ids, sim.n_pixels_dev, sim.waveforms, target_ids, target_waves,
                      state.resid, state.loss)
        ctx.state, ctx.n = state, n
        ctx.pdev = [v.device if torch.is_tensor(v) else None for v in (DL, DT, tau)]
        ctx.save_for_backward(z)
        return state.loss.to(torch.float32).reshape(())

    @staticmethod
    def backward(ctx, g):
        state, n = ctx.state, ctx.n
        (z,) = ctx.saved_tensors
        sim = state.sim
        tred_adjoint(sim.h, n, sim.deps, sim.block_ids, sim.dep_offsets, sim.dep_index, sim.n_blocks_dev,
                     sim.pixel_ids, sim.n_pixels_dev, state.resid, sim.qeff, state.grad7)
        tred_param_grads(sim.h, n, z, sim.deps, state.grad7, state.gin, state.gglob)
        gin = state.gin[:n] * g.to(state.gin.device)
        gg = (state.gglob * g.to(state.gglob.device).double()).to(torch.float32)
        gp = [gg[k].to(dv) if dv is not None else None for k, dv in enumerate(ctx.pdev)]
        return (None, None, None, gin[:, 0], gin[:, 1], None, gin[:, 2], gin[:, 3], gp[0], gp[1], gp[2])


# ----------------------------------------------------------------- batches of events
class BatchSimulator:
    """Many events of uneven size in one pass (Sec. III-B-2 hierarchical batching).

    Events are stacked along y (geometry n_events); every kernel runs once per step
    as a persistent grid over the global active-block list of all events.  With
    ``persistent`` (lt = 384 or 512, the FFT form) the effective charge and the convolution
    are one persistent launch over that list (tred_effq_convolve), Q^eff staged in one ring
    row per resident CTA; otherwise (and always with ``conv_mode`` 4, the direct spatial
    form) they run over sub-batches of ``chunk_blocks`` slots
    so that Q^eff never needs more than one chunk of device memory.  The launch
    sequence is fixed (the block count stays on the device), so ``capture()`` can
    record a step in a CUDA graph."""

    def __init__(self, cfg, resp: torch.Tensor, events, max_blocks: int, max_pixels: int,
                 chunk_blocks: int = 2048, max_hits: int | None = None, mpcp=1, device=None,
                 n_events: int | None = None, max_deposits: int | None = None, persistent: bool = False,
                 effq_skip_empty: int = 0, conv_mode: int = 0, fuse_gather: bool = False):
        self.cfg = cfg
        self.device = d = torch.device(device or "cuda")
        # fuse_gather (conv_mode 4): the chunks stop at the output spectra, kept for every
        # slot, and one launch inverts them per pixel tile into the waveforms
        self.fuse_gather = bool(fuse_gather) and conv_mode == 4 and not persistent
        if self.fuse_gather and not fused_gather_shape_ok(cfg, conv_mode):
            raise ValueError("fuse_gather needs conv_mode 4, lt 384 or 512, bp 8, kp 9, nr - 1 <= bt, nt / bt <= 128")
        self.n_events = n_events or len(events)
        cap = max_deposits or int(sum(len(e["x"]) for e in events))
        # the persistent launch runs the FFT form; the direct form (conv_mode 4) runs the
        # chunks and reads only the covered columns
        self.persistent = bool(persistent) and conv_mode == 0
        skip = 1 if (self.persistent or conv_mode == 4) else effq_skip_empty
        self.h = Handle(geometry(cfg, self.n_events),
                        params(cfg, mpcp=mpcp, effq_skip_empty=skip, conv_mode=conv_mode,
                               conv_keep_spectra=1 if self.fuse_gather else 0), max(cap, 1),
                        max_blocks, max_pixels)
        if self.fuse_gather and not tred_convolve_gather_supported(self.h):
            raise ValueError("fuse_gather needs conv_mode 4, bp 8, kp 9, nr - 1 <= bt and nt / bt <= 128")
        self.rp = readout_params(cfg)
        if self.persistent:
            # one Q^eff ring row per resident CTA of the persistent launch
            sms = torch.cuda.get_device_properties(d).multi_processor_count
            self.chunk = min(sms, max_blocks, 8192)
        else:
            self.chunk = min(chunk_blocks, max_blocks)
        self.max_blocks = max_blocks
        self.inputs = {k: torch.zeros(max(cap, 1), dtype=torch.float32, device=d)
                       for k in ("x", "y", "z", "t0", "ne")}
        self.inputs["event"] = torch.zeros(max(cap, 1), dtype=torch.int32, device=d)
        self.load(events)
        ns, bp, bt, lt = cfg.n_sub, cfg.bp, cfg.bt, cfg.lt
        self.deps = DepositBuffers(max(cap, 1), d)
        self.block_ids = torch.zeros(max_blocks, dtype=torch.int32, device=d)
        self.block_counts = torch.zeros(max_blocks, dtype=torch.int32, device=d)
        self.dep_offsets = torch.zeros(max_blocks + 1, dtype=torch.int32, device=d)
        # a support is shorter than a block on every axis, so a deposit meets at most
        # 2 x 2 x 2 blocks: 8 (deposit, block) pairs per deposit of the capacity
        self.dep_index = torch.zeros(8 * max(cap, 1), dtype=torch.int32, device=d)
        self.counts = torch.zeros(4, dtype=torch.int32, device=d)
        self.qeff = torch.empty((self.chunk, ns, ns, bp, bp, bt), dtype=torch.float32, device=d)
        self.out_blocks = torch.empty((1 if self.fuse_gather else max_blocks, 16, 16, lt), dtype=torch.float32,
                                      device=d)
        self.pixel_ids = torch.zeros(max_pixels, dtype=torch.int32, device=d)
        self.waveforms = torch.empty((max_pixels, cfg.nt), dtype=torch.float32, device=d)
        mh = max_hits or 4 * max_pixels
        self.hit_pixel = torch.zeros(mh, dtype=torch.int32, device=d)
        self.hit_tick = torch.zeros(mh, dtype=torch.int32, device=d)
        self.hit_charge = torch.zeros(mh, dtype=torch.float32, device=d)
        self.resp = resp.to(d, torch.float32).contiguous()
        tred_set_response(self.h, self.resp)
        self.graph = None

    def load(self, events):
        """Copy a batch of events (at most n_events, within the deposit capacity) into the
        input buffers; event i gets id i."""
        assert len(events) <= self.n_events
        n = int(sum(len(e["x"]) for e in events))
        assert n <= self.inputs["x"].numel()
        if n:
            for k in ("x", "y", "z", "t0", "ne"):
                self.inputs[k][:n].copy_(torch.from_numpy(
                    np.concatenate([e[k] for e in events]).astype(np.float32)))
            self.inputs["event"][:n].copy_(torch.from_numpy(
                np.concatenate([np.full(len(e["x"]), i, np.int32) for i, e in enumerate(events)])))
        self.n = n

    def step(self, stream=None, conv_events=None):
        """Enqueue one step.  conv_events: a list that receives a (start, end) pair of
        recorded CUDA events around every convolution launch (timing only)."""
        h, x, n = self.h, self.inputs, self.n
        nb_dev, np_dev, nh_dev = self.counts[0:1], self.counts[1:2], self.counts[2:3]
        tred_drift_events(h, n, x["x"], x["y"], x["z"], x["t0"], x["ne"], x["event"], self.deps, stream)
        tred_blockbin(h, n, self.deps, self.block_ids, self.block_counts, self.dep_offsets, self.dep_index,
                      nb_dev, stream)
        if self.persistent:
            ev = None
            if conv_events is not None:
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record()
            tred_effq_convolve(h, n, self.deps, self.block_ids, self.dep_offsets, self.dep_index, nb_dev, self.qeff,
                               self.out_blocks, stream)
            if ev is not None:
                ev[1].record()
                conv_events.append(ev)
        for base in range(0, self.max_blocks if not self.persistent else 0, self.chunk):
            tred_effq_range(h, n, self.deps, self.block_ids, self.dep_offsets, self.dep_index, nb_dev, base,
                            self.chunk, self.qeff, stream)
            ev = None
            if conv_events is not None:
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record()
            if self.fuse_gather:
                tred_convolve_spectra_range(h, self.block_ids, nb_dev, base, self.chunk, self.qeff, stream)
            else:
                tred_convolve_range(h, self.block_ids, nb_dev, base, self.chunk, self.qeff, self.out_blocks, stream)
            if ev is not None:
                ev[1].record()
                conv_events.append(ev)
        if self.fuse_gather:
            tred_wave_gather_readout(h, self.block_ids, nb_dev, self.pixel_ids, self.waveforms, np_dev, self.rp,
                                     self.hit_pixel, self.hit_tick, self.hit_charge, nh_dev, stream)
            return
        tred_gather_readout(h, self.block_ids, nb_dev, self.out_blocks, self.pixel_ids, self.waveforms, np_dev,
                            self.rp, self.hit_pixel, self.hit_tick, self.hit_charge, nh_dev, stream)

    def capture(self):
        """Record one step in a CUDA graph (call after a warm-up step)."""
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.step(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def status(self, stream=None):
        return tred_sync_status(self.h, stream)

    def event_of_pixel(self, pixel_ids):
        return np.asarray(pixel_ids) // (self.cfg.npx * self.cfg.npx)
