/*
 * libtred -- C ABI of the B300 (sm_103a) hot path of TRED (arXiv 2602.12052):
 * effective charge of drifted, diffused ionisation deposits on a sub-pixel x tick
 * grid, block-sparse binning, interlaced FFT convolution with the field response,
 * electrode gather and trigger-reset readout.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns int32_t: TRED_OK (0) or a TRED_ERR_* code; nothing throws.
 *    tred_last_error(h) returns a message for the last failing call on h.
 *  - Pointers named *_dev, and every array argument unless stated otherwise, are
 *    DEVICE pointers owned by the caller, 256-byte aligned (any cudaMalloc /
 *    torch allocation qualifies).  The handle owns only the response spectrum and
 *    internal scratch, allocated once in tred_create from the capacities.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is enqueued
 *    asynchronously; no call synchronises the host except tred_sync_status.
 *  - Counts produced on the device (active blocks, pixels, hits) stay on the device
 *    (*_dev arguments) so that a whole step can be captured in a CUDA graph.
 *    Downstream calls read them there.  Overflow of a capacity sets a bit of the
 *    device status word (TRED_ST_*) and truncates; read it with tred_sync_status.
 *  - Grid units: x, y in sub-cells of size h = pitch / n_sub with grid points at
 *    sub-cell centres (mu_x = x / h - 1/2); t in ticks with grid points at integer
 *    ticks.  Pixel id = py * npx_x + px.  Block id = (by * NBx + bx) * NBt + bt
 *    with NBx = npx_x / bp, NBt = nt / bt.
 */
#ifndef TRED_H
#define TRED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TRED_OK = 0,
    TRED_ERR_INVALID_ARG = 1,  /* bad pointer, size, geometry or parameter */
    TRED_ERR_CUDA = 2,         /* a CUDA runtime call failed (message has the name) */
    TRED_ERR_CAPACITY = 3,     /* a capacity given to tred_create is too small */
    TRED_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    TRED_ERR_NOT_READY = 5     /* call made before tred_set_response */
};

/* Bits of the device status word (host_status[0] of tred_sync_status). */
enum {
    TRED_ST_BLOCK_OVERFLOW = 1 << 0,   /* more active blocks than max_blocks */
    TRED_ST_PAIR_OVERFLOW = 1 << 1,    /* more (deposit, block) pairs than max_pairs */
    TRED_ST_PIXEL_OVERFLOW = 1 << 2,   /* more active pixels than max_pixels */
    TRED_ST_HIT_OVERFLOW = 1 << 3,     /* more hits than max_hits */
    TRED_ST_DRIFT_RANGE = 1 << 4,      /* a deposit drifted farther than max_drift_cm */
    TRED_ST_TIMEOUT = 1 << 5           /* a bounded device wait expired */
};

#define TRED_STATUS_WORDS 8
/* host_status layout: [0] status bits, [1] deposits dropped at drift (off the plane,
 * negative z or n_e, non-finite), [2] active blocks, [3] (deposit, block) pairs,
 * [4] active pixels, [5] hits, [6] reserved, [7] reserved. */

typedef struct tred_handle tred_handle;

/* Detector geometry and block decomposition (Sec. II-B, II-D, III-B).  All floating
 * constants are binary32; the window arithmetic promotes them exactly. */
typedef struct {
    float pitch_cm;      /* pixel pitch a */
    int32_t n_sub;       /* impact positions per pixel axis (even; grid G is n_sub x finer) */
    float tick_us;       /* sampling tick */
    int32_t npx_x, npx_y;/* plane size in pixels (multiples of bp) */
    int32_t nt;          /* readout window in ticks (multiple of bt) */
    int32_t bp, bt;      /* block shape: bp x bp pixels x bt ticks */
    int32_t kp, nr;      /* field response: kp x kp pixels (odd), nr ticks */
    int32_t lt;          /* FFT length along time: 384, 512, 768 or 1024, >= bt + nr - 1 */
    int32_t n_events;    /* independent events stacked along y (0 or 1: a single event).
                            Event e occupies pixel rows [e npx_y, (e + 1) npx_y); no support,
                            footprint or gather crosses an event boundary, so a batch of
                            events is simulated exactly as each event alone. */
} tred_geometry;

/* Transport and method switches. */
typedef struct {
    float v_cm_per_us;       /* drift velocity */
    float DL_cm2_per_s;      /* longitudinal diffusion coefficient */
    float DT_cm2_per_s;      /* transverse diffusion coefficient */
    float lifetime_us;       /* electron lifetime (attachment) */
    float sigma0_cells_xy;   /* diffusion floor (sub-cells), added in quadrature */
    float sigma0_ticks;      /* diffusion floor (ticks), added in quadrature */
    float nsigma;            /* raster half-width in units of sigma */
    float max_drift_cm;      /* largest drift distance the window capacity covers */
    int32_t gl_order;        /* Gauss-Legendre points per axis, 1..8 */
    int32_t effq_mode;       /* 0: Gauss-Legendre (FP32); 1: exact tent, FP64 erf tails */
    int32_t conv_mode;       /* 0: FP32 FFT (shared memory + tensor-memory accumulator);
                                1: time DFT as a tcgen05 GEMM in TF32 (tolerance 1e-4);
                                2: the same with split TF32, three products (FP32 grade);
                                3: the same with split BF16, three products (BF16 hi + lo
                                parts of both operands; tolerance 1e-4).
                                1, 2 and 3 need lt = 512 and bp = 8 (TRED_ERR_INVALID_ARG).
                                4: time DFT by FFT, then per time-frequency bin the sum over
                                impacts and response taps of the block pixels that hold
                                charge as a split-BF16 tcgen05 GEMM (three products, FP32
                                accumulation); needs lt = 384 or 512 and kp <= 9
                                (TRED_ERR_INVALID_ARG); reads only the columns whose
                                non-empty mask bit is set, so effq_skip_empty may be 1. */
    int32_t mpcp;            /* 1: mirror-pair complex packing (needs a mirror-
                                symmetric response); 0: one channel per FFT */
    int32_t compensated_gather; /* 1: accumulate overlapping blocks in FP64 */
    int32_t effq_skip_empty;    /* 1: tred_effq writes only the sub-cell columns that some
                                   deposit's support covers; the other columns of the qeff
                                   buffer are left as they were (conv_mode 0 reads only the
                                   columns whose non-empty mask bit is set).  0: every column
                                   is written (required by conv_mode 1, 2, 3; conv_mode 4
                                   reads only the non-empty columns, as conv_mode 0). */
    int32_t conv_rows_cap;      /* conv_mode 4: non-empty (block, pixel) rows per launch pair
                                   of its forward DFT and GEMM, a multiple of 128 (device
                                   memory 4 (lt/2 + 1) 2 n_sub^2 bytes per row); 0: 131072.
                                   Larger row sets run as several launch pairs. */
    int32_t conv_keep_spectra;  /* conv_mode 4: 1 = the handle keeps every slot's output
                                   spectrum (max_blocks (lt/2 + 1) 256 8 bytes) and pixel
                                   mask, indexed by absolute slot, so that the electrode gather
                                   can run once after tred_convolve_spectra_range has covered
                                   the slots in chunks (tred_wave_gather_readout); 0 = the
                                   spectra of one pass of at most 16384 slots. */
} tred_params;

/* Pixel readout (Sec. II-E): the trigger-reset scheme and the two variants the
 * section names.  A zero-initialised mode / n_samples selects trigger-reset. */
typedef struct {
    float threshold_e;       /* trigger threshold on the integrated charge; in mode 2 the
                                charge quantum */
    int32_t clock_ticks;     /* clock period: triggers are tested at multiples of it */
    int32_t hold_ticks;      /* charge is sampled hold_ticks after the trigger edge (mode 1:
                                spacing of the successive samples) */
    int32_t reset_ticks;     /* dead time after the (last) sample */
    int32_t mode;            /* 0 trigger-reset, 1 successive digitisations without
                                intervening resets, 2 fixed-charge integration */
    int32_t n_samples;       /* mode 1: digitisations per trigger (>= 1; 1 is mode 0) */
} tred_readout_params;

/* Drifted deposits, structure of arrays, caller-owned device arrays of length
 * >= n each.  Written by tred_drift, read by tred_blockbin and tred_effq.
 * cell = floor(mu), frac = mu - cell in [0,1) (computed in binary64, rounded),
 * sigma in grid units, [lo, hi] the quadrature cells (effective charge support is
 * [lo - 1, hi + 1]), q the electrons after attachment.  A dropped deposit has
 * q = 0 and lo > hi on every axis. */
typedef struct {
    int32_t *cell_x, *cell_y, *cell_t;
    float *frac_x, *frac_y, *frac_t;
    float *sigma_x, *sigma_y, *sigma_t;
    int32_t *lo_x, *lo_y, *lo_t;
    int32_t *hi_x, *hi_y, *hi_t;
    float *q;
} tred_deposits;

/* Create a handle on the current CUDA device.  Capacities: max_deposits per call,
 * max_blocks active blocks, max_pixels active pixels.  Allocates the response
 * spectrum and scratch (cudaMalloc).  On error *out is NULL. */
int32_t tred_create(const tred_geometry *geom, const tred_params *params,
                    int32_t max_deposits, int32_t max_blocks, int32_t max_pixels,
                    tred_handle **out);

/* Free the handle and its device memory (after the caller's streams are idle). */
int32_t tred_destroy(tred_handle *h);

/* Message of the last failing call on h (static storage owned by h). */
const char *tred_last_error(const tred_handle *h);

/* Device status word and counters (TRED_STATUS_WORDS int32 into host_status);
 * synchronises `stream`.  Does not clear them; tred_reset_status does. */
int32_t tred_sync_status(tred_handle *h, void *stream, int32_t *host_status);
int32_t tred_reset_status(tred_handle *h, void *stream);

/* Number of kernels this handle has launched so far (host-side counter, no device
 * access; diagnostics for benchmarks). */
int32_t tred_launch_count(const tred_handle *h, int64_t *count);

/* Per-kernel device time (diagnostics for benchmarks).  While enabled, the library
 * brackets every launch of the kernel classes below with a pair of CUDA events on the
 * launching stream (do not enable it during CUDA-graph capture).  tred_kernel_time waits
 * for the recorded events, returns the summed milliseconds and the launch count of class
 * `which` since the previous call for that class (or since enabling), and forgets them.
 *   which: TRED_KT_EFFQ (effective charge, k_effq_blocks), TRED_KT_DX_FWD, TRED_KT_DX_GEMM,
 *          TRED_KT_DX_INV (the forward DFT, GEMM and inverse DFT of conv_mode 4),
 *          TRED_KT_DX_WAVE (the inverse DFT fused with the gather, k_dx_wave, of
 *          tred_convolve_gather_readout).
 * TRED_ERR_INVALID_ARG for a class outside the list or null outputs. */
enum {
    TRED_KT_EFFQ = 0,
    TRED_KT_DX_FWD = 1,
    TRED_KT_DX_GEMM = 2,
    TRED_KT_DX_INV = 3,
    TRED_KT_DX_WAVE = 4,
    TRED_KT_CLASSES = 5
};
int32_t tred_set_kernel_timing(tred_handle *h, int32_t enable);
/* conv_mode 4 diagnostics: the non-empty (block, pixel) rows and the non-empty columns of
 * those rows summed over every tred_convolve / tred_convolve_range pass since the previous
 * call (which resets the sums; device counts copied to the host, so the call synchronises
 * the device); 0 and 0 for the other modes. */
int32_t tred_direct_counts(tred_handle *h, int64_t *rows, int64_t *columns);
int32_t tred_kernel_time(tred_handle *h, int32_t which, double *ms, int32_t *launches);

/* Failure-detection self-test of the bounded device waits (the paper has no
 * counterpart; this is the library's own fault path).  Enqueues one thread that
 * waits, for limit_cycles SM clock cycles (1 .. 2e9; about 1 s per 2e9 at the
 * maximum clock), on an mbarrier phase that nothing completes, exactly as the
 * tensor-core convolution waits on its copies; when the limit passes it sets
 * TRED_ST_TIMEOUT in the status word and returns, leaving the context usable.
 * Read it with tred_sync_status; clear it with tred_reset_status.
 * TRED_ERR_INVALID_ARG for a limit outside the range. */
int32_t tred_wait_selftest(tred_handle *h, int64_t limit_cycles, void *stream);

/* Measured FP32 FMA throughput of the current device (the paper has no counterpart:
 * the convolution is bound by the FP32 ALU, and this gives its roofline denominator).
 * Runs 8 CTAs of 256 threads per SM, each thread 8 independent FMA chains of
 * 16 * iters FMAs, once to warm up and once timed with CUDA events on `stream`
 * (synchronises it).  sink: caller-owned device float[sink_len] with sink_len >=
 * SMs * 2048 (TRED_ERR_CAPACITY otherwise), written with the chains' results.
 * *tflops = 2 * FMAs / time in TFLOP/s; *sms_out (if not null) = SM count.
 * TRED_ERR_INVALID_ARG for null outputs or iters < 1. */
int32_t tred_fp32_peak(float *sink, int64_t sink_len, int32_t iters, void *stream, double *tflops,
                       int32_t *sms_out);

/* a0. Response spectrum (Sec. III-A-2: the spectra of the per-impact responses are computed once; Eq. interlaced,
 * R[j, k] = i[j, -k]).  resp_dev: [kp][kp][n_sub][n_sub][nr] float32, index
 * [Ky + R][Kx + R][jy][jx][tau] = current on the central electrode from unit charge
 * at impact (jx, jy) of the pixel at offset K, tau ticks after crossing the
 * reference plane.  Computed once in FP64 (direct DFT) and stored in complex64,
 * pre-scaled by 1/(16*16*lt).  With mpcp=1 the response must be mirror symmetric,
 * i[-j][-K] = i[j][K] (Eq. multch); only one impact of each mirror pair is kept. */
int32_t tred_set_response(tred_handle *h, const float *resp_dev, void *stream);

/* a1. Transport (Sec. II-A; Fig. flowchart steps A, D).  Inputs x, y (cm, on the plane from
 * its lower corner), z (drift distance to the response reference plane, cm), t0
 * (us), ne (electrons), device float32[n].  Per deposit: t_d = z / v, arrival tick
 * mu_t = (t0 + t_d) / tick, mu_x = x / h - 1/2, sigma_xy = sqrt(2 DT t_d / h^2 +
 * s0^2), sigma_t = sqrt(2 DL t_d / (v tick)^2 + s0t^2), q = ne exp(-t_d / tau),
 * window lo = floor(mu - nsigma sigma), hi = ceil(mu + nsigma sigma).  The window is
 * one fixed sequence of correctly rounded binary64 operations (no contraction), so
 * any IEEE binary64 implementation of it gives the same integers. */
int32_t tred_drift(tred_handle *h, int32_t n, const float *x, const float *y,
                   const float *z, const float *t0, const float *ne,
                   const tred_deposits *out, void *stream);

/* tred_drift for a batch of events: event[n] (device int32) gives each deposit's
 * event in [0, n_events); x, y stay event-local.  The window is computed in
 * event-local coordinates and shifted by whole cells (e npx_y n_sub), so it equals
 * the single-event window bit for bit.  The handle remembers each deposit's event
 * for the later calls on the same deposits.  tred_drift = this with all events 0. */
int32_t tred_drift_events(tred_handle *h, int32_t n, const float *x, const float *y,
                          const float *z, const float *t0, const float *ne, const int32_t *event,
                          const tred_deposits *out, void *stream);

/* Line-shape track segments (Sec. II-C, Eq. qline; short segments).  Transport of
 * both endpoints (x0, y0, z0) and (x1, y1, z1) with one start time t0 and n_e
 * electrons per segment: cell/frac = the midpoint split as in tred_drift, sigma per
 * axis at the midpoint's drift time, q with attachment at the midpoint, window per
 * axis [floor(min endpoint - nsigma sigma), ceil(max endpoint + nsigma sigma)] (the
 * same binary64 sequence as tred_drift, so the oracle's windows agree bit for bit).
 * half[3 * n] (device, caller-owned): (p1 - p0) / 2 per axis in grid units, axis
 * major (x block, then y, then t).  A segment with an endpoint off the plane or
 * beyond max_drift_cm is dropped as in tred_drift.  Single event (event 0).  The
 * blockbin pair capacity assumes a segment's window is shorter than a block on every
 * axis (at most 2 blocks per axis). */
int32_t tred_drift_lines(tred_handle *h, int32_t n, const float *x0, const float *y0,
                         const float *z0, const float *x1, const float *y1, const float *z1,
                         const float *t0, const float *ne, const tred_deposits *out, float *half,
                         void *stream);

/* Effective charge of line segments (Eq. eff_q with the node charge
 * Q rho(node) w_l w_m w_n / 8, rho the diffused line density of Eq. qline with the
 * factor 1/2 in the exponent; segments shorter than 0.1 sigma on every axis use the
 * point Gaussian at the midpoint).  Same block list, CSR, qeff layout and column
 * masks as tred_effq; every column of every active block is written.  Needs
 * effq_mode 0, gl_order <= 4, (bp n_sub)^2 <= 8192 and bt a multiple of 16.  FP32
 * sums in the order of each block's segment list. */
int32_t tred_effq_lines(tred_handle *h, int32_t n, const tred_deposits *deps, const float *half,
                        const int32_t *block_ids, const int32_t *dep_offsets,
                        const int32_t *dep_index, const int32_t *n_blocks_dev, float *qeff,
                        void *stream);

/* a2. Block-sparse binning (Sec. III-B-1).  A block is active iff the clipped
 * support box of some deposit intersects it; its count is the number of such
 * deposits.  Output (device): block_ids[nb] ascending, block_counts[nb],
 * dep_offsets[nb + 1] (CSR), dep_index[pairs] (deposit ids of each block, ascending
 * within a block), n_blocks_dev[0] = nb.  Capacities: max_blocks (tred_create) and
 * max_pairs. */
int32_t tred_blockbin(tred_handle *h, int32_t n, const tred_deposits *deps,
                      int32_t *block_ids, int32_t *block_counts, int32_t *dep_offsets,
                      int32_t *dep_index, int32_t max_pairs, int32_t *n_blocks_dev,
                      void *stream);

/* a3. Effective charge (Sec. II-C, Eqs. cub, trilinear, eff_q; point-like charge):
 * per axis e[g] = sum_C sum_l (w_l / 2) phi(C + xi_l / 2) u_l(g - C) (Gauss-Legendre)
 * or the exact tent integral (effq_mode 1); Qeff = q e_x e_y e_t summed over the
 * block's deposits.  qeff_dev: [max_blocks][n_sub][n_sub][bp][bp][bt] float32,
 * index [slot][jy][jx][py][px][t], grid point gx = (bx bp + px) n_sub + jx.  Each
 * cell is summed in FP32 over the block's deposits in the order of dep_index (ascending
 * as tred_blockbin writes it), so the result is bitwise reproducible; a deposit's
 * contribution to a cell that stays below 2^-23 of the block's largest single
 * contribution over a 32-tick tile is left out. */
int32_t tred_effq(tred_handle *h, int32_t n, const tred_deposits *deps,
                  const int32_t *block_ids, const int32_t *dep_offsets,
                  const int32_t *dep_index, const int32_t *n_blocks_dev, float *qeff,
                  void *stream);

/* tred_effq restricted to the active-block slots [slot_base, slot_base + slot_count)
 * (clipped to the device count): the sub-batches of Sec. III-B-2, so that the
 * effective charge of a large batch is produced chunk by chunk.  qeff holds
 * slot_count blocks; slot s is written at row s - slot_base.  The call with
 * slot_base = 0 also computes the per-deposit weights that the later ranges of the
 * same pass reuse: call it first. */
int32_t tred_effq_range(tred_handle *h, int32_t n, const tred_deposits *deps,
                        const int32_t *block_ids, const int32_t *dep_offsets,
                        const int32_t *dep_index, const int32_t *n_blocks_dev, int32_t slot_base,
                        int32_t slot_count, float *qeff, void *stream);

/* a4. Interlaced convolution (Sec. II-D, Eq. interlaced; Sec. III-A-2, Eq. multch):
 *   I[P, t] = sum_j sum_K sum_tau Qeff[j, P + K, t - tau] i[j, K, tau]
 * for each active block, by FFT over the padded 16 x 16 x lt grid, with MPCP when
 * params.mpcp = 1.  out_blocks: [max_blocks][16][16][lt] float32, index
 * [slot][uy][ux][t]: block-local output pixel (by bp + uy - R, bx bp + ux - R) at
 * tick bt*bt_len + t, R = (kp - 1) / 2; only t < bt + nr - 1 is meaningful. */
int32_t tred_convolve(tred_handle *h, const int32_t *block_ids,
                      const int32_t *n_blocks_dev, const float *qeff, float *out_blocks,
                      void *stream);

/* tred_convolve restricted to slots [slot_base, slot_base + slot_count): qeff is
 * the chunk written by tred_effq_range with the same slot_base; out_blocks is
 * indexed by absolute slot. */
int32_t tred_convolve_range(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                            int32_t slot_base, int32_t slot_count, const float *qeff,
                            float *out_blocks, void *stream);

/* a3 + a4 in one persistent launch over the active-block queue (Sec. III-B-2: the
 * blocks of many events batched through the effective charge and the convolution).
 * One CTA per SM takes blocks from one device queue holding every active block (all
 * events of an n_events handle) and runs, per block: the effective charge (as
 * tred_effq computes it: Eq. eff_q, each cell's sum in the block's deposit order) into
 * its CTA's row of qeff_ring, then the convolution of every time-frequency class and
 * the inverse time transform (as tred_convolve) into out_blocks[slot].
 *  - qeff_ring: caller-owned device float32 [ring_rows][n_sub][n_sub][bp][bp][bt], the
 *    staging rows of the resident CTAs; ring_rows must be at least min(SMs,
 *    max_blocks, 8192) (TRED_ERR_CAPACITY otherwise).  Its contents afterwards are
 *    unspecified (each row holds the last block its CTA took).
 *  - out_blocks as tred_convolve: [max_blocks][16][16][lt], rows 0..n_blocks-1 written.
 *  - n, deps, block_ids, dep_offsets, dep_index, n_blocks_dev as tred_effq (the
 *    per-deposit weights are computed here too).
 *  - conv_mode 0 and lt = 384 or 512 only (TRED_ERR_INVALID_ARG otherwise); effq_skip_empty
 *    as the handle sets it.  Graph-capturable (counts stay on the device). */
int32_t tred_effq_convolve(tred_handle *h, int32_t n, const tred_deposits *deps, const int32_t *block_ids,
                           const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                           float *qeff_ring, int32_t ring_rows, float *out_blocks, void *stream);

/* a5. Electrode gather (Fig. flowchart: binning and accumulation onto the unique electrodes): every
 * in-plane pixel of an active block's output footprint is active; its waveform
 * [0, nt) is the sum, in a fixed order, of the overlapping blocks' outputs.
 * pixel_ids[npix] ascending, waveforms [max_pixels][nt], n_pixels_dev[0] = npix. */
int32_t tred_gather_pixels(tred_handle *h, const int32_t *block_ids,
                           const int32_t *n_blocks_dev, const float *out_blocks,
                           int32_t *pixel_ids, float *waveforms, int32_t *n_pixels_dev,
                           void *stream);

/* a6. Pixel readout (Sec. II-E, Fig. readout), per pixel over its waveform row.
 * mode 0, trigger-reset: C = running sum of the current since the end of the last
 *   reset; at clock edges k >= start, if C(k) >= threshold a hit (pixel, k + hold,
 *   C(k + hold)) is emitted when k + hold < nt and C restarts at k + hold + reset + 1.
 * mode 1, successive digitisations: a trigger at edge k gives n_samples hits
 *   (pixel, k + m hold, C(k + m hold)), m = 1..n_samples, with C not reset between
 *   them; C restarts at k + n_samples hold + reset + 1.  A sample at or beyond nt
 *   ends the pixel.
 * mode 2, fixed-charge integration: C = running sum from tick 0, never reset; at
 *   each clock edge k with C(k) >= threshold a hit (pixel, k, threshold) is emitted
 *   and the quantum is taken from C (no charge is lost).
 * All in FP32 running sums.  Hits sorted by (pixel, tick); n_hits_dev[0] = count
 * (capped at max_hits: TRED_ST_HIT_OVERFLOW in the status word beyond it).
 * TRED_ERR_INVALID_ARG for a null pointer, clock_ticks < 1, hold_ticks or
 * reset_ticks < 0, an unknown mode, or mode 1 with n_samples < 1 or hold_ticks < 1. */
int32_t tred_readout(tred_handle *h, const tred_readout_params *rp,
                     const int32_t *pixel_ids, const float *waveforms,
                     const int32_t *n_pixels_dev, int32_t *hit_pixel, int32_t *hit_tick,
                     float *hit_charge, int32_t *n_hits_dev, int32_t max_hits,
                     void *stream);

/* a5 + a6 in one call: the outputs of tred_gather_pixels followed by tred_readout on
 * its waveforms (same arguments, same results).  While the waveforms are written, the
 * gather records per pixel the sum of the positive current, which bounds the charge
 * any readout scheme integrates on the pixel; the readout then skips, without reading
 * them, the pixels whose bound stays below (1 - 1e-4) x threshold (they cannot reach
 * the threshold; the margin is far above the FP32 rounding of the sums). */
int32_t tred_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                            const float *out_blocks, int32_t *pixel_ids, float *waveforms,
                            int32_t *n_pixels_dev, const tred_readout_params *rp, int32_t *hit_pixel,
                            int32_t *hit_tick, float *hit_charge, int32_t *n_hits_dev, int32_t max_hits,
                            void *stream);

/* a4 + a5 (+ a6) for the direct spatial form without the per-block output buffer
 * (Sec. II-D, Eq. interlaced; Fig. flowchart: binning and accumulation onto the unique
 * electrodes).  The convolution runs as tred_convolve up to each block's output spectrum
 * Ihat[slot][f][P] (kept in the handle); the pixel list is built as tred_gather_pixels
 * builds it; then each 8 x 8 pixel tile offset by R from the block grid (all its pixels
 * lie in the footprints of the same 2 x 2 spatial blocks) sums, per time block, the
 * spectra of those blocks and takes one inverse DFT per pixel straight into the pixel's
 * waveform row, adding each time block's first nr - 1 ticks onto the previous one's tail.
 * The waveforms equal tred_convolve + tred_gather_pixels up to FP32 rounding order (the
 * spatial sum is taken on the spectra; every sum has a fixed order, so the result is
 * deterministic).  With rp non-null the readout (as tred_readout) follows; rp null
 * skips it (hit arguments may then be null).
 *  - qeff: as tred_convolve; pixel_ids [max_pixels], waveforms [max_pixels][nt],
 *    n_pixels_dev[0] = npix as tred_gather_pixels; hit buffers as tred_readout.
 *  - Shapes: conv_mode 4, bp = 8, kp = bp + 1, nr - 1 <= bt, nt / bt <= 128,
 *    max_blocks <= the direct form's slots per pass (16384, or any with
 *    conv_keep_spectra 1), compensated_gather 0;
 *    TRED_ERR_INVALID_ARG otherwise (tred_convolve_gather_supported says beforehand).
 *  Graph-capturable (counts stay on the device). */
int32_t tred_convolve_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                                     const float *qeff, int32_t *pixel_ids, float *waveforms,
                                     int32_t *n_pixels_dev, const tred_readout_params *rp, int32_t *hit_pixel,
                                     int32_t *hit_tick, float *hit_charge, int32_t *n_hits_dev, int32_t max_hits,
                                     void *stream);
/* 1 when the handle's shape allows tred_convolve_gather_readout, else 0 (-1 for null). */
int32_t tred_convolve_gather_supported(const tred_handle *h);

/* The two halves of tred_convolve_gather_readout, for slots processed in chunks (Sec.
 * III-B-2: many events batched through bounded Q^eff chunks).
 * tred_convolve_spectra_range: the direct form's convolution of slots [slot_base,
 *   slot_base + slot_count) up to their output spectra, kept in the handle; qeff is the
 *   chunk tred_effq_range wrote with the same slot_base.  slot_base > 0 needs
 *   conv_keep_spectra 1 (TRED_ERR_INVALID_ARG otherwise); the shape rules of
 *   tred_convolve_gather_readout apply.
 * tred_wave_gather_readout: once every active slot's spectra are in place (the ranges
 *   cover slots 0 .. n_blocks - 1), the pixel list, the inverse time DFT per pixel tile
 *   into the waveforms and, with rp non-null, the readout; arguments as
 *   tred_convolve_gather_readout without qeff.
 * Both graph-capturable. */
int32_t tred_convolve_spectra_range(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                                    int32_t slot_base, int32_t slot_count, const float *qeff, void *stream);
int32_t tred_wave_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                                 int32_t *pixel_ids, float *waveforms, int32_t *n_pixels_dev,
                                 const tred_readout_params *rp, int32_t *hit_pixel, int32_t *hit_tick,
                                 float *hit_charge, int32_t *n_hits_dev, int32_t max_hits, void *stream);

/* ---- Differentiable simulation (Sec. V-C).  Loss L = 1/2 sum (I - I*)^2 over
 * pixels and ticks; gradients through the whole path with the raster windows held
 * fixed (they are piecewise constant) and the quadrature recomputed, not stored.
 * Gauss-Legendre mode only. */

/* Replace the transport constants (v, DL, DT, lifetime, sigma floors, nsigma,
 * max_drift) of a handle, e.g. between gradient steps; every other field of params is
 * ignored and keeps the value tred_create set, except that the method switches
 * (gl_order, effq_mode, mpcp, conv_mode) must equal the handle's (TRED_ERR_INVALID_ARG
 * otherwise).  TRED_ERR_CAPACITY if the new diffusion needs wider windows than
 * tred_create provisioned (2x the diffusion constants given there). */
int32_t tred_set_transport(tred_handle *h, const tred_params *params);

/* resid = I - I* on the current pixel list (target rows matched by pixel id in the
 * ascending target_ids[n_target]; missing rows count as zero) and
 * loss_dev[0] = 1/2 sum over the union of both lists of (I - I*)^2 (FP64).
 * resid: [max_pixels][nt]. */
int32_t tred_residual(tred_handle *h, const int32_t *pixel_ids, const int32_t *n_pixels_dev,
                      const float *waveforms, const int32_t *target_ids, int32_t n_target,
                      const float *target_waves, float *resid, double *loss_dev, void *stream);

/* Adjoint of drift -> effq -> convolve -> gather for dL/dI = resid on the current
 * pixel list.  dL/dQeff[j, P', t'] = sum_K sum_tau r[P' - K, t' + tau] i[j, K, tau]
 * (the transpose of Eq. interlaced) is formed per active block by FFT with the
 * conjugate response spectrum (MPCP read backwards) into dqeff (the layout of
 * tred_effq's qeff; the forward's qeff buffer may be reused), then the chain rule
 * through the separable quadrature gives grad7[d][7] = dL/d(q, mu_x, mu_y, mu_t,
 * sigma_x, sigma_y, sigma_t) in grid units.  The first call allocates the adjoint
 * scratch (3 floats per weight of each deposit, a pixel map and 32 blocks of
 * spectra). */
int32_t tred_adjoint(tred_handle *h, int32_t n, const tred_deposits *deps, const int32_t *block_ids,
                     const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                     const int32_t *pixel_ids, const int32_t *n_pixels_dev, const float *resid,
                     float *dqeff, float *grad7, void *stream);

/* Chain rule through the transport step (Sec. II-A): grad_inputs[d][4] =
 * dL/d(x, y, t0, ne), grad_global[3] = dL/d(DL, DT, lifetime) (FP64).  z: the
 * drift distances given to tred_drift. */
int32_t tred_param_grads(tred_handle *h, int32_t n, const float *z, const tred_deposits *deps,
                         const float *grad7, float *grad_inputs, double *grad_global, void *stream);

/* Block-sparse binning without any device allocation (the paper has no
 * counterpart; this is a deployment variant of tred_blockbin).
 *
 * Some callers cannot call cudaMalloc once they are running: a host framework that
 * owns all device memory through its own pool and forbids direct allocations, or a
 * real-time acquisition loop where the implicit synchronisation of cudaMalloc would
 * stall the stream.  They need the binning without a tred_handle (tred_create
 * allocates).  This entry point computes exactly what tred_blockbin computes, from
 * the same caller-owned inputs into the same caller-owned outputs, and keeps its
 * scratch (per-block counts, block-to-slot map, CSR cursors, scan partials) in a
 * fixed array that the library reserves on each device it is loaded on and holds
 * until the process exits: 3 * TRED_NOALLOC_MAX_GRID_BLOCKS + 1032 int32
 * (6.3 MB).  It calls no cudaMalloc, cudaFree or allocating routine.
 *
 *  - The plane's block grid (npx_x/bp * npx_y/bp * nt/bt) and max_blocks must not
 *    exceed TRED_NOALLOC_MAX_GRID_BLOCKS; otherwise TRED_ERR_CAPACITY is returned
 *    (with a message on stderr) and nothing is enqueued.
 *  - status_dev: caller-owned device int32[TRED_STATUS_WORDS]; words 0 (bits), 2 and
 *    3 are written as by tred_blockbin; the caller clears it when it wants to.
 *  - The first call on a device looks up the array's device address on the current
 *    device (cudaGetSymbolAddress) and caches it.  With CUDA's lazy module loading
 *    (the default) that first call may also load the library's device code, which
 *    reserves the array and synchronises: make one warm-up call on each device before
 *    the region that must not allocate, and before any stream capture.
 *  - cudaDeviceReset unloads the array and leaves the cached address stale: do not
 *    call this entry point on a device after resetting it in the same process.
 *  - Every call reuses the same array and the array keeps the last call's contents
 *    (the counts are cleared at the start of each call).  Calls whose work overlaps
 *    on the GPU (several streams, or several host threads) race on it and give wrong
 *    results: serialise them on one stream.
 *  - Arguments otherwise as tred_blockbin.  The geometry gets tred_create's checks
 *    (and n_events must be 0 or 1); a failed check, a null array in *deps (when
 *    n > 0) or a null output gives TRED_ERR_INVALID_ARG with nothing enqueued. */
#define TRED_NOALLOC_MAX_GRID_BLOCKS (1 << 19)
int32_t tred_blockbin_noalloc(const tred_geometry *geom, int32_t n, const tred_deposits *deps,
                              int32_t *block_ids, int32_t *block_counts, int32_t *dep_offsets,
                              int32_t *dep_index, int32_t max_blocks, int32_t max_pairs,
                              int32_t *n_blocks_dev, int32_t *status_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TRED_H */
