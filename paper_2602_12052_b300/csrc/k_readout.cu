// a6. Pixel readout (Sec. II-E, Fig. readout: LArPix trigger-reset scheme, and the
// two variants the section names: successive digitisations without intervening
// resets, and fixed-charge integration).
//
// One warp per pixel walks the waveform 512 ticks at a time (the loads of a step in
// flight together), scanning it 128 ticks (4 per lane) at a time: lane and warp scans
// give the running charge inside the sub-step, the charge carried between sub-steps
// is added to it; all in FP32 (the rounding of a running sum over a 6400-tick
// window is a few 1e-7 of the charge, far inside the 1e-4 threshold band in which
// the FP64 oracle's hit lists may differ).  Clock edges k >= start with
// C(k) >= threshold are found with a ballot; the charge is sampled at k + hold, the
// hit (pixel, k + hold, C) is emitted, and integration restarts at
// k + hold + reset + 1.  Successive digitisations take n_samples samples hold apart
// before that restart; fixed-charge integration never restarts and, sub-step by
// sub-step, emits one quantum at every edge whose charge less the quanta already
// taken reaches the threshold.
//
//   k_ro_count   count hits per pixel; cache the first HIT_TMP hits
//   (scan)       hit offsets and the total
//   k_ro_emit    copy cached hits to their sorted position; pixels with more than
//                HIT_TMP hits are walked again and written directly
#include "tred_internal.cuh"

namespace tred {

int launch_scan_large(tred_handle *h, int64_t n, int32_t *part, int32_t *sums, int32_t cap, int32_t *count_dev,
                      int flag, int word, cudaStream_t s);

struct RoConst {
    int nt, clock, hold, reset, nsamp;
    float thr;
};

// Walk one pixel 512 ticks per step: the step's loads are issued together (4 ticks per
// lane in each of 4 sub-steps of 128 ticks), then the sub-steps are scanned in tick
// order.  For each hit call sink(index, tick, charge).  Returns the hit count.
// RM: readout mode (0 trigger-reset, 1 successive digitisations, 2 fixed charge).
template <int RM, typename Sink>
__device__ int walk_pixel(const float *__restrict__ I, const RoConst &c, int lane, Sink sink) {
    int nh = 0;
    int pos = 0;              // first tick of the current step
    float base = 0.f;         // charge integrated before the sub-step (since the last restart)
    int state = 0;            // 0: looking for a trigger; 1: waiting for the sample tick
    int ts = 0;               // next sample tick
    int left = 0;             // samples still to take after ts (mode 1)
    auto load = [&](float (&v)[4][4], int p) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int t = p + 128 * i + 4 * lane + e;
                v[i][e] = t < c.nt ? __ldg(I + t) : 0.f;
            }
    };
    float v[4][4];
    load(v, pos);
    while (pos < c.nt) {
        // the next step's loads are in flight while this step is scanned (a restart after a
        // hit reloads from the new position)
        float vn[4][4];
        load(vn, pos + 512);
        bool restart = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int spos = pos + 128 * i;
            if (spos >= c.nt) break;
            const int t0 = spos + 4 * lane;
            // an all-zero sub-step leaves the running charge at `base`: with no trigger
            // possible (idle and base below threshold) or the sample tick beyond it,
            // nothing changes, so it is skipped (the scan below would give C = base)
            const bool nz = (v[i][0] != 0.f) | (v[i][1] != 0.f) | (v[i][2] != 0.f) | (v[i][3] != 0.f);
            if (!__any_sync(0xffffffffu, nz) && ((state == 0 && !(base >= c.thr)) || (state == 1 && ts >= spos + 128)))
                continue;
            float w[4] = {v[i][0], v[i][1], v[i][2], v[i][3]};
            w[1] += w[0];
            w[2] += w[1];
            w[3] += w[2];
            float x = w[3];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            const float excl = x - w[3];
            float C[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) C[e] = base + (excl + w[e]);
            if (RM == 2) {
                // fixed charge: every edge with C >= threshold gives one quantum, taken
                // from C; the edges are visited in order, quanta already taken subtracted
                float sub = 0.f;
                int from = spos;
                for (;;) {
                    int first = 4;
                    int ph = t0 % c.clock;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (first == 4 && ph == 0 && t0 + e < c.nt && t0 + e >= from && C[e] - sub >= c.thr) first = e;
                        ph = ph + 1 == c.clock ? 0 : ph + 1;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, first < 4);
                    if (!bal) break;
                    const int src = __ffs(bal) - 1;
                    const int k = spos + 4 * src + __shfl_sync(0xffffffffu, first, src);
                    sink(nh, k, c.thr);
                    ++nh;
                    sub += c.thr;
                    from = k + 1;
                }
                base = __shfl_sync(0xffffffffu, C[3], 31) - sub;
                continue;
            }
            if (state == 0) {
                int first = 4;
                int ph = t0 % c.clock;                      // clock phase of tick t0
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (first == 4 && ph == 0 && t0 + e < c.nt && C[e] >= c.thr) first = e;
                    ph = ph + 1 == c.clock ? 0 : ph + 1;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, first < 4);
                if (bal) {
                    const int src = __ffs(bal) - 1;
                    const int fe = __shfl_sync(0xffffffffu, first, src);
                    const int k = spos + 4 * src + fe;
                    ts = k + c.hold;
                    if (ts >= c.nt) return nh;              // sample falls outside the window
                    left = RM == 1 ? c.nsamp - 1 : 0;
                    state = 1;
                }
            }
            // the samples that fall in this sub-step (several in mode 1 when hold < 128)
            while (state == 1 && ts < spos + 128) {
                const int off = ts - spos;
                const int e = off & 3;
                const float mine = e == 0 ? C[0] : e == 1 ? C[1] : e == 2 ? C[2] : C[3];
                const float Cs = __shfl_sync(0xffffffffu, mine, off >> 2);
                sink(nh, ts, Cs);
                ++nh;
                if (left > 0) {                             // next digitisation, no reset
                    --left;
                    ts += c.hold;
                    if (ts >= c.nt) return nh;
                    continue;
                }
                pos = ts + c.reset + 1;
                base = 0.f;
                state = 0;
                restart = true;
            }
            if (restart) break;
            base = __shfl_sync(0xffffffffu, C[3], 31);
        }
        if (!restart) {
            pos += 512;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) v[i][e] = vn[i][e];
        } else if (pos < c.nt) {
            load(v, pos);
        }
    }
    return nh;
}

// With `possum` given (the gather's per-row sum of the positive current), a row whose
// sum stays below `cut` (the threshold less a margin far above FP32 rounding) cannot reach
// the threshold in any scheme: its hit count is zero without reading the waveform.
template <int RM>
__global__ void __launch_bounds__(256, 2) k_ro_count(const float *__restrict__ wave,
                                                  const int32_t *__restrict__ n_pixels_dev, RoConst c,
                                                  int32_t *__restrict__ cnt, int32_t *__restrict__ tmp_t,
                                                  float *__restrict__ tmp_c, const float *__restrict__ possum,
                                                  float cut) {
    const int np = n_pixels_dev[0];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < np; row += nwarps) {
        if (possum && possum[row] < cut) {
            if (lane == 0) cnt[row] = 0;
            continue;
        }
        const float *I = wave + (size_t)row * c.nt;
        const int nh = walk_pixel<RM>(I, c, lane, [&](int k, int t, float q) {
            if (lane == 0 && k < HIT_TMP) {
                tmp_t[(size_t)row * HIT_TMP + k] = t;
                tmp_c[(size_t)row * HIT_TMP + k] = q;
            }
        });
        if (lane == 0) cnt[row] = nh;
    }
}

template <int RM>
__global__ void __launch_bounds__(256, 2) k_ro_emit(const float *__restrict__ wave,
                                                 const int32_t *__restrict__ pixel_ids,
                                                 const int32_t *__restrict__ n_pixels_dev, RoConst c,
                                                 const int32_t *__restrict__ off,
                                                 const int32_t *__restrict__ tmp_t,
                                                 const float *__restrict__ tmp_c, int32_t max_hits,
                                                 int32_t *__restrict__ hp, int32_t *__restrict__ ht,
                                                 float *__restrict__ hc) {
    const int np = n_pixels_dev[0];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < np; row += nwarps) {
        const int o = off[row], nh = off[row + 1] - o;
        const int pid = pixel_ids[row];
        if (nh <= HIT_TMP) {
            if (lane < nh && o + lane < max_hits) {
                hp[o + lane] = pid;
                ht[o + lane] = tmp_t[(size_t)row * HIT_TMP + lane];
                hc[o + lane] = tmp_c[(size_t)row * HIT_TMP + lane];
            }
        } else {
            walk_pixel<RM>(wave + (size_t)row * c.nt, c, lane, [&](int k, int t, float q) {
                if (lane == 0 && o + k < max_hits) {
                    hp[o + k] = pid;
                    ht[o + k] = t;
                    hc[o + k] = q;
                }
            });
        }
    }
}

int launch_readout(tred_handle *h, const tred_readout_params &rp, const int32_t *pixel_ids,
                   const float *wave, const int32_t *n_pixels_dev, int32_t *hit_pixel,
                   int32_t *hit_tick, float *hit_charge, int32_t *n_hits_dev, int32_t max_hits,
                   cudaStream_t s, const float *possum) {
    const float cut = rp.threshold_e > 0.f ? rp.threshold_e * (1.0f - 1e-4f) : -3.0e38f;
    RoConst c{h->g.nt, rp.clock_ticks, rp.hold_ticks, rp.reset_ticks, rp.mode == 1 ? rp.n_samples : 1, rp.threshold_e};
    const int sms = num_sms(h);
    const int ro_grid = min(sms * 8, (h->max_pixels + 7) / 8);   // a warp per pixel, 8 per CTA
    int rc = check_cuda(h, cudaMemsetAsync(h->hit_cnt, 0, sizeof(int32_t) * ((size_t)h->max_pixels + 1), s),
                        "clear hit counts");
    if (rc) return rc;
    auto count = [&](auto kern) {
        kern<<<ro_grid, 256, 0, s>>>(wave, n_pixels_dev, c, h->hit_cnt, h->hit_tmp, h->hit_tmpc, possum, cut);
    };
    if (rp.mode == 2) count(k_ro_count<2>);
    else if (rp.mode == 1) count(k_ro_count<1>);
    else count(k_ro_count<0>);
    // chunk sums after the counts and their total (max_pixels + 8 words)
    rc = launch_scan_large(h, h->max_pixels, h->hit_cnt, h->hit_cnt + (size_t)h->max_pixels + 8, max_hits, n_hits_dev,
                           TRED_ST_HIT_OVERFLOW, 5, s);
    if (rc) return rc;
    auto emit = [&](auto kern) {
        kern<<<ro_grid, 256, 0, s>>>(wave, pixel_ids, n_pixels_dev, c, h->hit_cnt, h->hit_tmp, h->hit_tmpc, max_hits,
                                     hit_pixel, hit_tick, hit_charge);
    };
    if (rp.mode == 2) emit(k_ro_emit<2>);
    else if (rp.mode == 1) emit(k_ro_emit<1>);
    else emit(k_ro_emit<0>);
    h->launches += 2;
    return check_cuda(h, cudaGetLastError(), "readout launch");
}

}  // namespace tred
