// a4. Interlaced convolution with the field response (Sec. II-D, Eq. interlaced)
// evaluated by FFT with Mirror-Pair Complex Packing (Sec. III-A-2, Eq. multch).
//
// Per active block and impact pair (j, j') with j' the mirror impact of j, the
// packed input is Z = Qeff[j] + i * flip(Qeff[j']) (flip = spatial reflection inside
// the block), zero padded to 16 x 16 x lt.  With the mirror symmetry i[-j, -K] =
// i[j, K] of the response, one complex FFT per pair, a product with the
// precomputed spectrum Rhat[j] and a single inverse FFT of the sum over pairs give
//     out[u] = Re C[(u - R) mod 16] + Im C[(bp - 1 + R - u) mod 16]   (per axis).
// Without MPCP each impact is its own (real) channel and out[u] = Re C[...].
//
// Work split (B300: 148 SMs, 227 KB shared memory per CTA):
//   k_conv_spec   one CTA (512 threads) per (block, time-frequency class k1), the
//                 persistent CTAs taking the items from a queue:
//                 the class owns the 64 bins f = k1 + G k2.  Stage A computes, per
//                 column, the time DFT restricted to the class (an in-lane
//                 pre-butterfly over the nonzero n1 = 0..bt/64-1 blocks of the
//                 input followed by a 64-point FFT across the warp); stage B does
//                 the 16 x 16 spatial FFT of every bin (8-point in-lane FFTs and a
//                 per-warp shared transpose) and accumulates Rhat * Z in tensor
//                 memory: each warp owns 64 TMEM columns of its lane quarter, one
//                 lane per (bin, kx) with the 16 ky values of two bins, read and
//                 written with tcgen05.ld / tcgen05.st, so the sum over channel pairs
//                 takes no shared-memory bandwidth.  The epilogue inverts the spatial
//                 FFT from the registers and writes the class's bins to the
//                 per-chunk spectrum buffer.
//   k_conv_itime  persistent CTAs over (block, mirror row pair, part) items of 16
//                 columns (8 mirror pairs; 8 columns at lt = 1024), one warp per
//                 column: inverse time FFT and the MPCP recombination, the next
//                 item's spectra streamed in by cp.async meanwhile.  At lt = 512 and
//                 384, k_conv_itime_mp takes the same items with one warp per mirror pair
//                 and no cross-lane butterflies (a shared transpose between a 16-point
//                 and a 32-point in-lane stage).
#include <utility>

#include "conv_item.cuh"

namespace tred {

// ZS: stage A reads the packed time spectra written by the tensor-core DFT
// (zspec[slot][k1][pair][k2][col], k_dftgemm.cu) instead of computing them.
// HZ: blocks of at most 4 x 4 pixels, so the rows and columns 4..7 of every packed input
// are zero: both spatial stages skip them (half-zero first butterfly stage).
template <int NB1, int G, bool ZS, bool HZ>
__global__ void __launch_bounds__(SPEC_THREADS, 1)
    k_conv_spec(const int32_t *__restrict__ n_blocks_dev, const float *__restrict__ qeff,
                const uint64_t *__restrict__ colmask, const float2 *__restrict__ rhat,
                const int32_t *__restrict__ pair_j, const float2 *__restrict__ tw, ConvConst c,
                float2 *__restrict__ yspec, int slot_base, int slot_count, int qbase,
                const float2 *__restrict__ zspec, int32_t *__restrict__ queue) {
    constexpr int LT = 64 * G;
    extern __shared__ float2 smem[];
    const SpecSmem sm(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid < 2) sm.s_ntask[tid] = 0;
    if (warp == 0) {
        tmem_alloc(sm.tslot, SPEC_TMEM_COLS);
        tmem_relinquish();
    }
    sm.load_tables(tw);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    // this warp's accumulator columns: lane quarter warp % 4, columns (warp / 4) * 64 + 32 it
    const uint32_t tbase = *sm.tslot;
    const uint32_t tacc = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));

    const int nb = n_blocks_dev[0];
    const int nloc = max(0, min(slot_count, nb - slot_base));
    const int slab = c.bp * c.bp * c.bt;
    const int ngrp = conv_round_groups(nloc, G, gridDim.x, slot_count);
    const int nrounds = (c.npairs + PG - 1) / PG;
    const int items = nloc * G * ngrp;

    // items are taken from a queue (their stage A cost varies with the block's non-empty columns)
    for (;;) {
        __syncthreads();
        if (tid == 0) sm.s_ntask[2] = atomicAdd(queue, 1);
        __syncthreads();
        const int item = sm.s_ntask[2];
        if (item >= items) break;
        const int grp = item % ngrp, sl = item / ngrp / G, k1 = (item / ngrp) % G;
        const int slot = slot_base + sl;
        const int p_beg = PG * (grp * nrounds / ngrp), p_end = min(c.npairs, PG * ((grp + 1) * nrounds / ngrp));
        conv_spec_item<NB1, G, ZS, HZ, false>(
            sm, tacc, c, k1, p_beg, p_end, qeff + (size_t)(slot - qbase) * c.nch * slab, colmask + (size_t)slot * c.nch,
            rhat, pair_j, tw, ZS ? zspec + ((size_t)sl * G + k1) * c.npairs * BINS * 64 : nullptr,
            yspec + (size_t)(grp * nloc + sl) * LT * (LP * LP));
    }
    // release the accumulator columns once every warp is done with them
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tbase, SPEC_TMEM_COLS);
    }
}

template <int G>
__global__ void __launch_bounds__(32 * itime_cols<G>(), 1)
    k_conv_itime(const int32_t *__restrict__ n_blocks_dev, const float2 *__restrict__ yspec,
                 const float2 *__restrict__ tw, ConvConst c, float *__restrict__ out, int slot_base,
                 int slot_count) {
    constexpr int LT = 64 * G;
    constexpr int NPL = LT / 32;          // values per lane
    constexpr int NC = itime_cols<G>();   // columns per item
    constexpr int HC = NC / 2;
    constexpr int PARTS = LP / HC;        // items per mirror row pair
    constexpr int NT = 32 * NC;
    constexpr int SROW = LT + 1;
    constexpr int IROW = 33;              // imaginary-part exchange: [column][bitrev(k)][lane group]
    extern __shared__ float2 sm[];
    float2 *S = sm;                                                   // [2][NC][SROW]
    float2 *wlt = S + 2 * NC * SROW;                                  // W_LT
    float2 *w32 = wlt + LT;
    float *Ib = reinterpret_cast<float *>(w32 + 32);                  // [NC][NPL][IROW]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = tid; k < LT; k += NT) wlt[k] = tw[TW_LT + k];
    if (tid < 32) w32[tid] = tw[TW_32 + tid];
    const int nb = n_blocks_dev[0];
    const int nloc = min(slot_count, nb - slot_base);
    if (nloc <= 0) return;
    const int items = nloc * 8 * PARTS;
    // the spectral kernel's grid is one CTA per SM, as this one's
    const int ngrp = conv_round_groups(nloc, G, gridDim.x, slot_count);
    // the rows of mirror row pair rp: the rp-th row a with a < m(a), and bro = m(a)
    auto rows_of = [&](int rp, int &a, int &bro) {
        a = -1;
        int cnt = 0;
        for (int r = 0; r < LP; ++r) {
            const int m = (c.bp - 1 - r + 2 * LP) % LP;
            if (r < m) {
                if (cnt == rp) {
                    a = r;
                    break;
                }
                ++cnt;
            }
        }
        bro = (c.bp - 1 - a + 2 * LP) % LP;
    };
    auto column = [&](int q, int part, int a, int bro, int &cy, int &cx) {
        const int cx0 = HC * part + (q % HC);
        cy = q < HC ? a : bro;
        cx = q < HC ? cx0 : (c.bp - 1 - cx0 + 2 * LP) % LP;
    };
    // thread tid copies column q = tid % NC at frequencies f = tid / NC + 32 j
    auto issue = [&](int it, int bsel) {
        const int sl = it / (8 * PARTS), rp = (it / PARTS) % 8, part = it % PARTS;
        int a, bro, cy, cx;
        rows_of(rp, a, bro);
        const int q = tid % NC;
        column(q, part, a, bro, cy, cx);
        const float2 *src = yspec + (size_t)sl * LT * (LP * LP) + cy * LP + cx;
        float2 *dst = S + (bsel * NC + q) * SROW;
#pragma unroll 4
        for (int f = tid / NC; f < LT; f += NT / NC) cp_async8(dst + f, src + (size_t)f * (LP * LP));
        cp_async_commit();
    };
    int it = blockIdx.x;
    if (it < items) issue(it, 0);
    for (int i = 0; it < items; ++i, it += gridDim.x) {
        const int cur = i & 1;
        if (it + (int)gridDim.x < items)
            issue(it + gridDim.x, cur ^ 1);       // that buffer's last readers passed the previous barrier
        else
            cp_async_commit();                    // empty group: keeps the wait count uniform
        cp_async_wait<1>();
        __syncthreads();                          // this item's columns (and W tables) are in place
        const int sl = it / (8 * PARTS), rp = (it / PARTS) % 8, part = it % PARTS;
        int a, bro, cy, cx;
        rows_of(rp, a, bro);
        const int q = warp;
        column(q, part, a, bro, cy, cx);
        itime_column<G>(S + (cur * NC + q) * SROW,
                        ngrp == 2 ? yspec + (size_t)(nloc + sl) * LT * (LP * LP) + cy * LP + cx : nullptr, Ib, wlt,
                        w32, c, q, cy, cx, out + (size_t)(slot_base + sl) * LP * LP * LT);
    }
    cp_async_wait<0>();
}

// Inverse time FFT + MPCP recombination at lt = 64 G = 32 NPL (NPL = 16 or 12: lt = 512
// or 384), two columns per warp: a column and its mirror partner.  The same (block,
// mirror row pair, part) items of 16 columns as k_conv_itime, 8 warps (items of 8 columns
// over two CTAs per SM read 32-byte runs and ran slower).  With n = l + 32 m (lane l,
// register m) the transform is an NPL-point in-lane DFT over m, the twiddles
// W_lt^(l k1), a per-warp shared transpose, then one 32-point in-lane DFT over l per
// lane (lane = (column, k1); at NPL = 12 lanes k1 = 12..15 idle), giving t = k1 + NPL k2.
// No cross-lane butterflies: the only shuffle fetches the partner column's imaginary
// parts from lane ^ 16, and each half warp stores a run of NPL consecutive ticks.
constexpr int IT5_WARPS = 8;   // warps per CTA (16-column items: 64-byte runs per row); one CTA per SM
template <int G>
constexpr size_t itime_mp_smem_bytes() {
    return sizeof(float2) * (2 * 2 * IT5_WARPS * (64 * G + 1) + 2 * G * 32 + IT5_WARPS * 2 * (2 * G) * 32);
}

template <int G>
__global__ void __launch_bounds__(32 * IT5_WARPS, 1)
    k_conv_itime_mp(const int32_t *__restrict__ n_blocks_dev, const float2 *__restrict__ yspec,
                    const float2 *__restrict__ tw, ConvConst c, float *__restrict__ out, int slot_base,
                    int slot_count) {
    constexpr int LT = 64 * G, NPL = 2 * G;
    static_assert(NPL == 16 || NPL == 12, "lt = 512 or 384");
    constexpr int HC = IT5_WARPS, NC = 2 * HC, PARTS = LP / HC, NT = 32 * IT5_WARPS, SROW = LT + 1;
    extern __shared__ float2 sm[];
    float2 *S = sm;                          // [2][NC][SROW] spectra, double buffered
    float2 *twl = S + 2 * NC * SROW;         // [k1][l] = conj(W_lt^(l k1))
    float2 *T = twl + NPL * 32;              // per warp [2 columns][k1][l ^ k1]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < NPL * 32; i += NT) {
        float2 w = tw[TW_LT + (i & 31) * (i >> 5)];
        w.y = -w.y;
        twl[i] = w;
    }
    const int nb = n_blocks_dev[0];
    const int nloc = min(slot_count, nb - slot_base);
    if (nloc <= 0) return;
    const int items = nloc * 8 * PARTS;
    const int ngrp = conv_round_groups(nloc, G, gridDim.x, slot_count);   // as the spectral kernel split
    // the rows of mirror row pair rp: the rp-th row a with a < m(a), and bro = m(a)
    auto rows_of = [&](int rp, int &a, int &bro) {
        a = -1;
        int cnt = 0;
        for (int r = 0; r < LP; ++r) {
            const int m = (c.bp - 1 - r + 2 * LP) % LP;
            if (r < m) {
                if (cnt == rp) {
                    a = r;
                    break;
                }
                ++cnt;
            }
        }
        bro = (c.bp - 1 - a + 2 * LP) % LP;
    };
    auto column = [&](int q, int part, int a, int bro, int &cy, int &cx) {
        const int cx0 = HC * part + (q % HC);
        cy = q < HC ? a : bro;
        cx = q < HC ? cx0 : (c.bp - 1 - cx0 + 2 * LP) % LP;
    };
    // thread tid copies column q = tid % NC at frequencies f = tid / NC + (NT / NC) j
    auto issue = [&](int it, int bsel) {
        const int sl = it / (8 * PARTS), rp = (it / PARTS) % 8, part = it % PARTS;
        int a, bro, cy, cx;
        rows_of(rp, a, bro);
        const int q = tid % NC;
        column(q, part, a, bro, cy, cx);
        const float2 *src = yspec + (size_t)sl * LT * (LP * LP) + cy * LP + cx;
        float2 *dst = S + (bsel * NC + q) * SROW;
#pragma unroll 4
        for (int f = tid / NC; f < LT; f += NT / NC) cp_async8(dst + f, src + (size_t)f * (LP * LP));
        cp_async_commit();
    };
    float2 *Ta = T + warp * 2 * NPL * 32;
    int it = blockIdx.x;
    if (it < items) issue(it, 0);
    for (int i = 0; it < items; ++i, it += gridDim.x) {
        const int cur = i & 1;
        cp_async_wait<0>();
        __syncthreads();                     // this item's columns are in place, the other buffer is free
        if (it + (int)gridDim.x < items) issue(it + gridDim.x, cur ^ 1);
        const int sl = it / (8 * PARTS), rp = (it / PARTS) % 8, part = it % PARTS;
        int a, bro, cya, cxa, cyb, cxb;
        rows_of(rp, a, bro);
        column(warp, part, a, bro, cya, cxa);          // column A
        column(warp + HC, part, a, bro, cyb, cxb);     // its mirror partner B
        {
            float2 va[NPL], vb[NPL];
            const float2 *sa = S + (cur * NC + warp) * SROW, *sb = S + (cur * NC + warp + HC) * SROW;
#pragma unroll
            for (int m = 0; m < NPL; ++m) {
                va[m] = sa[lane + 32 * m];
                vb[m] = sb[lane + 32 * m];
            }
            if (ngrp == 2) {   // the second half of the rounds' spectra, from its own plane
                const float2 *ga = yspec + (size_t)(nloc + sl) * LT * (LP * LP) + cya * LP + cxa;
                const float2 *gb = yspec + (size_t)(nloc + sl) * LT * (LP * LP) + cyb * LP + cxb;
#pragma unroll
                for (int m = 0; m < NPL; ++m) {
                    va[m] = cadd(va[m], __ldg(ga + (size_t)(lane + 32 * m) * (LP * LP)));
                    vb[m] = cadd(vb[m], __ldg(gb + (size_t)(lane + 32 * m) * (LP * LP)));
                }
            }
            fft_reg_any<NPL, true>(va);              // va[k] = sum over m at k1 = fft_perm(k)
            fft_reg_any<NPL, true>(vb);
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int k1 = fft_perm<NPL>(k);
                const float2 w = twl[k1 * 32 + lane];
                Ta[k1 * 32 + (lane ^ k1)] = cmul(va[k], w);
                Ta[NPL * 32 + k1 * 32 + (lane ^ k1)] = cmul(vb[k], w);
            }
        }
        __syncwarp();
        const int hcol = lane >> 4, k1 = lane & 15;
        const int kr = k1 < NPL ? k1 : NPL - 1;       // idle lanes re-read a valid row
        float2 y[32];
        {
            const float2 *tr = Ta + hcol * NPL * 32 + kr * 32;
#pragma unroll
            for (int l = 0; l < 32; ++l) y[l] = tr[l ^ kr];
        }
        fft_reg_dif_c<32, true>(y);                  // y[k] = x at t = k1 + NPL bitrev5(k)
        const int cy = hcol ? cyb : cya, cx = hcol ? cxb : cxa;
        const int uy = (cy + c.R) % LP, ux = (cx + c.R) % LP;
        float *o = out + (((size_t)(slot_base + sl) * LP + uy) * LP + ux) * LT + k1;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float im = __shfl_xor_sync(0xffffffffu, y[k].y, 16);   // the partner column, same t
            if (k1 < NPL) o[NPL * bitrev<32>(k)] = c.mpcp ? y[k].x + im : y[k].x;
        }
    }
    cp_async_wait<0>();
}

template <int NB1, int G, bool HZ>
static int run_conv_bp(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, float *out,
                    const ConvConst &c, int slot_base, int slot_count, cudaStream_t s) {
    static bool attr = false;
    const size_t itime_smem = itime_smem_bytes<G>();
    if (!attr) {
        cudaFuncSetAttribute(k_conv_spec<NB1, G, false, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SPEC_SMEM);
        if constexpr (G == 8)   // the tensor-core time DFT: lt = 512 only
            cudaFuncSetAttribute(k_conv_spec<NB1, G, true, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SPEC_SMEM);
        cudaFuncSetAttribute(k_conv_itime<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)itime_smem);
        if constexpr (G == 8 || G == 6) {
            cudaFuncSetAttribute(k_conv_itime_mp<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)itime_mp_smem_bytes<G>());
            cudaFuncSetAttribute(k_conv_itime_mp<G>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        attr = true;
    }
    const int sms = num_sms(h);
    const bool tc = h->p.conv_mode != 0;
    // the item queue counter: a word after the effective charge's per-CTA scratch
    int32_t *queue = h->effq_acc + (effq_scratch_bytes(h->g.bp * h->g.n_sub, sms) / sizeof(int32_t) - 48);
    const int chunk = tc ? h->zspec_blocks : h->yspec_blocks;
    const int end = slot_base + slot_count;
    for (int base = slot_base; base < end; base += chunk) {
        const int cnt = chunk < end - base ? chunk : end - base;
        if (tc) {
            if constexpr (G == 8) {   // the tensor-core time DFT: lt = 512 only
                int rc = launch_dft_gemm(h, n_blocks_dev, qeff, slot_count, base, cnt, slot_base, s);
                if (rc) return rc;
                rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "convolution queue reset");
                if (rc) return rc;
                k_conv_spec<NB1, G, true, HZ><<<sms, SPEC_THREADS, SPEC_SMEM, s>>>(
                    n_blocks_dev, qeff, h->colmask, h->rhat, h->pair_j, h->tw, c, h->yspec, base, cnt, slot_base,
                    h->zspec, queue);
            } else {
                return set_error(h, TRED_ERR_INVALID_ARG, "convolve: the tensor-core time DFT needs lt = 512");
            }
        } else {
            int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "convolution queue reset");
            if (rc) return rc;
            k_conv_spec<NB1, G, false, HZ><<<sms, SPEC_THREADS, SPEC_SMEM, s>>>(n_blocks_dev, qeff, h->colmask, h->rhat,
                                                                           h->pair_j, h->tw, c, h->yspec, base, cnt,
                                                                           slot_base, nullptr, queue);
        }
        if constexpr (G == 8 || G == 6)
            k_conv_itime_mp<G><<<sms, 32 * IT5_WARPS, itime_mp_smem_bytes<G>(), s>>>(n_blocks_dev, h->yspec, h->tw,
                                                                                  c, out, base, cnt);
        else
            k_conv_itime<G><<<sms, 32 * itime_cols<G>(), itime_smem, s>>>(n_blocks_dev, h->yspec, h->tw, c, out,
                                                                           base, cnt);
        h->launches += 2;
    }
    return check_cuda(h, cudaGetLastError(), "convolve launch");
}

template <int NB1, int G>
static int run_conv(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, float *out,
                    const ConvConst &c, int slot_base, int slot_count, cudaStream_t s) {
    return c.bp <= 4 ? run_conv_bp<NB1, G, true>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s)
                     : run_conv_bp<NB1, G, false>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
}

int launch_convolve(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                    const float *qeff, float *out, int slot_base, int slot_count, cudaStream_t s) {
    (void)block_ids;
    if (h->p.conv_mode == 4) return launch_direct(h, n_blocks_dev, qeff, out, slot_base, slot_count, slot_base, s);
    ConvConst c;
    c.ns = h->g.n_sub;
    c.bp = h->g.bp;
    c.bt = h->g.bt;
    c.nch = c.ns * c.ns;
    c.npairs = h->d.npairs;
    c.G = h->d.G;
    c.lt = h->g.lt;
    c.R = h->d.R;
    c.mpcp = h->p.mpcp;
    const int nb1 = h->g.bt / 64;
    if (c.G == 8) {
        switch (nb1) {
            case 1: return run_conv<1, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 2: return run_conv<2, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 3: return run_conv<3, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 4: return run_conv<4, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 5: return run_conv<5, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 6: return run_conv<6, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 7: return run_conv<7, 8>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            default: break;
        }
    } else if (c.G == 6) {   // lt = 384 = 3 x 128: the inverse time transform is mixed radix
        switch (nb1) {
            case 1: return run_conv<1, 6>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 2: return run_conv<2, 6>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            default: break;
        }
    } else if (c.G == 12) {   // lt = 768 = 3 x 256
        switch (nb1) {
            case 1: return run_conv<1, 12>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 2: return run_conv<2, 12>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 4: return run_conv<4, 12>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 5: return run_conv<5, 12>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 8: return run_conv<8, 12>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            default: break;
        }
    } else if (c.G == 16) {
        switch (nb1) {
            case 2: return run_conv<2, 16>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 4: return run_conv<4, 16>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 5: return run_conv<5, 16>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 8: return run_conv<8, 16>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            case 10: return run_conv<10, 16>(h, n_blocks_dev, qeff, out, c, slot_base, slot_count, s);
            default: break;
        }
    }
    return set_error(h, TRED_ERR_INVALID_ARG, "convolve: unsupported bt=%d lt=%d", h->g.bt, h->g.lt);
}

}  // namespace tred
