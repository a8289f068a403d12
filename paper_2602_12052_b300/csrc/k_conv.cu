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

#include "tred_internal.cuh"

namespace tred {

struct ConvConst {
    int ns, bp, bt, nch, npairs, G, lt, R, mpcp;
};

constexpr int SPEC_THREADS = 512;
constexpr int SPEC_WARPS = SPEC_THREADS / 32;
constexpr int SPEC_TMEM_COLS = 256;         // 4 warps per lane quarter x 64 columns
constexpr int PG = 5;                       // channel pairs per stage A / stage B round
constexpr int ZT_ROW = 9;                   // padded px row of the bin-major transpose
constexpr int ZT_BIN = 8 * ZT_ROW + 1;      // [py][px] for py, px < 8, odd stride
// Bin order inside the stage A buffer.  Stage A lane l stores bins k2 = a + 2 b
// with b = bitrev5(l): the 16 lanes of a half warp hold the even b, the other 16
// the odd ones.  k2 = 4 c + 2 d + a goes to slot 32 a + 16 d + (c ^ 8 a): each half
// warp's 16 stores land on 16 distinct 8-byte bank pairs (odd bin stride), and the
// row stage's two bins k2, k2 + 1 (k2 even) sit 8 bank pairs apart, so its 16
// distinct row addresses per warp are conflict-free too.
__device__ __forceinline__ int zt_slot(int k2) {
    const int a = k2 & 1;
    return (a << 5) | (((k2 >> 1) & 1) << 4) | ((k2 >> 2) ^ (a << 3));
}
// Per-warp transpose of the row-stage outputs: (kx = 2 r + h, py) at 17 r + 8 h + py, so
// that the row stage's stores (lanes py, h at fixed r) and the column stage's loads
// (lanes kx at fixed py) both fall on 16 distinct 8-byte bank pairs per half warp
// with compile-time offsets; the bins of a warp are 136 entries apart.
constexpr int TB_R = 17;
constexpr int TB_BIN = 8 * TB_R;

constexpr int EP_ROW = LP + 1;              // epilogue transpose [cy][kx + pad]
constexpr int EP_BIN = LP * EP_ROW;
static_assert(SPEC_WARPS * 2 * EP_BIN <= PG * BINS * ZT_BIN, "the epilogue transpose reuses the stage A buffers");
constexpr size_t SPEC_SMEM = sizeof(float2) * ((size_t)PG * BINS * ZT_BIN + (size_t)SPEC_WARPS * 2 * TB_BIN +
                                               32 + 16 + 8 + 64 + 2) +
                             sizeof(int) * (PG * 64 + 4);      // stage A task list and counters

// Rounds of channel pairs per (block, class) item: all of them, or half when the event has
// so few blocks that its items would leave most CTAs idle (then each half of the rounds is
// its own item, writing its partial spectra to a plane of its own, nloc planes further on,
// which the inverse time transform adds; two halves at most, and only while the spectrum
// buffer holds both planes).  Both kernels derive it from the same device-side count.
__host__ __device__ inline int conv_round_groups(int nloc, int G, int grid, int chunk) {
    return (nloc > 0 && 2 * nloc * G <= grid && 2 * nloc <= chunk) ? 2 : 1;
}

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
    float2 *zt = smem;                                // [PG][64][8][9]
    float2 *ebuf = smem;                              // [warps][2][16][17], epilogue only
    float2 *tbuf = zt + PG * BINS * ZT_BIN;           // [warps][2][16][9]
    float2 *w32 = tbuf + SPEC_WARPS * 2 * TB_BIN;     // W_32
    float2 *w16 = w32 + 32;                           // W_16
    float2 *w8 = w16 + 16;                            // W_8
    float2 *w64 = w8 + 8;                             // W_64
    uint32_t *tslot = reinterpret_cast<uint32_t *>(w64 + 64);
    int *s_task = reinterpret_cast<int *>(tslot + 4);         // [PG * 64] non-empty (pair, column)
    int *s_ntask = s_task + PG * 64;                          // [2] counters, one per round parity
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 2) s_ntask[tid] = 0;
    if (warp == 0) {
        tmem_alloc(tslot, SPEC_TMEM_COLS);
        tmem_relinquish();
    }
    if (tid < 32) w32[tid] = tw[TW_32 + tid];
    if (tid < 16) w16[tid] = tw[TW_16 + tid];
    if (tid < 8) w8[tid] = tw[TW_8 + tid];
    if (tid < 64) w64[tid] = tw[TW_64 + tid];
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    // this warp's accumulator columns: lane quarter warp % 4, columns (warp / 4) * 64 + 32 it
    const uint32_t tacc = *tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));

    const int nb = n_blocks_dev[0];
    const int nloc = max(0, min(slot_count, nb - slot_base));
    const int cols = c.bp * c.bp;
    const int slab = cols * c.bt;
    const int ngrp = conv_round_groups(nloc, G, gridDim.x, slot_count);
    const int nrounds = (c.npairs + PG - 1) / PG;
    const int items = nloc * G * ngrp;
    float2 *tb = tbuf + warp * 2 * TB_BIN;
    float2 *eb = ebuf + warp * 2 * EP_BIN;

    // items are taken from a queue (their stage A cost varies with the block's non-empty columns)
    for (;;) {
        __syncthreads();
        if (tid == 0) s_ntask[2] = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_ntask[2];
        if (item >= items) break;
        const int grp = item % ngrp, sl = item / ngrp / G, k1 = (item / ngrp) % G;
        const int slot = slot_base + sl;
        const int p_beg = PG * (grp * nrounds / ngrp), p_end = min(c.npairs, PG * ((grp + 1) * nrounds / ngrp));
        // zero the stage A buffers (the previous epilogue used them; rows and columns
        // beyond bp must read as zero)
        __syncthreads();
        for (int k = tid; k < PG * BINS * ZT_BIN; k += SPEC_THREADS) zt[k] = make_float2(0.f, 0.f);
        if (tid < 2) s_ntask[tid] = 0;                  // round counters start at zero per item
        __syncthreads();
        // per-lane stage A twiddles for this class
        float2 wg[NB1];
#pragma unroll
        for (int n1 = 0; n1 < NB1; ++n1) wg[n1] = tw[TW_LT + ((64 * k1 * n1) % LT)];
        const float2 wl0 = tw[TW_LT + (k1 * lane) % LT];
        const float2 wl1 = tw[TW_LT + (k1 * (lane + 32)) % LT];
        const float2 w64l = w64[lane];
        {
            float z[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) z[k] = 0.f;
            tmem_st32(tacc, z);
            tmem_st32(tacc + 32, z);
        }

        const float *qblk = qeff + (size_t)(slot - qbase) * c.nch * slab;
        const uint64_t *mrow = colmask + (size_t)slot * c.nch;
        for (int p0 = p_beg; p0 < p_end; p0 += PG) {
            const int ng = min(PG, p_end - p0);
            if (ZS) {
                // ---------------- stage A from the tensor-core spectra of the round's pairs
                const float2 *zsrc = zspec + (((size_t)sl * G + k1) * c.npairs + p0) * BINS * 64;
                for (int e = tid; e < ng * BINS * cols; e += SPEC_THREADS) {
                    const int g = e / (BINS * cols), r = e - g * (BINS * cols);
                    const int k2 = r / cols, col = r - k2 * cols;
                    const int py = col / c.bp, px = col - py * c.bp;
                    zt[g * (BINS * ZT_BIN) + zt_slot(k2) * ZT_BIN + py * ZT_ROW + px] =
                        zsrc[((size_t)g * BINS + k2) * 64 + col];
                }
            }
            // ---------------- stage A: class-restricted time DFT of the non-empty columns.
            // The round's buffers are zeroed and the non-empty (pair, column) tasks listed,
            // so that the warps share the few columns that carry charge evenly and each
            // warp issues the loads of two columns before computing either.
            if (!ZS) {
                const int par = (p0 / PG) & 1;
                float4 *z4 = reinterpret_cast<float4 *>(zt);
                for (int k = tid; k < ng * BINS * ZT_BIN / 2; k += SPEC_THREADS) z4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (tid == 0) s_ntask[par ^ 1] = 0;
                for (int task = tid; task < ng * cols; task += SPEC_THREADS) {
                    const int g = task / cols, col = task - g * cols;
                    const int p = p0 + g;
                    const int j1 = pair_j[2 * p], j2 = pair_j[2 * p + 1];
                    // each half of the packed column is read only where its own mask bit is
                    // set (a column that no support covers may not have been written)
                    const int h1 = (int)((mrow[j1] >> col) & 1ull);
                    const int h2 = j2 >= 0 ? (int)((mrow[j2] >> (cols - 1 - col)) & 1ull) : 0;
                    if (h1 | h2) s_task[atomicAdd(&s_ntask[par], 1)] = task | (h1 << 20) | (h2 << 21);
                }
                __syncthreads();
                const int ntask = s_ntask[par];
                const int b5 = bitrev<32>(lane);
                for (int t0 = warp; t0 < ntask; t0 += 2 * SPEC_WARPS) {
                    const int nt = t0 + SPEC_WARPS < ntask ? 2 : 1;
                    float2 za[2][NB1], zb[2][NB1];
                    int tk[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (u >= nt) break;
                        const int te = s_task[t0 + u * SPEC_WARPS];
                        const int task = te & 0xFFFFF;
                        tk[u] = task;
                        const int g = task / cols, col = task - g * cols;
                        const int p = p0 + g;
                        const int j1 = pair_j[2 * p], j2 = pair_j[2 * p + 1];
                        const float *q1 = (te >> 20) & 1 ? qblk + (size_t)j1 * slab + (size_t)col * c.bt : nullptr;
                        const float *q2 = (te >> 21) & 1 ? qblk + (size_t)j2 * slab + (size_t)(cols - 1 - col) * c.bt : nullptr;
#pragma unroll
                        for (int n1 = 0; n1 < NB1; ++n1) {
                            const int ta = lane + 64 * n1, tb = ta + 32;
                            za[u][n1] = make_float2(q1 ? __ldg(q1 + ta) : 0.f, q2 ? __ldg(q2 + ta) : 0.f);
                            zb[u][n1] = make_float2(q1 ? __ldg(q1 + tb) : 0.f, q2 ? __ldg(q2 + tb) : 0.f);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (u >= nt) break;
                        const int task = tk[u];
                        const int g = task / cols, col = task - g * cols;
                        const int py = col / c.bp, px = col - py * c.bp;
                        float2 *zdst = zt + g * (BINS * ZT_BIN) + py * ZT_ROW + px;
                        float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int n1 = 0; n1 < NB1; ++n1) {
                            y0 = cfma(za[u][n1], wg[n1], y0);
                            y1 = cfma(zb[u][n1], wg[n1], y1);
                        }
                        y0 = cmul(y0, wl0);
                        y1 = cmul(y1, wl1);
                        float2 v0 = cadd(y0, y1);
                        float2 v1 = cmul(csub(y0, y1), w64l);
                        v0 = fft32_lanes<false>(v0, w32, lane);
                        v1 = fft32_lanes<false>(v1, w32, lane);
                        zdst[zt_slot(2 * b5) * ZT_BIN] = v0;          // bin k2 = a + 2 b
                        zdst[zt_slot(2 * b5 + 1) * ZT_BIN] = v1;
                    }
                }
            }
            __syncthreads();
            // ---------------- stage B: spatial FFT per bin, product with Rhat, sum over the
            // round's pairs in registers, one accumulator update in tensor memory
#pragma unroll 1
            for (int it = 0; it < BINS / (2 * SPEC_WARPS); ++it) {
                const int b = lane >> 4;
                const int k2 = (BINS / SPEC_WARPS) * warp + 2 * it + b;
                const int kx = lane & 15;
                float a[32];                                   // columns 2 ky + {re, im}
                tmem_ld32(tacc + 32 * it, a);
#pragma unroll 1
                for (int g = 0; g < ng; ++g) {
                    // this lane's Rhat column (kx = lane & 15); the 16 lanes of a bin read
                    // one contiguous 128-byte ky row per load
                    float2 rr[LP];
                    const float2 *rsrc = rhat + rhat_bin(k1 + G * k2, p0 + g, c.npairs, 2 * G) + kx;
#pragma unroll
                    for (int ky = 0; ky < LP; ++ky) rr[ky] = __ldg(rsrc + ky * LP);
                    // x stage: lane = (b, py, h): 8-point FFT of the (twiddled) row
                    {
                        const int py = (lane >> 1) & 7, h = lane & 1;
                        const float2 *zrow = zt + g * (BINS * ZT_BIN) + zt_slot(k2) * ZT_BIN + py * ZT_ROW;
                        float2 v[8];
#pragma unroll
                        for (int x = 0; x < 8; ++x) {
                            if (HZ && x >= 4) {
                                v[x] = make_float2(0.f, 0.f);              // not read
                                continue;
                            }
                            const float2 z = zrow[x];
                            if (x == 0) {
                                v[x] = z;                                  // W_16^0
                            } else if (x == 4) {
                                v[x] = h ? make_float2(z.y, -z.x) : z;     // W_16^4 = -i
                            } else {
                                const float wr = h ? w32c(2 * x) : 1.f, wi = h ? w32s(2 * x) : 0.f;
                                v[x] = make_float2(z.x * wr - z.y * wi, z.x * wi + z.y * wr);
                            }
                        }
                        fft_reg_dif_c<8, false, HZ>(v);
                        float2 *dst = tb + b * TB_BIN + 8 * h + py;
#pragma unroll
                        for (int k = 0; k < 8; ++k) dst[TB_R * bitrev<8>(k)] = v[k];   // kx = 2 bitrev3(k) + h
                    }
                    __syncwarp();
                    // y stage: lane = (b, kx): 16-point FFT of 8 nonzero inputs
                    {
                        const float2 *src = tb + b * TB_BIN + TB_R * (kx >> 1) + 8 * (kx & 1);
                        float2 e[8], o[8];
#pragma unroll
                        for (int y = 0; y < 8; ++y) {
                            if (HZ && y >= 4) {
                                e[y] = o[y] = make_float2(0.f, 0.f);      // not read
                                continue;
                            }
                            e[y] = src[y];
                            o[y] = mul_w16(e[y], y);                       // e W_16^y
                        }
                        fft_reg_dif_c<8, false, HZ>(e);
                        fft_reg_dif_c<8, false, HZ>(o);
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int q = bitrev<8>(k);            // ky pair (2q, 2q + 1)
                            const float2 a0 = cfma(e[k], rr[2 * q], make_float2(a[4 * q], a[4 * q + 1]));
                            const float2 a1 = cfma(o[k], rr[2 * q + 1], make_float2(a[4 * q + 2], a[4 * q + 3]));
                            a[4 * q] = a0.x;
                            a[4 * q + 1] = a0.y;
                            a[4 * q + 2] = a1.x;
                            a[4 * q + 3] = a1.y;
                        }
                    }
                    __syncwarp();
                }
                tmem_st32(tacc + 32 * it, a);
            }
            __syncthreads();
        }
        // ---------------- epilogue: inverse spatial FFT of every bin from the accumulator
#pragma unroll 1
        for (int it = 0; it < BINS / (2 * SPEC_WARPS); ++it) {
            const int b = lane >> 4, r = lane & 15;
            const int k2 = (BINS / SPEC_WARPS) * warp + 2 * it + b;
            float a[32];
            tmem_ld32(tacc + 32 * it, a);
            float2 v[LP];
#pragma unroll
            for (int ky = 0; ky < LP; ++ky) v[ky] = make_float2(a[2 * ky], a[2 * ky + 1]);   // kx = r
            fft_reg_dif_c<LP, true>(v);                   // over ky: v[k] holds cy = bitrev16(k)
#pragma unroll
            for (int k = 0; k < LP; ++k) eb[b * EP_BIN + bitrev<LP>(k) * EP_ROW + r] = v[k];
            __syncwarp();
#pragma unroll
            for (int x = 0; x < LP; ++x) v[x] = eb[b * EP_BIN + r * EP_ROW + x];   // cy = r over kx
            fft_reg_dif_c<LP, true>(v);                   // v[k] holds cx = bitrev16(k)
            float2 o[LP];
#pragma unroll
            for (int k = 0; k < LP; ++k) o[bitrev<LP>(k)] = v[k];
            float4 *dst = reinterpret_cast<float4 *>(yspec + ((size_t)(grp * nloc + sl) * LT + (k1 + G * k2)) * (LP * LP) + r * LP);
#pragma unroll
            for (int x = 0; x < LP; x += 2) dst[x / 2] = make_float4(o[x].x, o[x].y, o[x + 1].x, o[x + 1].y);
            __syncwarp();
        }
    }
    // release the accumulator columns once every warp is done with them
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(*tslot, SPEC_TMEM_COLS);
    }
}

// 8-byte asynchronous copy global -> shared (through L1), committed per item
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Inverse time FFT + MPCP recombination.  An item is NC columns of one block: NC / 2
// columns (a, cx) of a row a and their mirrors (m(a), m(cx)), m(c) = (bp - 1 - c) mod 16.
// Persistent CTAs, one warp per column: the next item's spectra stream into the
// other half of a double buffer (cp.async) while the current item is transformed;
// mirror partners exchange their imaginary parts through shared memory.
template <int G>
__host__ __device__ constexpr int itime_cols() { return 64 * G <= 512 ? 16 : 8; }
template <int G>
constexpr size_t itime_smem_bytes() {
    return sizeof(float2) * (2 * itime_cols<G>() * (64 * G + 1) + 64 * G + 32) +
           sizeof(float) * itime_cols<G>() * (2 * G) * 33;
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
        float2 v[NPL];
        {
            const float2 *src = S + (cur * NC + q) * SROW;
#pragma unroll
            for (int m = 0; m < NPL; ++m) v[m] = src[lane + 32 * m];
            if (ngrp == 2) {   // the second half of the rounds' spectra, from its own plane
                const float2 *g2 = yspec + (size_t)(nloc + sl) * LT * (LP * LP) + cy * LP + cx;
#pragma unroll
                for (int m = 0; m < NPL; ++m) v[m] = cadd(v[m], __ldg(g2 + (size_t)(lane + 32 * m) * (LP * LP)));
            }
        }
        fft_reg_any<NPL, true>(v);                // v[k] = u[fft_perm(k)]
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            const int aa = fft_perm<NPL>(k);
            float2 w = wlt[(lane * aa) % LT];
            w.y = -w.y;
            v[k] = fft32_lanes<true>(cmul(v[k], w), w32, lane);
        }
        // lane holds t = NPL * bitrev5(lane) + fft_perm(k) in register k
        const int b5 = bitrev<32>(lane);
        float *ib = Ib + q * NPL * IROW;
#pragma unroll
        for (int k = 0; k < NPL; ++k) ib[fft_perm<NPL>(k) * IROW + b5] = v[k].y;
        __syncthreads();
        const float *pib = Ib + (q < HC ? q + HC : q - HC) * NPL * IROW;   // mirror partner
        const int uy = (cy + c.R) % LP, ux = (cx + c.R) % LP;
        float *o = out + (((size_t)(slot_base + sl) * LP + uy) * LP + ux) * LT + NPL * b5;
        float r[NPL];
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            const int t = fft_perm<NPL>(k);
            r[t] = c.mpcp ? v[k].x + pib[t * IROW + b5] : v[k].x;
        }
#pragma unroll
        for (int k = 0; k < NPL; k += 4) *reinterpret_cast<float4 *>(o + k) = make_float4(r[k], r[k + 1], r[k + 2], r[k + 3]);
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
