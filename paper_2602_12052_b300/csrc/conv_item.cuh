// Shared pieces of the convolution (a4, Sec. II-D Eq. interlaced, Sec. III-A-2 Eq.
// multch): the constants and shared-memory layout of the spectral stage, one (block,
// class) item of it, and one column of the inverse time transform.  k_conv.cu's
// kernels and the persistent block pipeline (k_pipeline.cu) are built from them.
#pragma once

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
                             sizeof(int) * (2 * PG * 64 + 4);      // stage A task lists (two rounds) and counters

// Rounds of channel pairs per (block, class) item: all of them, or half when the event has
// so few blocks that its items would leave most CTAs idle (then each half of the rounds is
// its own item, writing its partial spectra to a plane of its own, nloc planes further on,
// which the inverse time transform adds; two halves at most, and only while the spectrum
// buffer holds both planes).  Both kernels derive it from the same device-side count.
__host__ __device__ inline int conv_round_groups(int nloc, int G, int grid, int chunk) {
    return (nloc > 0 && 2 * nloc * G <= grid && 2 * nloc <= chunk) ? 2 : 1;
}

// Shared-memory carve-up of the spectral stage (stage A tiles, the per-warp transpose,
// twiddle tables, the TMEM address slot, the stage A task list and counters).
struct SpecSmem {
    float2 *zt, *ebuf, *tbuf, *w32, *w16, *w8, *w64;
    uint32_t *tslot;
    int *s_task, *s_ntask;
    __device__ explicit SpecSmem(float2 *smem) {
        zt = smem;                                // [PG][64][8][9]
        ebuf = smem;                              // [warps][2][16][17], epilogue only
        tbuf = zt + PG * BINS * ZT_BIN;           // [warps][2][16][9]
        w32 = tbuf + SPEC_WARPS * 2 * TB_BIN;     // W_32
        w16 = w32 + 32;                           // W_16
        w8 = w16 + 16;                            // W_8
        w64 = w8 + 8;                             // W_64
        tslot = reinterpret_cast<uint32_t *>(w64 + 64);
        s_task = reinterpret_cast<int *>(tslot + 4);   // [2][PG * 64] non-empty (pair, column), per round parity
        s_ntask = s_task + 2 * PG * 64;                // [2] counters, one per round parity, then the item
    }
    __device__ void load_tables(const float2 *__restrict__ tw) const {
        const int tid = threadIdx.x;
        if (tid < 32) w32[tid] = tw[TW_32 + tid];
        if (tid < 16) w16[tid] = tw[TW_16 + tid];
        if (tid < 8) w8[tid] = tw[TW_8 + tid];
        if (tid < 64) w64[tid] = tw[TW_64 + tid];
    }
};

// Loads of the effective charge: through the read-only path when another kernel wrote
// it; as ordinary cached loads (coherent with this SM's own stores, never the read-only
// path) when the same persistent CTA wrote it just before.
template <bool FUSED>
__device__ __forceinline__ float ldq(const float *p) {
    if constexpr (FUSED) return __ldca(p);
    else return __ldg(p);
}

// One (block, time-frequency class k1) item of the spectral stage over the channel pairs
// [p_beg, p_end): qblk is the block's effective charge [nch][bp][bp][bt], mrow its
// non-empty column masks, zplane (tensor-core form) its packed time spectra of class k1,
// yplane the block's [lt][16 * 16] spectrum plane that receives the class's 64 bins.
// tacc: this warp's TMEM accumulator columns.  All 512 threads take part.
template <int NB1, int G, bool ZS, bool HZ, bool FUSED>
__device__ __forceinline__ void conv_spec_item(const SpecSmem &sm, uint32_t tacc, const ConvConst &c, int k1,
                                               int p_beg, int p_end, const float *__restrict__ qblk,
                                               const uint64_t *__restrict__ mrow, const float2 *__restrict__ rhat,
                                               const int32_t *__restrict__ pair_j, const float2 *__restrict__ tw,
                                               const float2 *__restrict__ zplane, float2 *__restrict__ yplane) {
    constexpr int LT = 64 * G;
    float2 *zt = sm.zt, *ebuf = sm.ebuf, *tbuf = sm.tbuf, *w32 = sm.w32, *w64 = sm.w64;
    int *s_task = sm.s_task, *s_ntask = sm.s_ntask;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cols = c.bp * c.bp;
    const int slab = cols * c.bt;
    float2 *tb = tbuf + warp * 2 * TB_BIN;
    float2 *eb = ebuf + warp * 2 * EP_BIN;
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

    for (int p0 = p_beg; p0 < p_end; p0 += PG) {
        const int ng = min(PG, p_end - p0);
        if (ZS) {
            // ---------------- stage A from the tensor-core spectra of the round's pairs
            const float2 *zsrc = zplane + (size_t)p0 * BINS * 64;
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
            // the task lists of consecutive rounds alternate between two arrays; the
            // previous round's columns are the only non-zero ones of the buffers (the item
            // started from zeroed buffers), so zeroing them clears the buffers
            const int par = ((p0 - p_beg) / PG) & 1;
            int *s_cur = s_task + par * (PG * 64);
            const int nprev = s_ntask[par ^ 1];
            {
                const int *prev = s_task + (par ^ 1) * (PG * 64);
                for (int e = tid; e < nprev * BINS; e += SPEC_THREADS) {
                    const int task = prev[e / BINS] & 0xFFFFF, k2 = e % BINS;
                    const int g = task / cols, col = task - g * cols;
                    const int py = col / c.bp, px = col - py * c.bp;
                    zt[g * (BINS * ZT_BIN) + zt_slot(k2) * ZT_BIN + py * ZT_ROW + px] = make_float2(0.f, 0.f);
                }
            }
            for (int task = tid; task < ng * cols; task += SPEC_THREADS) {
                const int g = task / cols, col = task - g * cols;
                const int p = p0 + g;
                const int j1 = pair_j[2 * p], j2 = pair_j[2 * p + 1];
                // each half of the packed column is read only where its own mask bit is
                // set (a column that no support covers may not have been written)
                const int h1 = (int)((mrow[j1] >> col) & 1ull);
                const int h2 = j2 >= 0 ? (int)((mrow[j2] >> (cols - 1 - col)) & 1ull) : 0;
                if (h1 | h2) s_cur[atomicAdd(&s_ntask[par], 1)] = task | (h1 << 20) | (h2 << 21);
            }
            __syncthreads();
            const int ntask = s_ntask[par];
            if (tid == 0) s_ntask[par ^ 1] = 0;           // the next round's counter (read above by all)
            const int b5 = bitrev<32>(lane);
            for (int t0 = warp; t0 < ntask; t0 += 2 * SPEC_WARPS) {
                const int nt = t0 + SPEC_WARPS < ntask ? 2 : 1;
                float2 za[2][NB1], zb[2][NB1];
                int tk[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (u >= nt) break;
                    const int te = s_cur[t0 + u * SPEC_WARPS];
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
                        za[u][n1] = make_float2(q1 ? ldq<FUSED>(q1 + ta) : 0.f, q2 ? ldq<FUSED>(q2 + ta) : 0.f);
                        zb[u][n1] = make_float2(q1 ? ldq<FUSED>(q1 + tb) : 0.f, q2 ? ldq<FUSED>(q2 + tb) : 0.f);
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
                const float4 *rsrc = reinterpret_cast<const float4 *>(rhat + rhat_bin(k1 + G * k2, p0 + g, c.npairs, 2 * G) +
                                                                      rhat_kk(0, kx));
#pragma unroll
                for (int q = 0; q < LP / 2; ++q) {
                    const float4 v = __ldg(rsrc + q * LP);   // ky = 2q, 2q + 1
                    rr[2 * q] = make_float2(v.x, v.y);
                    rr[2 * q + 1] = make_float2(v.z, v.w);
                }
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
        float4 *dst = reinterpret_cast<float4 *>(yplane + (size_t)(k1 + G * k2) * (LP * LP) + r * LP);
#pragma unroll
        for (int x = 0; x < LP; x += 2) dst[x / 2] = make_float4(o[x].x, o[x].y, o[x + 1].x, o[x + 1].y);
        __syncwarp();
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

// One column of the inverse time transform with the MPCP recombination, one warp per
// column q of the item's NC (q and its mirror partner q +- NC/2 in the same CTA): the
// column's lt bins in shared memory at col (plus, if g2 is given, a second partial plane
// in global memory, lt bins at a stride of 16 * 16), the inverse FFT over time, and the
// output column (cy, cx) of the block written at oblk ([16][16][lt]) after adding the
// partner's imaginary parts.  Contains a CTA-wide barrier: every warp of the CTA calls it.
template <int G>
__device__ __forceinline__ void itime_column(const float2 *__restrict__ col, const float2 *__restrict__ g2, float *Ib,
                                             const float2 *__restrict__ wlt, const float2 *__restrict__ w32,
                                             const ConvConst &c, int q, int cy, int cx, float *__restrict__ oblk) {
    constexpr int LT = 64 * G;
    constexpr int NPL = LT / 32;          // values per lane
    constexpr int NC = itime_cols<G>();   // columns per item
    constexpr int HC = NC / 2;
    constexpr int IROW = 33;              // imaginary-part exchange: [column][bitrev(k)][lane group]
    const int lane = threadIdx.x & 31;
    float2 v[NPL];
#pragma unroll
    for (int m = 0; m < NPL; ++m) v[m] = col[lane + 32 * m];
    if (g2) {   // the second half of the rounds' spectra, from its own plane
#pragma unroll
        for (int m = 0; m < NPL; ++m) v[m] = cadd(v[m], __ldg(g2 + (size_t)(lane + 32 * m) * (LP * LP)));
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
    float *o = oblk + ((size_t)uy * LP + ux) * LT + NPL * b5;
    float r[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int t = fft_perm<NPL>(k);
        r[t] = c.mpcp ? v[k].x + pib[t * IROW + b5] : v[k].x;
    }
#pragma unroll
    for (int k = 0; k < NPL; k += 4) *reinterpret_cast<float4 *>(o + k) = make_float4(r[k], r[k + 1], r[k + 2], r[k + 3]);
}

// The rows of mirror row pair rp (the rp-th row a with a < m(a), m(r) = (bp - 1 - r) mod
// 16) and its mirror bro = m(a); and column q of part `part` of that row pair (hc
// columns per part of each row).
__device__ __forceinline__ void itime_rows_of(int bp, int rp, int &a, int &bro) {
    a = -1;
    int cnt = 0;
    for (int r = 0; r < LP; ++r) {
        const int m = (bp - 1 - r + 2 * LP) % LP;
        if (r < m) {
            if (cnt == rp) {
                a = r;
                break;
            }
            ++cnt;
        }
    }
    bro = (bp - 1 - a + 2 * LP) % LP;
}
__device__ __forceinline__ void itime_column_of(int bp, int hc, int q, int part, int a, int bro, int &cy, int &cx) {
    const int cx0 = hc * part + (q % hc);
    cy = q < hc ? a : bro;
    cx = q < hc ? cx0 : (bp - 1 - cx0 + 2 * LP) % LP;
}

}  // namespace tred
