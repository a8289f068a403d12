// Differentiable simulation (Sec. V-C): the adjoint of the hot path for a loss on
// the pixel currents, with the quadrature recomputed instead of stored.
//
//   k_resid         r = I - I* on the current pixel list (target matched by pixel id)
//                   and L = 1/2 sum over the union of both lists of (I - I*)^2
//   k_adj_spec      per (block, time-frequency class): the packed output-side
//                   gradient D = r[u(c)] + i r[mirror u(c)] of every cyclic column,
//                   its class-restricted time DFT and 16 x 16 spatial FFT, then per
//                   channel pair conj(Rhat) * Dhat and the inverse spatial FFT
//                   restricted to the block's bp x bp input pixels
//   k_adj_itime     inverse time FFT per (block, pair, input column): real part ->
//                   dL/dQeff of the first impact, imaginary part -> of the mirror
//                   impact at the flipped column (Eq. multch read backwards); at
//                   lt = 512 k_adj_itime512, two columns per warp and a shared transpose
//                   between in-lane stages instead of cross-lane butterflies
//   k_adj_weights   per deposit: the 1-D weights and their derivatives in mu, sigma
//   k_adj_chain     per (block, deposit): sums of dL/dQeff against the separable
//                   weights and derivatives -> dL/d(q, mu, sigma) (windows fixed), the
//                   lanes along time so that the gradient loads cover whole sectors
//   k_adj_params    chain rule through the transport step to dL/d(x, y, t0, ne) and
//                   the global dL/d(DL, DT, tau)
#include "tred_internal.cuh"

namespace tred {

// ------------------------------------------------------------------ residual and loss
__device__ __forceinline__ int find_sorted(const int32_t *__restrict__ a, int n, int key) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void __launch_bounds__(256) k_resid(const int32_t *__restrict__ pix, const int32_t *__restrict__ n_pix_dev,
                                               const float *__restrict__ wave, const int32_t *__restrict__ tpix,
                                               int n_target, const float *__restrict__ twave, int nt,
                                               float *__restrict__ resid, double *__restrict__ loss) {
    const int np = n_pix_dev[0];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    // rows of the current list: r = I - I*
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < np + n_target; row += nwarps) {
        if (row < np) {
            const int tr = find_sorted(tpix, n_target, pix[row]);
            const float *a = wave + (size_t)row * nt;
            const float *b = tr >= 0 ? twave + (size_t)tr * nt : nullptr;
            float *o = resid + (size_t)row * nt;
            // squares summed in FP32 eight at a time, the partial sums in FP64
            for (int t0 = lane; t0 < nt; t0 += 32 * 8) {
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + 32 * u;
                    if (t < nt) {
                        const float v = a[t] - (b ? b[t] : 0.f);
                        o[t] = v;
                        part = fmaf(v, v, part);
                    }
                }
                acc += 0.5 * (double)part;
            }
        } else {
            // target pixels the current pass does not reach: constant part of L
            const int tr = row - np;
            if (find_sorted(pix, np, tpix[tr]) >= 0) continue;
            const float *b = twave + (size_t)tr * nt;
            for (int t0 = lane; t0 < nt; t0 += 32 * 8) {
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + 32 * u;
                    if (t < nt) part = fmaf(b[t], b[t], part);
                }
                acc += 0.5 * (double)part;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(loss, acc);
}

// pixel -> row of the current list (or -1)
__global__ void k_row_map(const int32_t *__restrict__ pix, const int32_t *__restrict__ n_pix_dev,
                          int32_t *__restrict__ row_of) {
    const int np = n_pix_dev[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) row_of[pix[k]] = k;
}

// ------------------------------------------------------------------ adjoint convolution
struct AdjConst {
    int ns, bp, bt, nr, nt, nch, npairs, R, mpcp, nbx, nbt, npx_x, npx_y;
    int npy_e, nby_e;              // pixel rows and block rows of one event
};

constexpr int AS_THREADS = 512;
constexpr int AS_WARPS = AS_THREADS / 32;
constexpr int DH_ROW = 17;                  // [slot][ky][kx] rows padded
constexpr int DH_BIN = LP * DH_ROW + 1;     // odd bin stride
constexpr int AT_ROW = 18;                  // per-warp transpose [2][8 cy][16 kx + 2]
constexpr int AT_BIN = 8 * AT_ROW;
// Bin slot in the spectrum buffer: bin k2 = 4 c + 2 d + a at slot 32 a + 16 d + c.  Stage
// A's lane l holds bins 2 b + {0, 1}, b = bitrev5(l), so each half warp's 16 stores land
// on 16 distinct slots modulo 16, i.e. distinct bank pairs with the odd bin stride.
__device__ __forceinline__ int dh_slot(int k2) { return ((k2 & 1) << 5) | (((k2 >> 1) & 1) << 4) | (k2 >> 2); }
constexpr size_t ADJ_SPEC_SMEM = sizeof(float2) * ((size_t)BINS * DH_BIN + (size_t)AS_WARPS * 2 * AT_BIN);

template <int G>
__global__ void __launch_bounds__(AS_THREADS, 1)
    k_adj_spec(const int32_t *__restrict__ n_blocks_dev, const int32_t *__restrict__ block_ids,
               const float *__restrict__ resid, const int32_t *__restrict__ row_of,
               const float2 *__restrict__ tw, const float2 *__restrict__ rhat, AdjConst c,
               float2 *__restrict__ gspec, int slot_base, int slot_count, int32_t *__restrict__ queue) {
    constexpr int LT = 64 * G;
    extern __shared__ float2 sm_a[];
    __shared__ int s_item;
    float2 *dh = sm_a;                                  // [64][16][17]
    float2 *tbuf = dh + BINS * DH_BIN;                  // [warps][2][8][17]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = n_blocks_dev[0];
    const int nloc = min(slot_count, nb - slot_base);
    if (nloc <= 0) return;
    const int span = c.bt + c.nr - 1;
    float2 *tb = tbuf + warp * 2 * AT_BIN;
    for (;;) {   // (block, class) items from a queue
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nloc * G) break;
        const int sl = item / G, k1 = item % G;
        const int slot = slot_base + sl;
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int T0 = bt * c.bt;
        const int ylo = (by / c.nby_e) * c.npy_e, yhi = ylo + c.npy_e;   // the block's event band
        const float2 wl0 = tw[TW_LT + (k1 * lane) % LT];
        const float2 wl1 = tw[TW_LT + (k1 * (lane + 32)) % LT];
        const float2 w64l = tw[TW_64 + lane];
        // ---- stage A: class-restricted time DFT of the 256 packed columns
        for (int col = warp; col < LP * LP; col += AS_WARPS) {
            const int cy = col >> 4, cx = col & 15;
            // output pixels of the real and imaginary parts (block-local u = c + R, mirror)
            const int uy1 = (cy + c.R) % LP, ux1 = (cx + c.R) % LP;
            const int uy2 = (c.bp - 1 + c.R - cy + 2 * LP) % LP, ux2 = (c.bp - 1 + c.R - cx + 2 * LP) % LP;
            const int Y1 = by * c.bp + uy1 - c.R, X1 = bx * c.bp + ux1 - c.R;
            const int Y2 = by * c.bp + uy2 - c.R, X2 = bx * c.bp + ux2 - c.R;
            const int r1 = (uy1 < c.bp + 2 * c.R && ux1 < c.bp + 2 * c.R && Y1 >= ylo && Y1 < yhi && X1 >= 0 &&
                            X1 < c.npx_x) ? row_of[Y1 * c.npx_x + X1] : -1;
            const int r2 = (c.mpcp && uy2 < c.bp + 2 * c.R && ux2 < c.bp + 2 * c.R && Y2 >= ylo && Y2 < yhi &&
                            X2 >= 0 && X2 < c.npx_x) ? row_of[Y2 * c.npx_x + X2] : -1;
            const float *a1 = r1 >= 0 ? resid + (size_t)r1 * c.nt + T0 : nullptr;
            const float *a2 = r2 >= 0 ? resid + (size_t)r2 * c.nt + T0 : nullptr;
            float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
            if (a1 || a2) {
#pragma unroll
                for (int n1 = 0; n1 < G; ++n1) {
                    const float2 wg = tw[TW_LT + ((64 * k1 * n1) % LT)];
                    const int t0 = lane + 64 * n1, t1 = t0 + 32;
                    const bool ok0 = t0 < span && T0 + t0 < c.nt, ok1 = t1 < span && T0 + t1 < c.nt;
                    const float2 z0 = make_float2(ok0 && a1 ? a1[t0] : 0.f, ok0 && a2 ? a2[t0] : 0.f);
                    const float2 z1 = make_float2(ok1 && a1 ? a1[t1] : 0.f, ok1 && a2 ? a2[t1] : 0.f);
                    y0 = cfma(z0, wg, y0);
                    y1 = cfma(z1, wg, y1);
                }
            }
            y0 = cmul(y0, wl0);
            y1 = cmul(y1, wl1);
            float2 v0 = cadd(y0, y1);
            float2 v1 = cmul(csub(y0, y1), w64l);
            v0 = fft32_lanes<false>(v0, tw + TW_32, lane);
            v1 = fft32_lanes<false>(v1, tw + TW_32, lane);
            const int b5 = bitrev<32>(lane);
            dh[dh_slot(2 * b5) * DH_BIN + cy * DH_ROW + cx] = v0;
            dh[dh_slot(2 * b5 + 1) * DH_BIN + cy * DH_ROW + cx] = v1;
        }
        __syncthreads();
        // ---- forward 16 x 16 spatial FFT of every bin, in place -> [k2][ky][kx]
        for (int it = 0; it < BINS / (2 * AS_WARPS); ++it) {
            const int b = lane >> 4, r = lane & 15;
            const int k2 = (BINS / AS_WARPS) * warp + 2 * it + b;
            float2 *d = dh + dh_slot(k2) * DH_BIN;
            float2 v[LP];
#pragma unroll
            for (int x = 0; x < LP; ++x) v[x] = d[r * DH_ROW + x];          // row cy = r over cx
            fft_reg_dif_c<LP, false>(v);
#pragma unroll
            for (int k = 0; k < LP; ++k) d[r * DH_ROW + bitrev<LP>(k)] = v[k];   // [cy][kx]
            __syncwarp();
#pragma unroll
            for (int y = 0; y < LP; ++y) v[y] = d[y * DH_ROW + r];          // column kx = r over cy
            fft_reg_dif_c<LP, false>(v);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < LP; ++k) d[bitrev<LP>(k) * DH_ROW + r] = v[k];   // [ky][kx]
            __syncwarp();
        }
        __syncthreads();
        // ---- per channel pair: conj(Rhat) Dhat, inverse spatial FFT onto the bp x bp inputs
        for (int p = 0; p < c.npairs; ++p) {
            const float2 *rp = rhat;   // bin f = k1 + G k2 at rhat_bin(f, p, npairs, lt / 32)
            float2 *gdst = gspec + (((size_t)sl * c.npairs + p) * LT) * 64;
            for (int it = 0; it < BINS / (2 * AS_WARPS); ++it) {
                const int b = lane >> 4, kx = lane & 15;
                const int k2 = (BINS / AS_WARPS) * warp + 2 * it + b;
                const float2 *d = dh + dh_slot(k2) * DH_BIN + kx;
                const float4 *rsrc = reinterpret_cast<const float4 *>(rp + rhat_bin(k1 + G * k2, p, c.npairs, LT / 32) +
                                                                      rhat_kk(0, kx));
                float2 v[LP];
#pragma unroll
                for (int q = 0; q < LP / 2; ++q) {
                    const float4 r = __ldg(rsrc + q * LP);   // ky = 2q, 2q + 1
                    v[2 * q] = cmul(cconj(make_float2(r.x, r.y)), d[2 * q * DH_ROW]);
                    v[2 * q + 1] = cmul(cconj(make_float2(r.z, r.w)), d[(2 * q + 1) * DH_ROW]);
                }
                fft_reg_dif_c<LP, true>(v);                 // over ky -> cy (bit-reversed)
                float2 *t = tb + b * AT_BIN;
#pragma unroll
                for (int k = 0; k < LP; ++k) {
                    const int cy = bitrev<LP>(k);
                    if (cy < 8) t[cy * AT_ROW + kx] = v[k];
                }
                __syncwarp();
                // over kx -> cx for the 8 input rows: lane (b, cy, h): h selects even/odd kx
                {
                    const int cy = (lane >> 1) & 7, h = lane & 1;
                    const float2 *src = tb + b * AT_BIN + cy * AT_ROW;
                    float2 e[8];
#pragma unroll
                    for (int m = 0; m < 8; ++m) e[m] = src[2 * m + h];
                    fft_reg_dif_c<8, true>(e);              // e[k] = sum_m W[2m+h] W8^{-m cx}, cx = bitrev3(k)
                    float2 res[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int cx = bitrev<8>(k);
                        float2 val = e[k];
                        if (h) {                            // times W16^{-cx}
                            const float wr = w32c(2 * cx), wi = -w32s(2 * cx);
                            val = make_float2(val.x * wr - val.y * wi, val.x * wi + val.y * wr);
                        }
                        float2 o;
                        o.x = __shfl_xor_sync(0xffffffffu, val.x, 1);
                        o.y = __shfl_xor_sync(0xffffffffu, val.y, 1);
                        res[cx] = cadd(val, o);
                    }
                    if (h == 0 && cy < c.bp) {
                        float2 *g = gdst + (size_t)(k1 + G * k2) * 64 + cy * 8;
#pragma unroll
                        for (int cx = 0; cx < 8; ++cx) g[cx] = res[cx];
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

// 8-byte asynchronous copy global -> shared (through L1), committed per item
__device__ __forceinline__ void acp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void acp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void acp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int G>
__host__ __device__ constexpr int adj_itime_cols() { return G == 8 ? 16 : 8; }
template <int G>
constexpr size_t adj_itime_smem() {
    return sizeof(float2) * (2 * adj_itime_cols<G>() * (64 * G + 1) + 64 * G + 32);
}

// Inverse time FFT of the packed adjoint spectra; writes dL/dQeff of both impacts of
// each pair.  Persistent CTAs over (block, pair, group of NC input columns) items, one
// warp per column; the next item's spectra stream into the other half of a double
// buffer (cp.async) while the current item is transformed, and each lane writes its
// 16 (or 32) consecutive ticks as float4 stores.
template <int G>
__global__ void __launch_bounds__(32 * adj_itime_cols<G>(), 1)
    k_adj_itime(const int32_t *__restrict__ n_blocks_dev, const float2 *__restrict__ gspec,
                const int32_t *__restrict__ pair_j, const float2 *__restrict__ tw, AdjConst c,
                float *__restrict__ gq, int slot_base, int slot_count) {
    constexpr int LT = 64 * G;
    constexpr int NPL = LT / 32;
    constexpr int NC = adj_itime_cols<G>();
    constexpr int NT = 32 * NC;
    constexpr int SROW = LT + 1;
    extern __shared__ float2 sm_t[];
    float2 *S = sm_t;                      // [2][NC][LT + 1]
    float2 *wlt = S + 2 * NC * SROW;
    float2 *w32 = wlt + LT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = tid; k < LT; k += NT) wlt[k] = tw[TW_LT + k];
    if (tid < 32) w32[tid] = tw[TW_32 + tid];
    const int nb = n_blocks_dev[0];
    const int nloc = min(slot_count, nb - slot_base);
    if (nloc <= 0) return;
    const int cols = c.bp * c.bp;
    const int groups = (cols + NC - 1) / NC;
    const int items = nloc * c.npairs * groups;
    // thread tid copies column q = tid % NC of the item at frequencies f = tid / NC + 32 j
    auto issue = [&](int item, int bsel) {
        const int grp = item % groups;
        const int p = (item / groups) % c.npairs;
        const int sl = item / (groups * c.npairs);
        const int q = tid % NC, col = grp * NC + q;
        if (col < cols) {
            const int py = col / c.bp, px = col % c.bp;
            const float2 *src = gspec + ((size_t)sl * c.npairs + p) * LT * 64 + py * 8 + px;
            float2 *dst = S + (bsel * NC + q) * SROW;
#pragma unroll 4
            for (int f = tid / NC; f < LT; f += NT / NC) acp_async8(dst + f, src + (size_t)f * 64);
        }
        acp_commit();
    };
    int item = blockIdx.x;
    if (item < items) issue(item, 0);
    for (int i = 0; item < items; ++i, item += gridDim.x) {
        const int cur = i & 1;
        if (item + (int)gridDim.x < items)
            issue(item + gridDim.x, cur ^ 1);   // that buffer's last readers passed the previous barrier
        else
            acp_commit();                       // empty group: keeps the wait count uniform
        acp_wait<1>();
        __syncthreads();                        // this item's columns (and the W tables) are in place
        const int grp = item % groups;
        const int p = (item / groups) % c.npairs;
        const int sl = item / (groups * c.npairs);
        const int col = grp * NC + warp;
        if (col < cols) {
            float2 v[NPL];
#pragma unroll
            for (int m = 0; m < NPL; ++m) v[m] = S[(cur * NC + warp) * SROW + lane + 32 * m];
            fft_reg_dif_c<NPL, true>(v);
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int aa = bitrev<NPL>(k);
                float2 w = wlt[(lane * aa) % LT];
                w.y = -w.y;
                v[k] = fft32_lanes<true>(cmul(v[k], w), w32, lane);
            }
            // lane holds t = NPL * bitrev5(lane) + bitrev(k); bt is a multiple of NPL, so a
            // lane's NPL consecutive ticks are all inside [0, bt) or all beyond it
            const int tbase = NPL * bitrev<32>(lane);
            if (tbase < c.bt) {
                const int slot = slot_base + sl;
                const int j1 = pair_j[2 * p], j2 = pair_j[2 * p + 1];
                float *o1 = gq + (((size_t)slot * c.nch + j1) * cols + col) * c.bt + tbase;
#pragma unroll
                for (int k = 0; k < NPL; k += 4)        // tick k + e sits in register bitrev(k + e)
                    *reinterpret_cast<float4 *>(o1 + k) =
                        make_float4(v[bitrev<NPL>(k)].x, v[bitrev<NPL>(k + 1)].x, v[bitrev<NPL>(k + 2)].x,
                                    v[bitrev<NPL>(k + 3)].x);
                if (j2 >= 0) {
                    float *o2 = gq + (((size_t)slot * c.nch + j2) * cols + (cols - 1 - col)) * c.bt + tbase;
#pragma unroll
                    for (int k = 0; k < NPL; k += 4)
                        *reinterpret_cast<float4 *>(o2 + k) =
                            make_float4(v[bitrev<NPL>(k)].y, v[bitrev<NPL>(k + 1)].y, v[bitrev<NPL>(k + 2)].y,
                                        v[bitrev<NPL>(k + 3)].y);
                }
            }
        }
    }
    acp_wait<0>();
}

// The same transform at lt = 512 with two columns per warp (columns w and w + 8 of the
// item): a 16-point in-lane DFT over m (n = l + 32 m), the twiddles W_512^(l k1), a
// per-warp shared transpose and one 32-point in-lane DFT per lane (lane = (column, k1)),
// so t = k1 + 16 k2 with no cross-lane butterflies; each half warp stores 64-byte runs.
constexpr int AIT5_THREADS = 256;
constexpr size_t adj_itime512_smem() {
    return sizeof(float2) * (2 * 16 * 513 + 512 + (AIT5_THREADS / 32) * 2 * 512);
}

__global__ void __launch_bounds__(AIT5_THREADS, 1)
    k_adj_itime512(const int32_t *__restrict__ n_blocks_dev, const float2 *__restrict__ gspec,
                   const int32_t *__restrict__ pair_j, const float2 *__restrict__ tw, AdjConst c,
                   float *__restrict__ gq, int slot_base, int slot_count) {
    constexpr int LT = 512, NC = 16, HC = 8, NT = AIT5_THREADS, SROW = LT + 1;
    extern __shared__ float2 sm_t[];
    float2 *S = sm_t;                      // [2][NC][LT + 1]
    float2 *twl = S + 2 * NC * SROW;       // [k1][l] = conj(W_512^(l k1))
    float2 *T = twl + 512;                 // per warp [2 columns][k1][l ^ k1]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 512; i += NT) {
        float2 w = tw[TW_LT + (i & 31) * (i >> 5)];
        w.y = -w.y;
        twl[i] = w;
    }
    const int nb = n_blocks_dev[0];
    const int nloc = min(slot_count, nb - slot_base);
    if (nloc <= 0) return;
    const int cols = c.bp * c.bp;
    const int groups = (cols + NC - 1) / NC;
    const int items = nloc * c.npairs * groups;
    // thread tid copies column q = tid % NC of the item at frequencies f = tid / NC + 16 j
    auto issue = [&](int item, int bsel) {
        const int grp = item % groups;
        const int p = (item / groups) % c.npairs;
        const int sl = item / (groups * c.npairs);
        const int q = tid % NC, col = grp * NC + q;
        if (col < cols) {
            const int py = col / c.bp, px = col % c.bp;
            const float2 *src = gspec + ((size_t)sl * c.npairs + p) * LT * 64 + py * 8 + px;
            float2 *dst = S + (bsel * NC + q) * SROW;
#pragma unroll 4
            for (int f = tid / NC; f < LT; f += NT / NC) acp_async8(dst + f, src + (size_t)f * 64);
        }
        acp_commit();
    };
    float2 *Ta = T + warp * 2 * 512;
    int item = blockIdx.x;
    if (item < items) issue(item, 0);
    for (int i = 0; item < items; ++i, item += gridDim.x) {
        const int cur = i & 1;
        acp_wait<0>();
        __syncthreads();                        // this item's columns are in place, the other buffer is free
        if (item + (int)gridDim.x < items) issue(item + gridDim.x, cur ^ 1);
        const int grp = item % groups;
        const int p = (item / groups) % c.npairs;
        const int sl = item / (groups * c.npairs);
        const int cola = grp * NC + warp;
        if (cola >= cols) continue;             // warp-uniform; then column b is out of range too
        {
            float2 va[16], vb[16];
            const float2 *sa = S + (cur * NC + warp) * SROW, *sb = S + (cur * NC + warp + HC) * SROW;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                va[m] = sa[lane + 32 * m];
                vb[m] = sb[lane + 32 * m];
            }
            fft_reg_dif_c<16, true>(va);
            fft_reg_dif_c<16, true>(vb);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int k1 = bitrev<16>(k);
                const float2 w = twl[k1 * 32 + lane];
                Ta[k1 * 32 + (lane ^ k1)] = cmul(va[k], w);
                Ta[512 + k1 * 32 + (lane ^ k1)] = cmul(vb[k], w);
            }
        }
        __syncwarp();
        const int hcol = lane >> 4, k1 = lane & 15;
        float2 y[32];
        {
            const float2 *tr = Ta + hcol * 512 + k1 * 32;
#pragma unroll
            for (int l = 0; l < 32; ++l) y[l] = tr[l ^ k1];
        }
        fft_reg_dif_c<32, true>(y);             // y[k] = x at t = k1 + 16 bitrev5(k)
        const int col = cola + hcol * HC;
        if (col < cols) {
            const int slot = slot_base + sl;
            const int j1 = pair_j[2 * p], j2 = pair_j[2 * p + 1];
            float *o1 = gq + (((size_t)slot * c.nch + j1) * cols + col) * c.bt + k1;
            float *o2 = gq + (((size_t)slot * c.nch + (j2 >= 0 ? j2 : j1)) * cols + (cols - 1 - col)) * c.bt + k1;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int t = k1 + 16 * bitrev<32>(k);
                if (t < c.bt) {
                    o1[16 * bitrev<32>(k)] = y[k].x;
                    if (j2 >= 0) o2[16 * bitrev<32>(k)] = y[k].y;
                }
            }
        }
    }
    acp_wait<0>();
}

// ------------------------------------------------------------------ chain rule
struct ChainConst {
    int ns, bp, bt, ngx, ngy, nt, nbx, nbt, wx, wt, wstride, nch, gl;
    int ngy_e;                     // sub-cells of one event along y
    float xi[MAX_GL], wl[MAX_GL];
};

// value, d/dmu and d/dsigma of one GL weight (window fixed)
__device__ void weight_gl3(int g, int cell, float frac, float sig, int lo, int hi, const ChainConst &c,
                           float &e, float &dm, float &ds) {
    const float inv_sig = 1.0f / sig;
    const float norm = 0.3989422804014327f * inv_sig;
    e = dm = ds = 0.f;
#pragma unroll
    for (int dc = -1; dc <= 1; ++dc) {
        const int C = g + dc;
        if (C < lo || C > hi) continue;
        const float base = (float)(C - cell);
        for (int l = 0; l < c.gl; ++l) {
            const float s = 0.5f * c.xi[l];
            float u;
            if (dc == 0) u = 1.f - fabsf(s);
            else if (dc == -1) u = s > 0.f ? s : 0.f;
            else u = s < 0.f ? -s : 0.f;
            if (u == 0.f) continue;
            const float dist = base + (s - frac);           // node - mu
            const float zz = dist * inv_sig;
            const float ph = norm * expf(-0.5f * zz * zz);
            const float wgt = 0.5f * c.wl[l] * u;
            e = fmaf(wgt, ph, e);
            dm = fmaf(wgt, ph * dist * inv_sig * inv_sig, dm);
            ds = fmaf(wgt, ph * (zz * zz - 1.f) * inv_sig, ds);
        }
    }
}

// weights and derivatives per deposit: wts2[d][3][2 wx + wt] (value, d/dmu, d/dsigma)
__global__ void __launch_bounds__(256) k_adj_weights(int n, tred_deposits d, ChainConst c,
                                                     float *__restrict__ wts2) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int lo[3] = {d.lo_x[i], d.lo_y[i], d.lo_t[i]};
    const int hi[3] = {d.hi_x[i], d.hi_y[i], d.hi_t[i]};
    if (lo[0] > hi[0]) return;
    const int cell[3] = {d.cell_x[i], d.cell_y[i], d.cell_t[i]};
    const float frac[3] = {d.frac_x[i], d.frac_y[i], d.frac_t[i]};
    const float sig[3] = {d.sigma_x[i], d.sigma_y[i], d.sigma_t[i]};
    float *w = wts2 + (size_t)i * 3 * c.wstride;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int cap = ax < 2 ? c.wx : c.wt;
        const int off = ax == 0 ? 0 : ax == 1 ? c.wx : 2 * c.wx;
        const int len = min(hi[ax] - lo[ax] + 3, cap);
        for (int k = lane; k < len; k += 32) {
            float e, dm, ds;
            weight_gl3(lo[ax] - 1 + k, cell[ax], frac[ax], sig[ax], lo[ax], hi[ax], c, e, dm, ds);
            w[off + k] = e;
            w[c.wstride + off + k] = dm;
            w[2 * c.wstride + off + k] = ds;
        }
    }
}

// One warp per (block, deposit) pair of the CSR.  The lanes run along time (W
// consecutive ticks, W the window's length rounded up to a power of two, at most 32)
// and over 32 / W columns at once, so each load of dL/dQeff covers whole sectors; per
// pixel-row gy the sums over the row's columns are kept apart and multiplied by the
// row's y factors once:
//   s = sum_gy fy(gy) sum_gx fx(gx) sum_t dL/dQeff(gx, gy, t) ft(t)
// for the seven combinations of value and derivative factors.
constexpr int CH_MAX_SIDE = 128;   // bp * n_sub
__global__ void __launch_bounds__(256, 2) k_adj_chain(const int32_t *__restrict__ block_ids,
                                                   const int32_t *__restrict__ dep_offsets,
                                                   const int32_t *__restrict__ dep_index,
                                                   const int32_t *__restrict__ n_blocks_dev, tred_deposits d,
                                                   ChainConst c, const float *__restrict__ wts2,
                                                   const int32_t *__restrict__ dep_event,
                                                   const float *__restrict__ gq, float *__restrict__ grad7) {
    __shared__ int offx[CH_MAX_SIDE], offy[CH_MAX_SIDE];   // offsets of block-local gx and gy in a slot
    const int side = c.bp * c.ns, cols = c.bp * c.bp;
    for (int g = threadIdx.x; g < side; g += blockDim.x) {
        const int pg = g / c.ns, jg = g - pg * c.ns;
        offx[g] = (jg * cols + pg) * c.bt;                   // jx, px
        offy[g] = (jg * c.ns * cols + pg * c.bp) * c.bt;     // jy, py
    }
    __syncthreads();
    const int nb = n_blocks_dev[0];
    if (nb <= 0) return;
    const int total = dep_offsets[nb];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < total; k += nwarps) {
        // slot of CSR entry k: binary search in dep_offsets
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (dep_offsets[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        const int slot = lo;
        const int i = dep_index[k];
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int X0 = bx * side, Y0 = by * side, T0 = bt * c.bt;
        const int lox = d.lo_x[i], hix = d.hi_x[i], loy = d.lo_y[i], hiy = d.hi_y[i];
        const int lot = d.lo_t[i], hit = d.hi_t[i];
        const int xa = max(max(lox - 1, 0), X0), xb = min(min(hix + 1, c.ngx - 1), X0 + side - 1);
        const int ev = dep_event[i];
        const int ya = max(max(loy - 1, ev * c.ngy_e), Y0), yb = min(min(hiy + 1, (ev + 1) * c.ngy_e - 1), Y0 + side - 1);
        const int ta = max(max(lot - 1, 0), T0), tb = min(min(hit + 1, c.nt - 1), T0 + c.bt - 1);
        if (xa > xb || ya > yb || ta > tb) continue;
        const float *w = wts2 + (size_t)i * 3 * c.wstride;
        const float *ex = w, *ey = w + c.wx, *et = w + 2 * c.wx;
        const float *gblk = gq + (size_t)slot * c.nch * cols * c.bt - T0;
        const int ntw = tb - ta + 1, ncol = (xb - xa + 1) * (yb - ya + 1);
        // W = 2^lw lanes along time: the width with the fewest lane passes over the
        // window, ceil(ntw / W) time chunks times ceil(ncol W / 32) column groups
        int lw = 2, best = 1 << 30;
        for (int l = 2; l <= 5; ++l) {
            const int passes = ((ntw + (1 << l) - 1) >> l) * (((ncol << l) + 31) >> 5);
            if (passes < best) best = passes, lw = l;
        }
        const int W = 1 << lw, tl = lane & (W - 1), cl = lane >> lw, cpg = 32 >> lw;
        float s[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int t0 = ta; t0 <= tb; t0 += W) {
            const int t = t0 + tl;
            const bool tok = t <= tb;
            const int gi = t - (lot - 1);
            const float e0 = tok ? et[gi] : 0.f, e1 = tok ? et[c.wstride + gi] : 0.f, e2 = tok ? et[2 * c.wstride + gi] : 0.f;
            for (int gy = ya; gy <= yb; ++gy) {
                const float *grow = gblk + offy[gy - Y0] + t;
                float r0 = 0.f, r1 = 0.f, r2 = 0.f, rb = 0.f, rc = 0.f;
#pragma unroll 4
                for (int gx = xa + cl; gx <= xb; gx += cpg) {
                    const float gv = tok ? grow[offx[gx - X0]] : 0.f;
                    const float A = gv * e0, B = gv * e1, C = gv * e2;
                    const int ix = gx - (lox - 1);
                    const float vx = ex[ix], dmx = ex[c.wstride + ix], dsx = ex[2 * c.wstride + ix];
                    r0 = fmaf(vx, A, r0);
                    r1 = fmaf(dmx, A, r1);
                    r2 = fmaf(dsx, A, r2);
                    rb = fmaf(vx, B, rb);
                    rc = fmaf(vx, C, rc);
                }
                const int iy = gy - (loy - 1);
                const float vy = ey[iy], dmy = ey[c.wstride + iy], dsy = ey[2 * c.wstride + iy];
                s[0] = fmaf(vy, r0, s[0]);
                s[1] = fmaf(vy, r1, s[1]);
                s[2] = fmaf(dmy, r0, s[2]);
                s[3] = fmaf(vy, rb, s[3]);
                s[4] = fmaf(vy, r2, s[4]);
                s[5] = fmaf(dsy, r0, s[5]);
                s[6] = fmaf(vy, rc, s[6]);
            }
        }
#pragma unroll
        for (int q = 0; q < 7; ++q)
#pragma unroll
            for (int o = 16; o; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
        if (lane == 0) {
            const float q = d.q[i];
            atomicAdd(&grad7[(size_t)i * 7 + 0], s[0]);
#pragma unroll
            for (int qq = 1; qq < 7; ++qq) atomicAdd(&grad7[(size_t)i * 7 + qq], q * s[qq]);
        }
    }
}

struct ParamConst {
    double v, tick, h, tau, s0, s0t, DT, DL;
};

__global__ void __launch_bounds__(256) k_adj_params(int n, const float *__restrict__ z, tred_deposits d,
                                                    ParamConst c, const float *__restrict__ grad7,
                                                    float *__restrict__ gin, double *__restrict__ gglob) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0, e = 0.0;
    if (i < n) {
        const float *g = grad7 + (size_t)i * 7;
        float *o = gin + (size_t)i * 4;
        if (d.lo_x[i] > d.hi_x[i]) {
            o[0] = o[1] = o[2] = o[3] = 0.f;
        } else {
            const double td = (double)z[i] / c.v;
            o[0] = (float)(g[1] / c.h);
            o[1] = (float)(g[2] / c.h);
            o[2] = (float)(g[3] / c.tick);
            o[3] = (float)(g[0] * exp(-td / c.tau));
            e = (double)g[0] * d.q[i] * td / (c.tau * c.tau);
            b = ((double)g[4] + g[5]) * 1e-6 * td / (c.h * c.h * d.sigma_x[i]);
            a = (double)g[6] * 1e-6 * td / (c.v * c.tick * c.v * c.tick * d.sigma_t[i]);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&gglob[0], a);
        atomicAdd(&gglob[1], b);
        atomicAdd(&gglob[2], e);
    }
}

// ------------------------------------------------------------------ launchers
int launch_residual(tred_handle *h, const int32_t *pix, const int32_t *n_pix_dev, const float *wave,
                    const int32_t *tpix, int n_target, const float *twave, float *resid, double *loss,
                    cudaStream_t s) {
    int rc = check_cuda(h, cudaMemsetAsync(loss, 0, sizeof(double), s), "clear loss");
    if (rc) return rc;
    k_resid<<<num_sms(h) * 8, 256, 0, s>>>(pix, n_pix_dev, wave, tpix, n_target, twave, h->g.nt, resid, loss);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "residual launch");
}

template <int G>
static int run_adjoint_conv(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                            const float *resid, float *gq, const AdjConst &c, cudaStream_t s) {
    static bool attr = false;
    const size_t itime_smem = adj_itime_smem<G>();
    if (!attr) {
        cudaFuncSetAttribute(k_adj_spec<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ADJ_SPEC_SMEM);
        cudaFuncSetAttribute(k_adj_itime<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)itime_smem);
        if constexpr (G == 8)
            cudaFuncSetAttribute(k_adj_itime512, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)adj_itime512_smem());
        attr = true;
    }
    const int sms = num_sms(h);
    const int chunk = h->adj_chunk;
    // the item queue counter: a word after the effective charge's per-CTA scratch
    int32_t *queue = h->effq_acc + (effq_scratch_bytes(h->g.bp * h->g.n_sub, sms) / sizeof(int32_t) - 16);
    for (int base = 0; base < h->max_blocks; base += chunk) {
        int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "adjoint queue reset");
        if (rc) return rc;
        k_adj_spec<G><<<sms, AS_THREADS, ADJ_SPEC_SMEM, s>>>(n_blocks_dev, block_ids, resid, h->pix_row, h->tw,
                                                             h->rhat, c, h->gspec, base, chunk, queue);
        if constexpr (G == 8)
            k_adj_itime512<<<sms, AIT5_THREADS, adj_itime512_smem(), s>>>(n_blocks_dev, h->gspec, h->pair_j, h->tw,
                                                                          c, gq, base, chunk);
        else
            k_adj_itime<G><<<sms, 32 * adj_itime_cols<G>(), itime_smem, s>>>(n_blocks_dev, h->gspec, h->pair_j,
                                                                             h->tw, c, gq, base, chunk);
        h->launches += 2;
    }
    return check_cuda(h, cudaGetLastError(), "adjoint convolution launch");
}

int launch_adjoint(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                   const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                   const int32_t *pixel_ids, const int32_t *n_pixels_dev, const float *resid, float *gq,
                   float *grad7, cudaStream_t s) {
    const int64_t npx = (int64_t)h->g.npx_x * h->d.npy;
    int rc = check_cuda(h, cudaMemsetAsync(h->pix_row, 0xff, sizeof(int32_t) * npx, s), "clear rows");
    if (!rc) rc = check_cuda(h, cudaMemsetAsync(grad7, 0, sizeof(float) * 7 * (size_t)n, s), "clear grads");
    if (rc) return rc;
    const int sms = num_sms(h);
    k_row_map<<<sms * 2, 256, 0, s>>>(pixel_ids, n_pixels_dev, h->pix_row);
    h->launches += 1;
    AdjConst c{h->g.n_sub, h->g.bp, h->g.bt, h->g.nr, h->g.nt, h->g.n_sub * h->g.n_sub, h->d.npairs, h->d.R,
               h->p.mpcp, h->d.nbx, h->d.nbt, h->g.npx_x, h->d.npy, h->d.npy_e, h->d.nby_e};
    if (h->d.G == 8) rc = run_adjoint_conv<8>(h, block_ids, n_blocks_dev, resid, gq, c, s);
    else if (h->d.G == 16) rc = run_adjoint_conv<16>(h, block_ids, n_blocks_dev, resid, gq, c, s);
    else rc = set_error(h, TRED_ERR_INVALID_ARG, "adjoint: unsupported lt");
    if (rc) return rc;
    ChainConst cc;
    cc.ns = h->g.n_sub;
    cc.bp = h->g.bp;
    cc.bt = h->g.bt;
    cc.ngx = h->d.ngx;
    cc.ngy = h->d.ngy;
    cc.nt = h->g.nt;
    cc.nbx = h->d.nbx;
    cc.nbt = h->d.nbt;
    cc.wx = h->d.wx;
    cc.wt = h->d.wt;
    cc.wstride = h->d.wstride;
    cc.nch = h->g.n_sub * h->g.n_sub;
    cc.gl = h->p.gl_order;
    cc.ngy_e = h->d.ngy_e;
    for (int l = 0; l < MAX_GL; ++l) {
        cc.xi[l] = l < cc.gl ? h->gl_xi[l] : 0.f;
        cc.wl[l] = l < cc.gl ? h->gl_wi[l] : 0.f;
    }
    if (n > 0) {
        k_adj_weights<<<(unsigned)(((int64_t)n * 32 + 255) / 256), 256, 0, s>>>(n, deps, cc, h->wts2);
        k_adj_chain<<<sms * 16, 256, 0, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, deps, cc, h->wts2,
                                             h->dep_event, gq, grad7);
        h->launches += 2;
    }
    return check_cuda(h, cudaGetLastError(), "adjoint launch");
}

int launch_param_grads(tred_handle *h, int n, const float *z, const tred_deposits &deps, const float *grad7,
                       float *gin, double *gglob, cudaStream_t s) {
    int rc = check_cuda(h, cudaMemsetAsync(gglob, 0, 3 * sizeof(double), s), "clear global grads");
    if (rc) return rc;
    if (n == 0) return TRED_OK;
    ParamConst c{(double)h->p.v_cm_per_us, (double)h->g.tick_us, h->d.h, (double)h->p.lifetime_us,
                 (double)h->p.sigma0_cells_xy, (double)h->p.sigma0_ticks, (double)h->p.DT_cm2_per_s,
                 (double)h->p.DL_cm2_per_s};
    k_adj_params<<<(n + 255) / 256, 256, 0, s>>>(n, z, deps, c, grad7, gin, gglob);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "parameter gradient launch");
}

}  // namespace tred
