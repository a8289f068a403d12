// a3. Effective charge (Sec. II-C; Eqs. cub, trilinear, eff_q; point-like charge).
//
// For a point deposit the charge at the quadrature nodes is a product of 1-D
// Gaussians, and the trilinear coefficients are products of 1-D linear ones, so
// Eq. (eff_q) factorises per axis:
//     e[g] = sum_{C in [lo,hi]} sum_l (w_l / 2) phi(C + s_l) u_l(g - C),  s_l = xi_l / 2,
//     u_l(0) = 1 - |s_l|,  u_l(sign s_l) = |s_l|,
//     Qeff[gx, gy, gt] = q e_x[gx] e_y[gy] e_t[gt].
// The exact-tent mode replaces the per-cell quadrature by its limit, the integral of
// the Gaussian against the hat function, evaluated in FP64 with erf/erfc so that
// differences of tail probabilities do not cancel.
//
//   k_effq_weights  one warp per deposit: the three 1-D weight vectors over the
//                   support [lo-1, hi+1], stored contiguously per deposit
//   k_effq_blocks   persistent CTAs over active blocks, 8-tick tiles of all
//                   channels x columns in shared memory; each deposit is visited once
//                   per tile it overlaps; tiles written as full 32-byte sectors; plus
//                   the mask of non-empty (py, px) columns per channel
#include "tred_internal.cuh"

namespace tred {

// Per-deposit record for the block kernel (48 bytes), written by k_effq_weights.
struct DepRec {
    int gx0, gy0, gt0;             // lo - 1 per axis: index base of the weight vectors
    int x0, x1, y0, y1, t0, t1;    // support [lo - 1, hi + 1] clipped to the grid
    float q;
    int idx;                       // deposit index (row of the weight buffer)
    int pad;
};

static_assert(sizeof(DepRec) == 48, "record size is part of the scratch layout");

struct EffqConst {
    int ns, bp, bt, ngx, ngy, nt, nbx, nbt, wx, wt, wstride, gl, mode;
    int ngy_e;                     // sub-cells of one event along y
    int cols_log2;                 // log2(bp * bp)
    float xi[MAX_GL], wl[MAX_GL];
};

// Gaussian density at node offset d (grid units) for width sig.
__device__ __forceinline__ float gauss(float d, float inv_sig, float norm) {
    const float u = d * inv_sig;
    return norm * expf(-0.5f * u * u);
}

// GL weight of grid point g (offset k = g - (lo - 1)) for a deposit with
// mean cell + frac and width sig.
__device__ float weight_gl(int g, int cell, float frac, float sig, int lo, int hi,
                           const EffqConst &c) {
    const float inv_sig = 1.0f / sig;
    const float norm = 0.3989422804014327f * inv_sig;   // 1 / (sqrt(2 pi) sig)
    float e = 0.f;
#pragma unroll
    for (int dc = -1; dc <= 1; ++dc) {
        const int C = g + dc;
        if (C < lo || C > hi) continue;
        const float base = (float)(C - cell);
        for (int l = 0; l < c.gl; ++l) {
            const float s = 0.5f * c.xi[l];
            float u;
            if (dc == 0) u = 1.f - fabsf(s);
            else if (dc == -1) u = s > 0.f ? s : 0.f;      // node of C = g-1 right of centre
            else u = s < 0.f ? -s : 0.f;                  // node of C = g+1 left of centre
            if (u == 0.f) continue;
            const float dist = base + (s - frac);
            e = fmaf(0.5f * c.wl[l] * u, gauss(dist, inv_sig, norm), e);
        }
    }
    return e;
}

// Exact tent weight in FP64: integral over [lo - 1/2, hi + 1/2] of N(x) Lambda(x - g).
__device__ double normal_mass_d(double a, double b, double mu, double sig) {
    const double k = 0.70710678118654752440 / sig;
    const double za = (a - mu) * k, zb = (b - mu) * k;
    if (za >= 0.0) return 0.5 * (erfc(za) - erfc(zb));
    if (zb <= 0.0) return 0.5 * (erfc(-zb) - erfc(-za));
    return 0.5 * (erf(zb) - erf(za));
}
__device__ double pdf_d(double x, double mu, double sig) {
    const double u = (x - mu) / sig;
    return exp(-0.5 * u * u) * (0.39894228040143267794 / sig);
}
__device__ double moment_d(double a, double b, double m, double mu, double sig) {
    if (b <= a) return 0.0;
    return (mu - m) * normal_mass_d(a, b, mu, sig) - sig * sig * (pdf_d(b, mu, sig) - pdf_d(a, mu, sig));
}
__device__ float weight_tent(int g, int cell, float frac, float sig, int lo, int hi) {
    // work relative to the cell so that large coordinates lose nothing
    const double mu = (double)frac;
    const double gg = (double)(g - cell);
    const double A = (double)(lo - cell) - 0.5, B = (double)(hi - cell) + 0.5;
    const double s = (double)sig;
    double a = fmax(gg - 1.0, A), b = fmin(gg, B);
    const double left = moment_d(a, b, gg - 1.0, mu, s);
    a = fmax(gg, A);
    b = fmin(gg + 1.0, B);
    const double right = -moment_d(a, b, gg + 1.0, mu, s);
    return (float)(left + right);
}

__global__ void __launch_bounds__(256) k_effq_weights(int n, tred_deposits d, EffqConst c,
                                                      const int32_t *__restrict__ dep_event,
                                                      float *__restrict__ wts, DepRec *__restrict__ recs) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp;
    const int lo[3] = {d.lo_x[i], d.lo_y[i], d.lo_t[i]};
    const int hi[3] = {d.hi_x[i], d.hi_y[i], d.hi_t[i]};
    const int cell[3] = {d.cell_x[i], d.cell_y[i], d.cell_t[i]};
    const float frac[3] = {d.frac_x[i], d.frac_y[i], d.frac_t[i]};
    const float sig[3] = {d.sigma_x[i], d.sigma_y[i], d.sigma_t[i]};
    float *w = wts + (size_t)i * c.wstride;
    if (lane == 0) {
        DepRec r;
        r.gx0 = lo[0] - 1;
        r.gy0 = lo[1] - 1;
        r.gt0 = lo[2] - 1;
        r.x0 = max(lo[0] - 1, 0);
        r.x1 = min(hi[0] + 1, c.ngx - 1);
        const int ev = dep_event[i];
        r.y0 = max(lo[1] - 1, ev * c.ngy_e);
        r.y1 = min(hi[1] + 1, (ev + 1) * c.ngy_e - 1);
        r.t0 = max(lo[2] - 1, 0);
        r.t1 = min(hi[2] + 1, c.nt - 1);
        r.q = d.q[i];
        r.idx = i;
        r.pad = 0;
        recs[i] = r;
    }
    if (lo[0] > hi[0]) return;   // dropped deposit: never read
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int cap = ax < 2 ? c.wx : c.wt;
        float *wa = w + (ax == 0 ? 0 : ax == 1 ? c.wx : 2 * c.wx);
        const int len = min(hi[ax] - lo[ax] + 3, cap);
        for (int k = lane; k < len; k += 32) {
            const int g = lo[ax] - 1 + k;
            wa[k] = c.mode == 1 ? weight_tent(g, cell[ax], frac[ax], sig[ax], lo[ax], hi[ax])
                                : weight_gl(g, cell[ax], frac[ax], sig[ax], lo[ax], hi[ax], c);
        }
    }
}

// Persistent CTAs over active blocks, time-tiled.  One tile holds the block's whole
// sub-cell plane for EQ_TT consecutive ticks, indexed by sub-cell ([t][gy][gx],
// (bp n_sub)^2 x 8 words = 200 KB at 80 x 80 x 8), so each deposit is visited once
// per tile it overlaps and all its sub-cells are handled in that visit: lanes over
// two rows of 16 sub-cells (banks gx and gx + 16: no conflicts), 8 tick updates per
// lane from the tile's time weights held in registers.
//
// The tile accumulates in 32-bit fixed point.  Every contribution q e_x e_y e_t is
// non-negative and at most q m_x m_y m_t, where m_a is the deposit's largest weight
// on axis a inside this block, so no cell exceeds B = sum over the block's deposits
// of q m_x m_y m_t, and the scale S = 2^30 / B keeps every sum below 2^31.  B is
// formed without depending on the order of the block's deposit list (which comes
// from atomics), integer shared-memory additions are single fire-and-forget
// reductions (the float ones are compare-and-swap loops) whose sum does not depend
// on order, so the block's effective charge is bitwise reproducible.  Rounding: at
// most 0.5 / S per contribution.
//
// The write pass converts each (channel, column) segment's 8 ticks back to float
// (one 32-byte sector of the [jy][jx][py][px][t] layout) and zeroes the tile; the
// non-empty column masks come from the data written.
constexpr int EQ_THREADS = 1024;
constexpr int EQ_TT = 8;
constexpr int EQ_CACHE = 256;      // deposit records staged per pass

__global__ void __launch_bounds__(EQ_THREADS, 1) k_effq_blocks(const int32_t *__restrict__ block_ids,
                                                            const int32_t *__restrict__ dep_offsets,
                                                            const int32_t *__restrict__ dep_index,
                                                            const int32_t *__restrict__ n_blocks_dev,
                                                            EffqConst c, const float *__restrict__ wts,
                                                            const DepRec *__restrict__ recs,
                                                            float *__restrict__ qeff,
                                                            uint64_t *__restrict__ colmask, int slot_base,
                                                            int slot_count) {
    extern __shared__ float smem_e[];
    const int nch = c.ns * c.ns;
    const int cols = c.bp * c.bp;
    const int side = c.bp * c.ns;
    const int plane = side * side;                                            // == nch * cols
    unsigned *tile = reinterpret_cast<unsigned *>(smem_e);                    // [8][side][side]
    DepRec *rc = reinterpret_cast<DepRec *>(tile + plane * EQ_TT);            // [EQ_CACHE]
    unsigned long long *mask = reinterpret_cast<unsigned long long *>(rc + EQ_CACHE);  // [nch]
    float *s_part = reinterpret_cast<float *>(mask + nch);                    // [EQ_THREADS / 32] x 8 bytes
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = EQ_THREADS / 32;
    {
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
        for (int k = tid; k < plane * (EQ_TT / 4); k += EQ_THREADS) reinterpret_cast<uint4 *>(tile)[k] = z4;
    }
    const int nb = min(n_blocks_dev[0], slot_base + slot_count);
    for (int slot = slot_base + blockIdx.x; slot < nb; slot += gridDim.x) {
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int X0 = bx * side, Y0 = by * side, T0 = bt * c.bt;
        const size_t qslot = (size_t)(slot - slot_base);   // row of the caller's qeff buffer
        const int beg = dep_offsets[slot], end = dep_offsets[slot + 1];
        const int passes = max(1, (end - beg + EQ_CACHE - 1) / EQ_CACHE);
        for (int k = tid; k < nch; k += EQ_THREADS) mask[k] = 0ull;
        // B: every deposit's largest weight product inside the block (its bound term),
        // summed order-independently: the terms' maximum M, then an integer sum of the
        // terms rounded up to multiples of M / 2^20.
        auto term = [&](int k) -> float {
            const DepRec r = recs[dep_index[k]];
            const int xa = max(r.x0, X0), xb = min(r.x1, X0 + side - 1);
            const int ya = max(r.y0, Y0), yb = min(r.y1, Y0 + side - 1);
            const int ta = max(r.t0, T0), tb = min(r.t1, T0 + c.bt - 1);
            if (xa > xb || ya > yb || ta > tb) return 0.f;
            const float *w = wts + (size_t)r.idx * c.wstride;
            float mx = 0.f, my = 0.f, mt = 0.f;
            for (int g = xa; g <= xb; ++g) mx = fmaxf(mx, __ldg(w + (g - r.gx0)));
            for (int g = ya; g <= yb; ++g) my = fmaxf(my, __ldg(w + c.wx + (g - r.gy0)));
            for (int g = ta; g <= tb; ++g) mt = fmaxf(mt, __ldg(w + 2 * c.wx + (g - r.gt0)));
            return fmaxf(r.q, 0.f) * mx * my * mt;
        };
        float tmax = 0.f;
        for (int k = beg + tid; k < end; k += EQ_THREADS) tmax = fmaxf(tmax, term(k));
#pragma unroll
        for (int o = 16; o; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        if (lane == 0) s_part[warp] = tmax;
        __syncthreads();
        float M = 0.f;
#pragma unroll 8
        for (int k = 0; k < EQ_THREADS / 32; ++k) M = fmaxf(M, s_part[k]);
        unsigned long long units = 0ull;
        if (M > 0.f) {
            const float to_units = 1048576.0f / M;
            for (int k = beg + tid; k < end; k += EQ_THREADS) units += (unsigned long long)ceilf(term(k) * to_units) + 1ull;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) units += __shfl_xor_sync(0xffffffffu, units, o);
        __syncthreads();                                     // everyone has read M
        if (lane == 0) reinterpret_cast<unsigned long long *>(s_part)[warp] = units;
        __syncthreads();
        unsigned long long usum = 0ull;
#pragma unroll 8
        for (int k = 0; k < EQ_THREADS / 32; ++k) usum += reinterpret_cast<const unsigned long long *>(s_part)[k];
        const float bound = (float)usum * (M * (1.0f / 1048576.0f)) * 1.0001f + 1e-20f;
        const float scale = 1073741824.0f / bound;          // 2^30 / B
        const float inv_scale = bound * (1.0f / 1073741824.0f);
        uint32_t nz = 0u;                       // per-lane non-empty flags of its (col, ch) segments
        for (int tt = 0; tt < c.bt; tt += EQ_TT) {
            const int ta = T0 + tt, tb = ta + EQ_TT - 1;   // absolute ticks of the tile
            for (int pass = 0; pass < passes; ++pass) {
                const int pb = beg + pass * EQ_CACHE;
                const int pn = min(EQ_CACHE, end - pb);
                if (tt == 0 || passes > 1) {
                    __syncthreads();
                    for (int k = tid; k < pn; k += EQ_THREADS) rc[k] = recs[dep_index[pb + k]];
                }
                __syncthreads();
                for (int k = warp; k < pn; k += nwarps) {
                    const int rt0 = rc[k].t0, rt1 = rc[k].t1;
                    if (rt1 < ta || rt0 > tb) continue;
                    const DepRec r = rc[k];
                    const int xa = max(r.x0, X0) - X0, xb = min(r.x1, X0 + side - 1) - X0;
                    const int ya = max(r.y0, Y0) - Y0, yb = min(r.y1, Y0 + side - 1) - Y0;
                    if (xa > xb || ya > yb) continue;
                    const float *w = wts + (size_t)r.idx * c.wstride;
                    const float *wxv = w + (X0 - r.gx0);            // indexed by block-local gx
                    const float *wyv = w + c.wx + (Y0 - r.gy0);     // indexed by block-local gy
                    float wt[EQ_TT];
#pragma unroll
                    for (int e = 0; e < EQ_TT; ++e) {
                        const int t = ta + e;
                        wt[e] = (t >= r.t0 && t <= r.t1) ? __ldg(w + 2 * c.wx + (t - r.gt0)) : 0.f;
                    }
                    const float qs = r.q * scale;
                    for (int gy = ya + (lane >> 4); gy <= yb; gy += 2) {
                        const float ay = qs * __ldg(wyv + gy);
                        for (int gx = xa + (lane & 15); gx <= xb; gx += 16) {
                            const float a = ay * __ldg(wxv + gx);
                            unsigned *cell = tile + gy * side + gx;
#pragma unroll
                            for (int e = 0; e < EQ_TT; ++e) atomicAdd(cell + e * plane, __float2uint_rn(a * wt[e]));
                        }
                    }
                }
            }
            __syncthreads();
            // write the tile (one 32-byte sector per (channel, column) segment), zero it
            int bit = 0;
            for (int col = warp; col < cols; col += nwarps) {
                const int py = col / c.bp, px = col - py * c.bp;
                for (int ch = lane; ch < nch; ch += 32, ++bit) {
                    const int jy = ch / c.ns, jx = ch - jy * c.ns;
                    unsigned *cell = tile + (py * c.ns + jy) * side + px * c.ns + jx;
                    float v[EQ_TT];
                    unsigned any = 0u;
#pragma unroll
                    for (int e = 0; e < EQ_TT; ++e) {
                        const unsigned u = cell[e * plane];
                        cell[e * plane] = 0u;
                        any |= u;
                        v[e] = (float)u * inv_scale;
                    }
                    if (any) nz |= 1u << bit;
                    float4 *dst = reinterpret_cast<float4 *>(qeff + ((qslot * nch + ch) * cols + col) * c.bt + tt);
                    dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                    dst[1] = make_float4(v[4], v[5], v[6], v[7]);
                }
            }
            __syncthreads();
        }
        {
            int bit = 0;
            for (int col = warp; col < cols; col += nwarps)
                for (int ch = lane; ch < nch; ch += 32, ++bit)
                    if ((nz >> bit) & 1u) atomicOr(&mask[ch], 1ull << col);
        }
        __syncthreads();
        for (int k = tid; k < nch; k += EQ_THREADS) colmask[(size_t)slot * nch + k] = mask[k];
        __syncthreads();
    }
}

int launch_effq(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                float *qeff, int slot_base, int slot_count, cudaStream_t s) {
    EffqConst c;
    c.ns = h->g.n_sub;
    c.bp = h->g.bp;
    c.bt = h->g.bt;
    c.ngx = h->d.ngx;
    c.ngy = h->d.ngy;
    c.ngy_e = h->d.ngy_e;
    c.nt = h->g.nt;
    c.nbx = h->d.nbx;
    c.nbt = h->d.nbt;
    c.wx = h->d.wx;
    c.wt = h->d.wt;
    c.wstride = h->d.wstride;
    c.gl = h->p.gl_order;
    c.mode = h->p.effq_mode;
    c.cols_log2 = h->g.bp == 8 ? 6 : 4;
    for (int l = 0; l < MAX_GL; ++l) {
        c.xi[l] = l < c.gl ? h->gl_xi[l] : 0.f;
        c.wl[l] = l < c.gl ? h->gl_wi[l] : 0.f;
    }
    if (n > 0 && slot_base == 0) {   // once per pass: the range starting at slot 0 computes the weights
        const int threads = 256;
        const int64_t blocks = ((int64_t)n * 32 + threads - 1) / threads;
        k_effq_weights<<<(unsigned)blocks, threads, 0, s>>>(n, deps, c, h->dep_event, h->wts,
                                                             reinterpret_cast<DepRec *>(h->recs));
    }
    const int nch = c.ns * c.ns;
    const size_t smem = sizeof(float) * (size_t)nch * c.bp * c.bp * EQ_TT + sizeof(DepRec) * EQ_CACHE +
                        sizeof(unsigned long long) * nch + sizeof(unsigned long long) * (EQ_THREADS / 32);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_effq_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_set = true;
    }
    if (smem > 227 * 1024)
        return set_error(h, TRED_ERR_INVALID_ARG, "effq: tile of n_sub^2 bp^2 x 8 ticks exceeds shared memory");
    const int grid = num_sms(h);
    k_effq_blocks<<<grid, EQ_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, h->wts,
                                                 reinterpret_cast<const DepRec *>(h->recs), qeff, h->colmask,
                                                 slot_base, slot_count);
    h->launches += 1 + (n > 0 && slot_base == 0 ? 1 : 0);
    return check_cuda(h, cudaGetLastError(), "effq launch");
}

}  // namespace tred
