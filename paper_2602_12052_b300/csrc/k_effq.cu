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
//   k_effq_blocks   CTAs take active blocks from a queue; 32-tick tiles of the
//                   block's sub-cell plane accumulated in registers per 8 x 4 patch
//                   from the tile's deposit list, in the list's fixed order; plus the
//                   mask of non-empty (py, px) columns per channel
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
    int skip_empty;                // write only the columns some deposit's support covers
    float xi[MAX_GL], wl[MAX_GL];
};

// Gaussian density at node offset d (grid units) for width sig.
__device__ __forceinline__ float gauss(float d, float inv_sig, float norm) {
    const float u = d * inv_sig;
    return norm * expf(-0.5f * u * u);
}

// GL weight of grid point g for a deposit with mean cell + frac and width sig, for
// an order-GL rule (compile-time, so the nodes and weights stay in registers).
template <int GL>
__device__ float weight_gl(int g, int cell, float frac, float sig, int lo, int hi, const EffqConst &c) {
    const float inv_sig = 1.0f / sig;
    const float norm = 0.3989422804014327f * inv_sig;   // 1 / (sqrt(2 pi) sig)
    float e = 0.f;
#pragma unroll
    for (int dc = -1; dc <= 1; ++dc) {
        const int C = g + dc;
        if (C < lo || C > hi) continue;
        const float base = (float)(C - cell);
#pragma unroll
        for (int l = 0; l < GL; ++l) {
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

// GL = 0: exact-tent weights; otherwise the order-GL rule.
template <int GL>
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
            wa[k] = GL == 0 ? weight_tent(g, cell[ax], frac[ax], sig[ax], lo[ax], hi[ax])
                            : weight_gl<GL>(g, cell[ax], frac[ax], sig[ax], lo[ax], hi[ax], c);
        }
    }
}

// Effective charge of the active blocks: CTAs take blocks from a queue; per block,
// 32-tick tiles with the accumulation in registers.
//
// The block's sub-cell plane is cut into 8 x 4 patches (gx x gy); a lane owns one
// sub-cell of a patch with that cell's 32 ticks in registers, and the warps of the
// CTA take patches one by one.  Per tile the CTA lists, in shared memory, the deposits
// whose support meets the tile (clipped ranges, charge, the tile's 32 time weights,
// and the clipped x and y weight vectors copied into a pool).  A warp walks the list
// 32 entries at a time, keeps (ballot) the ones that reach its patch and adds
// q e_x e_y e_t of each to its cells with one FP32 FMA per tick (a zero factor outside
// the entry's support).  No cell is written by two threads: no atomics and no
// shared-memory tile; each lane writes its 32 ticks as four 32-byte sectors of the
// [jy][jx][py][px][t] layout.
//
// The order of every sum is fixed: the deposits of a block come sorted by index
// (tred_blockbin), the tile list keeps that order and each patch takes its deposits
// in list order, so Q^eff is bitwise reproducible.
//
// A tile whose list would exceed the shared-memory capacities (entries, pool) is
// processed in passes, each a contiguous run of the block's deposit list chosen by a
// block-wide scan; the partial sums of the cells are kept in a per-CTA global scratch
// between passes.
constexpr int EQ_TT = 32;
constexpr int EQ_WARPS = 8;
constexpr int EQ_THREADS = EQ_WARPS * 32;
constexpr int EQ_CTAS_PER_SM = 2;
constexpr int EQ_LIST = 256;                 // tile-list entries per pass
constexpr int EQ_POOL = 8192;                // weight-pool floats per pass
constexpr int EQ_PX = 8, EQ_PY = 4;          // patch: 8 gx x 4 gy sub-cells
constexpr int EQ_MAX_SIDE = 128;             // bp * n_sub
constexpr int EQ_MAX_PATCH = (EQ_MAX_SIDE / EQ_PX) * (EQ_MAX_SIDE / EQ_PY);

struct TileEnt {
    int y0, y1, x0, x1;          // block-local clipped ranges
    int q, wxo, wyo, wmax;       // charge (float bits); pool offsets of the x and y weights; largest
                                 // time weight of the tile (float bits)
    float wt[EQ_TT];             // time weights of the tile's ticks, zero outside the support
};
static_assert(sizeof(TileEnt) == 32 + 4 * EQ_TT, "tile list entry");

struct EffqShared {
    TileEnt list[EQ_LIST];
    int2 wsrc[EQ_LIST];                  // per entry: offsets of its clipped x and y weights in wts
    float pool[EQ_POOL];
    int wl[EQ_WARPS][32];                // per warp: the list entries of its patch in one 32-entry chunk
    uint32_t nzp[EQ_MAX_PATCH];          // per patch: cells that are non-zero in some tile
    int offx[EQ_MAX_SIDE], offy[EQ_MAX_SIDE];   // output offsets of block-local gx and gy
    unsigned long long mask[128];        // per channel: non-empty (py, px) columns (n_sub^2 <= 128)
    uint32_t cov[EQ_MAX_SIDE * EQ_MAX_SIDE / 32];   // sub-cell columns covered by a support
    uint8_t pcov[EQ_MAX_PATCH];                       // patch has a covered column
    uint16_t alist[EQ_MAX_PATCH];                     // the patches written at all, in order
    int nactive;
    unsigned long long part[EQ_WARPS * 3];
    int tot[4];                          // list entries, pool floats
    int slot, next;
    float flush;                         // contributions below this are left out
};

// two CTAs per SM: 228 KB of shared memory per SM, 1 KB reserved per CTA
static_assert(2 * (sizeof(EffqShared) + 1024) <= 233472, "effq shared memory must leave room for two CTAs per SM");

__global__ void __launch_bounds__(EQ_THREADS, EQ_CTAS_PER_SM) k_effq_blocks(
    const int32_t *__restrict__ block_ids, const int32_t *__restrict__ dep_offsets,
    const int32_t *__restrict__ dep_index, const int32_t *__restrict__ n_blocks_dev, EffqConst c,
    const float *__restrict__ wts, const DepRec *__restrict__ recs, float *__restrict__ qeff,
    uint64_t *__restrict__ colmask, int32_t *__restrict__ acc_scratch, int32_t *__restrict__ queue,
    int slot_base, int slot_count) {
    extern __shared__ __align__(16) unsigned char smem_e[];
    EffqShared &S = *reinterpret_cast<EffqShared *>(smem_e);
    const int nch = c.ns * c.ns;
    const int cols = c.bp * c.bp;
    const int side = c.bp * c.ns;
    const int npx = (side + EQ_PX - 1) / EQ_PX;
    const int npatch = npx * ((side + EQ_PY - 1) / EQ_PY);
    const int len_cap = min(c.wx, side);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lx = lane & (EQ_PX - 1), ly = lane >> 3;   // the lane's cell of a patch
    float *scratch = reinterpret_cast<float *>(acc_scratch) + (size_t)blockIdx.x * side * side * EQ_TT;
    for (int g = tid; g < side; g += EQ_THREADS) {
        const int pg = g / c.ns, jg = g - pg * c.ns;
        S.offx[g] = (jg * cols + pg) * c.bt;                   // jx, px
        S.offy[g] = (jg * c.ns * cols + pg * c.bp) * c.bt;     // jy, py
    }
    const int nb = min(n_blocks_dev[0], slot_base + slot_count);
    const int nloc = max(0, nb - slot_base);
    // An item is a run of tg of the block's 32-tick tiles: the whole block while there are
    // enough blocks to keep every CTA busy, fewer tiles when a small event has few blocks,
    // so that its blocks spread over more CTAs (every CTA derives the same tg from nb)
    const int ntiles = c.bt / EQ_TT;
    int tg = ntiles;
    while (tg > 1 && (long long)nloc * ((ntiles + tg - 1) / tg) < 2ll * gridDim.x) tg = (tg + 1) / 2;
    const int groups = (ntiles + tg - 1) / tg;
    for (;;) {
        __syncthreads();
        if (tid == 0) S.slot = atomicAdd(queue, 1);   // item index
        for (int k = tid; k < nch; k += EQ_THREADS) S.mask[k] = 0ull;
        for (int k = tid; k < npatch; k += EQ_THREADS) S.nzp[k] = 0u;
        __syncthreads();
        const int item = S.slot;
        if (item >= nloc * groups) break;
        const int slot = slot_base + item / groups, grp = item - (item / groups) * groups;
        const int tt_beg = grp * tg * EQ_TT, tt_end = min(c.bt, (grp + 1) * tg * EQ_TT);
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int X0 = bx * side, Y0 = by * side, T0 = bt * c.bt;
        float *qblk = qeff + (size_t)(slot - slot_base) * nch * cols * c.bt;   // the caller's buffer row
        const int beg = dep_offsets[slot], end = dep_offsets[slot + 1];
        // flush level: 2^-23 of the largest single contribution inside the block (|q| times
        // each axis' largest weight within the block); a deposit's contribution to a cell
        // that stays below it over a whole tile is under the FP32 resolution of the block's
        // sums and is left out, so that columns holding only such tails stay empty for the
        // convolution
        {
            float pm = 0.f;
            for (int k = beg + tid; k < end; k += EQ_THREADS) {
                const DepRec r = recs[dep_index[k]];
                const int xa = max(r.x0, X0), xb = min(r.x1, X0 + side - 1);
                const int ya = max(r.y0, Y0), yb = min(r.y1, Y0 + side - 1);
                const int ta = max(r.t0, T0), tb = min(r.t1, T0 + c.bt - 1);
                if (xa > xb || ya > yb || ta > tb) continue;
                const float *w = wts + (size_t)r.idx * c.wstride;
                float mx = 0.f, my = 0.f, mt = 0.f;
                for (int g = xa; g <= xb; ++g) mx = fmaxf(mx, fabsf(__ldg(w + (g - r.gx0))));
                for (int g = ya; g <= yb; ++g) my = fmaxf(my, fabsf(__ldg(w + c.wx + (g - r.gy0))));
                for (int g = ta; g <= tb; ++g) mt = fmaxf(mt, fabsf(__ldg(w + 2 * c.wx + (g - r.gt0))));
                pm = fmaxf(pm, fabsf(r.q) * mx * my * mt);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, o));
            float *pw = reinterpret_cast<float *>(S.part);
            if (lane == 0) pw[warp] = pm;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < EQ_WARPS; ++k) pm = fmaxf(pm, pw[k]);
            if (tid == 0) S.flush = pm * 1.1920928955078125e-7f;   // 2^-23 (read after later barriers)
        }
        if (c.skip_empty) {
            // columns (gy, gx) covered by some deposit's clipped support: the others stay
            // zero in every tile and are not written
            for (int k = tid; k < (side * side + 31) / 32; k += EQ_THREADS) S.cov[k] = 0u;
            __syncthreads();
            for (int k = beg + tid; k < end; k += EQ_THREADS) {
                const DepRec r = recs[dep_index[k]];
                const int xa = max(r.x0, X0) - X0, xb = min(r.x1, X0 + side - 1) - X0;
                const int ya = max(r.y0, Y0) - Y0, yb = min(r.y1, Y0 + side - 1) - Y0;
                for (int gy = ya; gy <= yb; ++gy) {
                    const int b0 = gy * side + xa, b1 = gy * side + xb;
                    for (int wd = b0 >> 5; wd <= (b1 >> 5); ++wd) {
                        const int lo = max(b0, wd << 5) & 31, hi = min(b1, (wd << 5) + 31) & 31;
                        const uint32_t m = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
                        atomicOr(&S.cov[wd], m);
                    }
                }
            }
            __syncthreads();
            for (int pt = tid; pt < npatch; pt += EQ_THREADS) {
                const int qy = pt / npx, qx = pt - qy * npx;
                int any = 0;
                for (int r = 0; r < EQ_PY; ++r) {
                    const int gy = qy * EQ_PY + r;
                    for (int cx = 0; cx < EQ_PX && gy < side; ++cx) {
                        const int gx = qx * EQ_PX + cx;
                        if (gx < side) {
                            const int cb = gy * side + gx;
                            any |= (S.cov[cb >> 5] >> (cb & 31)) & 1u;
                        }
                    }
                }
                S.pcov[pt] = (uint8_t)any;
            }
            __syncthreads();
        }
        // the patches written at all (every patch, or those with a covered column): the
        // warps of each tile take only these
        if (warp == 0) {
            int na = 0;
            for (int b0 = 0; b0 < npatch; b0 += 32) {
                const int pt = b0 + lane;
                const bool act = pt < npatch && (!c.skip_empty || S.pcov[pt]);
                const unsigned bal = __ballot_sync(0xffffffffu, act);
                if (act) S.alist[na + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)pt;
                na += __popc(bal);
            }
            if (lane == 0) S.nactive = na;
        }
        __syncthreads();
        for (int tt = tt_beg; tt < tt_end; tt += EQ_TT) {
            const int ta = T0 + tt, tb = ta + EQ_TT - 1;   // absolute ticks of the tile
            int cur = beg;
            bool first = true;
            do {   // one pass: a contiguous run [cur, ...) of the block's deposit list
                __syncthreads();                           // the previous pass is consumed
                if (tid < 2) S.tot[tid] = 0;
                if (tid == 0) S.next = 0;
                __syncthreads();
                bool full = false;
                while (cur < end && !full) {
                    // (1) evaluate one chunk of the list: overlap and pool floats
                    const int k = cur + tid;
                    DepRec r;
                    int xa = 0, xb = -1, ya = 0, yb = -1, cnt = 0, pl = 0;
                    if (k < end) {
                        r = recs[dep_index[k]];
                        if (!(r.t1 < ta || r.t0 > tb)) {
                            // clipped ranges, at most len_cap long (the weight capacity bounds
                            // every accepted support; the cap keeps the indexes in range anyway)
                            xa = max(r.x0, X0) - X0;
                            xb = min(min(r.x1, X0 + side - 1) - X0, xa + len_cap - 1);
                            ya = max(r.y0, Y0) - Y0;
                            yb = min(min(r.y1, Y0 + side - 1) - Y0, ya + len_cap - 1);
                            if (xa <= xb && ya <= yb) {
                                cnt = 1;
                                pl = (xb - xa + 1) + (yb - ya + 1);
                            }
                        }
                    }
                    // block-wide inclusive scan of (cnt, pl)
                    int c1 = cnt, c2 = pl;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u1 = __shfl_up_sync(0xffffffffu, c1, o);
                        const int u2 = __shfl_up_sync(0xffffffffu, c2, o);
                        if (lane >= o) { c1 += u1; c2 += u2; }
                    }
                    int *wp = reinterpret_cast<int *>(S.part);   // [EQ_WARPS][2]
                    if (lane == 31) { wp[2 * warp] = c1; wp[2 * warp + 1] = c2; }
                    __syncthreads();
                    for (int w2 = 0; w2 < warp; ++w2) { c1 += wp[2 * w2]; c2 += wp[2 * w2 + 1]; }
                    const int b1 = S.tot[0], b2 = S.tot[1];
                    const bool fits = (b1 + c1 <= EQ_LIST) && (b2 + c2 <= EQ_POOL);
                    const int acc_n = __syncthreads_count(fits);   // prefix: the totals only grow
                    if (fits && cnt) {
                        const int pos = b1 + c1 - 1, po = b2 + c2 - pl;
                        const size_t base = (size_t)r.idx * c.wstride;
                        TileEnt en;
                        en.y0 = ya;
                        en.y1 = yb;
                        en.x0 = xa;
                        en.x1 = xb;
                        en.q = __float_as_int(r.q);
                        en.wxo = po;
                        en.wyo = po + (xb - xa + 1);
                        S.wsrc[pos] = make_int2((int)(base + (X0 + xa - r.gx0)), (int)(base + c.wx + (Y0 + ya - r.gy0)));
                        float wm = 0.f;
#pragma unroll
                        for (int e = 0; e < EQ_TT; ++e) {
                            const int t = ta + e;
                            en.wt[e] = (t >= r.t0 && t <= r.t1) ? __ldg(wts + base + 2 * c.wx + (t - r.gt0)) : 0.f;
                            wm = fmaxf(wm, fabsf(en.wt[e]));
                        }
                        en.wmax = __float_as_int(wm);
                        int4 *dst = reinterpret_cast<int4 *>(&S.list[pos]);
                        const int4 *src = reinterpret_cast<const int4 *>(&en);
#pragma unroll
                        for (int q = 0; q < (int)(sizeof(TileEnt) / 16); ++q) dst[q] = src[q];
                    }
                    if (tid == acc_n - 1) { S.tot[0] = b1 + c1; S.tot[1] = b2 + c2; }
                    __syncthreads();
                    cur += acc_n;
                    full = acc_n < EQ_THREADS;             // chunk cut short: capacity reached
                }
                const int ne = S.tot[0];
                const bool last = cur >= end;
                // (2) the clipped x and y weight vectors of the entries, two entries' loads in
                // flight per warp (their source offsets were kept when the entries were made)
                for (int k0 = warp; k0 < ne; k0 += 2 * EQ_WARPS) {
                    float vx[2], vy[2];
                    int ox[2], oy[2], nxs[2], nys[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int k = k0 + u * EQ_WARPS;
                        nxs[u] = nys[u] = 0;
                        vx[u] = vy[u] = 0.f;
                        if (k < ne) {
                            const int4 hy = *reinterpret_cast<const int4 *>(&S.list[k].y0);   // y0 y1 x0 x1
                            const int2 src = S.wsrc[k];
                            nxs[u] = hy.w - hy.z + 1;
                            nys[u] = hy.y - hy.x + 1;
                            ox[u] = S.list[k].wxo;
                            oy[u] = S.list[k].wyo;
                            if (lane < nxs[u]) vx[u] = __ldg(wts + (size_t)(unsigned)src.x + lane);
                            if (lane < nys[u]) vy[u] = __ldg(wts + (size_t)(unsigned)src.y + lane);
                            for (int q = lane + 32; q < nxs[u]; q += 32) S.pool[ox[u] + q] = __ldg(wts + (size_t)(unsigned)src.x + q);
                            for (int q = lane + 32; q < nys[u]; q += 32) S.pool[oy[u] + q] = __ldg(wts + (size_t)(unsigned)src.y + q);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (lane < nxs[u]) S.pool[ox[u] + lane] = vx[u];
                        if (lane < nys[u]) S.pool[oy[u] + lane] = vy[u];
                    }
                }
                __syncthreads();
                // (3) patches, taken one by one by the warps from the list of written patches
                const int nact = S.nactive;
                const float flush = S.flush;
                int *wl = S.wl[warp];
                for (;;) {
                    int pi = 0;
                    if (lane == 0) pi = atomicAdd(&S.next, 1);
                    pi = __shfl_sync(0xffffffffu, pi, 0);
                    if (pi >= nact) break;
                    const int pt = S.alist[pi];
                    const int qy = pt / npx, qx = pt - qy * npx;
                    const int px0 = qx * EQ_PX, py0 = qy * EQ_PY;
                    const int gx = px0 + lx, gy = py0 + ly;
                    const bool own = gx < side && gy < side;
                    float *sc = scratch + ((size_t)gy * side + gx) * EQ_TT;
                    float acc[EQ_TT];
                    if (first || !own) {
#pragma unroll
                        for (int e = 0; e < EQ_TT; ++e) acc[e] = 0.f;
                    } else {
#pragma unroll
                        for (int e4 = 0; e4 < EQ_TT; e4 += 4) {
                            const float4 u = reinterpret_cast<const float4 *>(sc)[e4 / 4];
                            acc[e4] = u.x; acc[e4 + 1] = u.y; acc[e4 + 2] = u.z; acc[e4 + 3] = u.w;
                        }
                    }
                    // the tile list in order, 32 entries at a time: the ones that reach the
                    // patch, then each of them added to the lane's cell (zero outside its support)
                    for (int c0 = 0; c0 < ne; c0 += 32) {
                        const int k = c0 + lane;
                        bool ov = false;
                        if (k < ne) {
                            const int4 hy = *reinterpret_cast<const int4 *>(&S.list[k].y0);   // y0 y1 x0 x1
                            ov = hy.z <= px0 + EQ_PX - 1 && hy.w >= px0 && hy.x <= py0 + EQ_PY - 1 && hy.y >= py0;
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, ov);
                        if (!bal) continue;
                        if (ov) wl[__popc(bal & ((1u << lane) - 1u))] = k;
                        __syncwarp();
                        const int cnt = __popc(bal);
                        for (int s = 0; s < cnt; ++s) {
                            const TileEnt &en = S.list[wl[s]];
                            const int4 hy = *reinterpret_cast<const int4 *>(&en.y0);   // y0 y1 x0 x1
                            const int4 hq = *reinterpret_cast<const int4 *>(&en.q);    // q wxo wyo wmax
                            const bool in = gx >= hy.z && gx <= hy.w && gy >= hy.x && gy <= hy.y;
                            const float wx = S.pool[in ? hq.y + gx - hy.z : 0], wy = S.pool[in ? hq.z + gy - hy.x : 0];
                            const float a0 = __int_as_float(hq.x) * wx * wy;
                            // a contribution that stays below the flush level at every tick of the
                            // tile is under the FP32 resolution of the block's sums: left out
                            const float a = (in && fabsf(a0) * __int_as_float(hq.w) >= flush) ? a0 : 0.f;
#pragma unroll
                            for (int e4 = 0; e4 < EQ_TT; e4 += 4) {
                                const float4 w = *reinterpret_cast<const float4 *>(&en.wt[e4]);
                                acc[e4] = fmaf(a, w.x, acc[e4]);
                                acc[e4 + 1] = fmaf(a, w.y, acc[e4 + 1]);
                                acc[e4 + 2] = fmaf(a, w.z, acc[e4 + 2]);
                                acc[e4 + 3] = fmaf(a, w.w, acc[e4 + 3]);
                            }
                        }
                        __syncwarp();                          // wl is rewritten by the next chunk
                    }
                    if (!last) {
                        if (own) {
#pragma unroll
                            for (int e4 = 0; e4 < EQ_TT; e4 += 4)
                                reinterpret_cast<float4 *>(sc)[e4 / 4] = make_float4(acc[e4], acc[e4 + 1], acc[e4 + 2], acc[e4 + 3]);
                        }
                        continue;
                    }
                    bool any = false;
#pragma unroll
                    for (int e = 0; e < EQ_TT; ++e) any |= acc[e] != 0.f;
                    const uint32_t bal = __ballot_sync(0xffffffffu, own && any);
                    if (lane == 0 && bal) S.nzp[pt] |= bal;       // this warp alone holds patch pt now
                    const int cb = gy * side + gx;
                    if (own && (!c.skip_empty || ((S.cov[cb >> 5] >> (cb & 31)) & 1u))) {
                        float4 *dst = reinterpret_cast<float4 *>(qblk + S.offy[gy] + S.offx[gx] + tt);
#pragma unroll
                        for (int e4 = 0; e4 < EQ_TT; e4 += 4) dst[e4 / 4] = make_float4(acc[e4], acc[e4 + 1], acc[e4 + 2], acc[e4 + 3]);
                    }
                }
                first = false;
            } while (cur < end);
        }
        __syncthreads();
        for (int pt = warp; pt < npatch; pt += EQ_WARPS) {
            if (!((S.nzp[pt] >> lane) & 1u)) continue;
            const int qy = pt / npx, qx = pt - qy * npx;
            const int gx = qx * EQ_PX + lx, gy = qy * EQ_PY + ly;
            const int py = gy / c.ns, jy = gy - py * c.ns, px = gx / c.ns, jx = gx - px * c.ns;
            atomicOr(&S.mask[jy * c.ns + jx], 1ull << (py * c.bp + px));
        }
        __syncthreads();
        // the block's items each add their columns (the launch cleared the masks)
        for (int k = tid; k < nch; k += EQ_THREADS)
            if (S.mask[k]) atomicOr(reinterpret_cast<unsigned long long *>(&colmask[(size_t)slot * nch + k]), S.mask[k]);
    }
}

size_t effq_scratch_bytes(int side, int sms) {
    return sizeof(int32_t) * ((size_t)sms * EQ_CTAS_PER_SM * side * side * EQ_TT + 64);
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
    c.skip_empty = h->p.effq_skip_empty;
    for (int l = 0; l < MAX_GL; ++l) {
        c.xi[l] = l < c.gl ? h->gl_xi[l] : 0.f;
        c.wl[l] = l < c.gl ? h->gl_wi[l] : 0.f;
    }
    if (n > 0 && slot_base == 0) {   // once per pass: the range starting at slot 0 computes the weights
        const int threads = 256;
        const int64_t blocks = ((int64_t)n * 32 + threads - 1) / threads;
        auto go = [&](auto kern) {
            kern<<<(unsigned)blocks, threads, 0, s>>>(n, deps, c, h->dep_event, h->wts, reinterpret_cast<DepRec *>(h->recs));
        };
        switch (c.mode == 1 ? 0 : c.gl) {
        case 0: go(k_effq_weights<0>); break;
        case 1: go(k_effq_weights<1>); break;
        case 2: go(k_effq_weights<2>); break;
        case 3: go(k_effq_weights<3>); break;
        case 4: go(k_effq_weights<4>); break;
        case 5: go(k_effq_weights<5>); break;
        case 6: go(k_effq_weights<6>); break;
        case 7: go(k_effq_weights<7>); break;
        default: go(k_effq_weights<8>); break;
        }
    }
    const int nch = c.ns * c.ns;
    const int side = c.bp * c.ns;
    const int len_cap = c.wx < side ? c.wx : side;
    if ((size_t)h->max_deposits * (size_t)c.wstride >= ((size_t)1 << 32))
        return set_error(h, TRED_ERR_INVALID_ARG, "effq: %d deposits x %d weights exceed 32-bit offsets",
                         h->max_deposits, c.wstride);
    if (side > EQ_MAX_SIDE || nch > 128 || 2 * len_cap > EQ_POOL)
        return set_error(h, TRED_ERR_INVALID_ARG, "effq: bp * n_sub = %d sub-cells (weight length %d) exceeds the tile kernel",
                         side, c.wx);
    const size_t smem = sizeof(EffqShared);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_effq_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    // the block queue counter lives after the per-CTA scratch
    const int sms = num_sms(h);
    int32_t *queue = h->effq_acc + (size_t)sms * EQ_CTAS_PER_SM * side * side * EQ_TT;
    int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "effq queue reset");
    if (rc) return rc;
    {
        // the non-empty column masks of the slots this call covers are OR-ed by its items
        const int hi = slot_count < h->max_blocks - slot_base ? slot_base + slot_count : h->max_blocks;
        if (hi > slot_base) {
            rc = check_cuda(h, cudaMemsetAsync(h->colmask + (size_t)slot_base * nch, 0,
                                               sizeof(uint64_t) * (size_t)(hi - slot_base) * nch, s),
                            "effq mask reset");
            if (rc) return rc;
        }
    }
    k_effq_blocks<<<sms * EQ_CTAS_PER_SM, EQ_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, h->wts,
                                                 reinterpret_cast<const DepRec *>(h->recs), qeff, h->colmask,
                                                 h->effq_acc, queue, slot_base, slot_count);
    h->launches += 1 + (n > 0 && slot_base == 0 ? 1 : 0);
    return check_cuda(h, cudaGetLastError(), "effq launch");
}

}  // namespace tred
