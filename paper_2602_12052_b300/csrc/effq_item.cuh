// Shared pieces of the effective charge (a3; Sec. II-C, Eqs. trilinear, eff_q): the
// per-deposit record, the kernel constants, the shared-memory layout of the block kernel
// and one item of it (some 32-tick tiles of one active block).  k_effq.cu's block kernel
// and the persistent block pipeline (k_pipeline.cu) are built from them.
#pragma once

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

constexpr int EQ_TT = 32;
constexpr int EQ_WARPS = 8;
constexpr int EQ_THREADS = EQ_WARPS * 32;
// three CTAs per SM (80 registers, a smaller tile list and pool): 5.41 ms per module-plane
// step against 5.65 at two CTAs and 6.59 at four (64 registers, spills)
constexpr int EQ_CTAS_PER_SM = 3;
constexpr int EQ_LIST = 192;                 // tile-list entries per pass
constexpr int EQ_POOL = 6144;                // weight-pool floats per pass
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

template <int NW>
struct EffqSharedT {
    TileEnt list[EQ_LIST];
    int2 wsrc[EQ_LIST];                  // per entry: offsets of its clipped x and y weights in wts
    float pool[EQ_POOL];
    int wl[NW][32];                // per warp: the list entries of its patch in one 32-entry chunk
    uint32_t nzp[EQ_MAX_PATCH];          // per patch: cells that are non-zero in some tile
    int offx[EQ_MAX_SIDE], offy[EQ_MAX_SIDE];   // output offsets of block-local gx and gy
    unsigned long long mask[128];        // per channel: non-empty (py, px) columns (n_sub^2 <= 128)
    uint32_t cov[EQ_MAX_SIDE * EQ_MAX_SIDE / 32];   // sub-cell columns covered by a support
    uint8_t pcov[EQ_MAX_PATCH];                       // patch has a covered column
    uint16_t alist[EQ_MAX_PATCH];                     // the patches written at all, in order
    int nactive;
    unsigned long long part[NW * 3];
    int tot[4];                          // list entries, pool floats
    int slot, next;
    float flush;                         // contributions below this are left out
};

using EffqShared = EffqSharedT<EQ_WARPS>;

// EQ_CTAS_PER_SM CTAs per SM: 228 KB of shared memory per SM, 1 KB reserved per CTA
static_assert(EQ_CTAS_PER_SM * (sizeof(EffqShared) + 1024) <= 233472, "effq shared memory must leave room for EQ_CTAS_PER_SM CTAs per SM");

// Barrier of the threads that run one effective-charge item: the whole CTA, or one
// group of NT threads (warps NT/32 * g ...) synchronised by named barrier `id`, so that
// two groups of a larger CTA run independent items side by side.
struct CtaSync {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int count(int pred) const { return __syncthreads_count(pred); }
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
};
template <int NT>
struct GroupSync {
    int id;   // named barrier (1..15; 0 is __syncthreads')
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NT) : "memory"); }
    __device__ __forceinline__ int count(int pred) const {
        int r;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.popc.u32 %0, %2, %3, p;\n\t}"
            : "=r"(r)
            : "r"(pred), "r"(id), "n"(NT)
            : "memory");
        return r;
    }
    __device__ __forceinline__ int tid() const { return threadIdx.x % NT; }
};

// One item of the effective charge: the 32-tick tiles at tt_beg, tt_beg + tt_step, ...
// below tt_end of the block in `slot` of the active list, written into qblk (that block's [ns][ns][bp][bp][bt] row) and
// its non-empty columns OR-ed into mrow[ns * ns].  Every one of the CTA's NW warps takes
// part; scratch is the CTA's own multi-pass buffer.
template <int NW, class Sync = CtaSync>
__device__ __forceinline__ void effq_block_item(EffqSharedT<NW> &S, const EffqConst &c, int slot, int tt_beg,
                                                int tt_end, const int32_t *__restrict__ block_ids,
                                                const int32_t *__restrict__ dep_offsets,
                                                const int32_t *__restrict__ dep_index, const float *__restrict__ wts,
                                                const DepRec *__restrict__ recs, float *__restrict__ qblk,
                                                uint64_t *__restrict__ mrow, float *__restrict__ scratch,
                                                Sync bar = Sync(), int tt_step = EQ_TT) {
    constexpr int NT = NW * 32;
    const int nch = c.ns * c.ns;
    const int cols = c.bp * c.bp;
    const int side = c.bp * c.ns;
    const int npx = (side + EQ_PX - 1) / EQ_PX;
    const int npatch = npx * ((side + EQ_PY - 1) / EQ_PY);
    const int len_cap = min(c.wx, side);
    const int tid = bar.tid(), warp = tid >> 5, lane = tid & 31;
    const int lx = lane & (EQ_PX - 1), ly = lane >> 3;   // the lane's cell of a patch
    bar.sync();                                           // the shared state is free
    for (int g = tid; g < side; g += NT) {
        const int pg = g / c.ns, jg = g - pg * c.ns;
        S.offx[g] = (jg * cols + pg) * c.bt;                   // jx, px
        S.offy[g] = (jg * c.ns * cols + pg * c.bp) * c.bt;     // jy, py
    }
    for (int k = tid; k < nch; k += NT) S.mask[k] = 0ull;
    for (int k = tid; k < npatch; k += NT) S.nzp[k] = 0u;
    bar.sync();
    const int blk = block_ids[slot];
    const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
    const int X0 = bx * side, Y0 = by * side, T0 = bt * c.bt;
        const int beg = dep_offsets[slot], end = dep_offsets[slot + 1];
    // flush level: 2^-23 of the largest single contribution inside the block (|q| times
    // each axis' largest weight within the block); a deposit's contribution to a cell
    // that stays below it over a whole tile is under the FP32 resolution of the block's
    // sums and is left out, so that columns holding only such tails stay empty for the
    // convolution
    {
        float pm = 0.f;
        for (int k = beg + tid; k < end; k += NT) {
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
        bar.sync();
#pragma unroll
        for (int k = 0; k < NW; ++k) pm = fmaxf(pm, pw[k]);
        if (tid == 0) S.flush = pm * 1.1920928955078125e-7f;   // 2^-23 (read after later barriers)
    }
    if (c.skip_empty) {
        // columns (gy, gx) covered by some deposit's clipped support: the others stay
        // zero in every tile and are not written
        for (int k = tid; k < (side * side + 31) / 32; k += NT) S.cov[k] = 0u;
        bar.sync();
        for (int k = beg + tid; k < end; k += NT) {
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
        bar.sync();
        for (int pt = tid; pt < npatch; pt += NT) {
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
        bar.sync();
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
    bar.sync();
    for (int tt = tt_beg; tt < tt_end; tt += tt_step) {
        const int ta = T0 + tt, tb = ta + EQ_TT - 1;   // absolute ticks of the tile
        int cur = beg;
        bool first = true;
        do {   // one pass: a contiguous run [cur, ...) of the block's deposit list
            bar.sync();                           // the previous pass is consumed
            if (tid < 2) S.tot[tid] = 0;
            if (tid == 0) S.next = 0;
            bar.sync();
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
                int *wp = reinterpret_cast<int *>(S.part);   // [NW][2]
                if (lane == 31) { wp[2 * warp] = c1; wp[2 * warp + 1] = c2; }
                bar.sync();
                for (int w2 = 0; w2 < warp; ++w2) { c1 += wp[2 * w2]; c2 += wp[2 * w2 + 1]; }
                const int b1 = S.tot[0], b2 = S.tot[1];
                const bool fits = (b1 + c1 <= EQ_LIST) && (b2 + c2 <= EQ_POOL);
                const int acc_n = bar.count(fits);   // prefix: the totals only grow
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
                bar.sync();
                cur += acc_n;
                full = acc_n < NT;             // chunk cut short: capacity reached
            }
            const int ne = S.tot[0];
            const bool last = cur >= end;
            // (2) the clipped x and y weight vectors of the entries, two entries' loads in
            // flight per warp (their source offsets were kept when the entries were made)
            for (int k0 = warp; k0 < ne; k0 += 2 * NW) {
                float vx[2], vy[2];
                int ox[2], oy[2], nxs[2], nys[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = k0 + u * NW;
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
            bar.sync();
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
    bar.sync();
    for (int pt = warp; pt < npatch; pt += NW) {
        if (!((S.nzp[pt] >> lane) & 1u)) continue;
        const int qy = pt / npx, qx = pt - qy * npx;
        const int gx = qx * EQ_PX + lx, gy = qy * EQ_PY + ly;
        const int py = gy / c.ns, jy = gy - py * c.ns, px = gx / c.ns, jx = gx - px * c.ns;
        atomicOr(&S.mask[jy * c.ns + jx], 1ull << (py * c.bp + px));
    }
    bar.sync();
    // the block's items each add their columns
    for (int k = tid; k < nch; k += NT)
        if (S.mask[k]) atomicOr(reinterpret_cast<unsigned long long *>(&mrow[k]), S.mask[k]);
}

// the kernel constants of a handle; the per-deposit weights launch (k_effq_weights, once
// per pass before any block item); the shape checks of the block kernel
EffqConst effq_const_of(const tred_handle *h);
int launch_effq_weights(tred_handle *h, int n, const tred_deposits &deps, cudaStream_t s);
int effq_check_shape(tred_handle *h);

}  // namespace tred
