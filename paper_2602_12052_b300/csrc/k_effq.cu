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
#include "effq_item.cuh"

namespace tred {

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
    // the three vectors as one index range over the lanes (x, then y, then t), so that
    // the short x and y vectors do not leave most of a pass's lanes idle
    const int lx = min(hi[0] - lo[0] + 3, c.wx), ly = min(hi[1] - lo[1] + 3, c.wx);
    const int lt = min(hi[2] - lo[2] + 3, c.wt);
    for (int k = lane; k < lx + ly + lt; k += 32) {
        const int ax = k < lx ? 0 : k < lx + ly ? 1 : 2;
        const int kk = k - (ax == 0 ? 0 : ax == 1 ? lx : lx + ly);
        const int cl = ax == 0 ? cell[0] : ax == 1 ? cell[1] : cell[2];
        const float fr = ax == 0 ? frac[0] : ax == 1 ? frac[1] : frac[2];
        const float sg = ax == 0 ? sig[0] : ax == 1 ? sig[1] : sig[2];
        const int l0 = ax == 0 ? lo[0] : ax == 1 ? lo[1] : lo[2], h0 = ax == 0 ? hi[0] : ax == 1 ? hi[1] : hi[2];
        const int g = l0 - 1 + kk;
        w[(ax == 0 ? 0 : ax == 1 ? c.wx : 2 * c.wx) + kk] =
            GL == 0 ? weight_tent(g, cl, fr, sg, l0, h0) : weight_gl<GL>(g, cl, fr, sg, l0, h0, c);
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
    const int tid = threadIdx.x;
    float *scratch = reinterpret_cast<float *>(acc_scratch) + (size_t)blockIdx.x * side * side * EQ_TT;
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
        __syncthreads();
        const int item = S.slot;
        if (item >= nloc * groups) break;
        const int slot = slot_base + item / groups, grp = item - (item / groups) * groups;
        const int tt_beg = grp * tg * EQ_TT, tt_end = min(c.bt, (grp + 1) * tg * EQ_TT);
        effq_block_item<EQ_WARPS>(S, c, slot, tt_beg, tt_end, block_ids, dep_offsets, dep_index, wts, recs,
                                  qeff + (size_t)(slot - slot_base) * nch * cols * c.bt,   // the caller's buffer row
                                  colmask + (size_t)slot * nch, scratch);
    }
}

size_t effq_scratch_bytes(int side, int sms) {
    return sizeof(int32_t) * ((size_t)sms * EQ_CTAS_PER_SM * side * side * EQ_TT + 64);
}

EffqConst effq_const_of(const tred_handle *h) {
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
    return c;
}

int launch_effq_weights(tred_handle *h, int n, const tred_deposits &deps, cudaStream_t s) {
    if (n <= 0) return TRED_OK;
    const EffqConst c = effq_const_of(h);
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
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "effq weights launch");
}

int effq_check_shape(tred_handle *h) {
    const EffqConst c = effq_const_of(h);
    const int nch = c.ns * c.ns;
    const int side = c.bp * c.ns;
    const int len_cap = c.wx < side ? c.wx : side;
    if ((size_t)h->max_deposits * (size_t)c.wstride >= ((size_t)1 << 32))
        return set_error(h, TRED_ERR_INVALID_ARG, "effq: %d deposits x %d weights exceed 32-bit offsets",
                         h->max_deposits, c.wstride);
    if (side > EQ_MAX_SIDE || nch > 128 || 2 * len_cap > EQ_POOL)
        return set_error(h, TRED_ERR_INVALID_ARG, "effq: bp * n_sub = %d sub-cells (weight length %d) exceeds the tile kernel",
                         side, c.wx);
    return TRED_OK;
}

int launch_effq(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                float *qeff, int slot_base, int slot_count, cudaStream_t s) {
    const EffqConst c = effq_const_of(h);
    int rc = effq_check_shape(h);
    if (rc) return rc;
    if (n > 0 && slot_base == 0) {   // once per pass: the range starting at slot 0 computes the weights
        rc = launch_effq_weights(h, n, deps, s);
        if (rc) return rc;
    }
    const int nch = c.ns * c.ns;
    const int side = c.bp * c.ns;
    const size_t smem = sizeof(EffqShared);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_effq_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    // the block queue counter lives after the per-CTA scratch
    const int sms = num_sms(h);
    int32_t *queue = h->effq_acc + (size_t)sms * EQ_CTAS_PER_SM * side * side * EQ_TT;
    rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "effq queue reset");
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
    kt_begin(h, TRED_KT_EFFQ, s);
    k_effq_blocks<<<sms * EQ_CTAS_PER_SM, EQ_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, h->wts,
                                                 reinterpret_cast<const DepRec *>(h->recs), qeff, h->colmask,
                                                 h->effq_acc, queue, slot_base, slot_count);
    kt_end(h, TRED_KT_EFFQ, s);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "effq launch");
}

}  // namespace tred
