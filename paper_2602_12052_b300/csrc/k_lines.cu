// Line-shape track segments (Sec. II-C, "Calculation of Q for a line-shape track
// segment", Eq. qline, and the short-segment limit).
//
//   k_drift_lines   transport of both endpoints (the point drift's binary64 sequence);
//                   one width per axis at the midpoint's drift time, attachment at
//                   the midpoint, window [floor(min end - n_s s), ceil(max end + n_s s)]
//                   per axis; the midpoint is split exactly into cell + fraction and
//                   the half vector (p1 - p0) / 2 is kept in grid units.
//   k_effq_lines    Eq. eff_q with the node charge Q rho(node) w_l w_m w_n / 8, where rho
//                   is the diffused line density
//                     rho = exp(-gperp / 2)
//                           (erf((alpha - beta) / sqrt(2 alpha)) + erf(beta / sqrt(2 alpha)))
//                           / (4 pi Delta),
//                   gperp = gamma - beta^2 / alpha = sum (a_i - (beta / alpha) d_i)^2 / s_i^2
//                   (the weighted squared distance to the line, summed as squares so that
//                   long segments lose nothing to cancellation),
//                   alpha = sum d_i^2 / s_i^2, beta = sum a_i d_i / s_i^2,
//                   gamma = sum a_i^2 / s_i^2, d = p1 - p0, a = node - p0,
//                   Delta = s_x s_y s_z sqrt(alpha) (Eq. qline with the factor 1/2 in
//                   the exponent that the isotropic limit requires); segments shorter
//                   than 0.1 sigma on every axis use the point Gaussian at the midpoint.
//                   CTAs take active blocks from a queue and add the block's segments
//                   one after another: the density is evaluated once per quadrature
//                   node (with the time interpolation folded into a 16-tick profile
//                   per x-y node pair), then each sub-cell column adds the profiles
//                   of the node pairs that interpolate to it (per axis: its own
//                   cell's nodes and the neighbouring cells' nodes on its side).
//                   FP32 sums in a fixed order for a given segment list.
#include "tred_internal.cuh"

namespace tred {

struct LineDriftConst {
    double v, tick, h, width_x, width_y, DT, DL, s0, s0t, ns, tau, max_td;
};

__global__ void __launch_bounds__(256) k_drift_lines(int n, const float *__restrict__ x0, const float *__restrict__ y0,
                                                     const float *__restrict__ z0, const float *__restrict__ x1,
                                                     const float *__restrict__ y1, const float *__restrict__ z1,
                                                     const float *__restrict__ t0, const float *__restrict__ ne,
                                                     LineDriftConst c, tred_deposits out, float *__restrict__ half,
                                                     int32_t *__restrict__ dep_event, int32_t *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xa = x0[i], ya = y0[i], za = z0[i], xb = x1[i], yb = y1[i], zb = z1[i];
    const double t0d = t0[i], ned = ne[i];
    dep_event[i] = 0;
    const bool ok = isfinite(xa) && isfinite(ya) && isfinite(za) && isfinite(xb) && isfinite(yb) && isfinite(zb) &&
                    isfinite(t0d) && isfinite(ned) && za >= 0.0 && zb >= 0.0 && ned >= 0.0 && xa >= 0.0 &&
                    xa < c.width_x && ya >= 0.0 && ya < c.width_y && xb >= 0.0 && xb < c.width_x && yb >= 0.0 &&
                    yb < c.width_y;
    const double tda = __ddiv_rn(za, c.v), tdb = __ddiv_rn(zb, c.v);
    if (!ok || !(tda <= c.max_td) || !(tdb <= c.max_td)) {
        if (ok) atomicOr(&status[0], TRED_ST_DRIFT_RANGE);
        atomicAdd(&status[1], 1);
        out.cell_x[i] = out.cell_y[i] = out.cell_t[i] = 0;
        out.frac_x[i] = out.frac_y[i] = out.frac_t[i] = 0.f;
        out.sigma_x[i] = out.sigma_y[i] = out.sigma_t[i] = 1.f;
        out.lo_x[i] = out.lo_y[i] = out.lo_t[i] = 0;
        out.hi_x[i] = out.hi_y[i] = out.hi_t[i] = -1;
        out.q[i] = 0.f;
        half[i] = half[n + i] = half[2 * n + i] = 0.f;
        return;
    }
    const double p0[3] = {__dadd_rn(__ddiv_rn(xa, c.h), -0.5), __dadd_rn(__ddiv_rn(ya, c.h), -0.5),
                          __ddiv_rn(__dadd_rn(t0d, tda), c.tick)};
    const double p1[3] = {__dadd_rn(__ddiv_rn(xb, c.h), -0.5), __dadd_rn(__ddiv_rn(yb, c.h), -0.5),
                          __ddiv_rn(__dadd_rn(t0d, tdb), c.tick)};
    double zm = __dadd_rn(za, zb);
    zm = __dmul_rn(zm, 0.5);
    const double td = __ddiv_rn(zm, c.v);
    double a = __dmul_rn(c.DT, 2.0);
    a = __dmul_rn(a, 1e-6);
    a = __dmul_rn(a, td);
    double b = __dmul_rn(c.h, c.h);
    a = __ddiv_rn(a, b);
    double cc = __dmul_rn(c.s0, c.s0);
    const double sxy = __dsqrt_rn(__dadd_rn(a, cc));
    a = __dmul_rn(c.DL, 2.0);
    a = __dmul_rn(a, 1e-6);
    a = __dmul_rn(a, td);
    b = __dmul_rn(c.v, c.tick);
    b = __dmul_rn(b, b);
    a = __ddiv_rn(a, b);
    cc = __dmul_rn(c.s0t, c.s0t);
    const double st = __dsqrt_rn(__dadd_rn(a, cc));
    const double sg[3] = {sxy, sxy, st};
    int32_t *cell[3] = {out.cell_x, out.cell_y, out.cell_t};
    float *frac[3] = {out.frac_x, out.frac_y, out.frac_t};
    float *sig[3] = {out.sigma_x, out.sigma_y, out.sigma_t};
    int32_t *lo[3] = {out.lo_x, out.lo_y, out.lo_t};
    int32_t *hi[3] = {out.hi_x, out.hi_y, out.hi_t};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const double K = __dmul_rn(c.ns, sg[ax]);
        const double mid = __dmul_rn(0.5, __dadd_rn(p0[ax], p1[ax]));
        const double fl = floor(mid);
        const double mn = p0[ax] < p1[ax] ? p0[ax] : p1[ax];
        const double mx = p0[ax] < p1[ax] ? p1[ax] : p0[ax];
        cell[ax][i] = (int32_t)fl;
        frac[ax][i] = (float)(mid - fl);
        sig[ax][i] = (float)sg[ax];
        lo[ax][i] = (int32_t)floor(__dadd_rn(mn, -K));
        hi[ax][i] = (int32_t)ceil(__dadd_rn(mx, K));
        half[(size_t)ax * n + i] = (float)(0.5 * (p1[ax] - p0[ax]));
    }
    out.q[i] = (float)(ned * exp(-td / c.tau));
}

int launch_drift_lines(tred_handle *h, int n, const float *x0, const float *y0, const float *z0, const float *x1,
                       const float *y1, const float *z1, const float *t0, const float *ne, const tred_deposits &out,
                       float *half, cudaStream_t s) {
    LineDriftConst c;
    c.v = (double)h->p.v_cm_per_us;
    c.tick = (double)h->g.tick_us;
    c.h = h->d.h;
    c.width_x = (double)h->g.npx_x * (double)h->g.pitch_cm;
    c.width_y = (double)h->g.npx_y * (double)h->g.pitch_cm;
    c.DT = (double)h->p.DT_cm2_per_s;
    c.DL = (double)h->p.DL_cm2_per_s;
    c.s0 = (double)h->p.sigma0_cells_xy;
    c.s0t = (double)h->p.sigma0_ticks;
    c.ns = (double)h->p.nsigma;
    c.tau = (double)h->p.lifetime_us;
    c.max_td = (double)h->p.max_drift_cm / (double)h->p.v_cm_per_us;
    if (n > 0)
        k_drift_lines<<<(n + 255) / 256, 256, 0, s>>>(n, x0, y0, z0, x1, y1, z1, t0, ne, c, out, half, h->dep_event,
                                                     h->status);
    h->launches += n > 0 ? 1 : 0;
    return check_cuda(h, cudaGetLastError(), "k_drift_lines launch");
}

// ---------------------------------------------------------------- effective charge
constexpr int LN_THREADS = 256;
constexpr int LN_TC = 16;                 // ticks per time chunk
constexpr int LN_NODES = 32;              // quadrature nodes per axis per x-y chunk
constexpr int LN_CAP = 64;                // segment records staged per pass
constexpr float LN_SHORT = 0.1f;          // short-segment switch, in sigma per axis
constexpr int LN_MAX_SIDE = 128;          // bp * n_sub

struct LineConst {
    int ns, bp, bt, nbx, nbt, skip_empty;
    float xi[4], wl[4];
};

struct LineRec {
    int lo[3], hi[3], cell[3];
    float m[3];                           // midpoint - cell
    float hv[3];                          // (p1 - p0) / 2
    float isg2[3];                        // 1 / sigma^2
    float dw[3];                          // d_i / sigma_i^2
    float q, alpha, inva, rs2a, pref;
    int point;
};

struct LineShared {
    float P[LN_NODES * LN_NODES * LN_TC];          // time profiles of a chunk's node pairs
    LineRec S[LN_CAP];
    uint32_t cov[LN_MAX_SIDE * LN_MAX_SIDE / 32];  // sub-cell columns some support covers
    unsigned long long mask[128];
    int slot;
};

// density (normalised) at a node at offsets a = node - p0 (line) or node - midpoint
// (point form)
__device__ __forceinline__ float line_rho(const LineRec &s, float ax, float ay, float at) {
    if (s.point) return s.pref * __expf(-0.5f * (ax * ax * s.isg2[0] + ay * ay * s.isg2[1] + at * at * s.isg2[2]));
    const float bet = ax * s.dw[0] + ay * s.dw[1] + at * s.dw[2];
    const float lam = bet * s.inva;
    const float ex = ax - lam * 2.f * s.hv[0], ey = ay - lam * 2.f * s.hv[1], et = at - lam * 2.f * s.hv[2];
    const float gp = ex * ex * s.isg2[0] + ey * ey * s.isg2[1] + et * et * s.isg2[2];
    return s.pref * __expf(-0.5f * gp) * (erff((s.alpha - bet) * s.rs2a) + erff(bet * s.rs2a));
}

// offset of the node (cell C, rule point l) on axis ax from the segment's reference point
template <int NGL>
__device__ __forceinline__ float node_offset(const LineRec &s, int ax, int C, int l, const LineConst &c) {
    const float rel = (float)(C - s.cell[ax]) + 0.5f * c.xi[l];
    return s.point ? rel - s.m[ax] : rel - (s.m[ax] - s.hv[ax]);
}

// Eq. trilinear, one axis: the coefficient with which the node (cell C, point l) feeds
// grid point g, times w_l / 2 (zero when it does not feed g)
__device__ __forceinline__ float node_weight(int g, int C, float sl, float wl) {
    float u = 0.f;
    if (C == g) u = 1.f - fabsf(sl);
    else if (C == g - 1) u = sl > 0.f ? sl : 0.f;
    else if (C == g + 1) u = sl < 0.f ? -sl : 0.f;
    return 0.5f * wl * u;
}

// Effective charge of the active blocks for line segments.  CTAs take blocks from a
// queue.  The block's covered columns are cleared (all columns unless skip_empty),
// then the block's segments are added one after another in list order: per chunk of
// at most 32 x 32 x-y quadrature nodes and 16 ticks, phase A evaluates the density
// once per node and folds the time interpolation in (one 16-tick profile per node
// pair, in shared memory), and phase B gives each sub-cell column the node pairs
// that feed it with their x and y interpolation weights and adds the result to the
// column's 16 ticks in the output (one writer per column per phase: no atomics on
// data, a fixed order of the sums).
template <int NGL>
__global__ void __launch_bounds__(LN_THREADS) k_effq_lines(const int32_t *__restrict__ block_ids,
                                                           const int32_t *__restrict__ dep_offsets,
                                                           const int32_t *__restrict__ dep_index,
                                                           const int32_t *__restrict__ n_blocks_dev, LineConst c,
                                                           tred_deposits d, const float *__restrict__ half, int n,
                                                           float *__restrict__ qeff, uint64_t *__restrict__ colmask,
                                                           int32_t *__restrict__ queue) {
    extern __shared__ __align__(16) unsigned char smem_l[];
    LineShared &L = *reinterpret_cast<LineShared *>(smem_l);
    constexpr int CC = LN_NODES / NGL;          // cells per axis per x-y chunk
    const int nch = c.ns * c.ns, cols = c.bp * c.bp, side = c.bp * c.ns;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = n_blocks_dev[0];
    const int nwords = (side * side + 31) / 32;
    for (;;) {
        __syncthreads();
        if (tid == 0) L.slot = atomicAdd(queue, 1);
        for (int k = tid; k < nch; k += LN_THREADS) L.mask[k] = 0ull;
        for (int k = tid; k < nwords; k += LN_THREADS) L.cov[k] = c.skip_empty ? 0u : 0xffffffffu;
        __syncthreads();
        const int slot = L.slot;
        if (slot >= nb) break;
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int X0 = bx * side, Y0 = by * side, T0 = bt * c.bt;
        float *qblk = qeff + (size_t)slot * nch * cols * c.bt;
        const int beg = dep_offsets[slot], end = dep_offsets[slot + 1];
        auto column = [&](int gxl, int gyl) -> float * {
            const int py = gyl / c.ns, jy = gyl - py * c.ns, px = gxl / c.ns, jx = gxl - px * c.ns;
            return qblk + ((size_t)(jy * c.ns + jx) * cols + py * c.bp + px) * c.bt;
        };
        // covered columns: each segment's support [lo - 1, hi + 1] clipped to the block
        if (c.skip_empty) {
            for (int k = beg + tid; k < end; k += LN_THREADS) {
                const int i = dep_index[k];
                const int xa = max(d.lo_x[i] - 1, X0) - X0, xb = min(d.hi_x[i] + 1, X0 + side - 1) - X0;
                const int ya = max(d.lo_y[i] - 1, Y0) - Y0, yb = min(d.hi_y[i] + 1, Y0 + side - 1) - Y0;
                for (int gy = ya; gy <= yb; ++gy) {
                    const int b0 = gy * side + xa, b1 = gy * side + xb;
                    for (int wd = b0 >> 5; wd <= (b1 >> 5) && xa <= xb; ++wd) {
                        const int lo = max(b0, wd << 5) & 31, hi = min(b1, (wd << 5) + 31) & 31;
                        const uint32_t m = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
                        atomicOr(&L.cov[wd], m);
                    }
                }
            }
            __syncthreads();
        }
        // clear the covered columns (a warp per column)
        for (int cb = warp; cb < side * side; cb += LN_THREADS / 32) {
            if (!((L.cov[cb >> 5] >> (cb & 31)) & 1u)) continue;
            float4 *col4 = reinterpret_cast<float4 *>(column(cb % side, cb / side));
            for (int t4 = lane; t4 < c.bt / 4; t4 += 32) col4[t4] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int cb0 = beg; cb0 < end; cb0 += LN_CAP) {
            const int cnt = min(LN_CAP, end - cb0);
            __syncthreads();                     // the previous pass is consumed (and the clears done)
            for (int k = tid; k < cnt; k += LN_THREADS) {
                const int i = dep_index[cb0 + k];
                LineRec r;
                r.lo[0] = d.lo_x[i]; r.lo[1] = d.lo_y[i]; r.lo[2] = d.lo_t[i];
                r.hi[0] = d.hi_x[i]; r.hi[1] = d.hi_y[i]; r.hi[2] = d.hi_t[i];
                r.cell[0] = d.cell_x[i]; r.cell[1] = d.cell_y[i]; r.cell[2] = d.cell_t[i];
                r.m[0] = d.frac_x[i]; r.m[1] = d.frac_y[i]; r.m[2] = d.frac_t[i];
                const float sg[3] = {d.sigma_x[i], d.sigma_y[i], d.sigma_t[i]};
                r.q = d.q[i];
                bool shortseg = true;
                float alpha = 0.f;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    r.hv[ax] = half[(size_t)ax * n + i];
                    r.isg2[ax] = 1.f / (sg[ax] * sg[ax]);
                    const float dd = 2.f * r.hv[ax];
                    r.dw[ax] = dd * r.isg2[ax];
                    shortseg = shortseg && fabsf(dd) < LN_SHORT * sg[ax];
                    alpha += dd * dd * r.isg2[ax];
                }
                r.point = shortseg ? 1 : 0;
                r.alpha = alpha;
                if (shortseg) {
                    r.inva = 0.f;
                    r.rs2a = 0.f;
                    r.pref = 0.06349363593424097f / (sg[0] * sg[1] * sg[2]);   // (2 pi)^{-3/2}
                } else {
                    r.inva = 1.f / alpha;
                    r.rs2a = rsqrtf(2.f * alpha);
                    r.pref = 0.07957747154594767f / (sg[0] * sg[1] * sg[2] * sqrtf(alpha));   // 1 / (4 pi Delta)
                }
                L.S[k] = r;
            }
            __syncthreads();
            for (int k = 0; k < cnt; ++k) {
                const LineRec &s = L.S[k];
                // quadrature cells whose nodes reach the block's grid points, and the grid
                // points of the support inside the block
                const int cx0 = max(s.lo[0], X0 - 1), cx1 = min(s.hi[0], X0 + side);
                const int cy0 = max(s.lo[1], Y0 - 1), cy1 = min(s.hi[1], Y0 + side);
                const int ct0 = max(s.lo[2], T0 - 1), ct1 = min(s.hi[2], T0 + c.bt);
                const int gx0 = max(s.lo[0] - 1, X0), gx1 = min(s.hi[0] + 1, X0 + side - 1);
                const int gy0 = max(s.lo[1] - 1, Y0), gy1 = min(s.hi[1] + 1, Y0 + side - 1);
                const int gt0 = max(s.lo[2] - 1, T0), gt1 = min(s.hi[2] + 1, T0 + c.bt - 1);
                if (cx0 > cx1 || cy0 > cy1 || ct0 > ct1 || gx0 > gx1 || gy0 > gy1 || gt0 > gt1) continue;
                const float qs = s.q;
                for (int cya = cy0; cya <= cy1; cya += CC)
                    for (int cxa = cx0; cxa <= cx1; cxa += CC) {
                        const int cxb = min(cxa + CC - 1, cx1), cyb = min(cya + CC - 1, cy1);
                        const int NX = (cxb - cxa + 1) * NGL, NY = (cyb - cya + 1) * NGL;
                        // grid columns this chunk's nodes feed
                        const int fx0 = max(cxa - 1, gx0), fx1 = min(cxb + 1, gx1);
                        const int fy0 = max(cya - 1, gy0), fy1 = min(cyb + 1, gy1);
                        if (fx0 > fx1 || fy0 > fy1) continue;
                        const int ncx = fx1 - fx0 + 1, ncol = ncx * (fy1 - fy0 + 1);
                        for (int tc0 = T0 + ((gt0 - T0) / LN_TC) * LN_TC; tc0 <= gt1; tc0 += LN_TC) {
                            __syncthreads();     // the previous chunk's profiles are consumed
                            // phase A: one profile per x-y node pair over the chunk's ticks
                            const int ca = max(tc0 - 1, ct0), cb = min(tc0 + LN_TC, ct1);
                            for (int pi = tid; pi < NX * NY; pi += LN_THREADS) {
                                const int ny = pi / NX, nx = pi - ny * NX;
                                const float ax = node_offset<NGL>(s, 0, cxa + nx / NGL, nx % NGL, c);
                                const float ay = node_offset<NGL>(s, 1, cya + ny / NGL, ny % NGL, c);
                                float acc[LN_TC];
#pragma unroll
                                for (int e = 0; e < LN_TC; ++e) acc[e] = 0.f;
                                // time cells tc0 - 1 .. tc0 + 16 (those inside [ca, cb])
#pragma unroll
                                for (int kc = 0; kc < LN_TC + 2; ++kc) {
                                    const int C = tc0 - 1 + kc;
                                    if (C < ca || C > cb) continue;
                                    const int e0 = kc - 1;
#pragma unroll
                                    for (int l = 0; l < NGL; ++l) {
                                        const float sl = 0.5f * c.xi[l];
                                        const float w = qs * 0.5f * c.wl[l] * line_rho(s, ax, ay, node_offset<NGL>(s, 2, C, l, c));
                                        // own tick C (1 - |s|); the neighbour on the node's side
                                        if (e0 >= 0 && e0 < LN_TC) acc[e0] += w * (1.f - fabsf(sl));
                                        if (sl > 0.f && e0 + 1 < LN_TC) acc[e0 + 1] += w * sl;
                                        if (sl < 0.f && e0 - 1 >= 0) acc[e0 - 1] += w * (-sl);
                                    }
                                }
                                float4 *dst = reinterpret_cast<float4 *>(L.P + pi * LN_TC);
#pragma unroll
                                for (int e4 = 0; e4 < LN_TC; e4 += 4)
                                    dst[e4 / 4] = make_float4(acc[e4], acc[e4 + 1], acc[e4 + 2], acc[e4 + 3]);
                            }
                            __syncthreads();
                            // phase B: each fed column adds its node pairs' profiles
                            for (int ci = tid; ci < ncol; ci += LN_THREADS) {
                                const int gy = fy0 + ci / ncx, gx = fx0 + ci % ncx;
                                float acc[LN_TC];
#pragma unroll
                                for (int e = 0; e < LN_TC; ++e) acc[e] = 0.f;
                                for (int Cy = max(gy - 1, max(cya, s.lo[1])); Cy <= min(gy + 1, min(cyb, s.hi[1])); ++Cy)
#pragma unroll
                                    for (int ly = 0; ly < NGL; ++ly) {
                                        const float wy = node_weight(gy, Cy, 0.5f * c.xi[ly], c.wl[ly]);
                                        if (wy == 0.f) continue;
                                        const int ny = (Cy - cya) * NGL + ly;
                                        for (int Cx = max(gx - 1, max(cxa, s.lo[0])); Cx <= min(gx + 1, min(cxb, s.hi[0])); ++Cx)
#pragma unroll
                                            for (int lx = 0; lx < NGL; ++lx) {
                                                const float wx = node_weight(gx, Cx, 0.5f * c.xi[lx], c.wl[lx]);
                                                if (wx == 0.f) continue;
                                                const float wxy = wx * wy;
                                                const float4 *src = reinterpret_cast<const float4 *>(
                                                    L.P + (ny * NX + (Cx - cxa) * NGL + lx) * LN_TC);
#pragma unroll
                                                for (int e4 = 0; e4 < LN_TC; e4 += 4) {
                                                    const float4 v = src[e4 / 4];
                                                    acc[e4] += wxy * v.x;
                                                    acc[e4 + 1] += wxy * v.y;
                                                    acc[e4 + 2] += wxy * v.z;
                                                    acc[e4 + 3] += wxy * v.w;
                                                }
                                            }
                                    }
                                float4 *col4 = reinterpret_cast<float4 *>(column(gx - X0, gy - Y0) + (tc0 - T0));
#pragma unroll
                                for (int e4 = 0; e4 < LN_TC; e4 += 4) {
                                    float4 v = col4[e4 / 4];
                                    v.x += acc[e4];
                                    v.y += acc[e4 + 1];
                                    v.z += acc[e4 + 2];
                                    v.w += acc[e4 + 3];
                                    col4[e4 / 4] = v;
                                }
                            }
                        }
                    }
            }
        }
        __syncthreads();
        // non-empty columns of each channel: the covered ones
        for (int cb = tid; cb < side * side; cb += LN_THREADS) {
            if (!((L.cov[cb >> 5] >> (cb & 31)) & 1u)) continue;
            const int gyl = cb / side, gxl = cb - gyl * side;
            const int py = gyl / c.ns, jy = gyl - py * c.ns, px = gxl / c.ns, jx = gxl - px * c.ns;
            atomicOr(&L.mask[jy * c.ns + jx], 1ull << (py * c.bp + px));
        }
        __syncthreads();
        for (int k = tid; k < nch; k += LN_THREADS) colmask[(size_t)slot * nch + k] = L.mask[k];
    }
}

int launch_effq_lines(tred_handle *h, int n, const tred_deposits &deps, const float *half, const int32_t *block_ids,
                      const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev, float *qeff,
                      cudaStream_t s) {
    const int side = h->g.bp * h->g.n_sub;
    if (side > LN_MAX_SIDE || h->g.n_sub * h->g.n_sub > 128 || h->p.gl_order > 4 || h->g.bt % LN_TC)
        return set_error(h, TRED_ERR_INVALID_ARG,
                         "effq_lines: needs bp n_sub <= %d, n_sub^2 <= 128, gl_order <= 4, bt multiple of %d",
                         LN_MAX_SIDE, LN_TC);
    if (h->p.effq_mode != 0) return set_error(h, TRED_ERR_INVALID_ARG, "effq_lines: Gauss-Legendre mode only");
    LineConst c;
    c.ns = h->g.n_sub;
    c.bp = h->g.bp;
    c.bt = h->g.bt;
    c.nbx = h->d.nbx;
    c.nbt = h->d.nbt;
    c.skip_empty = h->p.effq_skip_empty;
    for (int l = 0; l < 4; ++l) {
        c.xi[l] = l < h->p.gl_order ? h->gl_xi[l] : 0.f;
        c.wl[l] = l < h->p.gl_order ? h->gl_wi[l] : 0.f;
    }
    const int sms = num_sms(h);
    // the block queue counter shares the effq scratch's reserved tail
    int32_t *queue = h->effq_acc + (effq_scratch_bytes(side, sms) / sizeof(int32_t) - 32);
    int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "effq_lines queue reset");
    if (rc) return rc;
    const size_t smem = sizeof(LineShared);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_effq_lines<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_effq_lines<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_effq_lines<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_effq_lines<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int grid = sms * 3;
    switch (h->p.gl_order) {
    case 1: k_effq_lines<1><<<grid, LN_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    case 2: k_effq_lines<2><<<grid, LN_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    case 3: k_effq_lines<3><<<grid, LN_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    default: k_effq_lines<4><<<grid, LN_THREADS, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    }
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "effq_lines launch");
}

}  // namespace tred
