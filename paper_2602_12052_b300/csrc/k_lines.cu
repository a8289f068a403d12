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
//                   CTAs take active blocks from a queue; a thread owns sub-cell
//                   columns (gx, gy) and accumulates 16-tick tiles in registers over the
//                   block's segments, each grid point summing the nodes of Eq.
//                   trilinear that interpolate to it (per axis: its own cell's nodes
//                   and the neighbouring cells' nodes on its side).  FP32 sums in the
//                   order of the block's segment list.
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
constexpr int LN_TT = 16;                 // ticks per register tile
constexpr int LN_CAP = 256;               // segments staged per pass
constexpr float LN_SHORT = 0.1f;          // short-segment switch, in sigma per axis

struct LineConst {
    int ns, bp, bt, nbx, nbt;
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

// density (normalised) at a node at offsets a = node - p0 (line) or node - midpoint
// (point form)
__device__ __forceinline__ float line_rho(const LineRec &s, float ax, float ay, float at) {
    if (s.point) return s.pref * __expf(-0.5f * (ax * ax * s.isg2[0] + ay * ay * s.isg2[1] + at * at * s.isg2[2]));
    const float bet = ax * s.dw[0] + ay * s.dw[1] + at * s.dw[2];
    const float lam = bet * s.inva;
    const float ex = ax - lam * 2.f * s.hv[0], ey = ay - lam * 2.f * s.hv[1], et = at - lam * 2.f * s.hv[2];
    const float gp = ex * ex * s.isg2[0] + ey * ey * s.isg2[1] + et * et * s.isg2[2];
    return s.pref * expf(-0.5f * gp) * (erff((s.alpha - bet) * s.rs2a) + erff(bet * s.rs2a));
}

template <int NGL>
__global__ void __launch_bounds__(LN_THREADS) k_effq_lines(const int32_t *__restrict__ block_ids,
                                                           const int32_t *__restrict__ dep_offsets,
                                                           const int32_t *__restrict__ dep_index,
                                                           const int32_t *__restrict__ n_blocks_dev, LineConst c,
                                                           tred_deposits d, const float *__restrict__ half, int n,
                                                           float *__restrict__ qeff, uint64_t *__restrict__ colmask,
                                                           int32_t *__restrict__ queue) {
    __shared__ LineRec S[LN_CAP];
    __shared__ unsigned long long mask[128];
    __shared__ int s_slot;
    const int nch = c.ns * c.ns, cols = c.bp * c.bp, side = c.bp * c.ns;
    const int tid = threadIdx.x;
    const int nb = n_blocks_dev[0];
    for (;;) {
        __syncthreads();
        if (tid == 0) s_slot = atomicAdd(queue, 1);
        for (int k = tid; k < nch; k += LN_THREADS) mask[k] = 0ull;
        __syncthreads();
        const int slot = s_slot;
        if (slot >= nb) break;
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int X0 = bx * side, Y0 = by * side, T0 = bt * c.bt;
        float *qblk = qeff + (size_t)slot * nch * cols * c.bt;
        const int beg = dep_offsets[slot], end = dep_offsets[slot + 1];
        uint32_t nzbits = 0u;                   // per owned column: any non-zero value
        for (int cb = beg; cb < end || cb == beg; cb += LN_CAP) {
            const int cnt = min(LN_CAP, end - cb);
            const bool first = cb == beg, last = cb + LN_CAP >= end;
            __syncthreads();
            for (int k = tid; k < cnt; k += LN_THREADS) {
                const int i = dep_index[cb + k];
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
                S[k] = r;
            }
            __syncthreads();
            int own = 0;
            for (int cell = tid; cell < side * side; cell += LN_THREADS, ++own) {
                const int gyl = cell / side, gxl = cell - gyl * side;
                const int gx = X0 + gxl, gy = Y0 + gyl;
                const int py = gyl / c.ns, jy = gyl - py * c.ns, px = gxl / c.ns, jx = gxl - px * c.ns;
                float *col = qblk + ((size_t)(jy * c.ns + jx) * cols + py * c.bp + px) * c.bt;
                for (int tt = 0; tt < c.bt; tt += LN_TT) {
                    const int ta = T0 + tt;
                    float acc[LN_TT];
                    if (first) {
#pragma unroll
                        for (int e = 0; e < LN_TT; ++e) acc[e] = 0.f;
                    } else {
#pragma unroll
                        for (int e = 0; e < LN_TT; ++e) acc[e] = col[tt + e];
                    }
                    for (int k = 0; k < cnt; ++k) {
                        const LineRec &s = S[k];
                        // support [lo - 1, hi + 1] of the segment covers (gx, gy) and the tile
                        if (gx < s.lo[0] - 1 || gx > s.hi[0] + 1 || gy < s.lo[1] - 1 || gy > s.hi[1] + 1 ||
                            ta + LN_TT - 1 < s.lo[2] - 1 || ta > s.hi[2] + 1)
                            continue;
                        // nodes of Eq. trilinear that interpolate to gx (and gy): factor (w/2) u,
                        // and their (gamma, beta) parts; the point form keeps a_i - m_i only
                        float fx[2 * NGL], axv[2 * NGL];
                        float fy[2 * NGL], ayv[2 * NGL];
                        int nxn = 0, nyn = 0;
#pragma unroll
                        for (int ax = 0; ax < 2; ++ax) {
                            const int g = ax == 0 ? gx : gy;
                            float *fv = ax == 0 ? fx : fy;
                            float *av = ax == 0 ? axv : ayv;
                            int nn = 0;
#pragma unroll
                            for (int dc = -1; dc <= 1; ++dc) {
                                const int C = g + dc;
                                if (C < s.lo[ax] || C > s.hi[ax]) continue;
#pragma unroll
                                for (int l = 0; l < NGL; ++l) {
                                    const float sl = 0.5f * c.xi[l];
                                    float u;
                                    if (dc == 0) u = 1.f - fabsf(sl);
                                    else if (dc == -1) u = sl > 0.f ? sl : 0.f;
                                    else u = sl < 0.f ? -sl : 0.f;
                                    if (u == 0.f) continue;
                                    const float rel = (float)(C - s.cell[ax]) + sl;
                                    const float aa = s.point ? rel - s.m[ax] : rel - (s.m[ax] - s.hv[ax]);
                                    fv[nn] = 0.5f * c.wl[l] * u;
                                    av[nn] = aa;
                                    ++nn;
                                }
                            }
                            if (ax == 0) nxn = nn;
                            else nyn = nn;
                        }
                        const float qs = s.q;
                        for (int ix = 0; ix < nxn; ++ix)
                            for (int iy = 0; iy < nyn; ++iy) {
                                const float fxy = qs * fx[ix] * fy[iy];
                                const float a0 = axv[ix], a1 = ayv[iy];
                                // time nodes of the cells ta - 1 .. ta + LN_TT
#pragma unroll
                                for (int kc = 0; kc < LN_TT + 2; ++kc) {
                                    const int C = ta - 1 + kc;
                                    if (C < s.lo[2] || C > s.hi[2]) continue;
#pragma unroll
                                    for (int l = 0; l < NGL; ++l) {
                                        const float sl = 0.5f * c.xi[l];
                                        const float rel = (float)(C - s.cell[2]) + sl;
                                        const float aa = s.point ? rel - s.m[2] : rel - (s.m[2] - s.hv[2]);
                                        const float rho = line_rho(s, a0, a1, aa);
                                        const float w = fxy * 0.5f * c.wl[l] * rho;
                                        // own cell: tick C (1 - |s|); neighbour on the node's side
                                        const int e0 = kc - 1;
                                        if (e0 >= 0 && e0 < LN_TT) acc[e0] += w * (1.f - fabsf(sl));
                                        if (sl > 0.f && e0 + 1 < LN_TT) acc[e0 + 1] += w * sl;
                                        if (sl < 0.f && e0 - 1 >= 0) acc[e0 - 1] += w * (-sl);
                                    }
                                }
                            }
                    }
                    int any = 0;
#pragma unroll
                    for (int e = 0; e < LN_TT; ++e) any |= acc[e] != 0.f;
                    if (last && any) nzbits |= 1u << own;
                    float4 *dst = reinterpret_cast<float4 *>(col + tt);
#pragma unroll
                    for (int e4 = 0; e4 < LN_TT; e4 += 4)
                        dst[e4 / 4] = make_float4(acc[e4], acc[e4 + 1], acc[e4 + 2], acc[e4 + 3]);
                }
            }
            if (cnt <= 0) break;
        }
        {
            int own = 0;
            for (int cell = tid; cell < side * side; cell += LN_THREADS, ++own) {
                if (!((nzbits >> own) & 1u)) continue;
                const int gyl = cell / side, gxl = cell - gyl * side;
                const int py = gyl / c.ns, jy = gyl - py * c.ns, px = gxl / c.ns, jx = gxl - px * c.ns;
                atomicOr(&mask[jy * c.ns + jx], 1ull << (py * c.bp + px));
            }
        }
        __syncthreads();
        for (int k = tid; k < nch; k += LN_THREADS) colmask[(size_t)slot * nch + k] = mask[k];
    }
}

int launch_effq_lines(tred_handle *h, int n, const tred_deposits &deps, const float *half, const int32_t *block_ids,
                      const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev, float *qeff,
                      cudaStream_t s) {
    const int side = h->g.bp * h->g.n_sub;
    if (side * side > 32 * LN_THREADS || h->g.n_sub * h->g.n_sub > 128 || h->p.gl_order > 4 || h->g.bt % LN_TT)
        return set_error(h, TRED_ERR_INVALID_ARG,
                         "effq_lines: needs (bp n_sub)^2 <= %d, n_sub^2 <= 128, gl_order <= 4, bt multiple of %d",
                         32 * LN_THREADS, LN_TT);
    if (h->p.effq_mode != 0) return set_error(h, TRED_ERR_INVALID_ARG, "effq_lines: Gauss-Legendre mode only");
    LineConst c;
    c.ns = h->g.n_sub;
    c.bp = h->g.bp;
    c.bt = h->g.bt;
    c.nbx = h->d.nbx;
    c.nbt = h->d.nbt;
    for (int l = 0; l < 4; ++l) {
        c.xi[l] = l < h->p.gl_order ? h->gl_xi[l] : 0.f;
        c.wl[l] = l < h->p.gl_order ? h->gl_wi[l] : 0.f;
    }
    const int sms = num_sms(h);
    // the block queue counter shares the effq scratch's reserved tail
    int32_t *queue = h->effq_acc + (effq_scratch_bytes(side, sms) / sizeof(int32_t) - 32);
    int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "effq_lines queue reset");
    if (rc) return rc;
    const int grid = sms * 4;
    switch (h->p.gl_order) {
    case 1: k_effq_lines<1><<<grid, LN_THREADS, 0, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    case 2: k_effq_lines<2><<<grid, LN_THREADS, 0, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    case 3: k_effq_lines<3><<<grid, LN_THREADS, 0, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    default: k_effq_lines<4><<<grid, LN_THREADS, 0, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, c, deps, half, n, qeff, h->colmask, queue); break;
    }
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "effq_lines launch");
}

}  // namespace tred
