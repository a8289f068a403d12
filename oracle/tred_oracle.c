/*
 * FP64 CPU oracle for the TRED hot path (arXiv 2602.12052).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and loaded by
 * tests/, by __graft_entry__.smoke() and by bench.py's cpu_baseline / reference leg.
 * The CUDA product path never links, loads or calls it, and it shares no code with
 * the CUDA path (no header, helper or table in common).
 *
 * Plain, slow, obviously correct.  Each function cites the passage it follows.
 * Compile with -O2 -ffp-contract=off (no FMA contraction): the window arithmetic
 * below is a fixed sequence of correctly rounded binary64 operations, and the CUDA
 * path evaluates the same sequence, so the integer windows (and hence the active
 * block list and its occupancy) agree bit for bit.
 *
 * Parity pins (tests/test_oracle_*.py): Gauss-Legendre polynomial exactness and
 * textbook nodes; charge conservation of the effective charge (partition of unity
 * of the linear interpolation); closed-form erf cell integrals (exact-tent mode vs
 * numerical quadrature, GL-N -> exact-tent as N grows); GL-1 == grid sampling;
 * sigma -> 0 limit giving the interpolated response at the impact position;
 * brute-force fine-grid correlation on tiny grids; translation and mirror symmetry;
 * hand-computed readout waveforms; brute-force block enumeration; finite differences
 * for the adjoint.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* All geometry and physics constants are binary32 values (as a caller would pass
 * them); the oracle promotes them exactly to binary64. */
typedef struct {
    float pitch_cm;
    int32_t n_sub;
    float tick_us;
    int32_t npx_x, npx_y, nt;
    int32_t bp, bt;
    float v_cm_per_us, DL_cm2_per_s, DT_cm2_per_s, lifetime_us;
    float sigma0_cells_xy, sigma0_ticks, nsigma;
    int32_t gl_order;
    int32_t effq_mode;   /* 0 = Gauss-Legendre, 1 = exact tent (closed-form erf) */
} orc_params;

/* Drifted deposit, all in grid units (sub-cells for x, y; ticks for t). */
typedef struct {
    double mu[3];     /* mean position: x, y in sub-cell units, t in ticks */
    double sig[3];    /* widths in the same units */
    double q;         /* electrons after attachment */
    int32_t lo[3];    /* quadrature cells [lo, hi] per axis (unclipped) */
    int32_t hi[3];
    int32_t valid;
} orc_dep;

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1, 1] (Sec. II-C: the N-point rule {xi_i, w_i}).   */
/* Newton iteration on the Legendre polynomial P_n, three-term recurrence.     */
/* Nodes returned in ascending order.                                          */
/* ------------------------------------------------------------------------- */
int orc_gl_rule(int n, double *xi, double *w)
{
    if (n < 1 || n > 64) return -1;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            if (n == 1) { p1 = x; p0 = 1.0; }
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(x), p0 = P_{n-1}(x) */
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        xi[n - 1 - i] = x;                   /* cos gives descending nodes */
        w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    if (n % 2 == 1) xi[n / 2] = 0.0;          /* exact centre node */
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Transport [A;D] (Sec. II-A; Fig. flowchart steps A and D): drift time, attachment,  */
/* diffusion width with a floor added in quadrature, and the raster window.    */
/* The window is a fixed sequence of correctly rounded binary64 operations.    */
/* ------------------------------------------------------------------------- */
void orc_drift(const orc_params *p, int n, const float *x, const float *y,
               const float *z, const float *t0, const float *ne, orc_dep *out)
{
    const double v = (double)p->v_cm_per_us;
    const double tick = (double)p->tick_us;
    const double h = (double)p->pitch_cm / (double)p->n_sub;
    const double width_x = (double)p->npx_x * (double)p->pitch_cm;
    const double width_y = (double)p->npx_y * (double)p->pitch_cm;
    const double DT = (double)p->DT_cm2_per_s, DL = (double)p->DL_cm2_per_s;
    const double s0 = (double)p->sigma0_cells_xy, s0t = (double)p->sigma0_ticks;
    const double ns = (double)p->nsigma;
    const double tau = (double)p->lifetime_us;
    for (int i = 0; i < n; ++i) {
        orc_dep *d = &out[i];
        const double xd = x[i], yd = y[i], zd = z[i], t0d = t0[i], ned = ne[i];
        int ok = isfinite(xd) && isfinite(yd) && isfinite(zd) && isfinite(t0d)
                 && isfinite(ned) && zd >= 0.0 && ned >= 0.0
                 && xd >= 0.0 && xd < width_x && yd >= 0.0 && yd < width_y;
        d->valid = ok;
        if (!ok) {
            memset(d, 0, sizeof(*d));
            for (int a = 0; a < 3; ++a) { d->lo[a] = 0; d->hi[a] = -1; }
            d->valid = 0;
            continue;
        }
        double td = zd / v;                   /* drift time (us) */
        double ta = t0d + td;                 /* arrival time at the reference plane */
        d->mu[2] = ta / tick;                 /* grid points at integer ticks */
        d->mu[0] = xd / h - 0.5;              /* grid points at sub-cell centres */
        d->mu[1] = yd / h - 0.5;
        double a = DT * 2.0;
        a = a * 1e-6;
        a = a * td;
        double b = h * h;
        a = a / b;
        double c = s0 * s0;
        double sxy = sqrt(a + c);
        a = DL * 2.0;
        a = a * 1e-6;
        a = a * td;
        b = v * tick;
        b = b * b;
        a = a / b;
        c = s0t * s0t;
        double st = sqrt(a + c);
        d->sig[0] = sxy;
        d->sig[1] = sxy;
        d->sig[2] = st;
        d->q = ned * exp(-td / tau);          /* finite electron lifetime */
        for (int ax = 0; ax < 3; ++ax) {
            double K = ns * d->sig[ax];
            d->lo[ax] = (int32_t)floor(d->mu[ax] - K);
            d->hi[ax] = (int32_t)ceil(d->mu[ax] + K);
        }
    }
}

/* Unit normal density in grid units. */
static double normal_pdf(double xx, double mu, double sig)
{
    double u = (xx - mu) / sig;
    return exp(-0.5 * u * u) / (sig * sqrt(2.0 * M_PI));
}

/* ------------------------------------------------------------------------- */
/* One-axis effective-charge weights, Gauss-Legendre form.                     */
/* Eq. (cub): quadrature inside each cell C; Eq. (trilinear): the response at a */
/* node is interpolated linearly between the centre of C and the neighbouring   */
/* centre on the node's side; Eq. (eff_q): regrouping by grid point gives       */
/*   e[g] = sum_C sum_l (w_l / 2) phi(C + s_l) u_l(g - C),  s_l = xi_l / 2,      */
/* with u_l(0) = 1 - |s_l| and u_l(sign s_l) = |s_l|.  For a point deposit the    */
/* 3-D effective charge is Q e_x[gx] e_y[gy] e_t[gt] (Sec. II-C, point-like     */
/* charge).  Output e has hi - lo + 3 entries, for g = lo - 1 .. hi + 1.         */
/* ------------------------------------------------------------------------- */
void orc_weights_gl(int nl, const double *xi, const double *wl, double mu,
                    double sig, int lo, int hi, double *e)
{
    int n = hi - lo + 3;
    for (int k = 0; k < n; ++k) e[k] = 0.0;
    for (int C = lo; C <= hi; ++C) {
        for (int l = 0; l < nl; ++l) {
            double s = 0.5 * xi[l];
            double val = 0.5 * wl[l] * normal_pdf((double)C + s, mu, sig);
            int k = C - (lo - 1);
            if (s > 0.0) {
                e[k] += val * (1.0 - s);
                e[k + 1] += val * s;
            } else if (s < 0.0) {
                e[k] += val * (1.0 + s);
                e[k - 1] += val * (-s);
            } else {
                e[k] += val;
            }
        }
    }
}

/* Normal CDF difference Phi(b) - Phi(a) for b >= a, evaluated with erfc in the
 * tails so that same-sign tails do not cancel. */
static double normal_mass(double a, double b, double mu, double sig)
{
    double za = (a - mu) / (sig * M_SQRT2), zb = (b - mu) / (sig * M_SQRT2);
    if (za >= 0.0) return 0.5 * (erfc(za) - erfc(zb));
    if (zb <= 0.0) return 0.5 * (erfc(-zb) - erfc(-za));
    return 0.5 * (erf(zb) - erf(za));
}

/* integral_a^b (x - m) N(x; mu, sig) dx = (mu - m)[Phi]_a^b - sig^2 [N]_a^b */
static double first_moment(double a, double b, double m, double mu, double sig)
{
    if (b <= a) return 0.0;
    return (mu - m) * normal_mass(a, b, mu, sig)
           - sig * sig * (normal_pdf(b, mu, sig) - normal_pdf(a, mu, sig));
}

/* ------------------------------------------------------------------------- */
/* One-axis effective-charge weights, exact-tent form: the continuum limit of   */
/* Eq. (eff_q) as the number of nodes grows.  Linear interpolation between grid */
/* points is the hat function Lambda, so                                        */
/*   e[g] = integral over [lo - 1/2, hi + 1/2] of N(x; mu, sig) Lambda(x - g) dx  */
/* in closed form with erf/erfc (cf. the erf cell integrals of Eq. (qline)).    */
/* ------------------------------------------------------------------------- */
void orc_weights_tent(double mu, double sig, int lo, int hi, double *e)
{
    double A = lo - 0.5, B = hi + 0.5;
    int n = hi - lo + 3;
    for (int k = 0; k < n; ++k) {
        double g = (double)(lo - 1 + k);
        /* left half [g-1, g]: Lambda = x - (g - 1) */
        double a = fmax(g - 1.0, A), b = fmin(g, B);
        double left = first_moment(a, b, g - 1.0, mu, sig);
        /* right half [g, g+1]: Lambda = (g + 1) - x */
        a = fmax(g, A);
        b = fmin(g + 1.0, B);
        double right = -first_moment(a, b, g + 1.0, mu, sig);
        e[k] = left + right;
    }
}

/* Weights of one deposit on one axis (dispatch on the mode). */
static void axis_weights(const orc_params *p, const double *xi, const double *wl,
                         const orc_dep *d, int ax, double *e)
{
    if (p->effq_mode == 1)
        orc_weights_tent(d->mu[ax], d->sig[ax], d->lo[ax], d->hi[ax], e);
    else
        orc_weights_gl(p->gl_order, xi, wl, d->mu[ax], d->sig[ax], d->lo[ax],
                       d->hi[ax], e);
}

/* Effective-charge support [lo - 1, hi + 1] of a deposit, clipped to the grid. */
static int support(const orc_params *p, const orc_dep *d, int ax, int *a, int *b)
{
    int n = ax == 0 ? p->npx_x * p->n_sub : ax == 1 ? p->npx_y * p->n_sub : p->nt;
    if (!d->valid) return 0;
    *a = d->lo[ax] - 1;
    *b = d->hi[ax] + 1;
    if (*a < 0) *a = 0;
    if (*b > n - 1) *b = n - 1;
    return *a <= *b;
}

/* ------------------------------------------------------------------------- */
/* Block-sparse binning (Sec. III-B-1): blocks of bp x bp pixels x bt ticks     */
/* aligned to the volume's bin boundaries; a block is active iff the clipped    */
/* support box of some deposit intersects it; its occupancy is the number of    */
/* such deposits.  Block id = (by * NBx + bx) * NBt + bt.                       */
/* counts must hold NBx*NBy*NBt entries (zeroed here).  Returns the number of   */
/* (deposit, block) incidences.                                                 */
/* ------------------------------------------------------------------------- */
long orc_block_counts(const orc_params *p, int n, const orc_dep *d, int32_t *counts)
{
    const int nbx = p->npx_x / p->bp, nby = p->npx_y / p->bp, nbt = p->nt / p->bt;
    memset(counts, 0, sizeof(int32_t) * (size_t)nbx * nby * nbt);
    long pairs = 0;
    for (int i = 0; i < n; ++i) {
        int ga[3], gb[3];
        int ok = 1;
        for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
        if (!ok) continue;
        int bx0 = (ga[0] / p->n_sub) / p->bp, bx1 = (gb[0] / p->n_sub) / p->bp;
        int by0 = (ga[1] / p->n_sub) / p->bp, by1 = (gb[1] / p->n_sub) / p->bp;
        int bt0 = ga[2] / p->bt, bt1 = gb[2] / p->bt;
        for (int by = by0; by <= by1; ++by)
            for (int bx = bx0; bx <= bx1; ++bx)
                for (int bt = bt0; bt <= bt1; ++bt) {
                    counts[((long)by * nbx + bx) * nbt + bt] += 1;
                    ++pairs;
                }
    }
    return pairs;
}

/* Deposit list of one block, ascending deposit index.  Returns the count. */
int orc_block_deposits(const orc_params *p, int n, const orc_dep *d, int32_t block,
                       int32_t *idx, int cap)
{
    const int nbx = p->npx_x / p->bp, nbt = p->nt / p->bt;
    int bt = block % nbt, bxy = block / nbt, bx = bxy % nbx, by = bxy / nbx;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int ga[3], gb[3];
        int ok = 1;
        for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
        if (!ok) continue;
        int x0 = bx * p->bp * p->n_sub, x1 = x0 + p->bp * p->n_sub - 1;
        int y0 = by * p->bp * p->n_sub, y1 = y0 + p->bp * p->n_sub - 1;
        int t0 = bt * p->bt, t1 = t0 + p->bt - 1;
        if (gb[0] < x0 || ga[0] > x1 || gb[1] < y0 || ga[1] > y1 || gb[2] < t0
            || ga[2] > t1)
            continue;
        if (m < cap) idx[m] = i;
        ++m;
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* Effective charge of the listed blocks (Eq. (eff_q), separable point form),   */
/* layout [block][jy][jx][py][px][t] with gx = (bx*bp + px)*n_sub + jx etc.     */
/* ------------------------------------------------------------------------- */
void orc_qeff_blocks(const orc_params *p, int n, const orc_dep *d, int nb,
                     const int32_t *blocks, double *qeff)
{
    const int ns = p->n_sub, bp = p->bp, btk = p->bt;
    const int nbx = p->npx_x / p->bp, nbt = p->nt / p->bt;
    const size_t per_block = (size_t)ns * ns * bp * bp * btk;
    double xi[64], wl[64];
    orc_gl_rule(p->gl_order, xi, wl);
    memset(qeff, 0, sizeof(double) * per_block * nb);
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < nb; ++b) {
        int blk = blocks[b];
        int bt = blk % nbt, bxy = blk / nbt, bx = bxy % nbx, by = bxy / nbx;
        int x0 = bx * bp * ns, y0 = by * bp * ns, t0 = bt * btk;
        double *Q = qeff + per_block * b;
        for (int i = 0; i < n; ++i) {
            int ga[3], gb[3];
            int ok = 1;
            for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
            if (!ok) continue;
            if (gb[0] < x0 || ga[0] > x0 + bp * ns - 1 || gb[1] < y0
                || ga[1] > y0 + bp * ns - 1 || gb[2] < t0 || ga[2] > t0 + btk - 1)
                continue;
            double *e[3];
            for (int ax = 0; ax < 3; ++ax) {
                e[ax] = (double *)malloc(sizeof(double) * (d[i].hi[ax] - d[i].lo[ax] + 3));
                axis_weights(p, xi, wl, &d[i], ax, e[ax]);
            }
            for (int gy = ga[1] > y0 ? ga[1] : y0; gy <= gb[1] && gy < y0 + bp * ns; ++gy)
                for (int gx = ga[0] > x0 ? ga[0] : x0; gx <= gb[0] && gx < x0 + bp * ns; ++gx) {
                    int jy = gy % ns, py = gy / ns - by * bp;
                    int jx = gx % ns, px = gx / ns - bx * bp;
                    double exy = d[i].q * e[1][gy - (d[i].lo[1] - 1)] * e[0][gx - (d[i].lo[0] - 1)];
                    double *col = Q + ((((size_t)jy * ns + jx) * bp + py) * bp + px) * btk;
                    for (int gt = ga[2] > t0 ? ga[2] : t0; gt <= gb[2] && gt < t0 + btk; ++gt)
                        col[gt - t0] += exy * e[2][gt - (d[i].lo[2] - 1)];
                }
            for (int ax = 0; ax < 3; ++ax) free(e[ax]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Induced current on listed pixels (Sec. II-D, Eq. (interlaced) before the     */
/* R = i[j, -k] relabelling):                                                   */
/*   I[P, t] = sum_j sum_K sum_tau Qeff[j, P + K, t - tau] i[j, K, tau]          */
/* a correlation over the pixel plane and a convolution along time.  The        */
/* effective charge is built locally on the sub-cells of pixels P + K,          */
/* K in [-R, R]^2, from every deposit whose support reaches them; output ticks  */
/* are [0, nt).  resp layout [Ky][Kx][jy][jx][tau], K index = K + R.            */
/* wave: [npix][nt].                                                            */
/* ------------------------------------------------------------------------- */
void orc_pixel_currents(const orc_params *p, int n, const orc_dep *d,
                        const float *resp, int kp, int nr, int npix,
                        const int32_t *pixel_ids, double *wave)
{
    const int ns = p->n_sub, R = (kp - 1) / 2;
    const int ngx = p->npx_x * ns, ngy = p->npx_y * ns, nt = p->nt;
    double xi[64], wl[64];
    orc_gl_rule(p->gl_order, xi, wl);
#pragma omp parallel for schedule(dynamic)
    for (int ip = 0; ip < npix; ++ip) {
        double *I = wave + (size_t)ip * nt;
        memset(I, 0, sizeof(double) * nt);
        int P = pixel_ids[ip];
        int Px = P % p->npx_x, Py = P / p->npx_x;
        /* source sub-cell region of pixels Px-R .. Px+R (clipped) */
        int gx0 = (Px - R) * ns, gx1 = (Px + R + 1) * ns - 1;
        int gy0 = (Py - R) * ns, gy1 = (Py + R + 1) * ns - 1;
        if (gx0 < 0) gx0 = 0;
        if (gy0 < 0) gy0 = 0;
        if (gx1 > ngx - 1) gx1 = ngx - 1;
        if (gy1 > ngy - 1) gy1 = ngy - 1;
        int W = gx1 - gx0 + 1, H = gy1 - gy0 + 1;
        /* time range of the deposits that reach the region */
        int tmin = nt, tmax = -1;
        for (int i = 0; i < n; ++i) {
            int ga[3], gb[3];
            int ok = 1;
            for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
            if (!ok || gb[0] < gx0 || ga[0] > gx1 || gb[1] < gy0 || ga[1] > gy1) continue;
            if (ga[2] < tmin) tmin = ga[2];
            if (gb[2] > tmax) tmax = gb[2];
        }
        if (tmax < tmin) continue;
        int T = tmax - tmin + 1;
        double *Q = (double *)calloc((size_t)W * H * T, sizeof(double));
        int *cmin = (int *)malloc(sizeof(int) * W * H);
        int *cmax = (int *)malloc(sizeof(int) * W * H);
        for (int k = 0; k < W * H; ++k) { cmin[k] = T; cmax[k] = -1; }
        for (int i = 0; i < n; ++i) {
            int ga[3], gb[3];
            int ok = 1;
            for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
            if (!ok || gb[0] < gx0 || ga[0] > gx1 || gb[1] < gy0 || ga[1] > gy1) continue;
            double *e[3];
            for (int ax = 0; ax < 3; ++ax) {
                e[ax] = (double *)malloc(sizeof(double) * (d[i].hi[ax] - d[i].lo[ax] + 3));
                axis_weights(p, xi, wl, &d[i], ax, e[ax]);
            }
            for (int gy = ga[1] > gy0 ? ga[1] : gy0; gy <= gb[1] && gy <= gy1; ++gy)
                for (int gx = ga[0] > gx0 ? ga[0] : gx0; gx <= gb[0] && gx <= gx1; ++gx) {
                    int c = (gy - gy0) * W + (gx - gx0);
                    double exy = d[i].q * e[1][gy - (d[i].lo[1] - 1)] * e[0][gx - (d[i].lo[0] - 1)];
                    double *col = Q + (size_t)c * T;
                    for (int gt = ga[2]; gt <= gb[2]; ++gt)
                        col[gt - tmin] += exy * e[2][gt - (d[i].lo[2] - 1)];
                    if (ga[2] - tmin < cmin[c]) cmin[c] = ga[2] - tmin;
                    if (gb[2] - tmin > cmax[c]) cmax[c] = gb[2] - tmin;
                }
            for (int ax = 0; ax < 3; ++ax) free(e[ax]);
        }
        for (int gy = gy0; gy <= gy1; ++gy)
            for (int gx = gx0; gx <= gx1; ++gx) {
                int c = (gy - gy0) * W + (gx - gx0);
                if (cmax[c] < cmin[c]) continue;
                int Ky = gy / ns - Py, Kx = gx / ns - Px;
                int jy = gy % ns, jx = gx % ns;
                const float *ir = resp + ((((size_t)(Ky + R) * kp + (Kx + R)) * ns + jy) * ns + jx) * nr;
                const double *col = Q + (size_t)c * T;
                for (int tl = cmin[c]; tl <= cmax[c]; ++tl) {
                    double q = col[tl];
                    if (q == 0.0) continue;
                    int ts = tl + tmin;
                    for (int tau = 0; tau < nr && ts + tau < nt; ++tau)
                        I[ts + tau] += q * (double)ir[tau];
                }
            }
        free(Q);
        free(cmin);
        free(cmax);
    }
}

/* ------------------------------------------------------------------------- */
/* Active pixels: every in-plane pixel in the output footprint of an active     */
/* block, i.e. pixels [bx*bp - R, bx*bp + bp + R) x (same in y), since the      */
/* convolution enlarges a block by the response half-width (Sec. III-B-1).      */
/* flags: [npx_y * npx_x] (written).  Returns the count.                        */
/* ------------------------------------------------------------------------- */
int orc_active_pixels(const orc_params *p, int nb, const int32_t *blocks, int kp,
                      uint8_t *flags)
{
    const int R = (kp - 1) / 2, nbx = p->npx_x / p->bp, nbt = p->nt / p->bt;
    memset(flags, 0, (size_t)p->npx_x * p->npx_y);
    for (int b = 0; b < nb; ++b) {
        int bxy = blocks[b] / nbt, bx = bxy % nbx, by = bxy / nbx;
        for (int y = by * p->bp - R; y < by * p->bp + p->bp + R; ++y)
            for (int x = bx * p->bp - R; x < bx * p->bp + p->bp + R; ++x)
                if (x >= 0 && x < p->npx_x && y >= 0 && y < p->npx_y)
                    flags[(size_t)y * p->npx_x + x] = 1;
    }
    int m = 0;
    for (size_t k = 0; k < (size_t)p->npx_x * p->npx_y; ++k) m += flags[k];
    return m;
}

/* ------------------------------------------------------------------------- */
/* Pixel readout (Sec. II-E), three schemes.  Per pixel the charge C is the running  */
/* sum of the current.  Also reports, per pixel, the first tested edge whose C  */
/* lies within tol of the threshold (-1 if none): hit lists may legitimately    */
/* differ from that edge on.  Returns the number of hits (written up to cap).   */
/*                                                                              */
/* mode 0, trigger-reset (Fig. readout): C counts from the end of the last      */
/*   reset.  At each clock edge k (k a multiple of clock) with k >= start: if    */
/*   C(k) >= threshold the channel triggers; the charge is sampled at k + hold   */
/*   and a hit (pixel, k + hold, C(k + hold)) is emitted if k + hold < nt; then  */
/*   C restarts at k + hold + reset + 1.                                        */
/* mode 1, successive digitisations without intervening resets: a trigger at   */
/*   edge k is followed by nsamp samples at k + m hold, m = 1..nsamp, each a hit */
/*   (pixel, k + m hold, C(k + m hold)) with C not reset between them; after    */
/*   the last, C restarts at k + nsamp hold + reset + 1.  A sample tick at or    */
/*   beyond nt ends the pixel.  nsamp = 1 is mode 0.                            */
/* mode 2, fixed-charge integration: C counts from tick 0 and is never reset;   */
/*   at each clock edge k with C(k) >= threshold a hit (pixel, k, threshold) is  */
/*   emitted and one quantum (the threshold) is taken from C, so no charge is    */
/*   lost: hits x threshold + C(nt - 1) is the total charge.                    */
/* ------------------------------------------------------------------------- */
long orc_readout(int npix, int nt, const int32_t *pixel_ids, const double *wave,
                 double thr, int clock, int hold, int reset, int mode, int nsamp, double tol,
                 int32_t *hit_pixel, int32_t *hit_tick, double *hit_charge, long cap,
                 int32_t *first_ambiguous)
{
    long m = 0;
#define ORC_EMIT(P, T, Q)                                                         \
    do {                                                                          \
        if (m < cap) { hit_pixel[m] = (P); hit_tick[m] = (T); hit_charge[m] = (Q); } \
        ++m;                                                                      \
    } while (0)
    for (int ip = 0; ip < npix; ++ip) {
        const double *I = wave + (size_t)ip * nt;
        first_ambiguous[ip] = -1;
        if (mode == 2) {
            double C = 0.0;
            int t = 0;
            for (int k = 0; k < nt; k += clock) {
                while (t <= k) C += I[t++];
                if (first_ambiguous[ip] < 0 && fabs(C - thr) <= tol) first_ambiguous[ip] = k;
                if (C >= thr) {
                    ORC_EMIT(pixel_ids[ip], k, thr);
                    C -= thr;
                }
            }
            continue;
        }
        const int ns = mode == 1 ? nsamp : 1;
        int start = 0;
        double C = 0.0;
        int t = 0;           /* next tick to add into C */
        int done = 0;
        while (!done) {
            int k = ((start + clock - 1) / clock) * clock;   /* first edge >= start */
            int fired = 0;
            for (; k < nt; k += clock) {
                while (t <= k) C += I[t++];
                if (first_ambiguous[ip] < 0 && fabs(C - thr) <= tol) first_ambiguous[ip] = k;
                if (C >= thr) { fired = 1; break; }
            }
            if (!fired) break;
            int ts = k;
            for (int s = 1; s <= ns; ++s) {
                ts = k + s * hold;
                if (ts >= nt) { done = 1; break; }
                while (t <= ts) C += I[t++];
                ORC_EMIT(pixel_ids[ip], ts, C);
            }
            if (done) break;
            start = ts + reset + 1;
            C = 0.0;
            t = start;
            if (start >= nt) break;
        }
    }
#undef ORC_EMIT
    return m;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ========================================================================= */
/* Differentiable simulation (Sec. V-C): gradient of L = 1/2 sum (I - I*)^2.    */
/* ========================================================================= */

/* Derivatives of the GL weights with respect to the mean and the width, with the
 * window [lo, hi] held fixed (it is piecewise constant in mu and sigma):
 *   d phi/d mu = phi (x - mu) / sig^2,  d phi/d sig = phi ((x - mu)^2 / sig^3 - 1/sig). */
void orc_weights_gl_grad(int nl, const double *xi, const double *wl, double mu, double sig,
                         int lo, int hi, double *e, double *de_dmu, double *de_dsig)
{
    int n = hi - lo + 3;
    for (int k = 0; k < n; ++k) e[k] = de_dmu[k] = de_dsig[k] = 0.0;
    for (int C = lo; C <= hi; ++C) {
        for (int l = 0; l < nl; ++l) {
            double s = 0.5 * xi[l];
            double xx = (double)C + s;
            double ph = normal_pdf(xx, mu, sig);
            double dm = ph * (xx - mu) / (sig * sig);
            double ds = ph * ((xx - mu) * (xx - mu) / (sig * sig * sig) - 1.0 / sig);
            double wv = 0.5 * wl[l];
            int k = C - (lo - 1);
            int k2 = s > 0.0 ? k + 1 : k - 1;
            double u0 = 1.0 - fabs(s), u1 = fabs(s);
            e[k] += wv * ph * u0;
            de_dmu[k] += wv * dm * u0;
            de_dsig[k] += wv * ds * u0;
            if (s != 0.0) {
                e[k2] += wv * ph * u1;
                de_dmu[k2] += wv * dm * u1;
                de_dsig[k2] += wv * ds * u1;
            }
        }
    }
}

typedef struct { int gy, gx, dep; } orc_cellref;

static int cmp_cellref(const void *a, const void *b)
{
    const orc_cellref *x = (const orc_cellref *)a, *y = (const orc_cellref *)b;
    if (x->gy != y->gy) return x->gy < y->gy ? -1 : 1;
    if (x->gx != y->gx) return x->gx < y->gx ? -1 : 1;
    return x->dep < y->dep ? -1 : (x->dep > y->dep);
}

/* Adjoint of the whole path for the loss L = 1/2 sum_{P in pixel_ids, t} r^2 with
 * r = dL/dI given per listed pixel (resid [npix][nt]; unlisted pixels have r = 0).
 *   G[j, P', t'] = dL/dQeff = sum_K sum_tau r[P' - K, t' + tau] i[j, K, tau]
 * (the transpose of the interlaced convolution, Sec. II-D), then the chain rule
 * through Qeff = q e_x e_y e_t with the windows held fixed.
 * Output per deposit, grad[d][7] = dL/d(q, mu_x, mu_y, mu_t, sig_x, sig_y, sig_t)
 * in grid units (GL mode). */
void orc_adjoint(const orc_params *p, int n, const orc_dep *d, const float *resp, int kp,
                 int nr, int npix, const int32_t *pixel_ids, const double *resid, double *grad)
{
    const int ns = p->n_sub, R = (kp - 1) / 2, nt = p->nt;
    const int ngx = p->npx_x * ns, ngy = p->npx_y * ns;
    double xi[64], wl[64];
    orc_gl_rule(p->gl_order, xi, wl);
    int32_t *row_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)p->npx_x * p->npx_y);
    for (size_t k = 0; k < (size_t)p->npx_x * p->npx_y; ++k) row_of[k] = -1;
    for (int i = 0; i < npix; ++i) row_of[pixel_ids[i]] = i;
    /* every (column, deposit) incidence, sorted by column */
    long m = 0;
    for (int i = 0; i < n; ++i) {
        int ga[3], gb[3], ok = 1;
        for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
        if (ok) m += (long)(gb[0] - ga[0] + 1) * (gb[1] - ga[1] + 1);
    }
    orc_cellref *refs = (orc_cellref *)malloc(sizeof(orc_cellref) * (m > 0 ? m : 1));
    m = 0;
    for (int i = 0; i < n; ++i) {
        int ga[3], gb[3], ok = 1;
        for (int ax = 0; ax < 3; ++ax) ok &= support(p, &d[i], ax, &ga[ax], &gb[ax]);
        if (!ok) continue;
        for (int gy = ga[1]; gy <= gb[1]; ++gy)
            for (int gx = ga[0]; gx <= gb[0]; ++gx) {
                refs[m].gy = gy;
                refs[m].gx = gx;
                refs[m].dep = i;
                ++m;
            }
    }
    qsort(refs, m, sizeof(orc_cellref), cmp_cellref);
    /* column runs */
    long nrun = 0;
    for (long k = 0; k < m; ++k)
        if (k == 0 || refs[k].gy != refs[k - 1].gy || refs[k].gx != refs[k - 1].gx) ++nrun;
    long *run_beg = (long *)malloc(sizeof(long) * (nrun + 1));
    nrun = 0;
    for (long k = 0; k < m; ++k)
        if (k == 0 || refs[k].gy != refs[k - 1].gy || refs[k].gx != refs[k - 1].gx) run_beg[nrun++] = k;
    run_beg[nrun] = m;
    for (int i = 0; i < n * 7; ++i) grad[i] = 0.0;
#pragma omp parallel
    {
        double *G = (double *)malloc(sizeof(double) * nt);
        double *gloc = (double *)calloc((size_t)n * 7, sizeof(double));
#pragma omp for schedule(dynamic)
        for (long c = 0; c < nrun; ++c) {
            const int gy = refs[run_beg[c]].gy, gx = refs[run_beg[c]].gx;
            const int Py = gy / ns, Px = gx / ns, jy = gy % ns, jx = gx % ns;
            /* time range of this column's deposits */
            int ta = nt, tb = -1;
            for (long k = run_beg[c]; k < run_beg[c + 1]; ++k) {
                int a, b;
                support(p, &d[refs[k].dep], 2, &a, &b);
                if (a < ta) ta = a;
                if (b > tb) tb = b;
            }
            for (int t = ta; t <= tb; ++t) G[t] = 0.0;
            for (int Ky = -R; Ky <= R; ++Ky)
                for (int Kx = -R; Kx <= R; ++Kx) {
                    int qy = Py - Ky, qx = Px - Kx;     /* electrode seeing this cell through i[j, K] */
                    if (qy < 0 || qy >= p->npx_y || qx < 0 || qx >= p->npx_x) continue;
                    int row = row_of[qy * p->npx_x + qx];
                    if (row < 0) continue;
                    const double *rr = resid + (size_t)row * nt;
                    const float *ir = resp + ((((size_t)(Ky + R) * kp + (Kx + R)) * ns + jy) * ns + jx) * nr;
                    for (int t = ta; t <= tb; ++t) {
                        double s = 0.0;
                        for (int tau = 0; tau < nr && t + tau < nt; ++tau) s += rr[t + tau] * (double)ir[tau];
                        G[t] += s;
                    }
                }
            for (long k = run_beg[c]; k < run_beg[c + 1]; ++k) {
                const int i = refs[k].dep;
                const orc_dep *dd = &d[i];
                int a, b;
                support(p, dd, 2, &a, &b);
                double e[3][3];   /* [axis][value, d/dmu, d/dsig] at this column / summed in t */
                /* x and y weights at this column */
                for (int ax = 0; ax < 2; ++ax) {
                    int len = dd->hi[ax] - dd->lo[ax] + 3;
                    double *w0 = (double *)malloc(sizeof(double) * len * 3);
                    orc_weights_gl_grad(p->gl_order, xi, wl, dd->mu[ax], dd->sig[ax], dd->lo[ax],
                                        dd->hi[ax], w0, w0 + len, w0 + 2 * len);
                    int g = (ax == 0 ? gx : gy) - (dd->lo[ax] - 1);
                    e[ax][0] = w0[g];
                    e[ax][1] = w0[len + g];
                    e[ax][2] = w0[2 * len + g];
                    free(w0);
                }
                int len = dd->hi[2] - dd->lo[2] + 3;
                double *w0 = (double *)malloc(sizeof(double) * len * 3);
                orc_weights_gl_grad(p->gl_order, xi, wl, dd->mu[2], dd->sig[2], dd->lo[2], dd->hi[2],
                                    w0, w0 + len, w0 + 2 * len);
                double st0 = 0, st1 = 0, st2 = 0;
                for (int t = a; t <= b; ++t) {
                    int g = t - (dd->lo[2] - 1);
                    st0 += G[t] * w0[g];
                    st1 += G[t] * w0[len + g];
                    st2 += G[t] * w0[2 * len + g];
                }
                free(w0);
                e[2][0] = st0;
                e[2][1] = st1;
                e[2][2] = st2;
                double *gd = gloc + (size_t)i * 7;
                const double q = dd->q;
                gd[0] += e[0][0] * e[1][0] * e[2][0];
                gd[1] += q * e[0][1] * e[1][0] * e[2][0];
                gd[2] += q * e[0][0] * e[1][1] * e[2][0];
                gd[3] += q * e[0][0] * e[1][0] * e[2][1];
                gd[4] += q * e[0][2] * e[1][0] * e[2][0];
                gd[5] += q * e[0][0] * e[1][2] * e[2][0];
                gd[6] += q * e[0][0] * e[1][0] * e[2][2];
            }
        }
#pragma omp critical
        for (int i = 0; i < n * 7; ++i) grad[i] += gloc[i];
        free(gloc);
        free(G);
    }
    free(run_beg);
    free(refs);
    free(row_of);
}

/* Chain rule from the per-deposit gradients dL/d(q, mu, sigma) (grid units) to the
 * inputs of the transport step (Sec. II-A) and its global constants:
 *   mu_x = x / h - 1/2, mu_t = (t0 + z / v) / tick, q = ne exp(-t_d / tau),
 *   sig_xy^2 = 2 DT 1e-6 t_d / h^2 + s0^2, sig_t^2 = 2 DL 1e-6 t_d / (v tick)^2 + s0t^2.
 * Per deposit out[d][4] = dL/d(x, y, t0, ne); glob[3] = dL/d(DL, DT, tau). */
void orc_param_grads(const orc_params *p, int n, const float *z, const float *ne, const orc_dep *d,
                     const double *grad7, double *out, double *glob)
{
    const double v = p->v_cm_per_us, tick = p->tick_us, tau = p->lifetime_us;
    const double h = (double)p->pitch_cm / (double)p->n_sub;
    double gDL = 0, gDT = 0, gtau = 0;
    for (int i = 0; i < n; ++i) {
        const double *g = grad7 + (size_t)i * 7;
        double *o = out + (size_t)i * 4;
        if (!d[i].valid) {
            o[0] = o[1] = o[2] = o[3] = 0.0;
            continue;
        }
        const double td = (double)z[i] / v;
        o[0] = g[1] / h;
        o[1] = g[2] / h;
        o[2] = g[3] / tick;
        o[3] = g[0] * exp(-td / tau);
        gtau += g[0] * d[i].q * td / (tau * tau);
        gDT += (g[4] + g[5]) * 1e-6 * td / (h * h * d[i].sig[0]);
        gDL += g[6] * 1e-6 * td / (v * tick * v * tick * d[i].sig[2]);
    }
    glob[0] = gDL;
    glob[1] = gDT;
    glob[2] = gtau;
    (void)ne;
}

/* ========================================================================= */
/* Line-shape track segments (Sec. II-C, "Calculation of Q for a line-shape      */
/* track segment", Eq. qline; "short track segments").                         */
/* ========================================================================= */

/* Drifted segment: both endpoints in grid units; one width per axis, taken at the
 * midpoint's drift time (the paper gives one sigma per segment); the window spans
 * both endpoints +- nsigma sigma; attachment at the midpoint's drift time. */
typedef struct {
    orc_dep d;          /* mu = midpoint, sig, q, lo/hi window, valid */
    double p0[3], p1[3];
} orc_line;

void orc_drift_lines(const orc_params *p, int n, const float *x0, const float *y0,
                     const float *z0, const float *x1, const float *y1, const float *z1,
                     const float *t0, const float *ne, orc_line *out)
{
    const double v = (double)p->v_cm_per_us;
    const double tick = (double)p->tick_us;
    const double h = (double)p->pitch_cm / (double)p->n_sub;
    const double width_x = (double)p->npx_x * (double)p->pitch_cm;
    const double width_y = (double)p->npx_y * (double)p->pitch_cm;
    const double DT = (double)p->DT_cm2_per_s, DL = (double)p->DL_cm2_per_s;
    const double s0 = (double)p->sigma0_cells_xy, s0t = (double)p->sigma0_ticks;
    const double ns = (double)p->nsigma;
    const double tau = (double)p->lifetime_us;
    for (int i = 0; i < n; ++i) {
        orc_line *L = &out[i];
        orc_dep *d = &L->d;
        const double xa = x0[i], ya = y0[i], za = z0[i], xb = x1[i], yb = y1[i], zb = z1[i];
        const double t0d = t0[i], ned = ne[i];
        int ok = isfinite(xa) && isfinite(ya) && isfinite(za) && isfinite(xb) && isfinite(yb)
                 && isfinite(zb) && isfinite(t0d) && isfinite(ned) && za >= 0.0 && zb >= 0.0
                 && ned >= 0.0 && xa >= 0.0 && xa < width_x && ya >= 0.0 && ya < width_y
                 && xb >= 0.0 && xb < width_x && yb >= 0.0 && yb < width_y;
        memset(L, 0, sizeof(*L));
        if (!ok) {
            for (int a = 0; a < 3; ++a) { d->lo[a] = 0; d->hi[a] = -1; }
            d->valid = 0;
            continue;
        }
        d->valid = 1;
        const double tda = za / v, tdb = zb / v;
        L->p0[0] = xa / h - 0.5;
        L->p0[1] = ya / h - 0.5;
        L->p0[2] = (t0d + tda) / tick;
        L->p1[0] = xb / h - 0.5;
        L->p1[1] = yb / h - 0.5;
        L->p1[2] = (t0d + tdb) / tick;
        double zm = za + zb;
        zm = zm * 0.5;
        const double td = zm / v;               /* midpoint drift time */
        double a = DT * 2.0;
        a = a * 1e-6;
        a = a * td;
        double b = h * h;
        a = a / b;
        double c = s0 * s0;
        const double sxy = sqrt(a + c);
        a = DL * 2.0;
        a = a * 1e-6;
        a = a * td;
        b = v * tick;
        b = b * b;
        a = a / b;
        c = s0t * s0t;
        const double st = sqrt(a + c);
        d->sig[0] = sxy;
        d->sig[1] = sxy;
        d->sig[2] = st;
        d->q = ned * exp(-td / tau);
        for (int ax = 0; ax < 3; ++ax) {
            d->mu[ax] = 0.5 * (L->p0[ax] + L->p1[ax]);
            const double K = ns * d->sig[ax];
            const double mn = L->p0[ax] < L->p1[ax] ? L->p0[ax] : L->p1[ax];
            const double mx = L->p0[ax] < L->p1[ax] ? L->p1[ax] : L->p0[ax];
            d->lo[ax] = (int32_t)floor(mn - K);
            d->hi[ax] = (int32_t)ceil(mx + K);
        }
    }
}

/* Normalised charge density of a uniform line from p0 to p1 diffused by an
 * axis-aligned Gaussian (Eq. qline divided by Q), in grid units, written with
 *     Delta^2 = S alpha,  A1 = -S beta,  A2 = S (alpha - beta),  B = S (alpha gamma - beta^2),
 *     S = sx^2 sy^2 sz^2, alpha = sum d_i^2 / s_i^2, beta = sum a_i d_i / s_i^2,
 *     gamma = sum a_i^2 / s_i^2, d = p1 - p0, a = x - p0,
 * so that rho = exp(-B / (2 Delta^2)) (erf(A2 / (sqrt2 Delta sx sy sz))
 *                - erf(A1 / (sqrt2 Delta sx sy sz))) / (4 pi Delta).
 * The exponent carries the factor 1/2 that the isotropic limit exp(-d_perp^2 / 2 s^2)
 * requires.  Segments shorter than frac * sigma on every axis use the point
 * Gaussian at the midpoint (the short-segment limit). */
double orc_line_density(const double *p0, const double *p1, const double *sig, double frac,
                        const double *x)
{
    int shortseg = 1;
    for (int i = 0; i < 3; ++i) shortseg &= fabs(p1[i] - p0[i]) < frac * sig[i];
    if (shortseg) {
        double r = 1.0;
        for (int i = 0; i < 3; ++i) {
            const double m = 0.5 * (p0[i] + p1[i]);
            const double u = (x[i] - m) / sig[i];
            r *= exp(-0.5 * u * u) / (sqrt(2.0 * M_PI) * sig[i]);
        }
        return r;
    }
    const double S = sig[0] * sig[0] * sig[1] * sig[1] * sig[2] * sig[2];
    double alpha = 0.0, beta = 0.0, gamma = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double di = p1[i] - p0[i], ai = x[i] - p0[i], w = 1.0 / (sig[i] * sig[i]);
        alpha += di * di * w;
        beta += ai * di * w;
        gamma += ai * ai * w;
    }
    const double Delta = sqrt(S * alpha);
    const double B = S * (alpha * gamma - beta * beta);
    const double A1 = -S * beta, A2 = S * (alpha - beta);
    const double den = sqrt(2.0) * Delta * sig[0] * sig[1] * sig[2];
    return exp(-B / (2.0 * Delta * Delta)) * (erf(A2 / den) - erf(A1 / den)) / (4.0 * M_PI * Delta);
}

/* Effective charge of the listed blocks from line segments (Eq. eff_q with the node
 * charge Q_{lmn,C} = Q rho(node) w_l w_m w_n / 8): every quadrature node of every cell
 * of the window is scattered to the grid points of Eq. trilinear (its cell centre
 * with 1 - |s| and the adjacent centre on its side with |s|, per axis).  The
 * support of the result is the window +- 1, as for points.  Layout as
 * orc_qeff_blocks. */
void orc_qeff_line_blocks(const orc_params *p, int n, const orc_line *L, double frac, int nb,
                          const int32_t *blocks, double *qeff)
{
    const int ns = p->n_sub, bp = p->bp, btk = p->bt, nl = p->gl_order;
    const int nbx = p->npx_x / p->bp, nbt = p->nt / p->bt;
    const size_t per_block = (size_t)ns * ns * bp * bp * btk;
    double xi[64], wl[64];
    orc_gl_rule(nl, xi, wl);
    memset(qeff, 0, sizeof(double) * per_block * nb);
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < nb; ++b) {
        int blk = blocks[b];
        int bt = blk % nbt, bxy = blk / nbt, bx = bxy % nbx, by = bxy / nbx;
        int X0 = bx * bp * ns, Y0 = by * bp * ns, T0 = bt * btk;
        double *Q = qeff + per_block * b;
        for (int i = 0; i < n; ++i) {
            const orc_dep *d = &L[i].d;
            int ga[3], gb[3];
            int ok = 1;
            for (int ax = 0; ax < 3; ++ax) ok &= support(p, d, ax, &ga[ax], &gb[ax]);
            if (!ok) continue;
            if (gb[0] < X0 || ga[0] > X0 + bp * ns - 1 || gb[1] < Y0 || ga[1] > Y0 + bp * ns - 1
                || gb[2] < T0 || ga[2] > T0 + btk - 1)
                continue;
            for (int cz = d->lo[2]; cz <= d->hi[2]; ++cz)
                for (int cy = d->lo[1]; cy <= d->hi[1]; ++cy)
                    for (int cx = d->lo[0]; cx <= d->hi[0]; ++cx)
                        for (int ln = 0; ln < nl; ++ln)
                            for (int lm = 0; lm < nl; ++lm)
                                for (int ll = 0; ll < nl; ++ll) {
                                    const double s[3] = {0.5 * xi[ll], 0.5 * xi[lm], 0.5 * xi[ln]};
                                    const double node[3] = {cx + s[0], cy + s[1], cz + s[2]};
                                    const double qn = d->q * 0.125 * wl[ll] * wl[lm] * wl[ln]
                                                      * orc_line_density(L[i].p0, L[i].p1, d->sig, frac, node);
                                    /* targets per axis: (grid point, coefficient) */
                                    int tg[3][2];
                                    double tc[3][2];
                                    int nt3[3];
                                    const int cc[3] = {cx, cy, cz};
                                    for (int ax = 0; ax < 3; ++ax) {
                                        if (s[ax] == 0.0) {
                                            tg[ax][0] = cc[ax]; tc[ax][0] = 1.0; nt3[ax] = 1;
                                        } else {
                                            tg[ax][0] = cc[ax]; tc[ax][0] = 1.0 - fabs(s[ax]);
                                            tg[ax][1] = cc[ax] + (s[ax] > 0 ? 1 : -1); tc[ax][1] = fabs(s[ax]);
                                            nt3[ax] = 2;
                                        }
                                    }
                                    for (int kz = 0; kz < nt3[2]; ++kz) {
                                        const int gt = tg[2][kz];
                                        if (gt < T0 || gt >= T0 + btk || gt < ga[2] || gt > gb[2]) continue;
                                        for (int ky = 0; ky < nt3[1]; ++ky) {
                                            const int gy = tg[1][ky];
                                            if (gy < Y0 || gy >= Y0 + bp * ns || gy < ga[1] || gy > gb[1]) continue;
                                            for (int kx = 0; kx < nt3[0]; ++kx) {
                                                const int gx = tg[0][kx];
                                                if (gx < X0 || gx >= X0 + bp * ns || gx < ga[0] || gx > gb[0]) continue;
                                                const int jy = gy % ns, py = gy / ns - by * bp;
                                                const int jx = gx % ns, px = gx / ns - bx * bp;
                                                Q[((((size_t)jy * ns + jx) * bp + py) * bp + px) * btk + (gt - T0)] +=
                                                    qn * tc[0][kx] * tc[1][ky] * tc[2][kz];
                                            }
                                        }
                                    }
                                }
        }
    }
}

/* Induced current on listed pixels from block-stored effective charge (Eq.
 * interlaced written out): I[P, t] = sum_j sum_K sum_tau Qeff[j, P + K, t - tau]
 * i[j, K, tau], summing over the listed blocks (which must cover the support).
 * qeff layout [block][jy][jx][py][px][t]; resp [Ky][Kx][jy][jx][tau]. */
void orc_currents_from_qeff(const orc_params *p, int nb, const int32_t *blocks, const double *qeff,
                            const float *resp, int kp, int nr, int npix, const int32_t *pixel_ids,
                            double *wave)
{
    const int ns = p->n_sub, bp = p->bp, btk = p->bt, R = (kp - 1) / 2, nt = p->nt;
    const int nbx = p->npx_x / p->bp, nbt = p->nt / p->bt;
    const size_t per_block = (size_t)ns * ns * bp * bp * btk;
#pragma omp parallel for schedule(dynamic)
    for (int ip = 0; ip < npix; ++ip) {
        double *I = wave + (size_t)ip * nt;
        memset(I, 0, sizeof(double) * nt);
        const int P = pixel_ids[ip], Px = P % p->npx_x, Py = P / p->npx_x;
        for (int b = 0; b < nb; ++b) {
            const int blk = blocks[b];
            const int bt = blk % nbt, bxy = blk / nbt, bx = bxy % nbx, by = bxy / nbx;
            const double *Q = qeff + per_block * b;
            for (int py = 0; py < bp; ++py)
                for (int px = 0; px < bp; ++px) {
                    const int Ky = by * bp + py - Py, Kx = bx * bp + px - Px;
                    if (Ky < -R || Ky > R || Kx < -R || Kx > R) continue;
                    for (int jy = 0; jy < ns; ++jy)
                        for (int jx = 0; jx < ns; ++jx) {
                            const double *col = Q + ((((size_t)jy * ns + jx) * bp + py) * bp + px) * btk;
                            const float *ir = resp + ((((size_t)(Ky + R) * kp + (Kx + R)) * ns + jy) * ns + jx) * nr;
                            for (int tl = 0; tl < btk; ++tl) {
                                const double q = col[tl];
                                if (q == 0.0) continue;
                                const int ts = bt * btk + tl;
                                for (int tau = 0; tau < nr && ts + tau < nt; ++tau) I[ts + tau] += q * (double)ir[tau];
                            }
                        }
                }
        }
    }
}
