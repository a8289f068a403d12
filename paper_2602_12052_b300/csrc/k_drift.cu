// a1. Transport: drift time, attachment, diffusion width and the raster window
// (Sec. II-A; Fig. flowchart steps A and D).  One thread per deposit.
//
// The integer window is produced by one fixed sequence of correctly rounded
// binary64 operations (__dadd_rn / __dmul_rn / __ddiv_rn / __dsqrt_rn: no
// contraction into FMA), so every IEEE binary64 evaluation of the same sequence
// yields the same cells and therefore the same active blocks.
#include "tred_internal.cuh"

namespace tred {

struct DriftConst {
    double v, tick, h, width_x, width_y, DT, DL, s0, s0t, ns, tau, max_td;
    int n_events, ngy_e;
};

__global__ void __launch_bounds__(256) k_drift(int n, const float *__restrict__ x,
                                               const float *__restrict__ y,
                                               const float *__restrict__ z,
                                               const float *__restrict__ t0,
                                               const float *__restrict__ ne,
                                               const int32_t *__restrict__ event, DriftConst c,
                                               tred_deposits out, int32_t *__restrict__ dep_event,
                                               int32_t *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xd = x[i], yd = y[i], zd = z[i], t0d = t0[i], ned = ne[i];
    const int ev = event ? event[i] : 0;
    dep_event[i] = ev;
    const bool ok = isfinite(xd) && isfinite(yd) && isfinite(zd) && isfinite(t0d) && isfinite(ned) &&
                    zd >= 0.0 && ned >= 0.0 && xd >= 0.0 && xd < c.width_x && yd >= 0.0 &&
                    yd < c.width_y && ev >= 0 && ev < c.n_events;
    const double td = __ddiv_rn(zd, c.v);
    if (!ok || !(td <= c.max_td)) {
        if (ok) atomicOr(&status[0], TRED_ST_DRIFT_RANGE);
        atomicAdd(&status[1], 1);
        out.cell_x[i] = out.cell_y[i] = out.cell_t[i] = 0;
        out.frac_x[i] = out.frac_y[i] = out.frac_t[i] = 0.f;
        out.sigma_x[i] = out.sigma_y[i] = out.sigma_t[i] = 1.f;
        out.lo_x[i] = out.lo_y[i] = out.lo_t[i] = 0;
        out.hi_x[i] = out.hi_y[i] = out.hi_t[i] = -1;
        out.q[i] = 0.f;
        return;
    }
    const double ta = __dadd_rn(t0d, td);
    const double mu_t = __ddiv_rn(ta, c.tick);
    const double mu_x = __dadd_rn(__ddiv_rn(xd, c.h), -0.5);
    const double mu_y = __dadd_rn(__ddiv_rn(yd, c.h), -0.5);
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
    const double mu[3] = {mu_x, mu_y, mu_t};
    const double sg[3] = {sxy, sxy, st};
    int32_t *cell[3] = {out.cell_x, out.cell_y, out.cell_t};
    float *frac[3] = {out.frac_x, out.frac_y, out.frac_t};
    float *sig[3] = {out.sigma_x, out.sigma_y, out.sigma_t};
    int32_t *lo[3] = {out.lo_x, out.lo_y, out.lo_t};
    int32_t *hi[3] = {out.hi_x, out.hi_y, out.hi_t};
    // event-local window; events are stacked along y by whole cells
    const int shift[3] = {0, ev * c.ngy_e, 0};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const double K = __dmul_rn(c.ns, sg[ax]);
        const double fl = floor(mu[ax]);
        cell[ax][i] = (int32_t)fl + shift[ax];
        frac[ax][i] = (float)(mu[ax] - fl);   // exact in binary64, then rounded
        sig[ax][i] = (float)sg[ax];
        lo[ax][i] = (int32_t)floor(__dadd_rn(mu[ax], -K)) + shift[ax];
        hi[ax][i] = (int32_t)ceil(__dadd_rn(mu[ax], K)) + shift[ax];
    }
    out.q[i] = (float)(ned * exp(-td / c.tau));
}

int launch_drift(tred_handle *h, int n, const float *x, const float *y, const float *z,
                 const float *t0, const float *ne, const int32_t *event, const tred_deposits &out,
                 cudaStream_t s) {
    DriftConst c;
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
    c.n_events = h->d.n_events;
    c.ngy_e = h->d.ngy_e;
    k_drift<<<(n + 255) / 256, 256, 0, s>>>(n, x, y, z, t0, ne, event, c, out, h->dep_event, h->status);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "k_drift launch");
}

}  // namespace tred
