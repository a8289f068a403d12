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
//   k_effq_blocks   persistent CTAs over (active block, impact channel) items: a
//                   bp x bp x bt slab accumulated in shared memory from the block's
//                   deposits, written once with 16-byte stores, plus the mask of
//                   its non-empty (py, px) columns
#include "tred_internal.cuh"

namespace tred {

struct EffqConst {
    int ns, bp, bt, ngx, ngy, nt, nbx, nbt, wx, wt, wstride, gl, mode;
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
                                                      float *__restrict__ wts) {
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

// Persistent CTAs over (slot, channel) items.  Shared slab [bp*bp][bt] floats.
__global__ void __launch_bounds__(256) k_effq_blocks(const int32_t *__restrict__ block_ids,
                                                     const int32_t *__restrict__ dep_offsets,
                                                     const int32_t *__restrict__ dep_index,
                                                     const int32_t *__restrict__ n_blocks_dev,
                                                     tred_deposits d, EffqConst c,
                                                     const float *__restrict__ wts,
                                                     float *__restrict__ qeff,
                                                     uint64_t *__restrict__ colmask) {
    extern __shared__ float slab[];
    __shared__ unsigned s_mask[2];
    const int nb = n_blocks_dev[0];
    const int nch = c.ns * c.ns;
    const int cols = c.bp * c.bp;
    const int slab_n = cols * c.bt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int64_t items = (int64_t)nb * nch;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int slot = (int)(item / nch), ch = (int)(item % nch);
        const int jy = ch / c.ns, jx = ch % c.ns;
        const int blk = block_ids[slot];
        const int bt = blk % c.nbt, bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int gx0 = bx * c.bp * c.ns + jx;    // sub-cell of px = 0 in this channel
        const int gy0 = by * c.bp * c.ns + jy;
        const int t0 = bt * c.bt;
        for (int k = threadIdx.x; k < slab_n; k += blockDim.x) slab[k] = 0.f;
        if (threadIdx.x < 2) s_mask[threadIdx.x] = 0u;
        __syncthreads();
        const int beg = dep_offsets[slot], end = dep_offsets[slot + 1];
        for (int k = beg + warp; k < end; k += nwarps) {
            const int i = dep_index[k];
            const int lox = d.lo_x[i], hix = d.hi_x[i], loy = d.lo_y[i], hiy = d.hi_y[i];
            const int lot = d.lo_t[i], hit = d.hi_t[i];
            const int xa = max(lox - 1, 0), xb = min(hix + 1, c.ngx - 1);
            const int ya = max(loy - 1, 0), yb = min(hiy + 1, c.ngy - 1);
            const int ta = max(max(lot - 1, 0), t0), tb = min(min(hit + 1, c.nt - 1), t0 + c.bt - 1);
            if (ta > tb) continue;
            const int px0 = max(0, -floordiv(gx0 - xa, c.ns)), px1 = min(c.bp - 1, floordiv(xb - gx0, c.ns));
            const int py0 = max(0, -floordiv(gy0 - ya, c.ns)), py1 = min(c.bp - 1, floordiv(yb - gy0, c.ns));
            if (px0 > px1 || py0 > py1) continue;
            const float q = d.q[i];
            const float *w = wts + (size_t)i * c.wstride;
            const float *wxv = w, *wyv = w + c.wx, *wtv = w + 2 * c.wx;
            for (int py = py0; py <= py1; ++py) {
                const float ay = q * wyv[gy0 + py * c.ns - (loy - 1)];
                for (int px = px0; px <= px1; ++px) {
                    const float a = ay * wxv[gx0 + px * c.ns - (lox - 1)];
                    float *col = slab + (py * c.bp + px) * c.bt - t0;
                    for (int t = ta + lane; t <= tb; t += 32)
                        atomicAdd(&col[t], a * wtv[t - (lot - 1)]);
                    if (lane == 0) {
                        const int bit = py * c.bp + px;
                        atomicOr(&s_mask[bit >> 5], 1u << (bit & 31));
                    }
                }
            }
        }
        __syncthreads();
        float4 *dst = reinterpret_cast<float4 *>(qeff + ((size_t)slot * nch + ch) * slab_n);
        const float4 *src = reinterpret_cast<const float4 *>(slab);
        for (int k = threadIdx.x; k < slab_n / 4; k += blockDim.x) dst[k] = src[k];
        if (threadIdx.x == 0)
            colmask[(size_t)slot * nch + ch] = ((uint64_t)s_mask[1] << 32) | s_mask[0];
        __syncthreads();
    }
}

int launch_effq(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                float *qeff, cudaStream_t s) {
    EffqConst c;
    c.ns = h->g.n_sub;
    c.bp = h->g.bp;
    c.bt = h->g.bt;
    c.ngx = h->d.ngx;
    c.ngy = h->d.ngy;
    c.nt = h->g.nt;
    c.nbx = h->d.nbx;
    c.nbt = h->d.nbt;
    c.wx = h->d.wx;
    c.wt = h->d.wt;
    c.wstride = h->d.wstride;
    c.gl = h->p.gl_order;
    c.mode = h->p.effq_mode;
    for (int l = 0; l < MAX_GL; ++l) {
        c.xi[l] = l < c.gl ? h->gl_xi[l] : 0.f;
        c.wl[l] = l < c.gl ? h->gl_wi[l] : 0.f;
    }
    if (n > 0) {
        const int threads = 256;
        const int64_t blocks = ((int64_t)n * 32 + threads - 1) / threads;
        k_effq_weights<<<(unsigned)blocks, threads, 0, s>>>(n, deps, c, h->wts);
    }
    const size_t smem = sizeof(float) * (size_t)c.bp * c.bp * c.bt;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_effq_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    if (smem > 200 * 1024) return set_error(h, TRED_ERR_INVALID_ARG, "effq slab too large");
    const int grid = num_sms(h) * 3;
    k_effq_blocks<<<grid, 256, smem, s>>>(block_ids, dep_offsets, dep_index, n_blocks_dev, deps, c,
                                          h->wts, qeff, h->colmask);
    h->launches += 1 + (n > 0 ? 1 : 0);
    return check_cuda(h, cudaGetLastError(), "effq launch");
}

}  // namespace tred
