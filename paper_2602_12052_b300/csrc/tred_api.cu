// libtred C ABI: handle life cycle, argument checks, status word, and dispatch to
// the kernel launchers.  No C++ exception crosses this boundary.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tred_internal.cuh"

namespace tred {

// An NVTX range over one ABI call (named after it), so that a profiler's timeline shows
// the path's steps around their kernels; a push and a pop when no tool is attached.
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};

int set_error(tred_handle *h, int code, const char *fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int check_cuda(tred_handle *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return TRED_OK;
    return set_error(h, TRED_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int num_sms(tred_handle *h) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, h->device);
    return n > 0 ? n : 148;
}

}  // namespace tred

// Event pairs of the timed launches, per kernel class; the events are pooled and reused.
struct KernelTimers {
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs[TRED_KT_CLASSES];
    cudaEvent_t open[TRED_KT_CLASSES] = {};
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    ~KernelTimers() {
        for (auto e : pool) cudaEventDestroy(e);
        for (auto &v : pairs)
            for (auto &p : v) {
                cudaEventDestroy(p.first);
                cudaEventDestroy(p.second);
            }
        for (auto e : open)
            if (e) cudaEventDestroy(e);
    }
};

namespace tred {

void kt_begin(tred_handle *h, int which, cudaStream_t s) {
    if (!h->kt || which < 0 || which >= TRED_KT_CLASSES) return;
    cudaEvent_t e = h->kt->take();
    cudaEventRecord(e, s);
    h->kt->open[which] = e;
}
void kt_end(tred_handle *h, int which, cudaStream_t s) {
    if (!h->kt || which < 0 || which >= TRED_KT_CLASSES || !h->kt->open[which]) return;
    cudaEvent_t e = h->kt->take();
    cudaEventRecord(e, s);
    h->kt->pairs[which].push_back({h->kt->open[which], e});
    h->kt->open[which] = nullptr;
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on the Legendre
// polynomial from Chebyshev-like starting points, derivative from the standard
// identity (1 - x^2) P_n' = n (P_{n-1} - x P_n).
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0, pd = 0;
        for (int it = 0; it < 200; ++it) {
            double a = 1.0, b = z;              // P_0, P_1
            if (n == 1) { pn = z; a = 1.0; }
            for (int k = 2; k <= n; ++k) {
                double c = ((2 * k - 1) * z * b - (k - 1) * a) / k;
                a = b;
                b = c;
            }
            pn = b;                               // P_n(z)
            pd = n * (a - z * b) / (1.0 - z * z); // P_n'(z)
            double dz = pn / pd;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        double a = 1.0, b = z;
        for (int k = 2; k <= n; ++k) {
            double c = ((2 * k - 1) * z * b - (k - 1) * a) / k;
            a = b;
            b = c;
        }
        pd = n * (a - z * b) / (1.0 - z * z);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pd * pd);
    }
    if (n % 2) x[n / 2] = 0.0;
}

}  // namespace tred

using namespace tred;

extern "C" {

const char *tred_last_error(const tred_handle *h) { return h ? h->err : "null handle"; }

}  // extern "C"

namespace tred {

bool deps_ok(const tred_deposits *d) {
    return d && d->cell_x && d->cell_y && d->cell_t && d->frac_x && d->frac_y && d->frac_t &&
           d->sigma_x && d->sigma_y && d->sigma_t && d->lo_x && d->lo_y && d->lo_t && d->hi_x &&
           d->hi_y && d->hi_t && d->q;
}

int validate_geometry(const tred_geometry *g, char *msg, size_t len) {
    auto bad = [&](const char *m) { snprintf(msg, len, "%s", m); return TRED_ERR_INVALID_ARG; };
    if (!g) return bad("null geometry");
    if (!(g->pitch_cm > 0 && g->tick_us > 0)) return bad("pitch and tick must be > 0");
    if (g->n_sub < 2 || g->n_sub % 2 || g->n_sub > 32) return bad("n_sub must be even, 2..32");
    if ((int64_t)g->n_sub * g->n_sub * g->bp * g->bp > 6400) return bad("n_sub^2 bp^2 must be <= 6400");
    if (g->bp != 4 && g->bp != 8) return bad("bp must be 4 or 8 (padded extent 16)");
    if (g->kp < 1 || g->kp % 2 == 0 || g->bp + g->kp - 1 > LP) return bad("kp odd with bp + kp - 1 <= 16");
    if (g->lt != 384 && g->lt != 512 && g->lt != 768 && g->lt != 1024) return bad("lt must be 384, 512, 768 or 1024");
    if (g->bt < 64 || g->bt % 64 || g->bt + g->nr - 1 > g->lt) return bad("bt multiple of 64 with bt + nr - 1 <= lt");
    if (g->bt / 64 > g->lt / 64) return bad("bt too large for lt");
    if (g->nr < 1) return bad("nr must be >= 1");
    if (g->npx_x < g->bp || g->npx_y < g->bp || g->npx_x % g->bp || g->npx_y % g->bp)
        return bad("plane must be a multiple of bp pixels");
    if (g->nt < g->bt || g->nt % g->bt) return bad("nt must be a multiple of bt");
    if (g->n_events < 0 || g->n_events > 4096) return bad("n_events must be in [0, 4096]");
    if ((int64_t)g->npx_x * g->n_sub > (1 << 28) ||
        (int64_t)g->npx_y * g->n_sub * (g->n_events > 1 ? g->n_events : 1) > (1 << 28))
        return bad("plane too large");
    return TRED_OK;
}

}  // namespace tred

extern "C" {

static int validate(const tred_geometry *g, const tred_params *p, char *msg, size_t len) {
    auto bad = [&](const char *m) { snprintf(msg, len, "%s", m); return TRED_ERR_INVALID_ARG; };
    if (validate_geometry(g, msg, len) != TRED_OK) return TRED_ERR_INVALID_ARG;
    if (!(p->v_cm_per_us > 0 && p->lifetime_us > 0 && p->DL_cm2_per_s >= 0 && p->DT_cm2_per_s >= 0))
        return bad("bad transport constants");
    if (!(p->sigma0_cells_xy > 0 && p->sigma0_ticks > 0)) return bad("sigma floors must be > 0");
    if (!(p->nsigma > 0 && p->nsigma <= 16)) return bad("nsigma must be in (0, 16]");
    if (!(p->max_drift_cm >= 0)) return bad("max_drift_cm must be >= 0");
    if (p->gl_order < 1 || p->gl_order > MAX_GL) return bad("gl_order must be 1..8");
    if (p->effq_mode != 0 && p->effq_mode != 1) return bad("effq_mode must be 0 or 1");
    if (p->conv_mode < 0 || p->conv_mode > 4) return bad("conv_mode must be 0, 1, 2, 3 or 4");
    if (p->conv_mode >= 1 && p->conv_mode <= 3 && (g->lt != 512 || g->bp != 8))
        return bad("the tensor-core convolution (conv_mode 1, 2, 3) needs lt = 512 and bp = 8");
    if (p->conv_mode == 4 && ((g->lt != 384 && g->lt != 512) || g->kp > 9 || g->n_sub > 10 ||
                             !dx_shape_ok(g->n_sub * g->n_sub, g->lt)))
        return bad("the direct spatial form (conv_mode 4) needs lt = 384 or 512, kp <= 9 and n_sub <= 10");
    if (p->mpcp != 0 && p->mpcp != 1) return bad("mpcp must be 0 or 1");
    if (p->effq_skip_empty != 0 && p->effq_skip_empty != 1) return bad("effq_skip_empty must be 0 or 1");
    if (p->conv_rows_cap < 0 || p->conv_rows_cap % 128) return bad("conv_rows_cap must be a non-negative multiple of 128");
    if (p->conv_keep_spectra != 0 && p->conv_keep_spectra != 1) return bad("conv_keep_spectra must be 0 or 1");
    if (p->effq_skip_empty && p->conv_mode >= 1 && p->conv_mode <= 3)
        return bad("the tensor-core time DFT reads every column: effq_skip_empty must be 0");
    return TRED_OK;
}

int32_t tred_create(const tred_geometry *geom, const tred_params *params, int32_t max_deposits,
                    int32_t max_blocks, int32_t max_pixels, tred_handle **out) {
    if (!out) return TRED_ERR_INVALID_ARG;
    *out = nullptr;
    if (!geom || !params || max_deposits < 1 || max_blocks < 1 || max_pixels < 1)
        return TRED_ERR_INVALID_ARG;
    char msg[256];
    if (validate(geom, params, msg, sizeof msg) != TRED_OK) {
        fprintf(stderr, "tred_create: %s\n", msg);
        return TRED_ERR_INVALID_ARG;
    }
    tred_handle *h = (tred_handle *)calloc(1, sizeof(tred_handle));
    if (!h) return TRED_ERR_CUDA;
    h->g = *geom;
    h->p = *params;
    h->max_deposits = max_deposits;
    h->max_blocks = max_blocks;
    h->max_pixels = max_pixels;
    cudaGetDevice(&h->device);
    Derived &d = h->d;
    d.h = (double)geom->pitch_cm / (double)geom->n_sub;
    d.ngx = geom->npx_x * geom->n_sub;
    d.n_events = geom->n_events > 1 ? geom->n_events : 1;
    d.ngy_e = geom->npx_y * geom->n_sub;
    d.nby_e = geom->npx_y / geom->bp;
    d.npy_e = geom->npx_y;
    d.npy = geom->npx_y * d.n_events;
    d.ngy = d.ngy_e * d.n_events;
    d.nbx = geom->npx_x / geom->bp;
    d.nby = d.nby_e * d.n_events;
    d.nbt = geom->nt / geom->bt;
    d.nblk = (int64_t)d.nbx * d.nby * d.nbt;
    d.R = (geom->kp - 1) / 2;
    d.G = geom->lt / BINS;
    d.npairs = params->mpcp ? geom->n_sub * geom->n_sub / 2 : geom->n_sub * geom->n_sub;
    // Window capacity from the largest drift: width = hi - lo + 3 <= 2 K + 5.  The
    // diffusion constants get a 2x margin so that tred_set_transport may raise them.
    {
        double td = (double)params->max_drift_cm / (double)params->v_cm_per_us;
        double sx = std::sqrt(2.0 * 2.0 * params->DT_cm2_per_s * 1e-6 * td / (d.h * d.h)
                              + (double)params->sigma0_cells_xy * params->sigma0_cells_xy);
        double vt = (double)params->v_cm_per_us * geom->tick_us;
        double st = std::sqrt(2.0 * 2.0 * params->DL_cm2_per_s * 1e-6 * td / (vt * vt)
                              + (double)params->sigma0_ticks * params->sigma0_ticks);
        d.wx = (int)std::ceil(2.0 * params->nsigma * sx * (1 + 1e-9)) + 6;
        d.wt = (int)std::ceil(2.0 * params->nsigma * st * (1 + 1e-9)) + 6;
        d.wx = (d.wx + 3) & ~3;
        d.wt = (d.wt + 3) & ~3;
        d.wstride = 2 * d.wx + d.wt;
    }
    {
        double xi[MAX_GL], wi[MAX_GL];
        gauss_legendre(params->gl_order, xi, wi);
        for (int i = 0; i < params->gl_order; ++i) {
            h->gl_xi[i] = (float)xi[i];
            h->gl_wi[i] = (float)wi[i];
        }
    }
    int rc = TRED_OK;
    auto alloc = [&](void **ptr, size_t bytes, const char *what) {
        if (rc != TRED_OK) return;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) rc = check_cuda(h, e, what);
    };
    const int G = d.G, NP = d.npairs, ns = geom->n_sub;
    alloc((void **)&h->rhat, sizeof(float2) * (size_t)G * NP * BINS * LP * LP, "alloc spectrum");
    alloc((void **)&h->pair_j, sizeof(int32_t) * 2 * NP, "alloc pairs");
    alloc((void **)&h->dep_event, sizeof(int32_t) * (size_t)max_deposits, "alloc deposit events");
    alloc((void **)&h->wts, sizeof(float) * (size_t)max_deposits * d.wstride, "alloc weights");
    alloc((void **)&h->recs, 48 * (size_t)max_deposits, "alloc deposit records");
    alloc((void **)&h->effq_acc, effq_scratch_bytes(geom->bp * ns, num_sms(h)), "alloc effq scratch");
    if (params->conv_mode >= 1 && params->conv_mode <= 3) {
        h->zspec_blocks = max_blocks < 256 ? max_blocks : 256;
        alloc((void **)&h->dft_hi, dft_basis_bytes(geom->bt), "alloc dft basis");
        alloc((void **)&h->dft_lo, dft_basis_bytes(geom->bt), "alloc dft basis");
        alloc((void **)&h->zspec, dft_zspec_bytes(h->zspec_blocks, NP, geom->lt), "alloc packed spectra");
        if (rc == TRED_OK) rc = dft_basis_build(h);
    }
    alloc((void **)&h->blk_count, sizeof(int32_t) * (size_t)d.nblk, "alloc block counts");
    alloc((void **)&h->blk_slot, sizeof(int32_t) * (size_t)d.nblk, "alloc block slots");
    alloc((void **)&h->blk_fill, sizeof(int32_t) * (size_t)max_blocks, "alloc fill");
    h->nchunks = (d.nblk + 1023) / 1024;
    alloc((void **)&h->scan_part, sizeof(int32_t) * (size_t)(2 * h->nchunks + 8), "alloc scan");
    alloc((void **)&h->colmask, sizeof(uint64_t) * (size_t)max_blocks * ns * ns, "alloc masks");
    // blocks per convolution launch pair: 8192 (8.6 GB of spectra at lt = 512) puts a
    // module plane in one launch, so the spectral kernel's last partial wave of
    // (block, class) items comes once per call rather than once per 1024 blocks
    if (params->conv_mode == 4) {
        const int kq = 32 * ((ns * ns + 15) / 16), npad = (geom->kp * geom->kp + 15) & ~15, nbins = geom->lt / 2 + 1;
        const int bp2 = geom->bp * geom->bp;
        h->dx_blocks = params->conv_keep_spectra ? max_blocks : dx_blocks_of(max_blocks);
        h->dx_rows_cap = dx_rows_cap_of(h->dx_blocks, bp2, params->conv_rows_cap);
        alloc((void **)&h->dx_bhi, dx_bytes_b(nbins, npad, kq), "alloc direct-form response");
        alloc((void **)&h->dx_blo, dx_bytes_b(nbins, npad, kq), "alloc direct-form response");
        alloc((void **)&h->dx_qhi, dx_bytes_q(nbins, h->dx_rows_cap, kq), "alloc direct-form spectra");
        alloc((void **)&h->dx_qlo, dx_bytes_q(nbins, h->dx_rows_cap, kq), "alloc direct-form spectra");
        // the K positions of the impacts past n_sub^2 (padding of the last group of 16) are
        // never written and must read as zero
        if (rc == TRED_OK) rc = check_cuda(h, cudaMemset(h->dx_qhi, 0, dx_bytes_q(nbins, h->dx_rows_cap, kq)), "clear spectra");
        if (rc == TRED_OK) rc = check_cuda(h, cudaMemset(h->dx_qlo, 0, dx_bytes_q(nbins, h->dx_rows_cap, kq)), "clear spectra");
        alloc((void **)&h->dx_y, sizeof(float2) * (size_t)h->dx_blocks * nbins * LP * LP, "alloc direct-form output");
        alloc((void **)&h->dx_rows, sizeof(int32_t) * (size_t)h->dx_blocks * bp2, "alloc direct-form rows");
        alloc((void **)&h->dx_rowstart, sizeof(int32_t) * ((size_t)h->dx_blocks + 2), "alloc direct-form rows");
        alloc((void **)&h->dx_meta, sizeof(int32_t) * 8, "alloc direct-form rows");
        if (rc == TRED_OK) rc = check_cuda(h, cudaMemset(h->dx_meta, 0, sizeof(int32_t) * 8), "clear direct-form rows");
        alloc((void **)&h->dx_pmask, sizeof(uint64_t) * (size_t)h->dx_blocks, "alloc direct-form masks");
        alloc((void **)&h->dx_pcnt, sizeof(int32_t) * (size_t)h->dx_blocks, "alloc direct-form counts");
        h->dx_ntiles = d.n_events * (d.nby_e + 1) * (d.nbx + 1);
        alloc((void **)&h->dx_tflag, sizeof(int32_t) * (size_t)h->dx_ntiles, "alloc direct-form tiles");
        alloc((void **)&h->dx_tpart, sizeof(int32_t) * ((size_t)h->dx_ntiles / 1024 + 8), "alloc direct-form tiles");
        alloc((void **)&h->dx_tlist, sizeof(int32_t) * (size_t)h->dx_ntiles, "alloc direct-form tiles");
        alloc((void **)&h->dx_tcount, sizeof(int32_t) * 8, "alloc direct-form tiles");
    } else {
        h->yspec_blocks = max_blocks < 8192 ? max_blocks : 8192;
        alloc((void **)&h->yspec, sizeof(float2) * (size_t)h->yspec_blocks * geom->lt * LP * LP, "alloc yspec");
    }
    alloc((void **)&h->pix_flag, sizeof(int32_t) * (size_t)geom->npx_x * d.npy, "alloc pixel flags");
    h->pix_chunks = ((int64_t)geom->npx_x * d.npy + 1023) / 1024;
    alloc((void **)&h->pix_part, sizeof(int32_t) * (size_t)(h->pix_chunks + 8), "alloc pixel scan");
    alloc((void **)&h->px_possum, sizeof(float) * ((size_t)max_pixels + 8), "alloc pixel bounds");
    alloc((void **)&h->hit_cnt, sizeof(int32_t) * ((size_t)max_pixels + 8 + (size_t)max_pixels / 1024 + 8),
          "alloc hit counts");   // counts and their scan, then the scan's chunk sums
    alloc((void **)&h->hit_tmp, sizeof(int32_t) * (size_t)max_pixels * HIT_TMP, "alloc hit cache");
    alloc((void **)&h->hit_tmpc, sizeof(float) * (size_t)max_pixels * HIT_TMP, "alloc hit cache");
    alloc((void **)&h->status, sizeof(int32_t) * TRED_STATUS_WORDS, "alloc status");
    alloc((void **)&h->tw, sizeof(float2) * TW_TOTAL, "alloc twiddles");
    if (rc == TRED_OK) {
        std::vector<float2> tw(TW_TOTAL, make_float2(0.f, 0.f));
        auto fill = [&](int off, int N) {
            for (int k = 0; k < N; ++k) {
                double a = 2.0 * M_PI * (double)k / (double)N;
                tw[off + k] = make_float2((float)std::cos(a), (float)-std::sin(a));
            }
        };
        fill(TW_32, 32);
        fill(TW_64, 64);
        fill(TW_16, 16);
        fill(TW_8, 8);
        fill(TW_LT, geom->lt);
        rc = check_cuda(h, cudaMemcpy(h->tw, tw.data(), sizeof(float2) * TW_TOTAL, cudaMemcpyHostToDevice), "copy twiddles");
        std::vector<int32_t> pj(2 * NP);
        int k = 0;
        for (int jy = 0; jy < ns; ++jy)
            for (int jx = 0; jx < ns; ++jx) {
                if (params->mpcp) {
                    if (jy >= ns / 2) continue;
                    pj[2 * k] = jy * ns + jx;
                    pj[2 * k + 1] = (ns - 1 - jy) * ns + (ns - 1 - jx);
                } else {
                    pj[2 * k] = jy * ns + jx;
                    pj[2 * k + 1] = -1;
                }
                ++k;
            }
        if (rc == TRED_OK)
            rc = check_cuda(h, cudaMemcpy(h->pair_j, pj.data(), sizeof(int32_t) * 2 * NP, cudaMemcpyHostToDevice), "copy pairs");
        if (rc == TRED_OK)
            rc = check_cuda(h, cudaMemset(h->status, 0, sizeof(int32_t) * TRED_STATUS_WORDS), "clear status");
    }
    if (rc != TRED_OK) {
        fprintf(stderr, "tred_create: %s\n", h->err);
        tred_destroy(h);
        return rc;
    }
    *out = h;
    return TRED_OK;
}

int32_t tred_destroy(tred_handle *h) {
    if (!h) return TRED_ERR_INVALID_ARG;
    void *ptrs[] = {h->dep_event, h->wts2, h->pix_row, h->gspec, h->rhat, h->pair_j, h->wts, h->recs, h->effq_acc, h->dft_hi, h->dft_lo, h->zspec, h->blk_count, h->blk_slot, h->blk_fill,
                    h->scan_part, h->colmask, h->yspec, h->pix_flag, h->pix_part, h->px_possum, h->hit_cnt,
                    h->hit_tmp, h->hit_tmpc, h->status, h->tw, h->dx_bhi, h->dx_blo, h->dx_qhi, h->dx_qlo,
                    h->dx_y, h->dx_rows, h->dx_rowstart, h->dx_meta, h->dx_pmask, h->dx_pcnt, h->dx_tflag,
                    h->dx_tpart, h->dx_tlist, h->dx_tcount};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete h->kt;
    free(h);
    return TRED_OK;
}

int32_t tred_sync_status(tred_handle *h, void *stream, int32_t *host_status) {
    if (!h || !host_status) return TRED_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_cuda(h, cudaMemcpyAsync(host_status, h->status, sizeof(int32_t) * TRED_STATUS_WORDS,
                                           cudaMemcpyDeviceToHost, s), "read status");
    if (rc) return rc;
    return check_cuda(h, cudaStreamSynchronize(s), "sync status");
}

int32_t tred_set_transport(tred_handle *h, const tred_params *params) {
    if (!h || !params) return TRED_ERR_INVALID_ARG;
    if (params->gl_order != h->p.gl_order || params->effq_mode != h->p.effq_mode || params->mpcp != h->p.mpcp ||
        params->conv_mode != h->p.conv_mode)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_set_transport: only transport constants may change");
    // the transport constants only: every other field keeps the value tred_create set
    tred_params np = h->p;
    np.v_cm_per_us = params->v_cm_per_us;
    np.DL_cm2_per_s = params->DL_cm2_per_s;
    np.DT_cm2_per_s = params->DT_cm2_per_s;
    np.lifetime_us = params->lifetime_us;
    np.sigma0_cells_xy = params->sigma0_cells_xy;
    np.sigma0_ticks = params->sigma0_ticks;
    np.nsigma = params->nsigma;
    np.max_drift_cm = params->max_drift_cm;
    char msg[256];
    if (validate(&h->g, &np, msg, sizeof msg) != TRED_OK) return set_error(h, TRED_ERR_INVALID_ARG, "%s", msg);
    const double td = (double)np.max_drift_cm / (double)np.v_cm_per_us;
    const double sx = std::sqrt(2.0 * np.DT_cm2_per_s * 1e-6 * td / (h->d.h * h->d.h) +
                                (double)np.sigma0_cells_xy * np.sigma0_cells_xy);
    const double vt = (double)np.v_cm_per_us * h->g.tick_us;
    const double st = std::sqrt(2.0 * np.DL_cm2_per_s * 1e-6 * td / (vt * vt) +
                                (double)np.sigma0_ticks * np.sigma0_ticks);
    if ((int)std::ceil(2.0 * np.nsigma * sx) + 6 > h->d.wx || (int)std::ceil(2.0 * np.nsigma * st) + 6 > h->d.wt)
        return set_error(h, TRED_ERR_CAPACITY, "tred_set_transport: diffusion beyond the window capacity of tred_create");
    h->p = np;
    return TRED_OK;
}

int32_t tred_residual(tred_handle *h, const int32_t *pixel_ids, const int32_t *n_pixels_dev, const float *waveforms,
                      const int32_t *target_ids, int32_t n_target, const float *target_waves, float *resid,
                      double *loss_dev, void *stream) {
    tred::CallRange range_("tred_residual");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!pixel_ids || !n_pixels_dev || !waveforms || !resid || !loss_dev || n_target < 0 ||
        (n_target > 0 && (!target_ids || !target_waves)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_residual: null pointer");
    return launch_residual(h, pixel_ids, n_pixels_dev, waveforms, target_ids, n_target, target_waves, resid, loss_dev,
                           (cudaStream_t)stream);
}

int32_t tred_adjoint(tred_handle *h, int32_t n, const tred_deposits *deps, const int32_t *block_ids,
                     const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                     const int32_t *pixel_ids, const int32_t *n_pixels_dev, const float *resid, float *dqeff,
                     float *grad7, void *stream) {
    tred::CallRange range_("tred_adjoint");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!h->response_ready) return set_error(h, TRED_ERR_NOT_READY, "tred_adjoint: call tred_set_response first");
    if (h->p.effq_mode != 0) return set_error(h, TRED_ERR_INVALID_ARG, "tred_adjoint: Gauss-Legendre mode only");
    if (n < 0 || n > h->max_deposits) return set_error(h, TRED_ERR_CAPACITY, "tred_adjoint: bad n");
    if ((n > 0 && (!deps_ok(deps) || !grad7)) || !block_ids || !dep_offsets || !dep_index || !n_blocks_dev ||
        !pixel_ids || !n_pixels_dev || !resid || !dqeff)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_adjoint: null pointer");
    if (!h->wts2) {   // first call: adjoint scratch
        // blocks per backward sub-batch: 256 keep every SM busy over ~14 waves of (block,
        // class) items (32 left the second of two waves three quarters full), 3.4 GB of spectra
        h->adj_chunk = h->max_blocks < 256 ? h->max_blocks : 256;
        const size_t b1 = sizeof(float) * 3 * (size_t)h->max_deposits * h->d.wstride;
        const size_t b2 = sizeof(int32_t) * (size_t)h->g.npx_x * h->d.npy;
        const size_t b3 = sizeof(float2) * (size_t)h->adj_chunk * h->d.npairs * h->g.lt * 64;
        int rc = check_cuda(h, cudaMalloc(&h->wts2, b1), "alloc adjoint weights");
        if (!rc) rc = check_cuda(h, cudaMalloc(&h->pix_row, b2), "alloc pixel rows");
        if (!rc) rc = check_cuda(h, cudaMalloc(&h->gspec, b3), "alloc adjoint spectra");
        if (rc) return rc;
    }
    return launch_adjoint(h, n, n > 0 ? *deps : tred_deposits{}, block_ids, dep_offsets, dep_index, n_blocks_dev,
                          pixel_ids, n_pixels_dev, resid, dqeff, grad7, (cudaStream_t)stream);
}

int32_t tred_param_grads(tred_handle *h, int32_t n, const float *z, const tred_deposits *deps, const float *grad7,
                         float *grad_inputs, double *grad_global, void *stream) {
    tred::CallRange range_("tred_param_grads");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits || (n > 0 && (!z || !deps_ok(deps) || !grad7 || !grad_inputs)) || !grad_global)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_param_grads: bad arguments");
    return launch_param_grads(h, n, z, n > 0 ? *deps : tred_deposits{}, grad7, grad_inputs, grad_global,
                              (cudaStream_t)stream);
}

int32_t tred_launch_count(const tred_handle *h, int64_t *count) {
    if (!h || !count) return TRED_ERR_INVALID_ARG;
    *count = h->launches;
    return TRED_OK;
}

int32_t tred_direct_counts(tred_handle *h, int64_t *rows, int64_t *columns) {
    if (!h || !rows || !columns) return TRED_ERR_INVALID_ARG;
    *rows = 0;
    *columns = 0;
    if (h->p.conv_mode != 4) return TRED_OK;
    unsigned long long acc[2] = {0, 0};
    int rc = check_cuda(h, cudaMemcpy(acc, h->dx_meta + 4, sizeof acc, cudaMemcpyDeviceToHost), "read direct-form counts");
    if (!rc) rc = check_cuda(h, cudaMemset(h->dx_meta + 4, 0, sizeof acc), "reset direct-form counts");
    if (rc) return rc;
    *rows = (int64_t)acc[0];
    *columns = (int64_t)acc[1];
    return TRED_OK;
}

int32_t tred_set_kernel_timing(tred_handle *h, int32_t enable) {
    if (!h) return TRED_ERR_INVALID_ARG;
    if (enable && !h->kt) h->kt = new KernelTimers();
    if (!enable && h->kt) {
        cudaDeviceSynchronize();   // the recorded events are complete before they go
        delete h->kt;
        h->kt = nullptr;
    }
    return TRED_OK;
}

int32_t tred_kernel_time(tred_handle *h, int32_t which, double *ms, int32_t *launches) {
    if (!h || !ms || !launches || which < 0 || which >= TRED_KT_CLASSES) return TRED_ERR_INVALID_ARG;
    *ms = 0.0;
    *launches = 0;
    if (!h->kt) return TRED_OK;
    auto &v = h->kt->pairs[which];
    for (auto &p : v) {
        int rc = check_cuda(h, cudaEventSynchronize(p.second), "kernel timing");
        if (rc) return rc;
        float t = 0.f;
        rc = check_cuda(h, cudaEventElapsedTime(&t, p.first, p.second), "kernel timing");
        if (rc) return rc;
        *ms += t;
        *launches += 1;
        h->kt->pool.push_back(p.first);
        h->kt->pool.push_back(p.second);
    }
    v.clear();
    return TRED_OK;
}

int32_t tred_reset_status(tred_handle *h, void *stream) {
    if (!h) return TRED_ERR_INVALID_ARG;
    return check_cuda(h, cudaMemsetAsync(h->status, 0, sizeof(int32_t) * TRED_STATUS_WORDS,
                                         (cudaStream_t)stream), "reset status");
}

int32_t tred_set_response(tred_handle *h, const float *resp_dev, void *stream) {
    tred::CallRange range_("tred_set_response");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!resp_dev) return set_error(h, TRED_ERR_INVALID_ARG, "tred_set_response: null response");
    int rc = launch_response(h, resp_dev, (cudaStream_t)stream);
    if (rc == TRED_OK && h->p.conv_mode == 4) rc = launch_direct_response(h, resp_dev, (cudaStream_t)stream);
    if (rc == TRED_OK) h->response_ready = true;
    return rc;
}


int32_t tred_drift(tred_handle *h, int32_t n, const float *x, const float *y, const float *z,
                   const float *t0, const float *ne, const tred_deposits *out, void *stream) {
    tred::CallRange range_("tred_drift");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_drift: n=%d outside [0, max_deposits=%d]", n, h->max_deposits);
    if (n > 0 && (!x || !y || !z || !t0 || !ne || !deps_ok(out)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_drift: null pointer");
    if (n == 0) return TRED_OK;
    return launch_drift(h, n, x, y, z, t0, ne, nullptr, *out, (cudaStream_t)stream);
}

int32_t tred_drift_lines(tred_handle *h, int32_t n, const float *x0, const float *y0, const float *z0,
                         const float *x1, const float *y1, const float *z1, const float *t0, const float *ne,
                         const tred_deposits *out, float *half, void *stream) {
    tred::CallRange range_("tred_drift_lines");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_drift_lines: n=%d outside [0, max_deposits=%d]", n, h->max_deposits);
    if (n > 0 && (!x0 || !y0 || !z0 || !x1 || !y1 || !z1 || !t0 || !ne || !half || !deps_ok(out)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_drift_lines: null pointer");
    if (h->d.n_events > 1) return set_error(h, TRED_ERR_INVALID_ARG, "tred_drift_lines: single-event handles only");
    if (n == 0) return TRED_OK;
    return launch_drift_lines(h, n, x0, y0, z0, x1, y1, z1, t0, ne, *out, half, (cudaStream_t)stream);
}

int32_t tred_effq_lines(tred_handle *h, int32_t n, const tred_deposits *deps, const float *half,
                        const int32_t *block_ids, const int32_t *dep_offsets, const int32_t *dep_index,
                        const int32_t *n_blocks_dev, float *qeff, void *stream) {
    tred::CallRange range_("tred_effq_lines");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_effq_lines: n=%d outside [0, max_deposits]", n);
    if ((n > 0 && (!deps_ok(deps) || !half)) || !block_ids || !dep_offsets || !dep_index || !n_blocks_dev || !qeff)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq_lines: null pointer");
    return launch_effq_lines(h, n, n > 0 ? *deps : tred_deposits{}, half, block_ids, dep_offsets, dep_index,
                             n_blocks_dev, qeff, (cudaStream_t)stream);
}

int32_t tred_drift_events(tred_handle *h, int32_t n, const float *x, const float *y, const float *z,
                          const float *t0, const float *ne, const int32_t *event, const tred_deposits *out,
                          void *stream) {
    tred::CallRange range_("tred_drift_events");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_drift_events: n=%d outside [0, max_deposits=%d]", n,
                         h->max_deposits);
    if (n > 0 && (!x || !y || !z || !t0 || !ne || !event || !deps_ok(out)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_drift_events: null pointer");
    if (n == 0) return TRED_OK;
    return launch_drift(h, n, x, y, z, t0, ne, event, *out, (cudaStream_t)stream);
}

int32_t tred_blockbin(tred_handle *h, int32_t n, const tred_deposits *deps, int32_t *block_ids,
                      int32_t *block_counts, int32_t *dep_offsets, int32_t *dep_index,
                      int32_t max_pairs, int32_t *n_blocks_dev, void *stream) {
    tred::CallRange range_("tred_blockbin");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_blockbin: n=%d outside [0, max_deposits]", n);
    if ((n > 0 && !deps_ok(deps)) || !block_ids || !block_counts || !dep_offsets || !n_blocks_dev ||
        (max_pairs > 0 && !dep_index) || max_pairs < 0)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_blockbin: null pointer or bad max_pairs");
    return launch_blockbin(h, n, n > 0 ? *deps : tred_deposits{}, block_ids, block_counts, dep_offsets,
                           dep_index, max_pairs, n_blocks_dev, (cudaStream_t)stream);
}

int32_t tred_effq(tred_handle *h, int32_t n, const tred_deposits *deps, const int32_t *block_ids,
                  const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                  float *qeff, void *stream) {
    tred::CallRange range_("tred_effq");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_effq: n=%d outside [0, max_deposits]", n);
    if ((n > 0 && !deps_ok(deps)) || !block_ids || !dep_offsets || !n_blocks_dev || !qeff)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq: null pointer");
    return launch_effq(h, n, n > 0 ? *deps : tred_deposits{}, block_ids, dep_offsets, dep_index,
                       n_blocks_dev, qeff, 0, h->max_blocks, (cudaStream_t)stream);
}

int32_t tred_effq_range(tred_handle *h, int32_t n, const tred_deposits *deps, const int32_t *block_ids,
                        const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                        int32_t slot_base, int32_t slot_count, float *qeff, void *stream) {
    tred::CallRange range_("tred_effq_range");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_effq_range: n=%d outside [0, max_deposits]", n);
    if ((n > 0 && !deps_ok(deps)) || !block_ids || !dep_offsets || !n_blocks_dev || !qeff || slot_base < 0 ||
        slot_count < 0)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq_range: bad arguments");
    return launch_effq(h, n, n > 0 ? *deps : tred_deposits{}, block_ids, dep_offsets, dep_index, n_blocks_dev,
                       qeff, slot_base, slot_count, (cudaStream_t)stream);
}

int32_t tred_effq_convolve(tred_handle *h, int32_t n, const tred_deposits *deps, const int32_t *block_ids,
                           const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                           float *qeff_ring, int32_t ring_rows, float *out_blocks, void *stream) {
    tred::CallRange range_("tred_effq_convolve");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!h->response_ready)
        return set_error(h, TRED_ERR_NOT_READY, "tred_effq_convolve: call tred_set_response first");
    if (n < 0 || n > h->max_deposits)
        return set_error(h, TRED_ERR_CAPACITY, "tred_effq_convolve: n=%d outside [0, max_deposits]", n);
    if ((n > 0 && !deps_ok(deps)) || !block_ids || !dep_offsets || !dep_index || !n_blocks_dev || !qeff_ring ||
        ring_rows < 1 || !out_blocks)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq_convolve: bad arguments");
    return launch_pipeline(h, n, n > 0 ? *deps : tred_deposits{}, block_ids, dep_offsets, dep_index, n_blocks_dev,
                           qeff_ring, ring_rows, out_blocks, (cudaStream_t)stream);
}

int32_t tred_convolve(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                      const float *qeff, float *out_blocks, void *stream) {
    tred::CallRange range_("tred_convolve");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!h->response_ready)
        return set_error(h, TRED_ERR_NOT_READY, "tred_convolve: call tred_set_response first");
    if (!block_ids || !n_blocks_dev || !qeff || !out_blocks)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_convolve: null pointer");
    return launch_convolve(h, block_ids, n_blocks_dev, qeff, out_blocks, 0, h->max_blocks, (cudaStream_t)stream);
}

int32_t tred_convolve_range(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                            int32_t slot_base, int32_t slot_count, const float *qeff, float *out_blocks,
                            void *stream) {
    tred::CallRange range_("tred_convolve_range");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!h->response_ready)
        return set_error(h, TRED_ERR_NOT_READY, "tred_convolve_range: call tred_set_response first");
    if (!block_ids || !n_blocks_dev || !qeff || !out_blocks || slot_base < 0 || slot_count < 0)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_convolve_range: bad arguments");
    return launch_convolve(h, block_ids, n_blocks_dev, qeff, out_blocks, slot_base, slot_count,
                           (cudaStream_t)stream);
}

int32_t tred_gather_pixels(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                           const float *out_blocks, int32_t *pixel_ids, float *waveforms,
                           int32_t *n_pixels_dev, void *stream) {
    tred::CallRange range_("tred_gather_pixels");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!block_ids || !n_blocks_dev || !out_blocks || !pixel_ids || !waveforms || !n_pixels_dev)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_gather_pixels: null pointer");
    return launch_gather(h, block_ids, n_blocks_dev, out_blocks, pixel_ids, waveforms, n_pixels_dev,
                         (cudaStream_t)stream);
}

int32_t tred_readout(tred_handle *h, const tred_readout_params *rp, const int32_t *pixel_ids,
                     const float *waveforms, const int32_t *n_pixels_dev, int32_t *hit_pixel,
                     int32_t *hit_tick, float *hit_charge, int32_t *n_hits_dev, int32_t max_hits,
                     void *stream) {
    tred::CallRange range_("tred_readout");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!rp || !pixel_ids || !waveforms || !n_pixels_dev || !n_hits_dev || max_hits < 0 ||
        (max_hits > 0 && (!hit_pixel || !hit_tick || !hit_charge)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_readout: null pointer");
    if (rp->clock_ticks < 1 || rp->hold_ticks < 0 || rp->reset_ticks < 0 || rp->mode < 0 || rp->mode > 2 ||
        (rp->mode == 1 && (rp->n_samples < 1 || rp->hold_ticks < 1)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_readout: bad readout parameters");
    return launch_readout(h, *rp, pixel_ids, waveforms, n_pixels_dev, hit_pixel, hit_tick, hit_charge,
                          n_hits_dev, max_hits, (cudaStream_t)stream);
}

int32_t tred_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                            const float *out_blocks, int32_t *pixel_ids, float *waveforms, int32_t *n_pixels_dev,
                            const tred_readout_params *rp, int32_t *hit_pixel, int32_t *hit_tick, float *hit_charge,
                            int32_t *n_hits_dev, int32_t max_hits, void *stream) {
    tred::CallRange range_("tred_gather_readout");
    if (!h) return TRED_ERR_INVALID_ARG;
    if (!block_ids || !n_blocks_dev || !out_blocks || !pixel_ids || !waveforms || !n_pixels_dev || !rp ||
        !n_hits_dev || max_hits < 0 || (max_hits > 0 && (!hit_pixel || !hit_tick || !hit_charge)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_gather_readout: null pointer");
    if (rp->clock_ticks < 1 || rp->hold_ticks < 0 || rp->reset_ticks < 0 || rp->mode < 0 || rp->mode > 2 ||
        (rp->mode == 1 && (rp->n_samples < 1 || rp->hold_ticks < 1)))
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_gather_readout: bad readout parameters");
    const cudaStream_t s = (cudaStream_t)stream;
    const int rc = launch_gather(h, block_ids, n_blocks_dev, out_blocks, pixel_ids, waveforms, n_pixels_dev, s,
                                 h->px_possum);
    if (rc) return rc;
    return launch_readout(h, *rp, pixel_ids, waveforms, n_pixels_dev, hit_pixel, hit_tick, hit_charge, n_hits_dev,
                          max_hits, s, h->px_possum);
}

int32_t tred_convolve_gather_supported(const tred_handle *h) {
    if (!h) return -1;
    return dx_wave_ok(h) ? 1 : 0;
}

static int wave_args_ok(tred_handle *h, const char *fn, const tred_readout_params *rp, int32_t *hit_pixel,
                        int32_t *hit_tick, float *hit_charge, int32_t *n_hits_dev, int32_t max_hits) {
    if (rp && (!n_hits_dev || max_hits < 0 || (max_hits > 0 && (!hit_pixel || !hit_tick || !hit_charge))))
        return set_error(h, TRED_ERR_INVALID_ARG, "%s: null hit buffers", fn);
    if (rp && (rp->clock_ticks < 1 || rp->hold_ticks < 0 || rp->reset_ticks < 0 || rp->mode < 0 || rp->mode > 2 ||
               (rp->mode == 1 && (rp->n_samples < 1 || rp->hold_ticks < 1))))
        return set_error(h, TRED_ERR_INVALID_ARG, "%s: bad readout parameters", fn);
    return TRED_OK;
}

static int wave_shape_ok(tred_handle *h, const char *fn) {
    if (!h->response_ready) return set_error(h, TRED_ERR_NOT_READY, "%s: call tred_set_response first", fn);
    if (!dx_wave_ok(h))
        return set_error(h, TRED_ERR_INVALID_ARG,
                         "%s: needs conv_mode 4, bp 8, kp 9, nr - 1 <= bt, nt / bt <= 128, max_blocks within one "
                         "pass (or conv_keep_spectra 1) and compensated_gather 0",
                         fn);
    return TRED_OK;
}

// pixel list, the fused inverse time DFT + gather, and the readout (rp non-null)
static int wave_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                               int32_t *pixel_ids, float *waveforms, int32_t *n_pixels_dev,
                               const tred_readout_params *rp, int32_t *hit_pixel, int32_t *hit_tick,
                               float *hit_charge, int32_t *n_hits_dev, int32_t max_hits, cudaStream_t s) {
    int32_t *queue = nullptr;
    int rc = launch_pixel_list(h, block_ids, n_blocks_dev, pixel_ids, n_pixels_dev, s, &queue);
    if (rc) return rc;
    rc = launch_direct_wave(h, block_ids, n_blocks_dev, queue, waveforms, h->px_possum, s);
    if (rc || !rp) return rc;
    return launch_readout(h, *rp, pixel_ids, waveforms, n_pixels_dev, hit_pixel, hit_tick, hit_charge, n_hits_dev,
                          max_hits, s, h->px_possum);
}

int32_t tred_convolve_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                                     const float *qeff, int32_t *pixel_ids, float *waveforms, int32_t *n_pixels_dev,
                                     const tred_readout_params *rp, int32_t *hit_pixel, int32_t *hit_tick,
                                     float *hit_charge, int32_t *n_hits_dev, int32_t max_hits, void *stream) {
    tred::CallRange range_("tred_convolve_gather_readout");
    const char *fn = "tred_convolve_gather_readout";
    if (!h) return TRED_ERR_INVALID_ARG;
    int rc = wave_shape_ok(h, fn);
    if (rc) return rc;
    if (!block_ids || !n_blocks_dev || !qeff || !pixel_ids || !waveforms || !n_pixels_dev)
        return set_error(h, TRED_ERR_INVALID_ARG, "%s: null pointer", fn);
    rc = wave_args_ok(h, fn, rp, hit_pixel, hit_tick, hit_charge, n_hits_dev, max_hits);
    if (rc) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    rc = launch_direct_spectra(h, n_blocks_dev, qeff, 0, h->max_blocks, s);
    if (rc) return rc;
    return wave_gather_readout(h, block_ids, n_blocks_dev, pixel_ids, waveforms, n_pixels_dev, rp, hit_pixel,
                               hit_tick, hit_charge, n_hits_dev, max_hits, s);
}

int32_t tred_convolve_spectra_range(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                                    int32_t slot_base, int32_t slot_count, const float *qeff, void *stream) {
    tred::CallRange range_("tred_convolve_spectra_range");
    const char *fn = "tred_convolve_spectra_range";
    if (!h) return TRED_ERR_INVALID_ARG;
    int rc = wave_shape_ok(h, fn);
    if (rc) return rc;
    if (!h->p.conv_keep_spectra && slot_base > 0)
        return set_error(h, TRED_ERR_INVALID_ARG, "%s: slot ranges past slot 0 need conv_keep_spectra 1", fn);
    if (!block_ids || !n_blocks_dev || !qeff || slot_base < 0 || slot_count < 0)
        return set_error(h, TRED_ERR_INVALID_ARG, "%s: bad arguments", fn);
    const int count = slot_count < h->max_blocks - slot_base ? slot_count : h->max_blocks - slot_base;
    if (count <= 0) return TRED_OK;
    return launch_direct_spectra(h, n_blocks_dev, qeff, slot_base, count, (cudaStream_t)stream);
}

int32_t tred_wave_gather_readout(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                                 int32_t *pixel_ids, float *waveforms, int32_t *n_pixels_dev,
                                 const tred_readout_params *rp, int32_t *hit_pixel, int32_t *hit_tick,
                                 float *hit_charge, int32_t *n_hits_dev, int32_t max_hits, void *stream) {
    tred::CallRange range_("tred_wave_gather_readout");
    const char *fn = "tred_wave_gather_readout";
    if (!h) return TRED_ERR_INVALID_ARG;
    int rc = wave_shape_ok(h, fn);
    if (rc) return rc;
    if (!block_ids || !n_blocks_dev || !pixel_ids || !waveforms || !n_pixels_dev)
        return set_error(h, TRED_ERR_INVALID_ARG, "%s: null pointer", fn);
    rc = wave_args_ok(h, fn, rp, hit_pixel, hit_tick, hit_charge, n_hits_dev, max_hits);
    if (rc) return rc;
    return wave_gather_readout(h, block_ids, n_blocks_dev, pixel_ids, waveforms, n_pixels_dev, rp, hit_pixel,
                               hit_tick, hit_charge, n_hits_dev, max_hits, (cudaStream_t)stream);
}

int32_t tred_wait_selftest(tred_handle *h, int64_t limit_cycles, void *stream) {
    if (!h) return TRED_ERR_INVALID_ARG;
    if (limit_cycles < 1 || limit_cycles > 2000000000ll)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_wait_selftest: limit must be in [1, 2e9] cycles");
    return launch_wait_selftest(h, (long long)limit_cycles, (cudaStream_t)stream);
}

}  // extern "C"
