// Internal declarations of libtred: the handle, launch helpers and the small
// in-register / cross-lane FFT building blocks the kernels share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "../../include/tred.h"

namespace tred {

constexpr int LP = 16;               // padded spatial FFT extent (pixels per axis)
constexpr int BINS = 64;             // time-frequency bins of one adjoint spectral CTA
constexpr int CBINS = 32;            // bins of one convolution class: f = k1 + G2 k2, G2 = lt / 32
// offset of bin f of channel pair p in the response spectrum rhat[f mod G2][p][f div G2][16 x 16]
// (the plane's order: rhat_kk)
__host__ __device__ inline size_t rhat_bin(int f, int p, int npairs, int G2) {
    return (((size_t)(f % G2) * npairs + p) * CBINS + f / G2) * (size_t)(LP * LP);
}
// position of (ky, kx) inside one bin's 16 x 16 plane of the response spectrum: the ky
// pairs (2q, 2q + 1) of one kx are adjacent, so that a lane holding one kx reads two ky
// values per 16-byte load and the 16 lanes of a bin read 256 contiguous bytes per load
__host__ __device__ constexpr int rhat_kk(int ky, int kx) { return (ky >> 1) * (2 * LP) + 2 * kx + (ky & 1); }
constexpr int MAX_GL = 8;

struct Derived {
    int ngx, ngy;          // sub-cell grid size (y: all events)
    int nbx, nby, nbt;     // blocks per axis (y: all events)
    int n_events;          // events stacked along y
    int ngy_e, nby_e, npy_e;  // sub-cells, blocks and pixels of one event along y
    int npy;               // pixel rows of all events
    int64_t nblk;          // blocks in the plane
    int R;                 // response half width in pixels
    int G;                 // time-frequency classes = lt / 64
    int npairs;            // packed channels (n_sub^2 / 2 with MPCP, else n_sub^2)
    int wx, wt;            // per-deposit weight capacity per axis (x/y, t)
    int wstride;           // floats per deposit in the weight buffer
    double h;              // sub-cell size (cm)
};

}  // namespace tred

struct tred_handle {
    tred_geometry g;
    tred_params p;
    int32_t max_deposits, max_blocks, max_pixels;
    tred::Derived d;
    int device;
    bool response_ready;
    // device memory owned by the handle
    float2 *rhat;          // [G][npairs][64][16*16] response spectrum
    int32_t *pair_j;       // [npairs][2] impact channel indices (second = -1 without MPCP)
    int32_t *dep_event;    // [max_deposits] event of each deposit (written by drift)
    float *wts;            // [max_deposits][wstride] per-deposit 1-D weights
    void *recs;            // [max_deposits] 48-byte per-deposit records for effq
    int32_t *effq_acc;     // per-CTA integer partial sums of multi-pass effq tiles + block queue
    float *dft_hi, *dft_lo;  // tensor-core form: [512][bt] real DFT basis, TF32 part and residual
    float2 *zspec;         // tensor-core form: [zspec_blocks][G][npairs][64][64] packed spectra
    int32_t zspec_blocks;
    // direct spatial form (conv_mode 4): per time frequency, the sum over impacts and
    // response taps as a split-BF16 tensor-core GEMM over the non-empty block pixels
    uint16_t *dx_bhi, *dx_blo;  // [nbins][npad][kq] response operand (BF16 hi and lo parts)
                                // (kq = 32 ceil(n_sub^2 / 16), npad = kp^2 rounded up to 16)
    uint16_t *dx_qhi, *dx_qlo;  // [nbins][dx_rows_cap][kq] charge spectra of the rows
    float2 *dx_y;               // [dx_blocks][nbins][16 * 16] block output spectra
    int32_t *dx_rows;           // [dx_blocks * bp^2] row records: local slot << 6 | pixel
    int32_t *dx_rowstart;       // [dx_blocks + 1] first row of each slot, then the row count
    int32_t *dx_meta;           // [8]: slots, rows and non-empty columns of the pass; at 4: running totals (2 x 64 bit)
    uint64_t *dx_pmask;         // [dx_blocks] non-empty pixels of each slot
    int32_t *dx_pcnt;           // [dx_blocks] non-empty columns of each slot
    int32_t dx_blocks, dx_rows_cap;
    int32_t *dx_tflag, *dx_tpart, *dx_tlist, *dx_tcount;   // fused gather: pixel tiles touched by active
                                                           // blocks (flags, scan scratch, list, count)
    int32_t dx_ntiles;                                     // n_events (nby_e + 1) (nbx + 1)
    int32_t *blk_count;    // [nblk] occupancy
    int32_t *blk_slot;     // [nblk] slot of an active block or -1
    int32_t *blk_fill;     // [max_blocks] CSR fill cursors
    int32_t *scan_part;    // [2 * nchunks + 4] scan partials
    int64_t nchunks;
    uint64_t *colmask;     // [max_blocks][n_sub^2] non-empty columns of each channel slab
    float2 *yspec;         // [yspec_blocks][lt][16*16] spatially inverted spectra
    int32_t yspec_blocks;
    int32_t *pix_flag;     // [npx_x * npx_y] active pixel flags, then row index
    int32_t *pix_part;     // pixel scan partials
    float *px_possum;      // [max_pixels] sum of the positive current per pixel row (fused readout)
    int64_t pix_chunks;
    int32_t *hit_cnt;      // [max_pixels + 1] hits per pixel then offsets; from max_pixels + 8 the scan's chunk sums
    int32_t *hit_tmp;      // [max_pixels][HIT_TMP] cached hits (tick)
    float *hit_tmpc;       // [max_pixels][HIT_TMP] cached hits (charge)
    int32_t *status;       // [TRED_STATUS_WORDS]
    float2 *tw;            // twiddle tables (see tred_api.cu)
    double *gl_x, *gl_w;   // host copies unused on device; kept for reference
    float gl_xi[tred::MAX_GL], gl_wi[tred::MAX_GL];
    // adjoint scratch (allocated on the first tred_adjoint call)
    float *wts2;           // [max_deposits][3][wstride] weights, d/dmu, d/dsigma
    int32_t *pix_row;      // [npx_x * npx_y] row of a pixel in the current list or -1
    float2 *gspec;         // [adj_chunk][npairs][lt][64] adjoint spectra of the input pixels
    int32_t adj_chunk;
    int64_t launches;      // kernels launched through this handle (diagnostics)
    struct KernelTimers *kt;   // per-kernel event pairs while timing is enabled (else null)
    char err[512];
};

namespace tred {

constexpr int HIT_TMP = 16;

// twiddle table offsets into h->tw (float2): W_N[k] = exp(-2 pi i k / N)
constexpr int TW_32 = 0;            // 32 entries
constexpr int TW_64 = 32;           // 64 entries
constexpr int TW_16 = 96;           // 16 entries
constexpr int TW_8 = 112;           // 8 entries
constexpr int TW_LT = 128;          // lt entries (<= 1024)
constexpr int TW_TOTAL = 128 + 1024;

int set_error(tred_handle *h, int code, const char *fmt, ...);
// argument checks shared by the handle path and the allocation-free binning: every
// device array of a deposit set present; the geometry accepted by tred_create (a
// message in msg otherwise)
bool deps_ok(const tred_deposits *d);
int validate_geometry(const tred_geometry *g, char *msg, size_t len);
int check_cuda(tred_handle *h, cudaError_t e, const char *what);

// kernel launchers (each .cu file)
int launch_drift(tred_handle *h, int n, const float *x, const float *y, const float *z,
                 const float *t0, const float *ne, const int32_t *event, const tred_deposits &out,
                 cudaStream_t s);
int launch_blockbin(tred_handle *h, int n, const tred_deposits &deps, int32_t *block_ids,
                    int32_t *block_counts, int32_t *dep_offsets, int32_t *dep_index,
                    int32_t max_pairs, int32_t *n_blocks_dev, cudaStream_t s);
size_t effq_scratch_bytes(int side, int grid);
int dft_basis_build(tred_handle *h);
int launch_drift_lines(tred_handle *h, int n, const float *x0, const float *y0, const float *z0, const float *x1,
                       const float *y1, const float *z1, const float *t0, const float *ne, const tred_deposits &out,
                       float *half, cudaStream_t s);
int launch_effq_lines(tred_handle *h, int n, const tred_deposits &deps, const float *half, const int32_t *block_ids,
                      const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev, float *qeff,
                      cudaStream_t s);
size_t dft_basis_bytes(int bt);
size_t dft_zspec_bytes(int blocks, int npairs, int lt);
int launch_dft_gemm(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, int qrows_blocks,
                    int slot_base, int slot_count, int qbase, cudaStream_t s);
int launch_effq(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                const int32_t *dep_offsets, const int32_t *dep_index,
                const int32_t *n_blocks_dev, float *qeff, int slot_base, int slot_count, cudaStream_t s);
int launch_response(tred_handle *h, const float *resp, cudaStream_t s);
int launch_pipeline(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                    const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev, float *qring,
                    int ring_rows, float *out, cudaStream_t s);
int launch_wait_selftest(tred_handle *h, long long limit, cudaStream_t s);
// direct spatial form (conv_mode 4): the response operand (once per response) and the
// convolution of slots [slot_base, slot_base + slot_count) with qeff rows from qbase
int launch_direct_response(tred_handle *h, const float *resp, cudaStream_t s);
int launch_direct(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, float *out, int slot_base,
                  int slot_count, int qbase, cudaStream_t s);
// fused inverse DFT + gather of conv_mode 4 (tred_convolve_gather_readout): the spectra of
// every slot in one pass, then k_dx_wave over the pixel list that launch_pixel_list built
bool dx_wave_ok(const tred_handle *h);
int launch_direct_spectra(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, int slot_base,
                          int slot_count, cudaStream_t s);
int launch_direct_wave(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev, int32_t *queue,
                       float *wave, float *possum, cudaStream_t s);
size_t dx_bytes_b(int nbins, int npad, int kq);
size_t dx_bytes_q(int nbins, int rows_cap, int kq);
int dx_rows_cap_of(int dx_blocks, int bp2, int cap_param);
int dx_blocks_of(int max_blocks);
bool dx_shape_ok(int nch, int lt);
// the driver entry point cuTensorMapEncodeTiled (nullptr when unavailable)
void *tensor_map_encoder();
int launch_convolve(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                    const float *qeff, float *out, int slot_base, int slot_count, cudaStream_t s);
// the gather's pixel list (pixel_ids, n_pixels_dev), pix_flag = row of each pixel or -1,
// blk_slot = slot of each active block or -1; returns the device word for a work queue
int launch_flag_list(tred_handle *h, int64_t n, int32_t *flags, int32_t *part, int32_t *ids, int32_t *count_dev,
                     cudaStream_t s);
int launch_pixel_list(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev, int32_t *pixel_ids,
                      int32_t *n_pixels_dev, cudaStream_t s, int32_t **queue);
int launch_gather(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                  const float *out, int32_t *pixel_ids, float *wave, int32_t *n_pixels_dev,
                  cudaStream_t s, float *possum = nullptr);
int launch_readout(tred_handle *h, const tred_readout_params &rp, const int32_t *pixel_ids,
                   const float *wave, const int32_t *n_pixels_dev, int32_t *hit_pixel,
                   int32_t *hit_tick, float *hit_charge, int32_t *n_hits_dev,
                   int32_t max_hits, cudaStream_t s, const float *possum = nullptr);

int launch_residual(tred_handle *h, const int32_t *pix, const int32_t *n_pix_dev, const float *wave,
                    const int32_t *tpix, int n_target, const float *twave, float *resid, double *loss,
                    cudaStream_t s);
int launch_adjoint(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                   const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev,
                   const int32_t *pixel_ids, const int32_t *n_pixels_dev, const float *resid, float *gq,
                   float *grad7, cudaStream_t s);
int launch_param_grads(tred_handle *h, int n, const float *z, const tred_deposits &deps, const float *grad7,
                       float *gin, double *gglob, cudaStream_t s);

int num_sms(tred_handle *h);

// Per-kernel event timing (tred_set_kernel_timing): kt_begin / kt_end bracket one launch
// of class `which` on stream s; no-ops while timing is disabled.
void kt_begin(tred_handle *h, int which, cudaStream_t s);
void kt_end(tred_handle *h, int which, cudaStream_t s);

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * b + c
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

__device__ __forceinline__ int floordiv(int a, int b) {  // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// In-register radix-2 decimation-in-frequency FFT of N = 2^k points with twiddles
// read from W (W[m] = exp(-2 pi i m / N), or its conjugate when INV).  Natural-order
// input; output v[k] = X[bitrev(k)].  Fully unrolled: all indices are constants.
template <int N, bool INV>
__device__ __forceinline__ void fft_reg_dif(float2 (&v)[N], const float2 *__restrict__ W) {
#pragma unroll
    for (int span = N / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int start = 0; start < N; start += 2 * span) {
#pragma unroll
            for (int i = 0; i < span; ++i) {
                float2 a = v[start + i], b = v[start + i + span];
                v[start + i] = cadd(a, b);
                float2 d = csub(a, b);
                const int m = i * (N / (2 * span));
                if (m == 0) {
                    v[start + i + span] = d;
                } else if (4 * m == N) {
                    v[start + i + span] = mul_mi<INV>(d);
                } else {
                    float2 w = W[m];
                    if (INV) w.y = -w.y;
                    v[start + i + span] = cmul(d, w);
                }
            }
        }
    }
}

// exp(-2 pi i m / 32) as compile-time constants (cos and -sin rounded to binary32),
// used by the in-register FFTs of size <= 32 so that twiddles fold into the code.
__host__ __device__ constexpr float w32c(int m) {
    constexpr float c[32] = {1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f, 7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f, 0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f, -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f, -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f, -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f, 0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f, 7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f};
    return c[m & 31];
}
__host__ __device__ constexpr float w32s(int m) {
    constexpr float s[32] = {0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f, -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f, -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f, -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f, 0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f, 7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f, 1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f, 7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f};
    return s[m & 31];
}

// Radix-2 DIF FFT in registers, N <= 32, twiddles as constants.  Output v[k] = X[bitrev(k)].
// HZ: the upper half of the input is zero (v[N/2 ..] are not read), so the first stage's
// butterflies reduce to a copy and a twiddled copy.
template <int N, bool INV, bool HZ = false>
__device__ __forceinline__ void fft_reg_dif_c(float2 (&v)[N]) {
    static_assert(N >= 2 && N <= 32 && (N & (N - 1)) == 0, "N must be a power of two <= 32");
#pragma unroll
    for (int span = N / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int start = 0; start < N; start += 2 * span) {
#pragma unroll
            for (int i = 0; i < span; ++i) {
                float2 a = v[start + i];
                float2 d;
                if (HZ && span == N / 2) {
                    d = a;
                } else {
                    const float2 b = v[start + i + span];
                    v[start + i] = cadd(a, b);
                    d = csub(a, b);
                }
                const int m = i * (N / (2 * span));        // exponent on W_N
                const int m32 = m * (32 / N);               // same angle on W_32
                if (m == 0) {
                    v[start + i + span] = d;
                } else if (4 * m == N) {
                    v[start + i + span] = mul_mi<INV>(d);
                } else {
                    const float wr = w32c(m32), wi = INV ? -w32s(m32) : w32s(m32);
                    v[start + i + span] = make_float2(d.x * wr - d.y * wi, d.x * wi + d.y * wr);
                }
            }
        }
    }
}

template <int N>
__host__ __device__ constexpr int bitrev(int x) {
    int r = 0;
    for (int b = 1; b < N; b <<= 1) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

// exp(-2 pi i m / 24) as compile-time constants (cos and -sin rounded to binary32), for the
// in-register transforms of 12 and 24 points
__host__ __device__ constexpr float w24c(int m) {
    constexpr float c[24] = {1.000000000e+00f, 9.659258263e-01f, 8.660254038e-01f, 7.071067812e-01f, 5.000000000e-01f, 2.588190451e-01f, 0.0f, -2.588190451e-01f, -5.000000000e-01f, -7.071067812e-01f, -8.660254038e-01f, -9.659258263e-01f, -1.000000000e+00f, -9.659258263e-01f, -8.660254038e-01f, -7.071067812e-01f, -5.000000000e-01f, -2.588190451e-01f, 0.0f, 2.588190451e-01f, 5.000000000e-01f, 7.071067812e-01f, 8.660254038e-01f, 9.659258263e-01f};
    return c[((m % 24) + 24) % 24];
}
__host__ __device__ constexpr float w24s(int m) {
    constexpr float s[24] = {0.0f, -2.588190451e-01f, -5.000000000e-01f, -7.071067812e-01f, -8.660254038e-01f, -9.659258263e-01f, -1.000000000e+00f, -9.659258263e-01f, -8.660254038e-01f, -7.071067812e-01f, -5.000000000e-01f, -2.588190451e-01f, 0.0f, 2.588190451e-01f, 5.000000000e-01f, 7.071067812e-01f, 8.660254038e-01f, 9.659258263e-01f, 1.000000000e+00f, 9.659258263e-01f, 8.660254038e-01f, 7.071067812e-01f, 5.000000000e-01f, 2.588190451e-01f};
    return s[((m % 24) + 24) % 24];
}

// In-register DFT of N = 3 M points (M = 4 or 8; N = 12 or 24), mixed radix: a radix-3
// butterfly over n = n2 + M n1 for each n2, the twiddles W_N^(n2 k1), then an M-point
// radix-2 DIF transform of each of the three rows k1.  Output register k1 M + j holds
// X[3 bitrev_M(j) + k1] (fft_perm gives that index).  INV: conjugate twiddles.
template <int N, bool INV>
__device__ __forceinline__ void fft_reg_mixed3(float2 (&v)[N]) {
    static_assert(N == 12 || N == 24, "N = 12 or 24");
    constexpr int M = N / 3;
    constexpr float C3 = 8.660254038e-01f;                  // sin(2 pi / 3)
#pragma unroll
    for (int n2 = 0; n2 < M; ++n2) {
        const float2 x0 = v[n2], x1 = v[n2 + M], x2 = v[n2 + 2 * M];
        const float2 sm = make_float2(x1.x + x2.x, x1.y + x2.y), df = make_float2(x1.x - x2.x, x1.y - x2.y);
        const float2 y0 = make_float2(x0.x + sm.x, x0.y + sm.y);
        const float2 t = make_float2(x0.x - 0.5f * sm.x, x0.y - 0.5f * sm.y);
        const float2 id = make_float2(-C3 * df.y, C3 * df.x);   // i sin(2 pi / 3) (x1 - x2)
        const float2 y1 = INV ? make_float2(t.x + id.x, t.y + id.y) : make_float2(t.x - id.x, t.y - id.y);
        const float2 y2 = INV ? make_float2(t.x - id.x, t.y - id.y) : make_float2(t.x + id.x, t.y + id.y);
        v[n2] = y0;
        const int m1 = n2 * (24 / N), m2 = 2 * n2 * (24 / N);     // W_N^(n2) and W_N^(2 n2) on W_24
        const float c1 = w24c(m1), s1 = INV ? -w24s(m1) : w24s(m1);
        const float c2 = w24c(m2), s2 = INV ? -w24s(m2) : w24s(m2);
        v[n2 + M] = n2 == 0 ? y1 : make_float2(y1.x * c1 - y1.y * s1, y1.x * s1 + y1.y * c1);
        v[n2 + 2 * M] = n2 == 0 ? y2 : make_float2(y2.x * c2 - y2.y * s2, y2.x * s2 + y2.y * c2);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        float2 r[M];
#pragma unroll
        for (int j = 0; j < M; ++j) r[j] = v[k1 * M + j];
        fft_reg_dif_c<M, INV>(r);
#pragma unroll
        for (int j = 0; j < M; ++j) v[k1 * M + j] = r[j];
    }
}

// Output index held in register k by fft_reg_any<N>: bit reversal for powers of two,
// 3 bitrev_M(k mod M) + k div M for N = 3 M.
template <int N>
__host__ __device__ constexpr int fft_perm(int k) {
    if constexpr ((N & (N - 1)) == 0) {
        return bitrev<N>(k);
    } else {
        return 3 * bitrev<N / 3>(k % (N / 3)) + k / (N / 3);
    }
}
template <int N, bool INV>
__device__ __forceinline__ void fft_reg_any(float2 (&v)[N]) {
    if constexpr ((N & (N - 1)) == 0) fft_reg_dif_c<N, INV>(v);
    else fft_reg_mixed3<N, INV>(v);
}

// Cross-lane 32-point DIF FFT (one value per lane, natural order in lane index);
// afterwards lane l holds X[bitrev5(l)].  w32: lane-independent table
// W32[m] = exp(-2 pi i m / 32) (shared or global memory).
template <bool INV>
__device__ __forceinline__ float2 fft32_lanes(float2 v, const float2 *__restrict__ w32, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        float2 p;
        p.x = __shfl_xor_sync(0xffffffffu, v.x, s);
        p.y = __shfl_xor_sync(0xffffffffu, v.y, s);
        const bool upper = (lane & s) != 0;
        // lower: v + p ; upper: (p - v) * W_{2s}^{lane mod s}
        float2 u = upper ? csub(p, v) : cadd(v, p);
        if (upper) {
            float2 w = w32[(lane & (s - 1)) * (16 / s)];
            if (INV) w.y = -w.y;
            u = cmul(u, w);
        }
        v = u;
    }
    return v;
}

// x * W_16^m (forward), m a compile-time constant after unrolling: the rotations by
// 0 and -i are exact swaps, the others one complex product
__device__ __forceinline__ float2 mul_w16(float2 x, int m) {
    if (m == 0) return x;
    if (m == 4) return make_float2(x.y, -x.x);
    const float wr = w32c(2 * m), wi = w32s(2 * m);
    return make_float2(x.x * wr - x.y * wi, x.x * wi + x.y * wr);
}

// ---------------------------------------------------------------- tensor memory (TMEM)
// Allocation by one full warp; the address (lane << 16 | column) lands in shared memory.
// ---------------------------------------------------------------- mbarriers
constexpr long long WAIT_CYCLES = 2000000000ll;   // bound of every mbarrier wait (~1 s at 2 GHz)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait for the phase with parity `phase` to complete; false once `limit` cycles
// have passed without it
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit = WAIT_CYCLES) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 consecutive 32-bit columns of this thread's lane (32x32b shape: the warp's 32
// lanes of its lane quarter), then wait for the load.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
                   "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]),
                   "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]),
                   "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]),
                   "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
                 : "r"(taddr)
                 : "memory");
}
// store 32 consecutive columns of this thread's lane, then wait for the store
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\t"
                 "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
                 "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]),
                 "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]),
                 "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
                 : "memory");
}

}  // namespace tred
