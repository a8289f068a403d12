// a4, tensor-core form with the spatial sum taken directly per time frequency (Sec.
// II-D, Eq. interlaced; Sec. III-A-2: the time axis by DFT, the pixel plane and the
// impacts by a GEMM on the tcgen05 tensor cores).
//
// The interlaced convolution of one active block,
//     I[P, t] = sum_j sum_K sum_tau Qeff[j, P + K, t - tau] i[j, K, tau],
// becomes after a length-lt DFT over time, for every bin f = 0 .. lt/2 (the data are
// real, so the other half of the spectrum is the conjugate),
//     Ihat[P, f] = sum_{p'} Z[p', p' - P, f],   Z[p', K, f] = sum_j Qhat[j, p', f] R[j, K, f]
// with Qhat the DFT of the block's column (impact j, pixel p') and R the DFT of the
// response column (j, K).  For each bin, Z is a complex matrix product over the impacts:
// rows = the block's pixels that hold charge (on a module plane about 10 of the 64),
// columns = the kp^2 response taps.  Batched over every non-empty (block, pixel) row of
// the pass, each bin is one complex GEMM with M = rows, K = nch impacts, N = kp^2 taps,
// run on the tensor cores as four real products per K step,
//     Re Z += Re Q Re R,  Re Z -= Im Q Im R,  Im Z += Re Q Im R,  Im Z += Im Q Re R
// (the minus by the instruction's negate-B bit), each as three split-BF16 products
// (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation in tensor memory).  The K axis is
// laid out in groups of 16 impacts, k = 32 g + 16 h + i for impact j = 16 g + i (h = 0:
// real part, 1: imaginary part), in both operands (B holds Re R and Im R), so that one
// 32-wide K chunk of A and of B serves all four products and B is stored once.
//
// Kernels of one pass over at most dx_blocks slots:
//  k_dx_pixmask / k_dx_rows  non-empty pixels of each slot (from the effective charge's
//                            column masks) and the row list, in slot then pixel order;
//  k_dx_fwd                  per row, the real DFT of its nch columns (two real columns
//                            per complex FFT in registers, split by Hermitian symmetry),
//                            transposed in shared memory and written as BF16 hi and lo
//                            parts [bin][row][k];
//  k_dx_gemm                 per (bin, 128-row tile): TMA (128-byte swizzle) of the two
//                            operands' parts, tcgen05.mma kind::f16 (M = 128, N = npad,
//                            K = 16) into one of two pairs of tensor-memory accumulators
//                            (Re Z, Im Z), and an
//                            epilogue that sums each block's rows into its 16 x 16 output
//                            spectrum Ihat[slot][f][P] in a fixed row order;
//  k_dx_inv                  per block, the inverse real DFT of the 256 output pixels
//                            (two per complex FFT) into out_blocks[slot][uy][ux][t].
// A block whose rows cross a 128-row tile boundary gets its two tiles' parts by two
// floating-point additions onto zero (the fixed summation order holds: a + b = b + a).
// Every mbarrier wait is bounded; an expired wait sets TRED_ST_TIMEOUT, and the CTA
// lets its copies and products in flight finish (bounded) before it frees the tensor
// memory and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tred_internal.cuh"

namespace tred {

constexpr int DX_M = 128;                // rows of one GEMM tile
constexpr int DX_KC = 64;                // K chunk: 64 BF16 = one 128-byte row (128-byte swizzle), two groups
constexpr int DX_STAGES = 2;             // operand stages
constexpr int DX_ROWS_MAX = 131072;      // rows per forward + GEMM launch pair
constexpr int DX_BLOCKS_MAX = 16384;     // slots per pass
constexpr int DX_FWD_THREADS = 256;
constexpr int DX_FWD_UNITS = 13;         // units of 4 impacts per forward item at most (26 pairs)
constexpr int DX_FWD_CTAS = 2;           // forward CTAs per SM (shared memory of 26 pairs each)
constexpr int DX_INV_THREADS = 256;
constexpr int DX_GEMM_THREADS = 320;     // warp 0 copies, warp 1 products, warps 2..9 epilogue
constexpr uint32_t DX_A_BYTES = DX_M * DX_KC * 2;   // 16 KB per part
constexpr int DX_TAPS_PER_LANE = 3;   // kp <= 9: at most 81 taps
constexpr int DX_YS = 25;            // output accumulator row stride (float2): 9 mod 16

struct DxConst {
    int nch, kq, ntap, npad, imoff, nparts, kp, R, bp, bpl, bp2, bt, lt, nbins, rows_cap;
};

__host__ __device__ constexpr int dx_round16(int x) { return (x + 15) & ~15; }
__host__ __device__ constexpr uint32_t dx_b_bytes(int npad) { return (uint32_t)npad * DX_KC * 2; }
__host__ __device__ constexpr uint32_t dx_stage_bytes(int npad) {
    return (2 * DX_A_BYTES + 2 * dx_b_bytes(npad) + 1023u) & ~1023u;
}
// column stride of the forward kernel's transposition buffer: at least nbins + 3 (room
// for the columns' skew of up to 3) and 1 mod 8, so that lanes reading the columns of
// distinct pairs of one bin hit distinct banks; the buffer holds the impacts of one item,
// at most 4 DX_FWD_UNITS, two columns per impact
__host__ __device__ constexpr int dx_tstride(int nbins) { return ((nbins + 10) & ~7) + 1; }
// A row's impacts in the GEMM's K groups of 16, cut into nparts items of whole groups
// (part q: groups [q ng / nparts, (q + 1) ng / nparts)), so that no 32-byte sector of a
// row's spectra is written by two CTAs; nparts is the least count whose parts hold at
// most DX_FWD_UNITS units of 4 impacts below nch (the pairs the shared buffer holds).
__host__ __device__ constexpr int dx_part_units(int nch, int np, int q) {
    const int ng = (nch + 15) / 16;
    const int j0 = 16 * (q * ng / np), j1 = 16 * ((q + 1) * ng / np) < nch ? 16 * ((q + 1) * ng / np) : nch;
    return j1 > j0 ? (j1 - j0 + 3) / 4 : 0;
}
static int dx_fwd_max_units(int nch, int np) {
    int mx = 0;
    for (int q = 0; q < np; ++q) mx = std::max(mx, dx_part_units(nch, np, q));
    return mx;
}
static int dx_fwd_parts(int nch) {
    int np = 1;
    while (dx_fwd_max_units(nch, np) > DX_FWD_UNITS) ++np;
    return np;
}
size_t dx_fwd_smem(int nch, int nbins) {
    return sizeof(float) * (size_t)(8 * dx_fwd_max_units(nch, dx_fwd_parts(nch))) * dx_tstride(nbins);
}
// epilogue staging row (floats): Re Z of the taps at 0, Im Z at imoff = ntap rounded up to
// 4; a multiple of 4 (16-byte stores) with an odd number of 16-byte chunks (the 32 lanes'
// rows start in distinct bank groups)
__host__ __device__ constexpr int dx_zstride(int ntap) { return (((2 * ((ntap + 3) & ~3)) / 4) | 1) * 4; }
static size_t dx_gemm_smem(int npad, int ntap) {
    return 1024 + DX_STAGES * (size_t)dx_stage_bytes(npad) + sizeof(float) * DX_M * dx_zstride(ntap) +
           sizeof(float2) * 8 * LP * DX_YS + sizeof(int32_t) * (3 * DX_M + 2 + 5) + 128;
}

// two binary32 values to their nearest BF16 (ties to even), lo in the low 16 bits
__device__ __forceinline__ uint32_t dx_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// nearest BF16 (ties to even) of a finite binary32 value, as its 16 bits, and its value
__host__ __device__ __forceinline__ uint32_t dx_bf16_bits(float x) {
#ifdef __CUDA_ARCH__
    const uint32_t u = __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
#endif
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
__host__ __device__ __forceinline__ float dx_bf16_value(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b << 16);
#else
    const uint32_t u = b << 16;
    float x;
    memcpy(&x, &u, 4);
    return x;
#endif
}

// ---------------------------------------------------------------- response operand
// R[j][n][f] = (1 / (2 lt)) sum_tau i[Ky][Kx][jy][jx][tau] exp(-2 pi i tau f / lt) in FP64
// (n = Ky kp + Kx, j = jy ns + jx; the 1/lt of the inverse DFT and the 1/2 of the
// forward kernel's Hermitian split folded in: it stores 2 Qhat).
__global__ void k_dx_resp_time(const float *__restrict__ resp, int nch, int ntap, int nr, int lt, int nbins,
                               const double2 *__restrict__ wlt, double2 *__restrict__ Rt) {
    const int64_t total = (int64_t)nch * ntap * nbins;
    const double scale = 0.5 / (double)lt;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(idx % nbins);
        const int64_t r = idx / nbins;
        const int n = (int)(r % ntap);
        const int j = (int)(r / ntap);
        // resp layout [Ky][Kx][jy][jx][tau] = [n][j][tau]
        const float *ir = resp + ((int64_t)n * nch + j) * nr;
        double re = 0.0, im = 0.0;
        for (int tau = 0; tau < nr; ++tau) {
            const double v = (double)ir[tau];
            const double2 w = wlt[((int64_t)tau * f) % lt];
            re = fma(v, w.x, re);
            im = fma(v, w.y, im);
        }
        Rt[idx] = make_double2(re * scale, im * scale);   // the forward kernel stores 2 Qhat
    }
}

// the GEMM's B operand [bin][tap][k] (k = 32 g + 16 h + i: Re R (h = 0) and Im R (h = 1)
// of impact 16 g + i), split into BF16 hi and lo parts
__global__ void k_dx_resp_pack(const double2 *__restrict__ Rt, DxConst c, uint16_t *__restrict__ bhi,
                               uint16_t *__restrict__ blo) {
    const int64_t total = (int64_t)c.nbins * c.npad * c.kq;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % c.kq);
        const int64_t r = idx / c.kq;
        const int n = (int)(r % c.npad);
        const int f = (int)(r / c.npad);
        const int j = 16 * (k >> 5) + (k & 15);
        const bool imr = ((k >> 4) & 1) != 0;   // the imaginary part of R
        double v = 0.0;
        if (n < c.ntap && j < c.nch) {
            const double2 R = Rt[((int64_t)j * c.ntap + n) * c.nbins + f];
            v = imr ? R.y : R.x;
        }
        const float x = (float)v;
        const uint32_t h = dx_bf16_bits(x);
        const uint32_t l = dx_bf16_bits((float)(v - (double)dx_bf16_value(h)));
        bhi[idx] = (uint16_t)h;
        blo[idx] = (uint16_t)l;
    }
}

static DxConst dx_const_of(const tred_handle *h) {
    DxConst c;
    c.nch = h->g.n_sub * h->g.n_sub;
    c.kq = 32 * ((c.nch + 15) / 16);
    c.nparts = dx_fwd_parts(c.nch);
    c.kp = h->g.kp;
    c.ntap = c.kp * c.kp;
    c.npad = dx_round16(c.ntap);
    c.imoff = (c.ntap + 3) & ~3;
    c.R = h->d.R;
    c.bp = h->g.bp;
    c.bpl = c.bp == 8 ? 3 : 2;   // bp is 4 or 8
    c.bp2 = c.bp * c.bp;
    c.bt = h->g.bt;
    c.lt = h->g.lt;
    c.nbins = c.lt / 2 + 1;
    c.rows_cap = h->dx_rows_cap;
    return c;
}

int launch_direct_response(tred_handle *h, const float *resp, cudaStream_t s) {
    const DxConst c = dx_const_of(h);
    std::vector<double2> wlt(c.lt);
    for (int k = 0; k < c.lt; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)c.lt;
        wlt[k] = make_double2(std::cos(a), -std::sin(a));
    }
    double2 *d_wlt = nullptr, *d_R = nullptr;
    int rc = check_cuda(h, cudaMalloc(&d_wlt, sizeof(double2) * c.lt), "alloc direct-form twiddles");
    if (!rc) rc = check_cuda(h, cudaMalloc(&d_R, sizeof(double2) * (size_t)c.nch * c.ntap * c.nbins), "alloc direct-form stage");
    if (!rc) rc = check_cuda(h, cudaMemcpyAsync(d_wlt, wlt.data(), sizeof(double2) * c.lt, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) {
        const int grid = num_sms(h) * 8;
        k_dx_resp_time<<<grid, 256, 0, s>>>(resp, c.nch, c.ntap, h->g.nr, c.lt, c.nbins, d_wlt, d_R);
        k_dx_resp_pack<<<grid, 256, 0, s>>>(d_R, c, h->dx_bhi, h->dx_blo);
        h->launches += 2;
        rc = check_cuda(h, cudaGetLastError(), "direct-form response launch");
    }
    cudaError_t e = cudaStreamSynchronize(s);   // set-up path, once per response
    if (!rc) rc = check_cuda(h, e, "direct-form response sync");
    cudaFree(d_wlt);
    cudaFree(d_R);
    return rc;
}

// ---------------------------------------------------------------- rows
// One warp per slot of the pass: the OR of its nch column masks = its non-empty pixels.
__global__ void k_dx_pixmask(const int32_t *__restrict__ n_blocks_dev, const uint64_t *__restrict__ colmask, int nch,
                             int bp2, int slot_base, int slot_count, uint64_t *__restrict__ pmask,
                             int32_t *__restrict__ pcnt) {
    const int nb = n_blocks_dev[0];
    const int cnt = max(0, min(slot_count, nb - slot_base));
    const int lane = threadIdx.x & 31;
    const uint64_t keep = bp2 >= 64 ? ~0ull : ((1ull << bp2) - 1ull);
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < cnt; s += (gridDim.x * blockDim.x) >> 5) {
        const uint64_t *m = colmask + (size_t)(slot_base + s) * nch;
        uint64_t v = 0;
        int nz = 0;   // non-empty columns of the slot
        for (int j = lane; j < nch; j += 32) {
            v |= m[j];
            nz += __popcll(m[j] & keep);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            v |= __shfl_xor_sync(0xffffffffu, v, o);
            nz += __shfl_xor_sync(0xffffffffu, nz, o);
        }
        if (lane == 0) {
            pmask[s] = v & keep;
            pcnt[s] = nz;
        }
    }
}

// One CTA: exclusive scan of the slots' pixel counts (rowstart), the row records in slot
// then pixel order, meta = {slots of the pass, rows of the pass, non-empty columns, -,
// running totals of rows and columns (two 64-bit words)}.
constexpr int DX_ROWS_THREADS = 1024;
__global__ void __launch_bounds__(DX_ROWS_THREADS) k_dx_rows(const int32_t *__restrict__ n_blocks_dev,
                                                              const uint64_t *__restrict__ pmask,
                                                              const int32_t *__restrict__ pcnt, int slot_base,
                                                              int slot_count, int32_t *__restrict__ rows,
                                                              int32_t *__restrict__ rowstart,
                                                              int32_t *__restrict__ meta) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    __shared__ long long wcol[32];
    const int nb = n_blocks_dev[0];
    const int cnt = max(0, min(slot_count, nb - slot_base));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    long long ncol = 0;   // this thread's non-empty columns
    __syncthreads();
    for (int base = 0; base < cnt; base += DX_ROWS_THREADS) {
        const int s = base + tid;
        const uint64_t m = s < cnt ? pmask[s] : 0ull;
        if (s < cnt) ncol += pcnt[s];
        const int n = __popcll(m);
        int x = n;   // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const int carry = carry_s;
        const int start = carry + (warp ? wsum[warp - 1] : 0) + x - n;
        if (s < cnt) {
            rowstart[s] = start;
            uint64_t mm = m;
            int r = start;
            while (mm) {
                const int p = __ffsll((long long)mm) - 1;
                rows[r++] = (s << 6) | p;
                mm &= mm - 1ull;
            }
        }
        __syncthreads();
        if (tid == 0) carry_s = carry + wsum[31];
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) ncol += __shfl_xor_sync(0xffffffffu, ncol, o);
    if (lane == 0) wcol[warp] = ncol;
    __syncthreads();
    if (tid == 0) {
        long long tot = 0;
        for (int w = 0; w < DX_ROWS_THREADS / 32; ++w) tot += wcol[w];
        rowstart[cnt] = carry_s;
        meta[0] = cnt;
        meta[1] = carry_s;
        meta[2] = (int32_t)min(tot, 2147483647ll);
        // running totals over the passes since the host last read them
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(meta + 4);
        atomicAdd(&acc[0], (unsigned long long)carry_s);
        atomicAdd(&acc[1], (unsigned long long)tot);
    }
}

// ---------------------------------------------------------------- forward time DFT
// index k with fft_perm<N>(k) == v (compile time)
template <int N>
__host__ __device__ constexpr int dx_perm_inv(int v) {
    for (int k = 0; k < N; ++k)
        if (fft_perm<N>(k) == v) return k;
    return 0;
}

// Zero the output spectra of the slots whose rows cross a 128-row tile boundary: the
// GEMM epilogue adds their two parts onto zero.
__device__ __forceinline__ void dx_zero_straddling(const int32_t *__restrict__ rowstart, int cnt, int nbins,
                                                   float2 *__restrict__ ybuf) {
    for (int s = blockIdx.x; s < cnt; s += gridDim.x) {
        const int rs = rowstart[s], re = rowstart[s + 1];
        if (re <= rs || (rs >> 7) == ((re - 1) >> 7)) continue;
        float4 *y = reinterpret_cast<float4 *>(ybuf + (size_t)s * nbins * (LP * LP));
        const int n4 = nbins * (LP * LP) / 2;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) y[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Items (row, part): the CTA transforms the impact pairs of one part of a row, whole
// groups of 16 impacts with at most 4 DX_FWD_UNITS impacts (two parts of a 10 x 10
// impact row, two CTAs per SM).  Parts that split a group put two CTAs' partial writes
// into one 32-byte sector of the spectra (the split at 52 instead of 48 impacts: 8.2
// against 6.8 ms on a module plane; four parts of 24 or 28 impacts at three CTAs per SM:
// 11.0 ms).  The last group's padding past nch is left as the buffer was cleared (writing
// it as zeros: 7.0 ms).
// Warp w takes the part's pairs
// q = w, w + 8, ...: the two real columns as one
// complex sequence z[t] = Q[2q][t] + i Q[2q+1][t] (t < bt, zero to lt), N = lt = 32 NPL:
//   pass 1  lane l holds z[l + 32 n1], n1 < NPL: an NPL-point DFT in registers, the
//           twiddles W_N^(l f1);
//   transpose through the pair's own columns of T (S[f1][n2 ^ f1]);
//   pass 2  lanes 2 d + e (d = f1 < NPL) hold the 16 samples n2 = 2 a + e of the 32-point
//           DFT over n2: a 16-point DFT in registers, the twiddles W_32^(e g), and one
//           radix-2 step across the lane pair, so that lane 2 d + e holds bin
//           f = d + NPL (g + 16 e) in register k (g = bitrev16(k));
// then Z[f] (f <= N/2) and Z[N - f] land in the pair's four columns.  A pair whose two
// columns are empty in the block's masks (or lie past the last impact) is written as
// zeros without a transform.  Then the CTA's threads take the (bin, unit of two pairs)
// items in order and write the Hermitian split of the unit's columns in BF16 hi and lo
// parts at the GEMM's K positions.
// Parts start at multiples of 4 impacts, so that each lane's four impacts lie in one
// group of 16.
// first float of pair q's region (4 ST floats: Z[f] then C[f] = Z[N - f] as complex
// numbers); the skew 2 ((q >> 3) & 3) keeps it 8-byte aligned and puts the regions of the
// pairs 2 c4 (c4 = 0 .. 15, one lane each) in distinct banks
__device__ __forceinline__ int dx_pbase(int q, int ST) { return 4 * q * ST + 2 * ((q >> 3) & 3); }

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned)
__device__ __forceinline__ void dx_cp16(float *smem, const float *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
template <int N, bool HZ>
__device__ __forceinline__ void dx_fft_fwd(float2 (&v)[N]) {
    if constexpr ((N & (N - 1)) == 0) fft_reg_dif_c<N, false, HZ>(v);
    else fft_reg_mixed3<N, false>(v);
}

template <int G>
__global__ void __launch_bounds__(DX_FWD_THREADS, DX_FWD_CTAS)
    k_dx_fwd(const float *__restrict__ qeff, const uint64_t *__restrict__ colmask, const int32_t *__restrict__ rows,
             const int32_t *__restrict__ rowstart, const int32_t *__restrict__ meta, const float2 *__restrict__ tw,
             DxConst c, int slot_base, int qbase, int row0, int zero_straddling, uint16_t *__restrict__ qhi,
             uint16_t *__restrict__ qlo, float2 *__restrict__ ybuf) {
    constexpr int LT = 64 * G;
    constexpr int NPL = LT / 32;
    constexpr int NW = DX_FWD_THREADS / 32;
    static_assert(NPL <= 16, "pass 2 holds 16 samples per lane");
    static_assert(2 * DX_FWD_UNITS <= 16 * NW, "a warp's pairs of one item fit one ballot");
    extern __shared__ float T[];   // per pair of the part 4 ST floats at dx_pbase(pair)
    const int ST = dx_tstride(c.nbins);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cnt = meta[0], nrows = meta[1];
    if (zero_straddling) dx_zero_straddling(rowstart, cnt, c.nbins, ybuf);
    const int nloc = min(c.rows_cap, nrows - row0);
    const float2 *wlt = tw + TW_LT;
    const int d = lane >> 1, e = lane & 1;
    const bool hz = 2 * c.bt <= LT;
    const int ng = (c.nch + 15) >> 4;
    // pass 1 twiddles W_N^(l f1), [f1][lane l], read from shared memory instead of through
    // the read-only cache (6.64 against 6.79 ms per module-plane step)
    __shared__ float2 twl[NPL][32];
    for (int i = tid; i < NPL * 32; i += DX_FWD_THREADS) twl[i >> 5][i & 31] = wlt[((i & 31) * (i >> 5)) % LT];
    __syncthreads();
    for (int item = blockIdx.x; item < c.nparts * nloc; item += gridDim.x) {
        const int rl = item / c.nparts, part = item - rl * c.nparts;
        // groups [g0, g1) of 16 impacts: nunit units of 4 hold impacts below nch (the
        // padding of the last group stays as the buffer was cleared)
        const int g0 = part * ng / c.nparts, g1 = (part + 1) * ng / c.nparts;
        const int j0 = 16 * g0;
        const int nunit = (min(16 * g1, c.nch) - j0 + 3) >> 2;
        const int nph = 2 * nunit;
        const int rec = rows[row0 + rl];
        const int s = rec >> 6, p = rec & 63;
        const uint64_t *mk = colmask + (size_t)(slot_base + s) * c.nch;
        const float *qs = qeff + (size_t)(slot_base + s - qbase) * c.nch * c.bp2 * c.bt + (size_t)p * c.bt;
        // the non-empty flags of this warp's pairs ql = warp + NW i, both columns: bits 2 i
        // and 2 i + 1, read in one round of loads ahead of the pairs (instead of one
        // dependent mask load before each pair's column loads)
        unsigned nzw;
        {
            const int ql = warp + NW * (lane >> 1), j = j0 + 2 * ql + (lane & 1);
            nzw = __ballot_sync(0xffffffffu, ql < nph && j < c.nch && ((mk[j] >> p) & 1ull));
        }
        // the non-empty columns of pair ql (the warp's i-th) copied into the front of the
        // pair's own shared region (16-byte aligned: column a at 0, b at bt), one copy
        // group per pair, so that the next pair's loads are in flight during this pair's
        // transform
        auto stage = [&](int ql, int i) {
            float *st = T + ((dx_pbase(ql, ST) + 3) & ~3);
            const float *ca = qs + (size_t)(j0 + 2 * ql) * c.bp2 * c.bt;
            const int nq = c.bt >> 2;   // bt is a multiple of 64
            for (int k = lane; k < 2 * nq; k += 32) {
                const int h = k >= nq;
                if ((nzw >> (2 * i + h)) & 1u) dx_cp16(st + 4 * k, ca + (size_t)h * c.bp2 * c.bt + 4 * (k - h * nq));
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        if (warp < nph) stage(warp, 0);
        for (int ql = warp, i = 0; ql < nph; ql += NW, ++i) {
            const bool nza = (nzw >> (2 * i)) & 1u;
            const bool nzb = (nzw >> (2 * i + 1)) & 1u;
            float2 *Zp = reinterpret_cast<float2 *>(T + dx_pbase(ql, ST));   // Z[f], f <= N/2
            float2 *Cp = Zp + ST;                                               // Z[N - f]
            if (ql + NW < nph) {
                stage(ql + NW, i + 1);
                asm volatile("cp.async.wait_group 1;" ::: "memory");   // this pair's copies are done
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncwarp();
            if (!(nza || nzb)) {
                for (int f = lane; f < c.nbins; f += 32) {
                    Zp[f] = make_float2(0.f, 0.f);
                    Cp[f] = make_float2(0.f, 0.f);
                }
                continue;
            }
            const float *st = T + ((dx_pbase(ql, ST) + 3) & ~3);
            float2 v[NPL];
#pragma unroll
            for (int n1 = 0; n1 < NPL; ++n1) {
                const int t = lane + 32 * n1;
                const bool in = t < c.bt;
                v[n1] = make_float2(nza && in ? st[t] : 0.f, nzb && in ? st[c.bt + t] : 0.f);
            }
            if (hz) dx_fft_fwd<NPL, true>(v);
            else dx_fft_fwd<NPL, false>(v);
            float2 *S = Zp;   // transpose scratch (NPL x 32 complex) in the pair's region
            __syncwarp();
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int f1 = fft_perm<NPL>(k);
                const float2 x = f1 ? cmul(v[k], twl[f1][lane]) : v[k];
                S[f1 * 32 + (lane ^ f1)] = x;
            }
            __syncwarp();
            float2 w[16];
#pragma unroll
            for (int a = 0; a < 16; ++a)
                w[a] = d < NPL ? S[d * 32 + ((2 * a + e) ^ d)] : make_float2(0.f, 0.f);
            __syncwarp();
            fft_reg_dif_c<16, false>(w);   // w[k] = E_e[bitrev16(k)]
#pragma unroll
            for (int k = 1; k < 16; ++k) {
                const int g = bitrev<16>(k);
                if (e) w[k] = cmul(w[k], make_float2(w32c(g), w32s(g)));
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float2 o;
                o.x = __shfl_xor_sync(0xffffffffu, w[k].x, 1);
                o.y = __shfl_xor_sync(0xffffffffu, w[k].y, 1);
                w[k] = e ? csub(o, w[k]) : cadd(w[k], o);
            }
            if (d < NPL) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int f = d + NPL * (bitrev<16>(k) + 16 * e);
                    if (2 * f <= LT) Zp[f] = w[k];
                    else Cp[LT - f] = w[k];
                }
            }
        }
        __syncthreads();
        // per (bin f, unit c4 = impacts j0 + 4 c4 .. + 3, two pairs): the Hermitian split
        // of each pair's Z[f] and Z[N - f], doubled (the 1/2 is folded into R),
        //     2 Qhat[2q][f] = Z[f] + conj Z[N - f],   2 Qhat[2q+1][f] = (Z[f] - conj Z[N - f]) / i,
        // then the four real parts at k = 32 g + i and the four imaginary parts at
        // k = 32 g + 16 + i (j = 16 g + i) as BF16 hi and lo parts (8 bytes each);
        // the (bin, unit) items flattened over the CTA's threads, so that every lane is busy
        // (16 lanes per bin, 12 or 13 of them with a unit: 6.47 ms per module-plane step,
        // against 6.35)
        // (f, c4) = divmod(idx, nunit), stepped by DX_FWD_THREADS items with one carry
        // instead of a division per item (6.36 -> 6.33 ms)
        const int fstep = DX_FWD_THREADS / nunit, cstep = DX_FWD_THREADS - fstep * nunit;
        int f = tid / nunit, c4 = tid - f * nunit;
        for (; f < c.nbins; f += fstep, c4 += cstep) {
            if (c4 >= nunit) {
                c4 -= nunit;
                ++f;
                if (f >= c.nbins) break;
            }
            const size_t o = ((size_t)f * c.rows_cap + rl) * c.kq;
            const bool self = f == 0 || 2 * f == LT;
            float re[4], im[4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const float2 *zq = reinterpret_cast<const float2 *>(T + dx_pbase(2 * c4 + h2, ST));
                const float2 z = zq[f];
                const float2 cz = self ? z : zq[ST + f];
                re[2 * h2] = z.x + cz.x;       // 2 Qhat[2q] (the 1/2 is in the response operand)
                im[2 * h2] = z.y - cz.y;
                re[2 * h2 + 1] = z.y + cz.y;   // 2 Qhat[2q + 1]
                im[2 * h2 + 1] = cz.x - z.x;
            }
            const int j = j0 + 4 * c4;
            const size_t kr = o + 32 * (j >> 4) + (j & 15);
            const uint32_t h01 = dx_bf16x2(re[0], re[1]), h23 = dx_bf16x2(re[2], re[3]);
            const uint32_t g01 = dx_bf16x2(im[0], im[1]), g23 = dx_bf16x2(im[2], im[3]);
            const uint32_t l01 = dx_bf16x2(re[0] - __uint_as_float(h01 << 16), re[1] - __uint_as_float(h01 & 0xFFFF0000u));
            const uint32_t l23 = dx_bf16x2(re[2] - __uint_as_float(h23 << 16), re[3] - __uint_as_float(h23 & 0xFFFF0000u));
            const uint32_t m01 = dx_bf16x2(im[0] - __uint_as_float(g01 << 16), im[1] - __uint_as_float(g01 & 0xFFFF0000u));
            const uint32_t m23 = dx_bf16x2(im[2] - __uint_as_float(g23 << 16), im[3] - __uint_as_float(g23 & 0xFFFF0000u));
            *reinterpret_cast<uint2 *>(qhi + kr) = make_uint2(h01, h23);
            *reinterpret_cast<uint2 *>(qlo + kr) = make_uint2(l01, l23);
            *reinterpret_cast<uint2 *>(qhi + kr + 16) = make_uint2(g01, g23);
            *reinterpret_cast<uint2 *>(qlo + kr + 16) = make_uint2(m01, m23);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- GEMM per bin
__device__ __forceinline__ void dx_tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// K-major operand with the 128-byte swizzle: rows of 128 B, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t dx_sdesc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= (uint64_t)2 << 61;                        // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void dx_mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void dx_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void dx_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void dx_epi_sync() { asm volatile("barrier.sync 1, 256;" ::: "memory"); }
// OR of a flag over the 256 epilogue threads (named barrier 1 with a reduction)
__device__ __forceinline__ int dx_epi_any(int flag) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, 1, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(flag)
        : "memory");
    return (int)r;
}

// Items (bin f, tile t) in bin-major order, strided over the persistent CTAs, so that the
// CTAs running at one time share the bin's B operand in L2.  Warp 0 (one lane) issues
// the copies of each item's K chunks into DX_STAGES stages; warp 1 (one lane) issues the
// products into accumulator (item index & 1) of tensor memory and commits; warps 2..9
// drain the accumulator into shared memory (row r = TMEM lane r), release it, and sum
// each block's rows into Ihat[slot][f][u]:
//     Ihat[u] = sum over the block's rows r (pixel p') of Z_r[K],  K = p' + 2R - u
// (u = (uy, ux) the block-local output pixel, tap index K per axis in [0, kp)), rows in
// ascending order.
__global__ void __launch_bounds__(DX_GEMM_THREADS, 1)
    k_dx_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
              const int32_t *__restrict__ rows, const int32_t *__restrict__ rowstart, const int32_t *__restrict__ meta,
              DxConst c, int row0, float2 *__restrict__ ybuf, int32_t *__restrict__ status) {
    extern __shared__ unsigned char dx_raw[];
    const uint32_t raw = smem_u32(dx_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = dx_raw + (base - raw);
    const uint32_t SB = dx_stage_bytes(c.npad);
    const uint32_t BB = dx_b_bytes(c.npad);
    const int SZ = dx_zstride(c.ntap);
    float *Zs = reinterpret_cast<float *>(gbase + DX_STAGES * SB);
    float2 *yacc_all = reinterpret_cast<float2 *>(Zs + DX_M * SZ);         // [8][16][DX_YS] block outputs
    int32_t *rowrec = reinterpret_cast<int32_t *>(yacc_all + 8 * LP * DX_YS);   // [DX_M + 2]
    int32_t *seg_slot = rowrec + DX_M + 2;                               // [DX_M]
    int32_t *seg_base = seg_slot + DX_M;                                 // [DX_M]
    int32_t *seg_cnt = seg_base + DX_M;                                  // [5]
    const uint32_t bar0 = (smem_u32(seg_cnt + 5) + 7u) & ~7u;
    auto bar_full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
    auto bar_empty = [&](int st) { return bar0 + 8u * (uint32_t)(DX_STAGES + st); };
    auto bar_accf = [&](int ab) { return bar0 + 8u * (uint32_t)(2 * DX_STAGES + ab); };
    auto bar_acce = [&](int ab) { return bar0 + 8u * (uint32_t)(2 * DX_STAGES + 2 + ab); };
    const uint32_t bar_done = bar0 + 8u * (uint32_t)(2 * DX_STAGES + 4);
    unsigned char *gb = gbase + (bar_done + 8u - base);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(gb);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gb + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int st = 0; st < DX_STAGES; ++st) {
            mbar_init(bar_full(st), 1);
            mbar_init(bar_empty(st), 1);
        }
        for (int ab = 0; ab < 2; ++ab) {
            mbar_init(bar_accf(ab), 1);
            mbar_init(bar_acce(ab), 8);
        }
        mbar_init(bar_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *tslot;

    const int nrows = meta[1];
    const int nloc = min(c.rows_cap, nrows - row0);
    const int ntiles = nloc > 0 ? (nloc + DX_M - 1) / DX_M : 0;
    const int nitems = ntiles * c.nbins;
    const int nkc = (c.kq + DX_KC - 1) / DX_KC;
    const uint32_t tx_bytes = 2 * DX_A_BYTES + 2 * BB;
    // D FP32, A and B BF16, both K-major, N = npad, M = 128; idesc_nb also negates B
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(c.npad >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t idesc_nb = idesc | (1u << 14);

    if (warp == 0) {
        // ------------------------------------------------ copies
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
                const int f = it / ntiles, t = it - f * ntiles;
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int st = g % DX_STAGES;
                    if (g >= DX_STAGES && !mbar_wait(bar_empty(st), (uint32_t)((g / DX_STAGES - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const uint32_t sb = base + (uint32_t)st * SB;
                    mbar_expect_tx(bar_full(st), tx_bytes);
                    const int ya = f * c.rows_cap + t * DX_M;
                    dx_tma_2d(sb, &tmAh, kc * DX_KC, ya, bar_full(st));
                    dx_tma_2d(sb + DX_A_BYTES, &tmAl, kc * DX_KC, ya, bar_full(st));
                    dx_tma_2d(sb + 2 * DX_A_BYTES, &tmBh, kc * DX_KC, f * c.npad, bar_full(st));
                    dx_tma_2d(sb + 2 * DX_A_BYTES + BB, &tmBl, kc * DX_KC, f * c.npad, bar_full(st));
                }
            }
            if (!ok) {
                atomicOr(&status[0], TRED_ST_TIMEOUT);
                *abort_flag = 1;
            }
            // the last copies into each stage have landed before the CTA ends
            for (int q = max(0, g - DX_STAGES); q < g; ++q)
                (void)mbar_wait(bar_full(q % DX_STAGES), (uint32_t)((q / DX_STAGES) & 1));
        }
    } else if (warp == 1) {
        // ------------------------------------------------ products
        if (lane == 0) {
            int g = 0, i = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++i) {
                const int ab = i & 1;
                if (i >= 2 && !mbar_wait(bar_acce(ab), (uint32_t)(((i >> 1) - 1) & 1))) {
                    ok = false;
                    break;
                }
                tmem_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * 256);
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int st = g % DX_STAGES;
                    if (!mbar_wait(bar_full(st), (uint32_t)((g / DX_STAGES) & 1)) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    tmem_fence_after();
                    const uint32_t sb = base + (uint32_t)st * SB;
                    // the chunk holds two groups of 16 impacts, 32 bytes per K step: group
                    // 2 kc at bytes 0 (real parts of Q and of R) and 32 (imaginary parts),
                    // group 2 kc + 1 at 64 and 96 (all zero past kq: its products are skipped)
                    const uint32_t dre = d, dim = d + 128;
#pragma unroll
                    for (int gi = 0; gi < 2; ++gi) {
                        if (kc * DX_KC + 32 * gi >= c.kq) break;
                        const uint32_t acc = (kc > 0 || gi > 0) ? 1u : 0u;
                        const uint32_t o = 64u * (uint32_t)gi;
                        const uint64_t aRh = dx_sdesc_sw128(sb + o), aIh = dx_sdesc_sw128(sb + o + 32);
                        const uint64_t aRl = dx_sdesc_sw128(sb + DX_A_BYTES + o), aIl = dx_sdesc_sw128(sb + DX_A_BYTES + o + 32);
                        const uint64_t bRh = dx_sdesc_sw128(sb + 2 * DX_A_BYTES + o);
                        const uint64_t bIh = dx_sdesc_sw128(sb + 2 * DX_A_BYTES + o + 32);
                        const uint64_t bRl = dx_sdesc_sw128(sb + 2 * DX_A_BYTES + BB + o);
                        const uint64_t bIl = dx_sdesc_sw128(sb + 2 * DX_A_BYTES + BB + o + 32);
                        dx_mma_bf16(dre, aRh, bRh, idesc, acc);      // Re Z += Re Q Re R
                        dx_mma_bf16(dim, aRh, bIh, idesc, acc);      // Im Z += Re Q Im R
                        dx_mma_bf16(dre, aRh, bRl, idesc, 1u);
                        dx_mma_bf16(dim, aRh, bIl, idesc, 1u);
                        dx_mma_bf16(dre, aRl, bRh, idesc, 1u);
                        dx_mma_bf16(dim, aRl, bIh, idesc, 1u);
                        dx_mma_bf16(dre, aIh, bIh, idesc_nb, 1u);    // Re Z -= Im Q Im R
                        dx_mma_bf16(dim, aIh, bRh, idesc, 1u);       // Im Z += Im Q Re R
                        dx_mma_bf16(dre, aIh, bIl, idesc_nb, 1u);
                        dx_mma_bf16(dim, aIh, bRl, idesc, 1u);
                        dx_mma_bf16(dre, aIl, bIh, idesc_nb, 1u);
                        dx_mma_bf16(dim, aIl, bRh, idesc, 1u);
                    }
                    dx_commit(bar_empty(st));
                }
                if (!ok) break;
                dx_commit(bar_accf(ab));
            }
            if (!ok) {
                atomicOr(&status[0], TRED_ST_TIMEOUT);
                *abort_flag = 1;
            }
            // every product issued has completed before the tensor memory goes
            dx_commit(bar_done);
            (void)mbar_wait(bar_done, 0);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..9)
        // warp w drains lane quarter w & 3 of accumulator Re Z (w < 6) or Im Z (w >= 6);
        // the first four warps list the tile's block segments (consecutive rows of one
        // slot: slot, first row); then each warp sums its segments' rows into the outputs:
        //     Ihat[u] = sum over the segment's rows r (pixel p') of Z_r[K],  K = p' + 2R - u
        const int te = tid - 64;
        const int ew = te >> 5;   // epilogue warp 0..7
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int R2 = 2 * c.R;
        const int ncc = (c.imoff + 31) / 32;   // 32-column loads per accumulator
        float2 *yacc = yacc_all + ew * (LP * DX_YS);
        // this lane's taps n = lane + 32 j and their output offsets (2R - K per axis)
        int tap_off[DX_TAPS_PER_LANE];
#pragma unroll
        for (int j = 0; j < DX_TAPS_PER_LANE; ++j) {
            const int n = lane + 32 * j;
            tap_off[j] = n < c.ntap ? (R2 - n / c.kp) * DX_YS + (R2 - n % c.kp) : -1;
        }
        int i = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++i) {
            const int f = it / ntiles, t = it - f * ntiles;
            const int ab = i & 1;
            const int nv = min(DX_M, nloc - t * DX_M);
            const int t0g = row0 + t * DX_M;
            if (te < DX_M) rowrec[te] = te < nv ? rows[t0g + te] : -1;
            // the slots of the rows just before and after the tile (a block with rows
            // there is split across tiles)
            if (te == DX_M) rowrec[DX_M] = t0g > 0 ? (rows[t0g - 1] >> 6) : -1;
            if (te == DX_M + 1) rowrec[DX_M + 1] = t0g + nv < nrows ? (rows[t0g + nv] >> 6) : -1;
            int bad = mbar_wait(bar_accf(ab), (uint32_t)((i >> 1) & 1)) ? 0 : 1;
            bad |= *abort_flag;
            if (dx_epi_any(bad)) {   // the eight epilogue warps leave together (and rowrec is complete)
                if (te == 0) {
                    atomicOr(&status[0], TRED_ST_TIMEOUT);
                    *abort_flag = 1;
                }
                break;
            }
            tmem_fence_after();
            const int r = 32 * quarter + lane;
            for (int cc = 0; cc < ncc; ++cc) {   // half 0: Re Z, half 1: Im Z
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(ab * 256 + 128 * half + 32 * cc), v);
                float *zd = Zs + r * SZ + half * c.imoff + 32 * cc;
#pragma unroll
                for (int e4 = 0; e4 < 8; ++e4)
                    if (32 * cc + 4 * e4 < c.imoff)
                        *reinterpret_cast<float4 *>(zd + 4 * e4) = make_float4(v[4 * e4], v[4 * e4 + 1], v[4 * e4 + 2], v[4 * e4 + 3]);
            }
            tmem_fence_before();
            __syncwarp();
            if (lane == 0) dx_arrive(bar_acce(ab));
            // segment starts: ballots of the first four epilogue warps (rows 0..127)
            unsigned sbal = 0u;
            int start = 0, rec = -1;
            if (te < DX_M) {
                rec = rowrec[te];
                start = te < nv && (te == 0 || (rowrec[te - 1] >> 6) != (rec >> 6));
                sbal = __ballot_sync(0xffffffffu, start);
                if (lane == 0) seg_cnt[te >> 5] = __popc(sbal);
            }
            dx_epi_sync();
            if (start) {
                int si = -1;
                for (int w = 0; w < (te >> 5); ++w) si += seg_cnt[w];
                si += __popc(sbal & (0xffffffffu >> (31 - lane)));
                seg_slot[si] = rec >> 6;
                seg_base[si] = te;
            }
            if (te == 0) seg_cnt[4] = seg_cnt[0] + seg_cnt[1] + seg_cnt[2] + seg_cnt[3];
            dx_epi_sync();
            const int nseg = seg_cnt[4];
            const int slot_before = rowrec[DX_M], slot_after = rowrec[DX_M + 1];
            // warp e takes segments e, e + 8, ... and adds its rows in ascending order
            // into the block's 16 x 16 output in its own shared-memory accumulator: row r at
            // pixel p' adds Z_r[K] at u = p' + 2R - K, one lane per tap (the taps of a row
            // reach distinct outputs; the accumulator's row stride 25 = 9 mod 16 puts the 16
            // taps n .. n + 15 a half-warp touches in distinct banks)
            for (int si = ew; si < nseg; si += 8) {
                const int sl = seg_slot[si], base = seg_base[si];
                const int end = si + 1 < nseg ? seg_base[si + 1] : nv;
#pragma unroll
                for (int j = 0; j < (LP * LP) / 32; ++j) {
                    const int u = lane + 32 * j;
                    yacc[(u >> 4) * DX_YS + (u & 15)] = make_float2(0.f, 0.f);
                }
                __syncwarp();
                for (int rr = base; rr < end; ++rr) {
                    const int pp = rowrec[rr] & 63;
                    const int pu = (pp >> c.bpl) * DX_YS + (pp & (c.bp - 1));
                    const float *zr = Zs + rr * SZ;
#pragma unroll
                    for (int j = 0; j < DX_TAPS_PER_LANE; ++j) {
                        if (tap_off[j] < 0) continue;
                        const int n = lane + 32 * j;
                        float2 *y = yacc + pu + tap_off[j];
                        float2 a = *y;
                        a.x += zr[n];
                        a.y += zr[c.imoff + n];
                        *y = a;
                    }
                    __syncwarp();
                }
                const bool split = (si == 0 && sl == slot_before) || (si == nseg - 1 && sl == slot_after);
                float2 *yb = ybuf + ((size_t)sl * c.nbins + f) * (LP * LP);
#pragma unroll
                for (int j = 0; j < (LP * LP) / 32; ++j) {
                    const int u = lane + 32 * j;
                    const float2 a = yacc[(u >> 4) * DX_YS + (u & 15)];
                    if (split) {
                        atomicAdd(&yb[u].x, a.x);
                        atomicAdd(&yb[u].y, a.y);
                    } else {
                        yb[u] = a;
                    }
                }
                __syncwarp();
            }
            dx_epi_sync();
        }
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- inverse time DFT
// Per block (persistent over the slots of the pass, two CTAs per SM), 16 output pixels at
// a time (8 columns of two adjacent rows): their lt/2 + 1 bins staged in shared memory
// pixel-major [u][f] (the next group's loads in flight in registers), then warp w inverts
// the vertical neighbours a = (uy, ux0 + w) and b = (uy + 1, ux0 + w) (of similar size,
// so that the rounding of one half of the packed sequence stays small against the other) as one complex sequence Z[f] = Ihat_a[f] + i Ihat_b[f] (the bins above lt/2 from
// the conjugate symmetry of real signals), N = lt = 32 NPL:
//   pass 1  lane l holds Z[l + 32 m], m < NPL: an NPL-point inverse DFT in registers, the
//           twiddles W_N^-(l t1);
//   transpose through the warp's scratch (S[t1][n2 ^ t1]);
//   pass 2  lanes 2 d + e (d = t1 < NPL) hold the 16 samples n2 = 2 a + e: a 16-point
//           inverse DFT in registers, the twiddles W_32^-(e g), one radix-2 step across
//           the lane pair: lane 2 d + e holds t = d + NPL (g + 16 e) in register k
//           (g = bitrev16(k)), Re z[t] = I_a[t] and Im z[t] = I_b[t].
// A slot with no rows is written as zeros.
constexpr int DX_INV_U = 16;   // output pixels per staged group
template <int G>
__global__ void __launch_bounds__(DX_INV_THREADS, 2)
    k_dx_inv(const float2 *__restrict__ ybuf, const int32_t *__restrict__ rowstart, const int32_t *__restrict__ meta,
             const float2 *__restrict__ tw, DxConst c, int slot_base, float *__restrict__ out) {
    constexpr int LT = 64 * G;
    constexpr int NPL = LT / 32;
    constexpr int NB = LT / 2 + 1;
    constexpr int NW = DX_INV_THREADS / 32;
    constexpr int NLD = (NB * (DX_INV_U / 2) + DX_INV_THREADS - 1) / DX_INV_THREADS;   // 16-byte loads per thread
    static_assert(NW * 2 == DX_INV_U, "one pixel pair per warp");
    extern __shared__ float2 dxs[];
    float2 *Ys = dxs;                                  // [DX_INV_U][NB]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *S = dxs + DX_INV_U * NB + warp * (NPL * 32);   // per-warp transpose scratch
    const int cnt = meta[0];
    const float2 *wlt = tw + TW_LT;
    const int d = lane >> 1, e = lane & 1;
    constexpr int NG = (LP * LP) / DX_INV_U;
    __shared__ float2 twl[NPL][32];   // pass 1 twiddles conj W_N^(l t1), [t1][lane l]
    for (int i = tid; i < NPL * 32; i += DX_INV_THREADS) {
        const float2 w = wlt[((i & 31) * (i >> 5)) % LT];
        twl[i >> 5][i & 31] = make_float2(w.x, -w.y);
    }
    __syncthreads();
    for (int s = blockIdx.x; s < cnt; s += gridDim.x) {
        float *ob = out + (size_t)(slot_base + s) * (LP * LP) * LT;
        if (rowstart[s + 1] == rowstart[s]) {
            float4 *o4 = reinterpret_cast<float4 *>(ob);
            for (int i = tid; i < (LP * LP) * LT / 4; i += DX_INV_THREADS) o4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float4 *yb = reinterpret_cast<const float4 *>(ybuf + (size_t)s * NB * (LP * LP));
        float4 pre[NLD];
        auto load = [&](int ug) {
#pragma unroll
            for (int i = 0; i < NLD; ++i) {
                const int idx = tid + i * DX_INV_THREADS;   // (bin, pixel pair)
                const int f = idx / (DX_INV_U / 2), up = idx - f * (DX_INV_U / 2);
                // group ug: rows 2 (ug >> 1) and 2 (ug >> 1) + 1, columns 8 (ug & 1) .. + 7
                const int u = (2 * (ug >> 1) + (up >> 2)) * LP + 8 * (ug & 1) + 2 * (up & 3);
                pre[i] = f < NB ? __ldg(yb + ((size_t)f * (LP * LP) + u) / 2) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        load(0);
        for (int ug = 0; ug < NG; ++ug) {
            __syncthreads();   // the previous group's reads of Ys are done
#pragma unroll
            for (int i = 0; i < NLD; ++i) {
                const int idx = tid + i * DX_INV_THREADS;
                const int f = idx / (DX_INV_U / 2), up = idx - f * (DX_INV_U / 2);
                if (f < NB) {
                    Ys[(2 * up) * NB + f] = make_float2(pre[i].x, pre[i].y);
                    Ys[(2 * up + 1) * NB + f] = make_float2(pre[i].z, pre[i].w);
                }
            }
            __syncthreads();
            if (ug + 1 < NG) load(ug + 1);
            const float2 *ya = Ys + warp * NB, *ybb = Ys + (warp + NW) * NB;
            float2 v[NPL];
#pragma unroll
            for (int m = 0; m < NPL; ++m) {
                const int f = lane + 32 * m;
                float2 A, B;
                if (f < NB) {
                    A = ya[f];
                    B = ybb[f];
                } else {
                    A = cconj(ya[LT - f]);
                    B = cconj(ybb[LT - f]);
                }
                v[m] = make_float2(A.x - B.y, A.y + B.x);
            }
            fft_reg_any<NPL, true>(v);   // v[k] = U[fft_perm(k)]
            __syncwarp();
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int t1 = fft_perm<NPL>(k);
                const float2 x = t1 ? cmul(v[k], twl[t1][lane]) : v[k];
                S[t1 * 32 + (lane ^ t1)] = x;
            }
            __syncwarp();
            float2 w[16];
#pragma unroll
            for (int a = 0; a < 16; ++a) w[a] = d < NPL ? S[d * 32 + ((2 * a + e) ^ d)] : make_float2(0.f, 0.f);
            fft_reg_dif_c<16, true>(w);   // w[k] = E_e[bitrev16(k)]
#pragma unroll
            for (int k = 1; k < 16; ++k) {
                const int g = bitrev<16>(k);
                if (e) w[k] = cmul(w[k], make_float2(w32c(g), -w32s(g)));
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float2 o;
                o.x = __shfl_xor_sync(0xffffffffu, w[k].x, 1);
                o.y = __shfl_xor_sync(0xffffffffu, w[k].y, 1);
                w[k] = e ? csub(o, w[k]) : cadd(w[k], o);
            }
            if (d < NPL) {
                const int ua = (2 * (ug >> 1)) * LP + 8 * (ug & 1) + warp;
                float *oa = ob + (size_t)ua * LT;
                float *obb = ob + (size_t)(ua + LP) * LT;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int t = d + NPL * (bitrev<16>(k) + 16 * e);
                    oa[t] = w[k].x;
                    obb[t] = w[k].y;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- inverse time DFT + gather
// The inverse time DFT and the electrode gather (a5) in one kernel, for block shapes with
// kp = bp + 1 (R = bp / 2; bp = 8) and nr - 1 <= bt.  The pixel plane is cut into 8 x 8
// tiles offset by R from the block grid; every pixel of a tile lies in the output
// footprints of the same 2 x 2 spatial blocks (bx, by) in {tx, tx + 1} x {ty, ty + 1}, at
// u = pixel - (bp b - R).  CTAs take tiles from a queue over the list of tiles some active
// block meets (k_dx_tile_mark and a ballot / scan compaction).  Per tile, 16 pixels at a time
// (group g: the 8 columns of rows 2 g and 2 g + 1) and per time block bt in ascending
// order: the spectra of the active blocks of the 2 x 2 set are summed per bin (first the
// lowest-numbered active block, then the others in order; the first one's loads are issued
// while the previous item is transformed) and staged [pixel][f]; warp w inverts its two
// vertical neighbours (column w) as one complex sequence (the two-pass FFT of k_dx_inv).
// Ticks t < bt of the result, plus what time block bt - 1 left for t < nr - 1, are the
// final values of ticks bt bt_len + t: assembled in the warp's tick buffer (shared memory)
// and written to the waveform rows once, with 16-byte stores; ticks bt .. bt + nr - 2 (the
// tail) then move to the front of the buffer for time block bt + 1.  Time blocks with no
// active block in the set cost no transform: their ticks are the previous tail or zero.  Every tick of an active pixel's row is written; each pixel belongs to one
// warp, so every sum has a fixed order.  The per-pixel sum of the positive current
// (readout bound) is kept per lane and reduced per pixel in a fixed order.
constexpr int DX_NBT_MAX = 128;   // time blocks per event the fused gather handles
struct DxWaveConst {
    int npx_x, npy_e, nby_e, nbx, nbt, n_events, bp, bt, nr, nt;
};
// per-warp tick buffer of one pixel: lt ticks (bt <= lt) and a 16-float gap after the
// first 16 NPL ticks, so that the lanes of the two halves of a transform (ticks t and
// t + 16 NPL) write distinct banks
#define DX_BUFW(G) (64 * (G) + 16)
template <int NPL>
__device__ __forceinline__ int dx_bpos(int t) { return t + (t >= 16 * NPL ? 16 : 0); }
// k_dx_wave CTAs per SM (three, with the transpose scratch over the staged spectra
// behind one more barrier and 80 registers: 6.0 against 3.1 ms on a module plane;
// 128-thread CTAs on half a tile's columns, four per SM: 3.8 ms)
constexpr int DX_WAVE_CTAS = 2;
__host__ __device__ constexpr size_t dx_wave_smem(int G) {
    // staged spectra [16][32 G + 1], transpose scratch [8 warps][64 G], tick buffers [8][2][64 G + 16]
    return sizeof(float2) * ((size_t)16 * (32 * G + 1) + (size_t)8 * 64 * G) + sizeof(float) * (size_t)8 * 2 * DX_BUFW(G);
}
// flag the four pixel tiles each active block's footprint meets: tile (tx, ty) holds the
// blocks {tx, tx + 1} x {ty, ty + 1}, so block (bx, by) meets tiles bx - 1, bx and by - 1, by
__global__ void k_dx_tile_mark(const int32_t *__restrict__ block_ids, const int32_t *__restrict__ n_blocks_dev,
                               DxWaveConst c, int32_t *__restrict__ tflag) {
    const int nb = n_blocks_dev[0];
    const int ntx = c.nbx + 1, nty = c.nby_e + 1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 4 * nb; k += gridDim.x * blockDim.x) {
        const int blk = block_ids[k >> 2], q = k & 3;
        const int bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int ev = by / c.nby_e, byl = by - ev * c.nby_e;
        const int tx = bx - (q & 1), ty = byl - (q >> 1);
        tflag[(ev * nty + ty + 1) * ntx + tx + 1] = 1;
    }
}

template <int G>
__global__ void __launch_bounds__(DX_INV_THREADS, DX_WAVE_CTAS)
    k_dx_wave(const float2 *__restrict__ ybuf, const int32_t *__restrict__ slot_of, const int32_t *__restrict__ pix_row,
              const uint64_t *__restrict__ pmask, const float2 *__restrict__ tw, DxWaveConst c,
              const int32_t *__restrict__ tile_list, const int32_t *__restrict__ tile_count,
              int32_t *__restrict__ queue, float *__restrict__ wave, float *__restrict__ possum) {
    constexpr int LT = 64 * G;
    constexpr int NPL = LT / 32;
    constexpr int NB = LT / 2 + 1;
    constexpr int NW = DX_INV_THREADS / 32;
    constexpr int NLD = (NB * 8 + DX_INV_THREADS - 1) / DX_INV_THREADS;   // 16-byte loads per thread and block
    static_assert(NW == 8, "one column of the 8-pixel tile per warp");
    extern __shared__ float2 dxs[];
    __shared__ int tslot[4][DX_NBT_MAX];
    __shared__ int nzbt[DX_NBT_MAX];   // the tile's time blocks with an active block, ascending
    __shared__ int s_tile, s_nnz;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *Ys = dxs;                                       // [16][NB]
    float2 *S = dxs + 16 * NB + warp * (NPL * 32);          // per-warp transpose scratch
    float *bufa = reinterpret_cast<float *>(dxs + 16 * NB + NW * NPL * 32) + warp * (2 * DX_BUFW(G));
    float *bufb = bufa + DX_BUFW(G);   // per warp: the two pixels' tick buffers
    const float2 *wlt = tw + TW_LT;
    const int d = lane >> 1, e = lane & 1;
    const int half = c.bp >> 1;
    const int ntx = c.nbx + 1, nty = c.nby_e + 1;
    const int ntile = tile_count[0];   // the tiles some active block meets (tile_list)
    const int span = c.bt + c.nr - 1;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // pass 1 twiddles conj W_N^(l t1), [t1][lane l], in shared memory (3.02 against 3.13 ms
    // per module-plane step through the read-only cache); the item loop's first barrier
    // orders them before their use
    __shared__ float2 twl[NPL][32];
    for (int i = tid; i < NPL * 32; i += DX_INV_THREADS) {
        const float2 w = wlt[((i & 31) * (i >> 5)) % LT];
        twl[i >> 5][i & 31] = make_float2(w.x, -w.y);
    }
    // this thread's 16-byte loads of item (g, bt), block k of the 2 x 2 set (slot sl)
    auto load_block = [&](int g, int k, int sl, float4 *dst, bool add) {
#pragma unroll
        for (int i = 0; i < NLD; ++i) {
            const int idx = tid + i * DX_INV_THREADS;   // (bin, pixel pair)
            const int f = idx >> 3, up = idx & 7;
            if (f < NB) {
                // tile row 2 g + (up >> 2), columns 2 (up & 3) and + 1
                const int uy = 2 * g + (up >> 2) + (k >> 1 ? 0 : c.bp), ux = 2 * (up & 3) + (k & 1 ? 0 : c.bp);
                const float4 v = __ldg(reinterpret_cast<const float4 *>(
                    ybuf + ((size_t)sl * NB + f) * (LP * LP) + uy * LP + ux));
                if (add) {
                    dst[i].x += v.x;
                    dst[i].y += v.y;
                    dst[i].z += v.z;
                    dst[i].w += v.w;
                } else {
                    dst[i] = v;
                }
            }
        }
    };
    // items: whole tiles, or (tile, group of 16 pixels) when there are fewer than two
    // tiles per CTA (a small event), so that its few tiles spread over more CTAs (the
    // groups of a tile are independent; every CTA derives the same choice)
    const bool split = ntile < 2 * (int)gridDim.x;
    const int nitem = split ? 4 * ntile : ntile;
    __shared__ int s_g0;
    for (;;) {   // items from a queue: their cost varies with the number of active blocks
        if (tid == 0) {
            const int q = atomicAdd(queue, 1);
            s_tile = q < nitem ? tile_list[split ? q >> 2 : q] : -1;
            s_g0 = split ? (q & 3) : 0;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) break;
        const int g0 = s_g0, g1 = split ? g0 + 1 : 4;   // the item's groups [g0, g1)
        const int ev = tile / (nty * ntx), rem = tile - ev * (nty * ntx);
        const int ty = rem / ntx - 1, tx = rem % ntx - 1;
        int found = 0;
        for (int i = tid; i < 4 * c.nbt; i += DX_INV_THREADS) {
            const int k = i / c.nbt, bt = i - k * c.nbt;
            const int bx = tx + (k & 1), byl = ty + (k >> 1);
            int sl = -1;
            if (bx >= 0 && bx < c.nbx && byl >= 0 && byl < c.nby_e) {
                sl = slot_of[((int64_t)(ev * c.nby_e + byl) * c.nbx + bx) * c.nbt + bt];
                found |= sl >= 0;   // its pixels are active: their rows are written, zeros if need be
                if (sl >= 0 && pmask[sl] == 0ull) sl = -1;   // no pixel holds charge: no spectrum written
            }
            tslot[k][bt] = sl;
        }
        if (!__syncthreads_or(found)) continue;
        if (warp == 0) {   // the time blocks with a spectrum, ascending
            int base = 0;
            for (int b0 = 0; b0 < c.nbt; b0 += 32) {
                const int bt = b0 + lane;
                const bool on = bt < c.nbt && (tslot[0][bt] >= 0 || tslot[1][bt] >= 0 || tslot[2][bt] >= 0 ||
                                               tslot[3][bt] >= 0);
                const unsigned bal = __ballot_sync(0xffffffffu, on);
                if (on) nzbt[base + __popc(bal & ((1u << lane) - 1u))] = bt;
                base += __popc(bal);
            }
            if (lane == 0) s_nnz = base;
        }
        __syncthreads();
        const int nnz = s_nnz;
        // the first active block of item (g, bt), issued ahead into pre (pre_k: its index)
        float4 pre[NLD];
        int pre_k = -1;
        auto prefetch = [&](int g, int bt) {
            pre_k = tslot[0][bt] >= 0 ? 0 : tslot[1][bt] >= 0 ? 1 : tslot[2][bt] >= 0 ? 2 : 3;
            load_block(g, pre_k, tslot[pre_k][bt], pre, false);
        };
        if (nnz > 0) prefetch(g0, nzbt[0]);
        // this warp's pixels: column w of the tile, rows 2 g (a) and 2 g + 1 (b)
        const int x = c.bp * tx + half + warp;
#pragma unroll 1
        for (int g = g0; g < g1; ++g) {
            int ra = -1, rb = -1;
            {
                const int ya = c.bp * ty + half + 2 * g, yb = ya + 1;
                const bool inx = x >= 0 && x < c.npx_x;
                if (inx && ya >= 0 && ya < c.npy_e) ra = pix_row[(int64_t)(ev * c.npy_e + ya) * c.npx_x + x];
                if (inx && yb >= 0 && yb < c.npy_e) rb = pix_row[(int64_t)(ev * c.npy_e + yb) * c.npx_x + x];
            }
            float *wa = ra >= 0 ? wave + (size_t)ra * c.nt : nullptr;
            float *wb = rb >= 0 ? wave + (size_t)rb * c.nt : nullptr;
            float pa = 0.f, pb = 0.f;
            bool live = false;   // the buffer's front holds time block bt - 1's tail
            int jn = 0;          // next entry of nzbt
            for (int bt = 0; bt < c.nbt; ++bt) {
                const bool act = jn < nnz && nzbt[jn] == bt;
                float2 w[16];
                if (act) {
                    ++jn;
                    __syncthreads();   // the previous item's reads of Ys are done
#pragma unroll
                    for (int k = 1; k < 4; ++k) {   // the other active blocks, in order
                        const int sl = tslot[k][bt];
                        if (k > pre_k && sl >= 0) load_block(g, k, sl, pre, true);
                    }
#pragma unroll
                    for (int i = 0; i < NLD; ++i) {
                        const int idx = tid + i * DX_INV_THREADS;
                        const int f = idx >> 3, up = idx & 7;
                        if (f < NB) {
                            const int pr = (up >> 2) * 8 + 2 * (up & 3);   // staged row of the first pixel
                            Ys[pr * NB + f] = make_float2(pre[i].x, pre[i].y);
                            Ys[(pr + 1) * NB + f] = make_float2(pre[i].z, pre[i].w);
                        }
                    }
                    __syncthreads();
                    {   // the next item's first block, in flight during this transform
                        const int gn = jn < nnz ? g : g + 1, jj = jn < nnz ? jn : 0;
                        if (gn < g1) prefetch(gn, nzbt[jj]);
                    }
                    const float2 *ya = Ys + warp * NB, *ybb = Ys + (warp + 8) * NB;
                    float2 v[NPL];
#pragma unroll
                    for (int m = 0; m < NPL; ++m) {
                        const int f = lane + 32 * m;
                        float2 A, B;
                        if (f < NB) {
                            A = ya[f];
                            B = ybb[f];
                        } else {
                            A = cconj(ya[LT - f]);
                            B = cconj(ybb[LT - f]);
                        }
                        v[m] = make_float2(A.x - B.y, A.y + B.x);
                    }
                    fft_reg_any<NPL, true>(v);
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < NPL; ++k) {
                        const int t1 = fft_perm<NPL>(k);
                        float2 xv = v[k];
                        if (t1) xv = cmul(xv, twl[t1][lane]);
                        S[t1 * 32 + (lane ^ t1)] = xv;
                    }
                    __syncwarp();
#pragma unroll
                    for (int a = 0; a < 16; ++a) w[a] = d < NPL ? S[d * 32 + ((2 * a + e) ^ d)] : make_float2(0.f, 0.f);
                    fft_reg_dif_c<16, true>(w);
#pragma unroll
                    for (int k = 1; k < 16; ++k) {
                        const int gg = bitrev<16>(k);
                        if (e) w[k] = cmul(w[k], make_float2(w32c(gg), -w32s(gg)));
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        float2 o;
                        o.x = __shfl_xor_sync(0xffffffffu, w[k].x, 1);
                        o.y = __shfl_xor_sync(0xffffffffu, w[k].y, 1);
                        w[k] = e ? csub(o, w[k]) : cadd(w[k], o);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) w[k] = make_float2(0.f, 0.f);
                }
                // ticks t < bt: the transform plus, for t < nr - 1, time block bt - 1's tail
                // (held at the front of the warp's buffer), assembled in the buffer and
                // written to the rows with 16-byte stores; then the new tail moves to the front
                __syncwarp();   // the previous item's buffer reads and tail writes are done
                if (act && d < NPL) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int t = d + NPL * (bitrev<16>(k) + 16 * e);
                        if (t < c.bt) {
                            float va = w[k].x, vb = w[k].y;
                            if (live && t < c.nr - 1) {
                                va += bufa[dx_bpos<NPL>(t)];
                                vb += bufb[dx_bpos<NPL>(t)];
                            }
                            bufa[dx_bpos<NPL>(t)] = va;
                            bufb[dx_bpos<NPL>(t)] = vb;
                        }
                    }
                }
                __syncwarp();
                {
                    const int lim = act ? c.bt : live ? c.nr - 1 : 0;   // buffer ticks below lim are valid
                    float *oa = wa ? wa + (size_t)bt * c.bt : nullptr;
                    float *ob = wb ? wb + (size_t)bt * c.bt : nullptr;
                    for (int t0 = 4 * lane; t0 < c.bt; t0 += 128) {
                        float4 va = zero4, vb = zero4;
                        if (t0 < lim) {
                            va = *reinterpret_cast<const float4 *>(bufa + dx_bpos<NPL>(t0));
                            vb = *reinterpret_cast<const float4 *>(bufb + dx_bpos<NPL>(t0));
                            if (t0 + 4 > lim) {   // the tail ends inside this quad
                                if (t0 + 1 >= lim) va.y = vb.y = 0.f;
                                if (t0 + 2 >= lim) va.z = vb.z = 0.f;
                                va.w = vb.w = 0.f;
                            }
                            pa += fmaxf(va.x, 0.f) + fmaxf(va.y, 0.f) + fmaxf(va.z, 0.f) + fmaxf(va.w, 0.f);
                            pb += fmaxf(vb.x, 0.f) + fmaxf(vb.y, 0.f) + fmaxf(vb.z, 0.f) + fmaxf(vb.w, 0.f);
                        }
                        if (oa) *reinterpret_cast<float4 *>(oa + t0) = va;
                        if (ob) *reinterpret_cast<float4 *>(ob + t0) = vb;
                    }
                }
                __syncwarp();   // the buffer is read before the tail replaces its front
                if (act && d < NPL) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int t = d + NPL * (bitrev<16>(k) + 16 * e);
                        if (t >= c.bt && t < span) {
                            bufa[dx_bpos<NPL>(t - c.bt)] = w[k].x;
                            bufb[dx_bpos<NPL>(t - c.bt)] = w[k].y;
                        }
                    }
                }
                live = act;
            }
            if (possum) {
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    pa += __shfl_xor_sync(0xffffffffu, pa, o);
                    pb += __shfl_xor_sync(0xffffffffu, pb, o);
                }
                if (lane == 0) {
                    if (ra >= 0) possum[ra] = pa;
                    if (rb >= 0) possum[rb] = pb;
                }
            }
        }
        __syncthreads();   // tslot, nzbt and Ys are reused by the next tile
    }
}

// ---------------------------------------------------------------- host side
// 2-D BF16 tensor [rows][inner], box [box_rows][64] (128 bytes), 128-byte swizzle; columns
// past inner read as zero
static int dx_make_map(tred_handle *h, CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t rows,
                       uint32_t box_rows) {
    auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!fn) return set_error(h, TRED_ERR_CUDA, "direct form: cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {(cuuint32_t)DX_KC, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(h, TRED_ERR_CUDA, "direct form: tensor map encode failed (%d)", (int)r);
    return TRED_OK;
}

template <int G>
static int run_direct(tred_handle *h, const DxConst &c, const int32_t *n_blocks_dev, const float *qeff, float *out,
                      int slot_base, int slot_count, int qbase, cudaStream_t s, bool inverse) {
    const size_t fwd_smem = dx_fwd_smem(c.nch, c.nbins);
    const size_t gemm_smem = dx_gemm_smem(c.npad, c.ntap);
    const size_t inv_smem = sizeof(float2) * ((size_t)DX_INV_U * (32 * G + 1) + (size_t)(DX_INV_THREADS / 32) * 64 * G);
    // the largest dynamic shared memory asked for so far (shapes differ between handles)
    static size_t set_fwd = 0, set_inv = 0;
    static size_t set_gemm = 0;
    if (fwd_smem > set_fwd) {
        cudaFuncSetAttribute(k_dx_fwd<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem);
        cudaFuncSetAttribute(k_dx_fwd<G>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        set_fwd = fwd_smem;
    }
    if (gemm_smem > set_gemm) {
        cudaFuncSetAttribute(k_dx_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem);
        set_gemm = gemm_smem;
    }
    if (inv_smem > set_inv) {
        cudaFuncSetAttribute(k_dx_inv<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem);
        cudaFuncSetAttribute(k_dx_inv<G>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        set_inv = inv_smem;
    }
    CUtensorMap tah, tal, tbh, tbl;
    int rc = dx_make_map(h, &tah, h->dx_qhi, (uint64_t)c.kq, (uint64_t)c.nbins * c.rows_cap, DX_M);
    if (!rc) rc = dx_make_map(h, &tal, h->dx_qlo, (uint64_t)c.kq, (uint64_t)c.nbins * c.rows_cap, DX_M);
    if (!rc) rc = dx_make_map(h, &tbh, h->dx_bhi, (uint64_t)c.kq, (uint64_t)c.nbins * c.npad, (uint32_t)c.npad);
    if (!rc) rc = dx_make_map(h, &tbl, h->dx_blo, (uint64_t)c.kq, (uint64_t)c.nbins * c.npad, (uint32_t)c.npad);
    if (rc) return rc;
    const int sms = num_sms(h);
    const int end = slot_base + slot_count;
    for (int base = slot_base; base < end; base += h->dx_blocks) {
        const int cnt = h->dx_blocks < end - base ? h->dx_blocks : end - base;
        // with conv_keep_spectra the pixel masks and the spectra are stored at absolute
        // slots (one pass covers the call), otherwise relative to the pass
        const size_t ao = h->p.conv_keep_spectra ? (size_t)base : 0;
        float2 *ybase = h->dx_y + ao * c.nbins * (LP * LP);
        k_dx_pixmask<<<sms * 4, 256, 0, s>>>(n_blocks_dev, h->colmask, c.nch, c.bp2, base, cnt, h->dx_pmask + ao,
                                             h->dx_pcnt + ao);
        k_dx_rows<<<1, DX_ROWS_THREADS, 0, s>>>(n_blocks_dev, h->dx_pmask + ao, h->dx_pcnt + ao, base, cnt,
                                                h->dx_rows, h->dx_rowstart, h->dx_meta);
        h->launches += 2;
        const int64_t max_rows = (int64_t)cnt * c.bp2;
        const int nrc = (int)((max_rows + c.rows_cap - 1) / c.rows_cap);
        for (int k = 0; k < nrc; ++k) {
            const int row0 = k * c.rows_cap;
            kt_begin(h, TRED_KT_DX_FWD, s);
            k_dx_fwd<G><<<DX_FWD_CTAS * sms, DX_FWD_THREADS, fwd_smem, s>>>(qeff, h->colmask, h->dx_rows, h->dx_rowstart, h->dx_meta,
                                                             h->tw, c, base, qbase, row0, k == 0 ? 1 : 0, h->dx_qhi,
                                                             h->dx_qlo, ybase);
            kt_end(h, TRED_KT_DX_FWD, s);
            kt_begin(h, TRED_KT_DX_GEMM, s);
            k_dx_gemm<<<sms, DX_GEMM_THREADS, gemm_smem, s>>>(tah, tal, tbh, tbl, h->dx_rows, h->dx_rowstart,
                                                              h->dx_meta, c, row0, ybase, h->status);
            kt_end(h, TRED_KT_DX_GEMM, s);
            h->launches += 2;
        }
        if (!inverse) continue;   // the spectra stay in dx_y for k_dx_wave (a single pass)
        kt_begin(h, TRED_KT_DX_INV, s);
        k_dx_inv<G><<<2 * sms, DX_INV_THREADS, inv_smem, s>>>(ybase, h->dx_rowstart, h->dx_meta, h->tw, c, base, out);
        kt_end(h, TRED_KT_DX_INV, s);
        h->launches += 1;
    }
    return check_cuda(h, cudaGetLastError(), "direct-form launch");
}

int launch_direct(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, float *out, int slot_base,
                  int slot_count, int qbase, cudaStream_t s) {
    const DxConst c = dx_const_of(h);
    if (c.lt == 512) return run_direct<8>(h, c, n_blocks_dev, qeff, out, slot_base, slot_count, qbase, s, true);
    if (c.lt == 384) return run_direct<6>(h, c, n_blocks_dev, qeff, out, slot_base, slot_count, qbase, s, true);
    return set_error(h, TRED_ERR_INVALID_ARG, "direct form: lt must be 384 or 512");
}

// the shapes the fused inverse + gather covers: every slot in one pass (the spectra of
// all blocks resident at once), 8 x 8 pixel tiles (bp = 8, kp = bp + 1), a block's tail
// overlapping only the next time block, FP32 sums
bool dx_wave_ok(const tred_handle *h) {
    return h->p.conv_mode == 4 && h->g.bp == 8 && h->g.kp == h->g.bp + 1 && h->d.R == h->g.bp / 2 &&
           h->g.nr - 1 <= h->g.bt && h->d.nbt <= DX_NBT_MAX && h->max_blocks <= h->dx_blocks &&
           !h->p.compensated_gather && (h->g.lt == 512 || h->g.lt == 384);
}

template <int G>
static int run_wave(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev, int32_t *queue, float *wave,
                    float *possum, cudaStream_t s) {
    const size_t smem = dx_wave_smem(G);
    static size_t set = 0;
    if (smem > set) {
        cudaFuncSetAttribute(k_dx_wave<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_dx_wave<G>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        set = smem;
    }
    const DxWaveConst c{h->g.npx_x, h->d.npy_e, h->d.nby_e, h->d.nbx, h->d.nbt, h->d.n_events,
                        h->g.bp,    h->g.bt,    h->g.nr,    h->g.nt};
    int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "tile queue reset");
    if (!rc) rc = check_cuda(h, cudaMemsetAsync(h->dx_tflag, 0, sizeof(int32_t) * (size_t)h->dx_ntiles, s),
                             "tile flags reset");
    if (rc) return rc;
    // the list of tiles some active block meets (the others hold no active pixel)
    k_dx_tile_mark<<<num_sms(h) * 2, 256, 0, s>>>(block_ids, n_blocks_dev, c, h->dx_tflag);
    h->launches += 1;
    rc = launch_flag_list(h, h->dx_ntiles, h->dx_tflag, h->dx_tpart, h->dx_tlist, h->dx_tcount, s);
    if (rc) return rc;
    kt_begin(h, TRED_KT_DX_WAVE, s);
    k_dx_wave<G><<<DX_WAVE_CTAS * num_sms(h), DX_INV_THREADS, smem, s>>>(h->dx_y, h->blk_slot, h->pix_flag, h->dx_pmask, h->tw,
                                                               c, h->dx_tlist, h->dx_tcount, queue, wave, possum);
    kt_end(h, TRED_KT_DX_WAVE, s);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "direct-form inverse + gather launch");
}

// a4 up to the per-block spectra of slots [slot_base, slot_base + slot_count) (no inverse;
// qeff rows from slot_base), then, once every active slot's spectra are in place and the
// pixel list and the slot map are built (launch_pixel_list), the inverse time DFT of each
// tile straight into the waves
int launch_direct_spectra(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, int slot_base,
                          int slot_count, cudaStream_t s) {
    const DxConst c = dx_const_of(h);
    if (c.lt == 512) return run_direct<8>(h, c, n_blocks_dev, qeff, nullptr, slot_base, slot_count, slot_base, s, false);
    if (c.lt == 384) return run_direct<6>(h, c, n_blocks_dev, qeff, nullptr, slot_base, slot_count, slot_base, s, false);
    return set_error(h, TRED_ERR_INVALID_ARG, "direct form: lt must be 384 or 512");
}
int launch_direct_wave(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev, int32_t *queue,
                       float *wave, float *possum, cudaStream_t s) {
    if (h->g.lt == 512) return run_wave<8>(h, block_ids, n_blocks_dev, queue, wave, possum, s);
    if (h->g.lt == 384) return run_wave<6>(h, block_ids, n_blocks_dev, queue, wave, possum, s);
    return set_error(h, TRED_ERR_INVALID_ARG, "direct form: lt must be 384 or 512");
}

// sizes of the direct form's buffers (tred_create)
size_t dx_bytes_b(int nbins, int npad, int kq) { return 2 * (size_t)nbins * npad * kq; }
size_t dx_bytes_q(int nbins, int rows_cap, int kq) { return 2 * (size_t)nbins * rows_cap * kq; }
int dx_rows_cap_of(int dx_blocks, int bp2, int cap_param) {
    const int64_t want = (int64_t)dx_blocks * bp2;
    const int64_t lim = cap_param > 0 ? cap_param : DX_ROWS_MAX;
    const int64_t cap = want < lim ? want : lim;
    return (int)((cap + DX_M - 1) / DX_M * DX_M);
}
int dx_blocks_of(int max_blocks) { return max_blocks < DX_BLOCKS_MAX ? max_blocks : DX_BLOCKS_MAX; }
// the forward kernel's transposition buffer must fit in one CTA's shared memory
bool dx_shape_ok(int nch, int lt) { return dx_fwd_smem(nch, lt / 2 + 1) <= 227 * 1024; }

}  // namespace tred
