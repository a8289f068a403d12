// a4, tensor-core form: the time DFT of the interlaced convolution (Sec. II-D, Eq.
// interlaced; Sec. III-A-2, Eq. multch) as a GEMM on the tcgen05 tensor cores.
//
// For one active block and one channel pair (j, j') the 128 rows of the A operand are
// the bp^2 = 64 time columns of impact j followed by the 64 columns of j' (FP32 Q^eff,
// t fastest, straight from the effective-charge buffer), and the 512 rows of the B
// operand are a real DFT basis of length lt = 512 over the block's bt ticks:
//     row 2f:   cos(2 pi f t / lt),  f = 0..255
//     row 2f+1: -sin(2 pi f t / lt), f = 1..255;  row 1: cos(pi t) (the f = 256 bin)
// so D = A B^T (128 x 512, FP32 in tensor memory) holds the half spectra of the 128
// real columns.  The epilogue forms the MPCP-packed spectrum of every bin,
//     Z[f]       = X_j[c][f] + i X_j'[flip c][f]
//     Z[lt - f]  = conj(X_j[c][f]) + i conj(X_j'[flip c][f]),
// and writes it in the order the spatial stage of k_conv_spec reads:
// zspec[slot][k1][pair][k2][c] with f = k1 + G k2 (G = lt / 64).
//
// Precision forms: TF32 (conv_mode 1): both operands rounded to the nearest TF32 (A in
// shared memory after the copy, the basis on the host), one product, FP32
// accumulation.  Split TF32 (conv_mode 2): A = A_hi + A_lo and B = B_hi + B_lo, three
// products A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation.  Split BF16 (conv_mode
// 3): the same three products with BF16 parts (8 significant bits each, so hi + lo
// carries 16 of FP32's 24), kind::f16 products of 16 ticks, K chunks of 64 ticks: the
// FP32 A chunk lands by TMA in a staging tile and is split into BF16 hi and lo tiles in
// shared memory; the basis parts are BF16 on the device.  BF16 keeps FP32's exponent
// range, so the split needs no per-block scaling.
//
// Data movement: TMA (cp.async.bulk.tensor, 128-byte swizzle) brings 32-tick chunks of
// A (two boxes of 64 rows) and B (two boxes of 256 rows) into shared memory, one
// elected thread issues tcgen05.mma (M = 128, N = 256, K = 8 per instruction, two N
// halves) and commits to an mbarrier; four warps drain the accumulator with
// tcgen05.ld.  Every mbarrier wait is bounded (clock64), sets TRED_ST_TIMEOUT when it
// expires, waits once more (bounded) for the copies or products in flight, frees the
// tensor memory and returns.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "tred_internal.cuh"

namespace tred {

constexpr int DG_THREADS = 128;
constexpr int DG_KC = 32;                       // K chunk: 32 FP32 = one 128-byte row
constexpr int DG_N = 512;                       // accumulator columns
constexpr int DG_ROWS = 128;                    // A rows: 64 columns of j, 64 of j'
constexpr int DG_SROW = 33;                     // epilogue staging row (floats)
constexpr uint32_t DG_A_BYTES = DG_ROWS * DG_KC * 4;          // 16 KB
constexpr uint32_t DG_B_BYTES = DG_N * DG_KC * 4;             // 64 KB
// one operand stage: A_hi [A_lo] B_hi [B_lo]; TF32 keeps two stages, split TF32 one
template <bool SPLIT> struct DgStage {
    static constexpr int STAGES = SPLIT ? 1 : 2;
    static constexpr uint32_t OFF_AHI = 0;
    static constexpr uint32_t OFF_ALO = DG_A_BYTES;
    static constexpr uint32_t OFF_BHI = SPLIT ? 2 * DG_A_BYTES : DG_A_BYTES;
    static constexpr uint32_t OFF_BLO = OFF_BHI + DG_B_BYTES;
    static constexpr uint32_t BYTES = SPLIT ? 2 * (DG_A_BYTES + DG_B_BYTES) : DG_A_BYTES + DG_B_BYTES;
    static constexpr uint32_t OFF_STAGE = STAGES * BYTES;                  // epilogue staging
    static constexpr uint32_t OFF_BAR = OFF_STAGE + DG_ROWS * DG_SROW * 4;
    static constexpr size_t SMEM = OFF_BAR + 64 + 1024;                    // + alignment slack
};

struct DgConst {
    int nch, cols, bt, npairs, G, mpcp;
};


// Bounded-wait self-test: one thread initialises an mbarrier that expects one arrival
// which never comes, waits on it for `limit` cycles and reports the expiry in the status
// word exactly as the tensor-core convolution's waits do (TRED_ST_TIMEOUT).  Nothing is
// left in flight: the barrier is plain shared memory, released when the CTA exits.
__global__ void k_wait_selftest(long long limit, int32_t *__restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    if (!mbar_wait(b, 0, limit)) atomicOr(&status[0], TRED_ST_TIMEOUT);
}

int launch_wait_selftest(tred_handle *h, long long limit, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(limit, h->status);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "wait self-test launch");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// K-major operand with 128-byte swizzle: rows of 128 B, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= (uint64_t)2 << 61;                        // 128-byte swizzle
    return d;
}
// instruction descriptor: D FP32, A and B TF32, both K-major, N = 256, M = 128
constexpr uint32_t DG_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(DG_IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// round to the nearest TF32 (10 explicit mantissa bits), ties away from zero
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <bool SPLIT>
__global__ void __launch_bounds__(DG_THREADS, 1)
    k_dft_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
               const __grid_constant__ CUtensorMap tmBlo, const int32_t *__restrict__ n_blocks_dev,
               const int32_t *__restrict__ pair_j, DgConst c, float2 *__restrict__ zspec,
               int32_t *__restrict__ status, int slot_base, int slot_count, int qbase) {
    using L = DgStage<SPLIT>;
    constexpr int ST = L::STAGES;
    extern __shared__ unsigned char dg_raw[];
    const uint32_t raw = smem_u32(dg_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = dg_raw + (base - raw);
    float *stage = reinterpret_cast<float *>(gbase + L::OFF_STAGE);
    // barriers: full[s] (copies landed), mma[s] (products that read stage s done)
    const uint32_t bar0 = base + L::OFF_BAR;
    auto bar_full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
    auto bar_mma = [&](int st) { return bar0 + 16u + 8u * (uint32_t)st; };
    uint32_t *tslot = reinterpret_cast<uint32_t *>(gbase + L::OFF_BAR + 32);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        tmem_alloc(tslot, DG_N);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int st = 0; st < ST; ++st) {
            mbar_init(bar_full(st), 1);
            mbar_init(bar_mma(st), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *tslot;

    const int nb = n_blocks_dev[0];
    const int nloc = max(0, min(slot_count, nb - slot_base));
    const int tiles = nloc * c.npairs;
    const int nkc = c.bt / DG_KC;
    const int my_tiles = tiles > (int)blockIdx.x ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Q = my_tiles * nkc;                      // this CTA's chunk stream
    const uint32_t tx_bytes = DG_A_BYTES + DG_B_BYTES * (SPLIT ? 2u : 1u);
    // chunk q uses stage q % ST for the (q / ST)-th time: its copies and its products
    // complete the phase of parity (q / ST) & 1 of that stage's two barriers
    auto par = [&](int q) { return (uint32_t)((q / ST) & 1); };
    int bad = 0;        // 1: a copy wait expired, 2: a product wait expired
    int last_q = -1;    // last chunk whose products were issued

    auto tile_of = [&](int q) { return (int)blockIdx.x + (q / nkc) * (int)gridDim.x; };
    auto issue = [&](int q) {          // thread 0: copies of chunk q into stage q % ST
        const int st = q % ST, tile = tile_of(q), kc = q % nkc;
        const int sl = tile / c.npairs, p = tile - sl * c.npairs;
        const int slot = slot_base + sl;
        const int j1 = pair_j[2 * p], j2r = pair_j[2 * p + 1];
        const int j2 = j2r >= 0 ? j2r : j1;            // without MPCP the upper rows are unused
        const int row1 = ((slot - qbase) * c.nch + j1) * c.cols;
        const int row2 = ((slot - qbase) * c.nch + j2) * c.cols;
        const uint32_t sb = base + (uint32_t)st * L::BYTES;
        mbar_expect_tx(bar_full(st), tx_bytes);
        tma_load_2d(sb + L::OFF_AHI, &tmA, kc * DG_KC, row1, bar_full(st));
        tma_load_2d(sb + L::OFF_AHI + 64 * 128, &tmA, kc * DG_KC, row2, bar_full(st));
        tma_load_2d(sb + L::OFF_BHI, &tmBhi, kc * DG_KC, 0, bar_full(st));
        tma_load_2d(sb + L::OFF_BHI + 256 * 128, &tmBhi, kc * DG_KC, 256, bar_full(st));
        if (SPLIT) {
            tma_load_2d(sb + L::OFF_BLO, &tmBlo, kc * DG_KC, 0, bar_full(st));
            tma_load_2d(sb + L::OFF_BLO + 256 * 128, &tmBlo, kc * DG_KC, 256, bar_full(st));
        }
    };
    if (tid == 0)
        for (int q = 0; q < ST && q < Q; ++q) issue(q);

    for (int q = 0; q < Q; ++q) {
        const int st = q % ST, kc = q % nkc;
        const uint32_t sb = base + (uint32_t)st * L::BYTES;
        float *a_hi = reinterpret_cast<float *>(gbase + (size_t)st * L::BYTES + L::OFF_AHI);
        float *a_lo = reinterpret_cast<float *>(gbase + (size_t)st * L::BYTES + L::OFF_ALO);
        int w = mbar_wait(bar_full(st), par(q)) ? 0 : 1;
        if (__syncthreads_or(w)) {
            bad = 1;
            break;
        }
        // A to TF32 in place (elementwise, so the swizzled order does not matter)
        for (int i = tid; i < DG_ROWS * DG_KC; i += DG_THREADS) {
            const float a = a_hi[i];
            const float hsel = tf32_rna(a);
            a_hi[i] = hsel;
            if (SPLIT) a_lo[i] = a - hsel;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < DG_KC / 8; ++ks) {
                const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                const uint64_t ah = sdesc_sw128(sb + L::OFF_AHI + 32 * ks);
                const uint64_t b0 = sdesc_sw128(sb + L::OFF_BHI + 32 * ks);
                const uint64_t b1 = sdesc_sw128(sb + L::OFF_BHI + 256 * 128 + 32 * ks);
                mma_tf32(tmem, ah, b0, acc);
                mma_tf32(tmem + 256, ah, b1, acc);
                if (SPLIT) {
                    const uint64_t al = sdesc_sw128(sb + L::OFF_ALO + 32 * ks);
                    const uint64_t l0 = sdesc_sw128(sb + L::OFF_BLO + 32 * ks);
                    const uint64_t l1 = sdesc_sw128(sb + L::OFF_BLO + 256 * 128 + 32 * ks);
                    mma_tf32(tmem, ah, l0, 1u);
                    mma_tf32(tmem + 256, ah, l1, 1u);
                    mma_tf32(tmem, al, b0, 1u);
                    mma_tf32(tmem + 256, al, b1, 1u);
                }
            }
            mma_commit(bar_mma(st));
            // refill the stage of chunk q + 1 once the products that last read it
            // (those of chunk q + 1 - ST) are done
            const int qn = q + 1;
            if (qn >= ST && qn < Q) {
                w = mbar_wait(bar_mma(qn % ST), par(qn - ST)) ? 0 : 2;
                if (!w) issue(qn);
            }
        }
        last_q = q;
        if (__syncthreads_or(w)) {
            bad = 2;
            break;
        }
        if (kc != nkc - 1) continue;
        // ---- last chunk of a tile: wait for its products, then the epilogue
        w = mbar_wait(bar_mma(st), par(q)) ? 0 : 2;
        if (__syncthreads_or(w)) {
            bad = 2;
            break;
        }
        tmem_fence_after();
        const int tile = tile_of(q);
        const int sl = tile / c.npairs, p = tile - sl * c.npairs;
        const bool mp = c.mpcp && pair_j[2 * p + 1] >= 0;
        float2 *zb = zspec + ((size_t)sl * c.G * c.npairs) * 64 * 64;
        for (int cc = 0; cc < DG_N / 32; ++cc) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * cc), v);
#pragma unroll
            for (int k = 0; k < 32; ++k) stage[tid * DG_SROW + k] = v[k];
            __syncthreads();
            for (int idx = tid; idx < 16 * 64; idx += DG_THREADS) {
                const int fb = idx >> 6, cp = idx & 63;
                const int f = cc * 16 + fb;
                const float *ra = stage + cp * DG_SROW + 2 * fb;
                const float *rb = stage + (127 - cp) * DG_SROW + 2 * fb;
                const float ar = ra[0], ai = ra[1];
                const float br = mp ? rb[0] : 0.f, bi = mp ? rb[1] : 0.f;
                auto put = [&](int ff, float re, float im) {
                    const int k1 = ff % c.G, k2 = ff / c.G;
                    zb[(((size_t)k1 * c.npairs + p) * 64 + k2) * 64 + cp] = make_float2(re, im);
                };
                if (f == 0) {
                    put(0, ar, br);                      // column 0: X[0] (real)
                    put(256, ai, bi);                    // column 1: X[256] (real)
                } else {
                    put(f, ar - bi, ai + br);
                    put(512 - f, ar + bi, br - ai);
                }
            }
            __syncthreads();
        }
        tmem_fence_before();
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicOr(&status[0], TRED_ST_TIMEOUT);
        // let the copies and products in flight finish (bounded) before the memory goes
        if (last_q >= 0) (void)mbar_wait(bar_mma(last_q % ST), par(last_q));
        for (int q = last_q + 1; q < Q && q <= last_q + ST; ++q) (void)mbar_wait(bar_full(q % ST), par(q));
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tmem, DG_N);
    }
}

// ---------------------------------------------------------------- split BF16
// Stage layout (one stage): A FP32 staging [2 K halves][128 rows][128 B] (TMA, 128-byte
// swizzle), A hi and A lo BF16 [128 rows][128 B], B hi and B lo BF16 [512 rows][128 B]
// (TMA, 128-byte swizzle); 64 ticks per chunk.
constexpr int DB_KC = 64;
constexpr uint32_t DB_AF_BYTES = DG_ROWS * DB_KC * 4;         // 32 KB
constexpr uint32_t DB_A_BYTES = DG_ROWS * DB_KC * 2;          // 16 KB
constexpr uint32_t DB_B_BYTES = DG_N * DB_KC * 2;             // 64 KB
constexpr uint32_t DB_OFF_AF = 0;
constexpr uint32_t DB_OFF_AHI = DB_OFF_AF + DB_AF_BYTES;
constexpr uint32_t DB_OFF_ALO = DB_OFF_AHI + DB_A_BYTES;
constexpr uint32_t DB_OFF_BHI = DB_OFF_ALO + DB_A_BYTES;
constexpr uint32_t DB_OFF_BLO = DB_OFF_BHI + DB_B_BYTES;
constexpr uint32_t DB_OFF_STAGE = DB_OFF_BLO + DB_B_BYTES;    // epilogue staging
constexpr uint32_t DB_OFF_BAR = DB_OFF_STAGE + DG_ROWS * DG_SROW * 4;
constexpr size_t DB_SMEM = DB_OFF_BAR + 64 + 1024;
static_assert(DB_SMEM <= 232448, "split-BF16 stage fits shared memory");
// instruction descriptor: D FP32, A and B BF16, both K-major, N = 256, M = 128
constexpr uint32_t DB_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(DB_IDESC), "r"(acc)
        : "memory");
}
// nearest BF16 (ties to even) of a finite FP32 value, as its 16 bits
__device__ __forceinline__ uint32_t bf16_rn_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
// byte offset of 16-byte chunk c of row r in a tile of 128-byte rows with the 128-byte
// swizzle (chunks XOR-ed with the row's position in its 8-row atom)
__device__ __forceinline__ uint32_t sw128_chunk(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__global__ void __launch_bounds__(DG_THREADS, 1)
    k_dft_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                    const __grid_constant__ CUtensorMap tmBlo, const int32_t *__restrict__ n_blocks_dev,
                    const int32_t *__restrict__ pair_j, DgConst c, float2 *__restrict__ zspec,
                    int32_t *__restrict__ status, int slot_base, int slot_count, int qbase) {
    extern __shared__ unsigned char dg_raw[];
    const uint32_t raw = smem_u32(dg_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = dg_raw + (base - raw);
    float *stage = reinterpret_cast<float *>(gbase + DB_OFF_STAGE);
    const uint32_t bar_full = base + DB_OFF_BAR, bar_mma = base + DB_OFF_BAR + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(gbase + DB_OFF_BAR + 32);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        tmem_alloc(tslot, DG_N);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_full, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *tslot;

    const int nb = n_blocks_dev[0];
    const int nloc = max(0, min(slot_count, nb - slot_base));
    const int tiles = nloc * c.npairs;
    const int nkc = c.bt / DB_KC;
    const int my_tiles = tiles > (int)blockIdx.x ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Q = my_tiles * nkc;
    const uint32_t tx_bytes = DB_AF_BYTES + 2 * DB_B_BYTES;
    int bad = 0;
    int last_q = -1;     // last chunk whose products were issued
    int copied = -1;     // last chunk whose copies were issued
    auto tile_of = [&](int q) { return (int)blockIdx.x + (q / nkc) * (int)gridDim.x; };
    auto issue = [&](int q) {          // thread 0: copies of chunk q (one stage: phase q & 1)
        const int tile = tile_of(q), kc = q % nkc;
        const int sl = tile / c.npairs, p = tile - sl * c.npairs;
        const int slot = slot_base + sl;
        const int j1 = pair_j[2 * p], j2r = pair_j[2 * p + 1];
        const int j2 = j2r >= 0 ? j2r : j1;
        const int row1 = ((slot - qbase) * c.nch + j1) * c.cols;
        const int row2 = ((slot - qbase) * c.nch + j2) * c.cols;
        mbar_expect_tx(bar_full, tx_bytes);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {   // K halves of 32 FP32 ticks
            const uint32_t af = base + DB_OFF_AF + (uint32_t)hh * (DG_ROWS * 128);
            tma_load_2d(af, &tmA, kc * DB_KC + 32 * hh, row1, bar_full);
            tma_load_2d(af + 64 * 128, &tmA, kc * DB_KC + 32 * hh, row2, bar_full);
        }
        tma_load_2d(base + DB_OFF_BHI, &tmBhi, kc * DB_KC, 0, bar_full);
        tma_load_2d(base + DB_OFF_BHI + 256 * 128, &tmBhi, kc * DB_KC, 256, bar_full);
        tma_load_2d(base + DB_OFF_BLO, &tmBlo, kc * DB_KC, 0, bar_full);
        tma_load_2d(base + DB_OFF_BLO + 256 * 128, &tmBlo, kc * DB_KC, 256, bar_full);
    };
    if (Q > 0) {
        if (tid == 0) issue(0);
        copied = 0;
    }

    for (int q = 0; q < Q; ++q) {
        const int kc = q % nkc;
        const uint32_t ph = (uint32_t)(q & 1);
        int w = mbar_wait(bar_full, ph) ? 0 : 1;
        if (__syncthreads_or(w)) {
            bad = 1;
            break;
        }
        // A: FP32 staging -> BF16 hi and lo tiles; each thread one 8-tick group (16 B of
        // BF16) of a row at a time: two 16-byte FP32 chunks of one K half
        for (int i = tid; i < DG_ROWS * (DB_KC / 8); i += DG_THREADS) {
            const int r = i >> 3, g = i & 7;            // row, 8-tick group (ticks 8g .. 8g + 7)
            const int hh = g >> 2, c4 = (g & 3) * 2;    // K half, first FP32 chunk in it
            const unsigned char *fp = gbase + DB_OFF_AF + hh * (DG_ROWS * 128);
            const float4 v0 = *reinterpret_cast<const float4 *>(fp + sw128_chunk(r, c4));
            const float4 v1 = *reinterpret_cast<const float4 *>(fp + sw128_chunk(r, c4 + 1));
            const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t h0 = bf16_rn_bits(x[2 * k]), h1 = bf16_rn_bits(x[2 * k + 1]);
                const uint32_t l0 = bf16_rn_bits(x[2 * k] - __uint_as_float(h0 << 16));
                const uint32_t l1 = bf16_rn_bits(x[2 * k + 1] - __uint_as_float(h1 << 16));
                hi[k] = h0 | (h1 << 16);
                lo[k] = l0 | (l1 << 16);
            }
            *reinterpret_cast<uint4 *>(gbase + DB_OFF_AHI + sw128_chunk(r, g)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(gbase + DB_OFF_ALO + sw128_chunk(r, g)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < DB_KC / 16; ++ks) {      // 16 ticks (32 bytes) per product
                const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                const uint64_t ah = sdesc_sw128(base + DB_OFF_AHI + 32 * ks);
                const uint64_t al = sdesc_sw128(base + DB_OFF_ALO + 32 * ks);
                const uint64_t b0 = sdesc_sw128(base + DB_OFF_BHI + 32 * ks);
                const uint64_t b1 = sdesc_sw128(base + DB_OFF_BHI + 256 * 128 + 32 * ks);
                const uint64_t l0 = sdesc_sw128(base + DB_OFF_BLO + 32 * ks);
                const uint64_t l1 = sdesc_sw128(base + DB_OFF_BLO + 256 * 128 + 32 * ks);
                mma_bf16(tmem, ah, b0, acc);
                mma_bf16(tmem + 256, ah, b1, acc);
                mma_bf16(tmem, ah, l0, 1u);
                mma_bf16(tmem + 256, ah, l1, 1u);
                mma_bf16(tmem, al, b0, 1u);
                mma_bf16(tmem + 256, al, b1, 1u);
            }
            mma_commit(bar_mma);
        }
        last_q = q;
        // one stage: the next chunk's copies wait for these products
        w = 0;
        if (tid == 0) {
            w = mbar_wait(bar_mma, ph) ? 0 : 2;
            if (!w && q + 1 < Q) issue(q + 1);
        }
        if (__syncthreads_or(w)) {
            bad = 2;
            break;
        }
        if (q + 1 < Q) copied = q + 1;
        if (kc != nkc - 1) continue;
        // ---- last chunk of a tile (its products are done): the epilogue
        tmem_fence_after();
        const int tile = tile_of(q);
        const int sl = tile / c.npairs, p = tile - sl * c.npairs;
        const bool mp = c.mpcp && pair_j[2 * p + 1] >= 0;
        float2 *zb = zspec + ((size_t)sl * c.G * c.npairs) * 64 * 64;
        for (int cc = 0; cc < DG_N / 32; ++cc) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * cc), v);
#pragma unroll
            for (int k = 0; k < 32; ++k) stage[tid * DG_SROW + k] = v[k];
            __syncthreads();
            for (int idx = tid; idx < 16 * 64; idx += DG_THREADS) {
                const int fb = idx >> 6, cp = idx & 63;
                const int f = cc * 16 + fb;
                const float *ra = stage + cp * DG_SROW + 2 * fb;
                const float *rb = stage + (127 - cp) * DG_SROW + 2 * fb;
                const float ar = ra[0], ai = ra[1];
                const float br = mp ? rb[0] : 0.f, bi = mp ? rb[1] : 0.f;
                auto put = [&](int ff, float re, float im) {
                    const int k1 = ff % c.G, k2 = ff / c.G;
                    zb[(((size_t)k1 * c.npairs + p) * 64 + k2) * 64 + cp] = make_float2(re, im);
                };
                if (f == 0) {
                    put(0, ar, br);
                    put(256, ai, bi);
                } else {
                    put(f, ar - bi, ai + br);
                    put(512 - f, ar + bi, br - ai);
                }
            }
            __syncthreads();
        }
        tmem_fence_before();
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicOr(&status[0], TRED_ST_TIMEOUT);
        // let the copies and products in flight finish (bounded) before the memory goes
        if (bad == 2 && last_q >= 0) (void)mbar_wait(bar_mma, (uint32_t)(last_q & 1));
        if (bad == 1 && copied >= 0) (void)mbar_wait(bar_full, (uint32_t)(copied & 1));
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tmem, DG_N);
    }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

void *tensor_map_encoder() { return reinterpret_cast<void *>(encode_fn()); }

// 2-D FP32 tensor [rows][inner], box [box_rows][32], 128-byte swizzle
static int make_map(tred_handle *h, CUtensorMap *m, const float *ptr, uint64_t inner, uint64_t rows,
                    uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(h, TRED_ERR_CUDA, "dft-gemm: cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)DG_KC, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(h, TRED_ERR_CUDA, "dft-gemm: tensor map encode failed (%d)", (int)r);
    return TRED_OK;
}

// 2-D BF16 tensor [rows][inner], box [box_rows][64] (128 bytes), 128-byte swizzle
static int make_map_bf16(tred_handle *h, CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t rows,
                         uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return set_error(h, TRED_ERR_CUDA, "dft-gemm: cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {(cuuint32_t)DB_KC, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(h, TRED_ERR_CUDA, "dft-gemm: bf16 tensor map encode failed (%d)", (int)r);
    return TRED_OK;
}

// nearest BF16 (ties to even) of a finite binary32 value, on the host
static uint16_t bf16_rn_host(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
static float bf16_value_host(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float x;
    memcpy(&x, &u, 4);
    return x;
}

// DFT basis (hi, lo parts) for bt ticks and lt = 512, on the host in FP64: TF32 parts in
// FP32 words (conv_mode 1, 2) or BF16 parts (conv_mode 3)
int dft_basis_build(tred_handle *h) {
    const int bt = h->g.bt, lt = h->g.lt;
    if (h->p.conv_mode == 3) {
        std::vector<uint16_t> bh((size_t)DG_N * bt), bl((size_t)DG_N * bt);
        for (int n = 0; n < DG_N; ++n) {
            const int f = n / 2;
            for (int t = 0; t < bt; ++t) {
                double v;
                if (n == 1) v = (t & 1) ? -1.0 : 1.0;
                else if (n % 2 == 0) v = std::cos(2.0 * M_PI * (double)(((int64_t)f * t) % lt) / lt);
                else v = -std::sin(2.0 * M_PI * (double)(((int64_t)f * t) % lt) / lt);
                const uint16_t xh = bf16_rn_host((float)v);
                bh[(size_t)n * bt + t] = xh;
                bl[(size_t)n * bt + t] = bf16_rn_host((float)(v - (double)bf16_value_host(xh)));
            }
        }
        int rc = check_cuda(h, cudaMemcpy(h->dft_hi, bh.data(), 2 * bh.size(), cudaMemcpyHostToDevice), "copy dft basis");
        if (!rc) rc = check_cuda(h, cudaMemcpy(h->dft_lo, bl.data(), 2 * bl.size(), cudaMemcpyHostToDevice), "copy dft basis");
        return rc;
    }
    std::vector<float> hi((size_t)DG_N * bt), lo((size_t)DG_N * bt);
    auto tf32 = [](float x) {
        uint32_t u;
        memcpy(&u, &x, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        float y;
        memcpy(&y, &u, 4);
        return y;
    };
    for (int n = 0; n < DG_N; ++n) {
        const int f = n / 2;
        for (int t = 0; t < bt; ++t) {
            double v;
            if (n == 1) v = (t & 1) ? -1.0 : 1.0;                                   // f = lt / 2
            else if (n % 2 == 0) v = std::cos(2.0 * M_PI * (double)(((int64_t)f * t) % lt) / lt);
            else v = -std::sin(2.0 * M_PI * (double)(((int64_t)f * t) % lt) / lt);
            const float x = (float)v;
            const float xh = tf32(x);
            hi[(size_t)n * bt + t] = xh;
            lo[(size_t)n * bt + t] = (float)(v - (double)xh);
        }
    }
    int rc = check_cuda(h, cudaMemcpy(h->dft_hi, hi.data(), sizeof(float) * hi.size(), cudaMemcpyHostToDevice),
                        "copy dft basis");
    if (!rc)
        rc = check_cuda(h, cudaMemcpy(h->dft_lo, lo.data(), sizeof(float) * lo.size(), cudaMemcpyHostToDevice),
                        "copy dft basis");
    return rc;
}

size_t dft_basis_bytes(int bt) { return sizeof(float) * (size_t)DG_N * bt; }
size_t dft_zspec_bytes(int blocks, int npairs, int lt) { return sizeof(float2) * (size_t)blocks * npairs * lt * 64; }

int launch_dft_gemm(tred_handle *h, const int32_t *n_blocks_dev, const float *qeff, int qrows_blocks,
                    int slot_base, int slot_count, int qbase, cudaStream_t s) {
    CUtensorMap ta, tbh, tbl;
    const int nch = h->g.n_sub * h->g.n_sub, cols = h->g.bp * h->g.bp;
    int rc = make_map(h, &ta, qeff, (uint64_t)h->g.bt, (uint64_t)qrows_blocks * nch * cols, 64);
    if (rc) return rc;
    DgConst c{nch, cols, h->g.bt, h->d.npairs, h->g.lt / 64, h->p.mpcp};
    if (h->p.conv_mode == 3) {
        if (h->g.bt % DB_KC) return set_error(h, TRED_ERR_INVALID_ARG, "dft-gemm: split BF16 needs bt a multiple of 64");
        rc = make_map_bf16(h, &tbh, h->dft_hi, (uint64_t)h->g.bt, DG_N, 256);
        if (!rc) rc = make_map_bf16(h, &tbl, h->dft_lo, (uint64_t)h->g.bt, DG_N, 256);
        if (rc) return rc;
        static bool attr_b = false;
        if (!attr_b) {
            cudaFuncSetAttribute(k_dft_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DB_SMEM);
            attr_b = true;
        }
        k_dft_gemm_bf16<<<num_sms(h), DG_THREADS, DB_SMEM, s>>>(ta, tbh, tbl, n_blocks_dev, h->pair_j, c, h->zspec,
                                                               h->status, slot_base, slot_count, qbase);
        h->launches += 1;
        return check_cuda(h, cudaGetLastError(), "dft-gemm launch");
    }
    rc = make_map(h, &tbh, h->dft_hi, (uint64_t)h->g.bt, DG_N, 256);
    if (!rc) rc = make_map(h, &tbl, h->dft_lo, (uint64_t)h->g.bt, DG_N, 256);
    if (rc) return rc;
    const bool split = h->p.conv_mode == 2;
    static bool attr[2] = {false, false};
    const size_t smem = split ? DgStage<true>::SMEM : DgStage<false>::SMEM;
    if (!attr[split]) {
        cudaFuncSetAttribute(split ? k_dft_gemm<true> : k_dft_gemm<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr[split] = true;
    }
    const int grid = num_sms(h);
    if (split)
        k_dft_gemm<true><<<grid, DG_THREADS, smem, s>>>(ta, tbh, tbl, n_blocks_dev, h->pair_j, c, h->zspec,
                                                        h->status, slot_base, slot_count, qbase);
    else
        k_dft_gemm<false><<<grid, DG_THREADS, smem, s>>>(ta, tbh, tbl, n_blocks_dev, h->pair_j, c, h->zspec,
                                                         h->status, slot_base, slot_count, qbase);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "dft-gemm launch");
}

}  // namespace tred
