// a3 + a4 in one persistent launch over the active-block queue (Sec. III-B-2: the
// blocks of many events batched through the effective charge and the convolution).
//
// CTAs (one per SM) take active blocks from one device queue that holds every event's
// blocks.  Each block then goes through three phases inside the CTA that took it:
//   1. its effective charge (Eq. eff_q; the block kernel's item, as two groups of 8
//      warps over the even and odd tiles of the block) into the CTA's own row of a
//      Q^eff ring (rows = resident CTAs);
//   2. the spectral stage of every time-frequency class (MPCP packing, class-restricted
//      time DFT, 16 x 16 spatial FFT, product with the response spectrum summed over the
//      channel pairs in tensor memory, inverse spatial FFT) into the CTA's spectrum row;
//   3. the inverse time transform and the MPCP recombination into the block's output
//      [16][16][lt].
// Q^eff and the spectra are written and read back by the same SM a few microseconds
// apart, mostly out of L2 (coherent loads: never the read-only path); no
// launch per chunk of blocks and no buffer sized by the number of blocks.  Nothing
// waits on another CTA: the queue is the only shared state.
#include "conv_item.cuh"
#include "effq_item.cuh"

namespace tred {

// The effective charge of a block runs as two independent groups of 8 warps, each with
// its own shared state and named barrier, over the even and the odd 32-tick tiles of the
// block (a track's charge spans several consecutive tiles, so the two share it evenly):
// like the two CTAs per SM of the standalone kernel, one group's barrier and load waits
// are covered by the other's work.
constexpr int PIPE_EQ_WARPS = 8;
constexpr size_t PIPE_EQ_BYTES = (sizeof(EffqSharedT<PIPE_EQ_WARPS>) + 127) / 128 * 128;
static_assert(2 * PIPE_EQ_BYTES <= SPEC_SMEM, "two effective-charge groups fit the spectral stage's memory");
static_assert(SPEC_THREADS == 2 * PIPE_EQ_WARPS * 32, "two groups make the CTA");

template <int NB1, int G, bool HZ>
__global__ void __launch_bounds__(SPEC_THREADS, 1)
    k_block_pipeline(const int32_t *__restrict__ n_blocks_dev, const int32_t *__restrict__ block_ids,
                     const int32_t *__restrict__ dep_offsets, const int32_t *__restrict__ dep_index, EffqConst ec,
                     const float *__restrict__ wts, const DepRec *__restrict__ recs, float *__restrict__ qring,
                     uint64_t *__restrict__ mring, int32_t *__restrict__ eff_scratch, const float2 *__restrict__ rhat,
                     const int32_t *__restrict__ pair_j, const float2 *__restrict__ tw, ConvConst c,
                     float2 *__restrict__ yring, float *__restrict__ out, int32_t *__restrict__ queue) {
    constexpr int LT = 64 * G;
    constexpr int NC = itime_cols<G>();
    static_assert(NC * 32 == SPEC_THREADS, "one warp per column of a 16-column item");
    constexpr int HC = NC / 2, PARTS = LP / HC, SROW = LT + 1, ITEMS = 8 * PARTS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    const SpecSmem sm(smem);
    __shared__ uint32_t s_tslot;
    __shared__ int s_item;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tmem_alloc(&s_tslot, SPEC_TMEM_COLS);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tbase = s_tslot;
    const uint32_t tacc = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));

    const int nb = n_blocks_dev[0];
    const int nch = ec.ns * ec.ns;
    const int side = ec.bp * ec.ns;
    float *qblk = qring + (size_t)blockIdx.x * nch * ec.bp * ec.bp * ec.bt;   // this CTA's ring row
    uint64_t *mrow = mring + (size_t)blockIdx.x * nch;
    float2 *yplane = yring + (size_t)blockIdx.x * LT * (LP * LP);
    // effective-charge group of this thread: its shared state, barrier, scratch and tiles
    const int grp = warp / PIPE_EQ_WARPS;
    EffqSharedT<PIPE_EQ_WARPS> &ES = *reinterpret_cast<EffqSharedT<PIPE_EQ_WARPS> *>(smem_raw + grp * PIPE_EQ_BYTES);
    const GroupSync<PIPE_EQ_WARPS * 32> gsync{1 + grp};
    float *scratch = reinterpret_cast<float *>(eff_scratch) + (size_t)(2 * blockIdx.x + grp) * side * side * EQ_TT;
    // inverse time phase: double-buffered spectra of 16-column items, twiddles, exchange buffer
    float2 *S = smem;                                   // [2][NC][SROW]
    float2 *wlt = S + 2 * NC * SROW;
    float2 *w32 = wlt + LT;
    float *Ib = reinterpret_cast<float *>(w32 + 32);   // [NC][NPL][33]
    auto issue = [&](int it, int bsel) {   // thread tid copies column tid % NC of item it
        const int rp = it / PARTS, part = it % PARTS;
        int a, bro, cy, cx;
        itime_rows_of(c.bp, rp, a, bro);
        const int q = tid % NC;
        itime_column_of(c.bp, HC, q, part, a, bro, cy, cx);
        const float2 *src = yplane + cy * LP + cx;
        float2 *dst = S + (bsel * NC + q) * SROW;
#pragma unroll 4
        for (int f = tid / NC; f < LT; f += SPEC_THREADS / NC) cp_async8(dst + f, src + (size_t)f * (LP * LP));
        cp_async_commit();
    };
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(queue, 1);
        // 1. effective charge of block b into the ring row (masks cleared first), two groups
        for (int k = tid; k < nch; k += SPEC_THREADS) mrow[k] = 0ull;
        __syncthreads();
        const int b = s_item;
        if (b >= nb) break;
        effq_block_item<PIPE_EQ_WARPS>(ES, ec, b, grp * EQ_TT, ec.bt, block_ids, dep_offsets, dep_index, wts, recs,
                                       qblk, mrow, scratch, gsync, 2 * EQ_TT);
        // 2. the spectral stage, class by class (each item starts with a barrier)
        __syncthreads();
        sm.load_tables(tw);
        for (int k1 = 0; k1 < G; ++k1)
            conv_spec_item<NB1, G, false, HZ, true>(sm, tacc, c, k1, 0, c.npairs, qblk, mrow, rhat, pair_j, tw,
                                                   nullptr, yplane);
        // 3. inverse time transform of the block's 16-column items, the next item's spectra
        //    streamed in while the current one is transformed
        __syncthreads();
        for (int k = tid; k < LT; k += SPEC_THREADS) wlt[k] = tw[TW_LT + k];
        if (tid < 32) w32[tid] = tw[TW_32 + tid];
        float *oblk = out + (size_t)b * LP * LP * LT;
        issue(0, 0);
        for (int it = 0; it < ITEMS; ++it) {
            const int cur = it & 1;
            if (it + 1 < ITEMS)
                issue(it + 1, cur ^ 1);            // that buffer's last readers passed the previous barrier
            else
                cp_async_commit();                 // empty group: keeps the wait count uniform
            cp_async_wait<1>();
            __syncthreads();                       // this item's columns (and the tables) are in place
            const int rp = it / PARTS, part = it % PARTS;
            int a, bro, cy, cx;
            itime_rows_of(c.bp, rp, a, bro);
            itime_column_of(c.bp, HC, warp, part, a, bro, cy, cx);
            itime_column<G>(S + (cur * NC + warp) * SROW, nullptr, Ib, wlt, w32, c, warp, cy, cx, oblk);
        }
        cp_async_wait<0>();
    }
    (void)lane;
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tbase, SPEC_TMEM_COLS);
    }
}

template <int NB1, int G, bool HZ>
static int run_pipeline(tred_handle *h, const int32_t *n_blocks_dev, const int32_t *block_ids,
                        const int32_t *dep_offsets, const int32_t *dep_index, const EffqConst &ec, const ConvConst &c,
                        float *qring, int grid, float *out, cudaStream_t s) {
    static_assert(itime_smem_bytes<G>() <= SPEC_SMEM, "the inverse time phase fits the spectral stage's memory");
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_block_pipeline<NB1, G, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SPEC_SMEM);
        attr = true;
    }
    const int sms = num_sms(h);
    int32_t *queue = h->effq_acc + (effq_scratch_bytes(h->g.bp * h->g.n_sub, sms) / sizeof(int32_t) - 40);
    int rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "pipeline queue reset");
    if (rc) return rc;
    k_block_pipeline<NB1, G, HZ><<<grid, SPEC_THREADS, SPEC_SMEM, s>>>(
        n_blocks_dev, block_ids, dep_offsets, dep_index, ec, h->wts, reinterpret_cast<const DepRec *>(h->recs), qring,
        h->colmask, h->effq_acc, h->rhat, h->pair_j, h->tw, c, h->yspec, out, queue);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "pipeline launch");
}

template <int G>
static int run_pipeline_g(tred_handle *h, int nb1, const int32_t *n_blocks_dev, const int32_t *block_ids,
                          const int32_t *dep_offsets, const int32_t *dep_index, const EffqConst &ec, const ConvConst &c,
                          float *qring, int grid, float *out, cudaStream_t s) {
    const bool hz = c.bp <= 4;
#define TRED_PIPE_CASE(N)                                                                                          \
    case N:                                                                                                        \
        return hz ? run_pipeline<N, G, true>(h, n_blocks_dev, block_ids, dep_offsets, dep_index, ec, c, qring, grid, \
                                             out, s)                                                               \
                  : run_pipeline<N, G, false>(h, n_blocks_dev, block_ids, dep_offsets, dep_index, ec, c, qring, grid, \
                                              out, s);
    if constexpr (G == 8) {
        switch (nb1) {
            TRED_PIPE_CASE(1)
            TRED_PIPE_CASE(2)
            TRED_PIPE_CASE(4)
            default: break;
        }
    } else {
        switch (nb1) {
            TRED_PIPE_CASE(1)
            TRED_PIPE_CASE(2)
            default: break;
        }
    }
#undef TRED_PIPE_CASE
    return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq_convolve: unsupported bt=%d lt=%d", h->g.bt, h->g.lt);
}

int launch_pipeline(tred_handle *h, int n, const tred_deposits &deps, const int32_t *block_ids,
                    const int32_t *dep_offsets, const int32_t *dep_index, const int32_t *n_blocks_dev, float *qring,
                    int ring_rows, float *out, cudaStream_t s) {
    if (h->p.conv_mode != 0)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq_convolve: the FFT convolution (conv_mode 0) only");
    if (h->g.lt != 384 && h->g.lt != 512)
        return set_error(h, TRED_ERR_INVALID_ARG, "tred_effq_convolve: lt must be 384 or 512");
    int rc = effq_check_shape(h);
    if (rc) return rc;
    const int sms = num_sms(h);
    // one CTA per SM, at most one per ring row, spectrum row and mask row
    int grid = sms;
    if (grid > h->max_blocks) grid = h->max_blocks;
    if (grid > h->yspec_blocks) grid = h->yspec_blocks;
    if (ring_rows < grid)
        return set_error(h, TRED_ERR_CAPACITY, "tred_effq_convolve: %d ring rows for %d resident CTAs", ring_rows, grid);
    rc = launch_effq_weights(h, n, deps, s);
    if (rc) return rc;
    const EffqConst ec = effq_const_of(h);
    ConvConst c;
    c.ns = h->g.n_sub;
    c.bp = h->g.bp;
    c.bt = h->g.bt;
    c.nch = c.ns * c.ns;
    c.npairs = h->d.npairs;
    c.G = h->d.G;
    c.lt = h->g.lt;
    c.R = h->d.R;
    c.mpcp = h->p.mpcp;
    const int nb1 = h->g.bt / 64;
    return c.G == 8 ? run_pipeline_g<8>(h, nb1, n_blocks_dev, block_ids, dep_offsets, dep_index, ec, c, qring, grid, out, s)
                    : run_pipeline_g<6>(h, nb1, n_blocks_dev, block_ids, dep_offsets, dep_index, ec, c, qring, grid, out, s);
}

}  // namespace tred
