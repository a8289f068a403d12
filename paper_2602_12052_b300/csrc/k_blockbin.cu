// a2. Block-sparse binning (Sec. III-B-1): occupancy of every block, warp-ballot
// + prefix-scan compaction into the ascending active-block list, block -> slot map
// and the per-block deposit CSR.
//
//   k_bb_count   one thread per deposit: clipped support box -> touched blocks,
//                atomicAdd on the block's count
//   k_bb_chunk   one 1024-wide chunk of blocks per CTA: ballot/popc counts of
//                active blocks and their occupancy sum
//   k_bb_top     one CTA: exclusive scan of the chunk totals; writes nb
//   k_bb_emit    per chunk: ballot + warp/CTA prefix -> slot of each active block
//   k_bb_fill    one thread per deposit: CSR fill through per-slot cursors
//   k_bb_sort    one CTA per active block: the block's deposit ids in ascending order
//                (the fill leaves them in arrival order), so that every later sum
//                over a block's deposits runs in one fixed order
#include "tred_internal.cuh"

namespace tred {

struct BinGeom {
    int ns, bp, bt, ngx, ngy, nt, nbx, nby, nbt;
    int ngy_e;                      // sub-cells of one event along y
    const int32_t *event;           // event of each deposit (nullptr: one event)
};

__device__ __forceinline__ bool support_box(const tred_deposits &d, int i, const BinGeom &g,
                                            int &bx0, int &bx1, int &by0, int &by1, int &bt0,
                                            int &bt1) {
    const int ev = g.event ? g.event[i] : 0;
    int xa = d.lo_x[i] - 1, xb = d.hi_x[i] + 1;
    int ya = d.lo_y[i] - 1, yb = d.hi_y[i] + 1;
    int ta = d.lo_t[i] - 1, tb = d.hi_t[i] + 1;
    if (d.lo_x[i] > d.hi_x[i]) return false;   // dropped deposit
    xa = max(xa, 0);
    ya = max(ya, ev * g.ngy_e);
    ta = max(ta, 0);
    xb = min(xb, g.ngx - 1);
    yb = min(yb, (ev + 1) * g.ngy_e - 1);
    tb = min(tb, g.nt - 1);
    if (xa > xb || ya > yb || ta > tb) return false;
    bx0 = (xa / g.ns) / g.bp;
    bx1 = (xb / g.ns) / g.bp;
    by0 = (ya / g.ns) / g.bp;
    by1 = (yb / g.ns) / g.bp;
    bt0 = ta / g.bt;
    bt1 = tb / g.bt;
    return true;
}

__global__ void __launch_bounds__(256) k_bb_count(int n, tred_deposits d, BinGeom g,
                                                  int32_t *__restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bx0, bx1, by0, by1, bt0, bt1;
    if (!support_box(d, i, g, bx0, bx1, by0, by1, bt0, bt1)) return;
    for (int by = by0; by <= by1; ++by)
        for (int bx = bx0; bx <= bx1; ++bx)
            for (int bt = bt0; bt <= bt1; ++bt)
                atomicAdd(&count[((int64_t)by * g.nbx + bx) * g.nbt + bt], 1);
}

// Per 1024-block chunk: number of active blocks and sum of their counts.
__global__ void __launch_bounds__(1024) k_bb_chunk(int64_t nblk, const int32_t *__restrict__ count,
                                                   int32_t *__restrict__ part, int64_t nchunks) {
    __shared__ int s_act[32], s_sum[32];
    const int64_t id = blockIdx.x * 1024ll + threadIdx.x;
    const int c = id < nblk ? count[id] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, c > 0);
    int sum = c;
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_act[warp] = __popc(bal);
        s_sum[warp] = sum;
    }
    __syncthreads();
    if (warp == 0) {
        int a = s_act[lane], s = s_sum[lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (lane == 0) {
            part[blockIdx.x] = a;
            part[nchunks + blockIdx.x] = s;
        }
    }
}

// Exclusive scan of the chunk totals in place (one CTA, any number of chunks);
// part[2*nchunks + 0] = active blocks, part[2*nchunks + 1] = pairs.
__global__ void __launch_bounds__(1024) k_bb_top(int64_t nchunks, int32_t *__restrict__ part,
                                                 int32_t max_blocks, int32_t max_pairs,
                                                 int32_t *__restrict__ n_blocks_dev,
                                                 int32_t *__restrict__ status) {
    __shared__ int s_a[32], s_s[32];
    __shared__ int carry_a, carry_s;
    if (threadIdx.x == 0) carry_a = carry_s = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t base = 0; base < nchunks; base += 1024) {
        const int64_t i = base + threadIdx.x;
        int a = i < nchunks ? part[i] : 0;
        int s = i < nchunks ? part[nchunks + i] : 0;
        int ia = a, is = s;   // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int ta = __shfl_up_sync(0xffffffffu, ia, o), ts = __shfl_up_sync(0xffffffffu, is, o);
            if (lane >= o) { ia += ta; is += ts; }
        }
        if (lane == 31) { s_a[warp] = ia; s_s[warp] = is; }
        __syncthreads();
        if (warp == 0) {
            int wa = s_a[lane], wsum = s_s[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int ta = __shfl_up_sync(0xffffffffu, wa, o), ts = __shfl_up_sync(0xffffffffu, wsum, o);
                if (lane >= o) { wa += ta; wsum += ts; }
            }
            s_a[lane] = wa;
            s_s[lane] = wsum;
        }
        __syncthreads();
        const int wa = warp ? s_a[warp - 1] : 0, wsum = warp ? s_s[warp - 1] : 0;
        if (i < nchunks) {
            part[i] = carry_a + wa + ia - a;
            part[nchunks + i] = carry_s + wsum + is - s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_a += s_a[31];
            carry_s += s_s[31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int nb = carry_a;
        if (nb > max_blocks) {
            atomicOr(&status[0], TRED_ST_BLOCK_OVERFLOW);
            nb = max_blocks;
        }
        if (carry_s > max_pairs) atomicOr(&status[0], TRED_ST_PAIR_OVERFLOW);
        n_blocks_dev[0] = nb;
        status[2] = carry_a;
        status[3] = carry_s;
        part[2 * nchunks] = carry_a;
        part[2 * nchunks + 1] = carry_s;
    }
}

__global__ void __launch_bounds__(1024) k_bb_emit(int64_t nblk, const int32_t *__restrict__ count,
                                                  const int32_t *__restrict__ part, int64_t nchunks,
                                                  int32_t max_blocks, int32_t max_pairs,
                                                  int32_t *__restrict__ slot_of,
                                                  int32_t *__restrict__ block_ids,
                                                  int32_t *__restrict__ block_counts,
                                                  int32_t *__restrict__ dep_offsets,
                                                  int32_t *__restrict__ fill) {
    __shared__ int s_a[32], s_s[32];
    const int64_t id = blockIdx.x * 1024ll + threadIdx.x;
    const int c = id < nblk ? count[id] : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, c > 0);
    const int rank = __popc(bal & ((1u << lane) - 1u));
    int is = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, is, o);
        if (lane >= o) is += t;
    }
    if (lane == 31) {
        s_a[warp] = __popc(bal);
        s_s[warp] = is;
    }
    __syncthreads();
    if (warp == 0) {
        int a = s_a[lane], s = s_s[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int ta = __shfl_up_sync(0xffffffffu, a, o), ts = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) { a += ta; s += ts; }
        }
        s_a[lane] = a - s_a[lane];   // exclusive
        s_s[lane] = s - s_s[lane];
    }
    __syncthreads();
    if (id >= nblk) return;
    if (c == 0) {
        slot_of[id] = -1;
        return;
    }
    const int slot = part[blockIdx.x] + s_a[warp] + rank;
    const int off = part[nchunks + blockIdx.x] + s_s[warp] + is - c;
    if (slot >= max_blocks) {
        slot_of[id] = -1;
        return;
    }
    slot_of[id] = slot;
    block_ids[slot] = (int32_t)id;
    block_counts[slot] = c;
    // offsets are clamped to max_pairs so that an overflowing CSR (status bit set)
    // never sends a reader past the dep_index capacity
    dep_offsets[slot] = min(off, max_pairs);
    fill[slot] = 0;
    // the CSR end of the last kept slot
    const int nb = min(part[2 * nchunks], max_blocks);
    if (slot == nb - 1) dep_offsets[nb] = min(off + c, max_pairs);
}

__global__ void __launch_bounds__(256) k_bb_fill(int n, tred_deposits d, BinGeom g,
                                                 const int32_t *__restrict__ slot_of,
                                                 const int32_t *__restrict__ dep_offsets,
                                                 int32_t *__restrict__ fill,
                                                 int32_t *__restrict__ dep_index, int32_t max_pairs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bx0, bx1, by0, by1, bt0, bt1;
    if (!support_box(d, i, g, bx0, bx1, by0, by1, bt0, bt1)) return;
    for (int by = by0; by <= by1; ++by)
        for (int bx = bx0; bx <= bx1; ++bx)
            for (int bt = bt0; bt <= bt1; ++bt) {
                const int s = slot_of[((int64_t)by * g.nbx + bx) * g.nbt + bt];
                if (s < 0) continue;
                const int pos = dep_offsets[s] + atomicAdd(&fill[s], 1);
                if (pos < max_pairs) dep_index[pos] = i;
            }
}

// Ascending sort of each block's deposit ids: a bitonic network whose comparators all
// point the same way (the first step of each merge pairs mirrored positions), so the
// list can stand for its power-of-two padding with +infinity that never moves: a
// comparator whose upper element lies past the end is simply skipped.  A warp sorts a
// list of up to BB_SORT_WARP ids in its part of shared memory; the CTA then sorts its
// longer lists together, in shared memory up to BB_SORT_CTA ids, else in place in global
// memory (the CTA alone owns the list and synchronises between steps).
constexpr int BB_SORT_THREADS = 256;
constexpr int BB_SORT_WARP = 1024;
constexpr int BB_SORT_CTA = (BB_SORT_THREADS / 32) * BB_SORT_WARP;

// threads t = 0 .. nt - 1 of the calling group sort key[0 .. n); sync() separates the steps
template <typename Sync>
__device__ void bitonic_ascending(int32_t *key, int n, int t, int nt, Sync sync) {
    int P = 1;
    while (P < n) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1, lj = __ffs(k) - 2; j >= 1; j >>= 1, --lj) {   // j = 2^lj
            for (int i = t; i < P / 2; i += nt) {
                const int lo = ((i >> lj) << (lj + 1)) | (i & (j - 1));
                const int hi = j == (k >> 1) ? (lo ^ (k - 1)) : lo + j;   // mirror pair on a merge's first step
                if (hi < n) {
                    const int32_t a = key[lo], b = key[hi];
                    if (b < a) {
                        key[lo] = b;
                        key[hi] = a;
                    }
                }
            }
            sync();
        }
    }
}

__global__ void __launch_bounds__(BB_SORT_THREADS) k_bb_sort(const int32_t *__restrict__ n_blocks_dev,
                                                            const int32_t *__restrict__ dep_offsets,
                                                            int32_t *__restrict__ dep_index, int32_t max_pairs,
                                                            int32_t max_blocks) {
    __shared__ int32_t key[BB_SORT_CTA];
    __shared__ int big[BB_SORT_THREADS / 32 * 8];
    __shared__ int nbig;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = min(n_blocks_dev[0], max_blocks);
    const int per = gridDim.x * (BB_SORT_THREADS / 32);
    for (int base = blockIdx.x * (BB_SORT_THREADS / 32); base < nb; base += per) {
        if (threadIdx.x == 0) nbig = 0;
        __syncthreads();
        // one list per warp
        const int slot = base + warp;
        if (slot < nb) {
            const int beg = min(dep_offsets[slot], max_pairs), end = min(dep_offsets[slot + 1], max_pairs);
            const int n = end - beg;
            if (n > BB_SORT_WARP) {
                if (lane == 0) big[atomicAdd(&nbig, 1)] = slot;
            } else if (n > 1) {
                int32_t *kw = key + warp * BB_SORT_WARP;
                for (int i = lane; i < n; i += 32) kw[i] = dep_index[beg + i];
                __syncwarp();
                bitonic_ascending(kw, n, lane, 32, [] { __syncwarp(); });
                for (int i = lane; i < n; i += 32) dep_index[beg + i] = kw[i];
            }
        }
        __syncthreads();
        // the longer lists, one at a time by the whole CTA
        for (int q = 0; q < nbig; ++q) {
            const int sl = big[q];
            const int beg = min(dep_offsets[sl], max_pairs), end = min(dep_offsets[sl + 1], max_pairs);
            const int n = end - beg;
            auto bar = [] { __syncthreads(); };
            if (n <= BB_SORT_CTA) {
                for (int i = threadIdx.x; i < n; i += BB_SORT_THREADS) key[i] = dep_index[beg + i];
                __syncthreads();
                bitonic_ascending(key, n, threadIdx.x, BB_SORT_THREADS, bar);
                for (int i = threadIdx.x; i < n; i += BB_SORT_THREADS) dep_index[beg + i] = key[i];
                __syncthreads();
            } else {
                bitonic_ascending(dep_index + beg, n, threadIdx.x, BB_SORT_THREADS, bar);
            }
        }
    }
}

// Zero-block case: dep_offsets[0] = 0 must still hold.
__global__ void k_bb_offsets0(int32_t *dep_offsets, const int32_t *n_blocks_dev) {
    if (n_blocks_dev[0] == 0) dep_offsets[0] = 0;
}

int launch_blockbin(tred_handle *h, int n, const tred_deposits &deps, int32_t *block_ids,
                    int32_t *block_counts, int32_t *dep_offsets, int32_t *dep_index,
                    int32_t max_pairs, int32_t *n_blocks_dev, cudaStream_t s) {
    BinGeom g{h->g.n_sub, h->g.bp, h->g.bt, h->d.ngx, h->d.ngy, h->g.nt, h->d.nbx, h->d.nby, h->d.nbt,
              h->d.ngy_e, h->dep_event};
    int rc = check_cuda(h, cudaMemsetAsync(h->blk_count, 0, sizeof(int32_t) * h->d.nblk, s), "clear counts");
    if (rc) return rc;
    if (n > 0) k_bb_count<<<(n + 255) / 256, 256, 0, s>>>(n, deps, g, h->blk_count);
    k_bb_chunk<<<(unsigned)h->nchunks, 1024, 0, s>>>(h->d.nblk, h->blk_count, h->scan_part, h->nchunks);
    k_bb_top<<<1, 1024, 0, s>>>(h->nchunks, h->scan_part, h->max_blocks, max_pairs, n_blocks_dev, h->status);
    k_bb_emit<<<(unsigned)h->nchunks, 1024, 0, s>>>(h->d.nblk, h->blk_count, h->scan_part, h->nchunks,
                                                    h->max_blocks, max_pairs, h->blk_slot, block_ids,
                                                    block_counts, dep_offsets, h->blk_fill);
    k_bb_offsets0<<<1, 1, 0, s>>>(dep_offsets, n_blocks_dev);
    if (n > 0)
        k_bb_fill<<<(n + 255) / 256, 256, 0, s>>>(n, deps, g, h->blk_slot, dep_offsets, h->blk_fill,
                                                  dep_index, max_pairs);
    if (n > 0)
        // eight lists per CTA: no more CTAs than the block capacity can use
        k_bb_sort<<<min(num_sms(h) * 4, (h->max_blocks + 7) / 8), BB_SORT_THREADS, 0, s>>>(n_blocks_dev, dep_offsets,
                                                                                      dep_index, max_pairs,
                                                                                      h->max_blocks);
    h->launches += 4 + (n > 0 ? 3 : 0);
    return check_cuda(h, cudaGetLastError(), "blockbin launch");
}

}  // namespace tred

// ---------------------------------------------------------------------------
// tred_blockbin_noalloc: the same binning for callers that may not allocate
// device memory themselves (see include/tred.h).  Its scratch lives in this
// file-scope array, reserved when the library's device code is loaded onto a
// device (with CUDA's lazy module loading, possibly during the first call) and
// held until the process exits.
// ---------------------------------------------------------------------------
namespace tred {

constexpr int64_t NOALLOC_MAX_GRID_BLOCKS = TRED_NOALLOC_MAX_GRID_BLOCKS;
constexpr int64_t NOALLOC_MAX_CHUNKS = (NOALLOC_MAX_GRID_BLOCKS + 1023) / 1024;
// count[grid] | slot_of[grid] | fill[grid] | scan partials[2 chunks + 8]
constexpr int64_t NOALLOC_WORDS = 3 * NOALLOC_MAX_GRID_BLOCKS + 2 * NOALLOC_MAX_CHUNKS + 8;

static __device__ __align__(256) int32_t g_noalloc_scratch[NOALLOC_WORDS];

// Device address of g_noalloc_scratch per device, looked up on the first call made
// with that device current.  A cudaDeviceReset unloads the module and makes the cached
// address stale: the header tells callers not to use this entry point after a reset.
static int32_t *g_noalloc_ptr[64];

static int noalloc_scratch(int32_t **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TRED_ERR_CUDA;
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "tred_blockbin_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return TRED_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return TRED_OK;
}

}  // namespace tred

extern "C" int32_t tred_blockbin_noalloc(const tred_geometry *geom, int32_t n, const tred_deposits *deps,
                                         int32_t *block_ids, int32_t *block_counts, int32_t *dep_offsets,
                                         int32_t *dep_index, int32_t max_blocks, int32_t max_pairs,
                                         int32_t *n_blocks_dev, int32_t *status_dev, void *stream) {
    using namespace tred;
    if (!geom || n < 0 || !block_ids || !block_counts || !dep_offsets || !n_blocks_dev || !status_dev ||
        max_blocks < 1 || max_pairs < 0 || (max_pairs > 0 && !dep_index) || (n > 0 && !deps_ok(deps)))
        return TRED_ERR_INVALID_ARG;
    const tred_geometry &g = *geom;
    char msg[256];
    if (validate_geometry(&g, msg, sizeof msg) != TRED_OK) {   // the checks of tred_create
        fprintf(stderr, "tred_blockbin_noalloc: %s\n", msg);
        return TRED_ERR_INVALID_ARG;
    }
    if (g.n_events > 1) return TRED_ERR_INVALID_ARG;   // single event only
    const int64_t nbx = g.npx_x / g.bp, nby = g.npx_y / g.bp, nbt = g.nt / g.bt;
    const int64_t nblk = nbx * nby * nbt;
    if (nblk > NOALLOC_MAX_GRID_BLOCKS || max_blocks > NOALLOC_MAX_GRID_BLOCKS) {
        fprintf(stderr,
                "tred_blockbin_noalloc: the plane has %lld blocks (max_blocks %d); this entry point's "
                "static scratch holds at most %lld\n",
                (long long)nblk, max_blocks, (long long)NOALLOC_MAX_GRID_BLOCKS);
        return TRED_ERR_CAPACITY;
    }
    int32_t *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != TRED_OK) return rc;
    int32_t *count = scratch;
    int32_t *slot_of = count + NOALLOC_MAX_GRID_BLOCKS;
    int32_t *fill = slot_of + NOALLOC_MAX_GRID_BLOCKS;
    int32_t *part = fill + NOALLOC_MAX_GRID_BLOCKS;
    const int64_t nchunks = (nblk + 1023) / 1024;
    cudaStream_t s = (cudaStream_t)stream;
    BinGeom bg{g.n_sub, g.bp, g.bt, g.npx_x * g.n_sub, g.npx_y * g.n_sub, g.nt, (int)nbx, (int)nby, (int)nbt,
               g.npx_y * g.n_sub, nullptr};
    if (cudaMemsetAsync(count, 0, sizeof(int32_t) * nblk, s) != cudaSuccess) return TRED_ERR_CUDA;
    if (n > 0) k_bb_count<<<(n + 255) / 256, 256, 0, s>>>(n, *deps, bg, count);
    k_bb_chunk<<<(unsigned)nchunks, 1024, 0, s>>>(nblk, count, part, nchunks);
    k_bb_top<<<1, 1024, 0, s>>>(nchunks, part, max_blocks, max_pairs, n_blocks_dev, status_dev);
    k_bb_emit<<<(unsigned)nchunks, 1024, 0, s>>>(nblk, count, part, nchunks, max_blocks, max_pairs, slot_of,
                                                 block_ids, block_counts, dep_offsets, fill);
    k_bb_offsets0<<<1, 1, 0, s>>>(dep_offsets, n_blocks_dev);
    if (n > 0)
        k_bb_fill<<<(n + 255) / 256, 256, 0, s>>>(n, *deps, bg, slot_of, dep_offsets, fill, dep_index,
                                                  max_pairs);
    if (n > 0) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return TRED_ERR_CUDA;
        k_bb_sort<<<min(sms * 4, (max_blocks + 7) / 8), BB_SORT_THREADS, 0, s>>>(n_blocks_dev, dep_offsets, dep_index,
                                                                                max_pairs, max_blocks);
    }
    return cudaGetLastError() == cudaSuccess ? TRED_OK : TRED_ERR_CUDA;
}
