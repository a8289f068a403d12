// a5. Electrode gather (Fig. flowchart: binning and accumulation onto the unique electrodes).
//
//   k_px_mark    flag every in-plane pixel of each active block's output footprint
//                [bx bp - R, bx bp + bp + R) x (same in y)
//   k_px_chunk / k_px_top / k_px_emit
//                ballot + prefix compaction of the flags into the ascending pixel
//                list; the flag array then holds each pixel's row (or -1)
//   k_px_wave    one warp per active pixel: the pixel's contributing blocks are
//                listed once in shared memory, then the window is swept 512 ticks
//                per step (4 float4 per lane): sum, in a fixed order (by, bx, bt
//                ascending), the outputs of the overlapping blocks; deterministic,
//                no atomics.  Optional FP64 accumulation (compensated mode).
#include <type_traits>

#include "tred_internal.cuh"

namespace tred {

struct GatherConst {
    int npx_x, npx_y, nt, bp, bt, nr, lt, R, nbx, nby, nbt, comp;
    int npy_e, nby_e;              // pixel rows and block rows of one event
};

__global__ void k_px_mark(const int32_t *__restrict__ block_ids, const int32_t *__restrict__ n_blocks_dev,
                          GatherConst c, int32_t *__restrict__ flags) {
    const int nb = n_blocks_dev[0];
    const int side = c.bp + 2 * c.R;
    const int64_t total = (int64_t)nb * side * side;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int slot = (int)(k / (side * side));
        const int r = (int)(k % (side * side));
        const int blk = block_ids[slot];
        const int bxy = blk / c.nbt, bx = bxy % c.nbx, by = bxy / c.nbx;
        const int x = bx * c.bp - c.R + r % side, y = by * c.bp - c.R + r / side;
        const int ev = by / c.nby_e;
        if (x >= 0 && x < c.npx_x && y >= ev * c.npy_e && y < (ev + 1) * c.npy_e) flags[(int64_t)y * c.npx_x + x] = 1;
    }
}

__global__ void __launch_bounds__(1024) k_px_chunk(int64_t n, const int32_t *__restrict__ flags,
                                                   int32_t *__restrict__ part) {
    __shared__ int s[32];
    const int64_t id = blockIdx.x * 1024ll + threadIdx.x;
    const unsigned bal = __ballot_sync(0xffffffffu, id < n && flags[id] != 0);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    if (threadIdx.x < 32) {
        int a = s[threadIdx.x];
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) part[blockIdx.x] = a;
    }
}

// Generic single-CTA exclusive scan of part[0..n) in place; total to part[n] and,
// capped at cap, to *count_dev; sets status bit `flag` and word `word` on overflow.
__global__ void __launch_bounds__(1024) k_scan_small(int64_t n, int32_t *__restrict__ part, int32_t cap,
                                                     int32_t *__restrict__ count_dev,
                                                     int32_t *__restrict__ status, int flag, int word) {
    __shared__ int s[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int v = i < n ? part[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            s[lane] = w;
        }
        __syncthreads();
        if (i < n) part[i] = carry + (warp ? s[warp - 1] : 0) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += s[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[n] = carry;
        int m = carry;
        if (m > cap) {
            atomicOr(&status[0], flag);
            m = cap;
        }
        *count_dev = m;
        if (word >= 0) status[word] = carry;
    }
}

__global__ void __launch_bounds__(1024) k_px_emit(int64_t n, int32_t *__restrict__ flags,
                                                  const int32_t *__restrict__ part, int32_t cap,
                                                  int32_t *__restrict__ pixel_ids) {
    __shared__ int s[32];
    const int64_t id = blockIdx.x * 1024ll + threadIdx.x;
    const bool on = id < n && flags[id] != 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) s[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        int a = s[lane];
        int x = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        s[lane] = x - a;
    }
    __syncthreads();
    if (id >= n) return;
    if (!on) {
        flags[id] = -1;
        return;
    }
    const int row = part[blockIdx.x] + s[warp] + __popc(bal & ((1u << lane) - 1u));
    if (row < cap) {
        pixel_ids[row] = (int32_t)id;
        flags[id] = row;
    } else {
        flags[id] = -1;
    }
}

constexpr int PXW_THREADS = 256;
constexpr int PXW_WARPS = PXW_THREADS / 32;
constexpr int PXW_MAXE = 128;               // contributing (block column, time block) entries per pixel
constexpr int PXW_CHUNK = 512;              // ticks per step of a warp (4 float4 per lane)

// The output column of entry (slot, uy, ux) and its time block's first tick.
struct PxEntry {
    long long off;
    int t0;
};

// The output of an entry at ticks t = T0 + 128 i + 4 lane + (0..3), i < 4 (zero outside its
// range [t0, t0 + span)).
__device__ __forceinline__ void px_load(const float *__restrict__ out, long long off, int t0e, int T0, int lane,
                                        int span, float4 (&v)[4]) {
    const float *src = out + off;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int tl = T0 + 128 * i + 4 * lane - t0e;     // multiple of 4
        if (tl >= 0 && tl + 3 < span) {
            v[i] = *reinterpret_cast<const float4 *>(src + tl);
        } else if (tl + 3 < 0 || tl >= span) {
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            v[i].x = (tl >= 0 && tl < span) ? src[tl] : 0.f;
            v[i].y = (tl + 1 >= 0 && tl + 1 < span) ? src[tl + 1] : 0.f;
            v[i].z = (tl + 2 >= 0 && tl + 2 < span) ? src[tl + 2] : 0.f;
            v[i].w = (tl + 3 >= 0 && tl + 3 < span) ? src[tl + 3] : 0.f;
        }
    }
}
template <typename Acc>
__device__ __forceinline__ void px_add(Acc (&acc)[4][4], const float4 (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        acc[i][0] += v[i].x;
        acc[i][1] += v[i].y;
        acc[i][2] += v[i].z;
        acc[i][3] += v[i].w;
    }
}

// Sum, for ticks t = T0 + 128 i + 4 lane + (0..3), i < 4, the listed entries' outputs in
// list order (entries whose range [t0, t0 + span) misses the chunk add nothing).
template <typename Acc>
__device__ __forceinline__ void px_accumulate(const float *__restrict__ out, long long off, int t0e, int T0,
                                              int lane, int span, Acc (&acc)[4][4]) {
    const float *src = out + off;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int tl = T0 + 128 * i + 4 * lane - t0e;     // multiple of 4
        float4 v;
        if (tl >= 0 && tl + 3 < span) {
            v = *reinterpret_cast<const float4 *>(src + tl);
        } else if (tl + 3 < 0 || tl >= span) {
            continue;
        } else {
            v.x = (tl >= 0 && tl < span) ? src[tl] : 0.f;
            v.y = (tl + 1 >= 0 && tl + 1 < span) ? src[tl + 1] : 0.f;
            v.z = (tl + 2 >= 0 && tl + 2 < span) ? src[tl + 2] : 0.f;
            v.w = (tl + 3 >= 0 && tl + 3 < span) ? src[tl + 3] : 0.f;
        }
        acc[i][0] += v.x;
        acc[i][1] += v.y;
        acc[i][2] += v.z;
        acc[i][3] += v.w;
    }
}

// One warp per active pixel.  The pixel's contributing entries -- every active block
// whose output footprint covers it, in (by, bx, bt) order -- are listed once in shared
// memory; then the warp sweeps the window 512 ticks per step, summing per tick, in
// list order, the entries that overlap the step (a fixed order: deterministic, no
// atomics), and writes every tick of the row (zeros where no block contributes).
// Optional FP64 accumulation (compensated mode).  A pixel with more than PXW_MAXE
// entries reads the block map per step instead, in the same order.  With `possum` given,
// also records per row the sum of the positive current (FP32), a bound on the charge
// any readout scheme can integrate on the pixel.
template <bool COMP>
__global__ void __launch_bounds__(PXW_THREADS) k_px_wave(const int32_t *__restrict__ pixel_ids,
                                                         const int32_t *__restrict__ n_pixels_dev,
                                                         const int32_t *__restrict__ slot_of,
                                                         const float *__restrict__ out, GatherConst c,
                                                         float *__restrict__ wave, float *__restrict__ possum,
                                                         int32_t *__restrict__ queue) {
    using Acc = typename std::conditional<COMP, double, float>::type;
    __shared__ PxEntry s_e[PXW_WARPS][PXW_MAXE];
    const int np = n_pixels_dev[0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int span = c.bt + c.nr - 1;      // meaningful ticks of a block's output
    PxEntry *E = s_e[warp];
    (void)nwarps;
    for (;;) {   // rows from a queue: their cost varies with the number of contributing blocks
        int row = 0;
        if (lane == 0) row = atomicAdd(queue, 1);
        row = __shfl_sync(0xffffffffu, row, 0);
        if (row >= np) break;
        const int pid = pixel_ids[row];
        const int x = pid % c.npx_x, y = pid / c.npx_x;
        const int bx_lo = max(0, floordiv(x - c.bp - c.R, c.bp) + 1), bx_hi = min(c.nbx - 1, floordiv(x + c.R, c.bp));
        const int ev = y / c.npy_e;
        const int by_lo = max(ev * c.nby_e, floordiv(y - c.bp - c.R, c.bp) + 1);
        const int by_hi = min((ev + 1) * c.nby_e - 1, floordiv(y + c.R, c.bp));
        // list the entries (ballot compaction over time blocks, columns in order)
        __syncwarp();
        int ne = 0;
        for (int by = by_lo; by <= by_hi; ++by)
            for (int bx = bx_lo; bx <= bx_hi; ++bx) {
                const int uy = y - by * c.bp + c.R, ux = x - bx * c.bp + c.R;
                for (int b0 = 0; b0 < c.nbt; b0 += 32) {
                    const int bt = b0 + lane;
                    const int slot = bt < c.nbt ? slot_of[((int64_t)by * c.nbx + bx) * c.nbt + bt] : -1;
                    const unsigned bal = __ballot_sync(0xffffffffu, slot >= 0);
                    if (slot >= 0) {
                        const int idx = ne + __popc(bal & ((1u << lane) - 1u));
                        if (idx < PXW_MAXE) E[idx] = {(((long long)slot * LP + uy) * LP + ux) * c.lt, bt * c.bt};
                    }
                    ne += __popc(bal);
                }
            }
        __syncwarp();
        float *dst = wave + (size_t)row * c.nt;
        float pos = 0.f;
        for (int T0 = 0; T0 < c.nt; T0 += PXW_CHUNK) {
            Acc acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[i][e] = 0;
            if (ne <= PXW_MAXE) {
                // the entries that overlap the step, two at a time with all eight loads in
                // flight before either is added (still in list order)
                int k = 0;
                for (;;) {
                    while (k < ne && (E[k].t0 >= T0 + PXW_CHUNK || E[k].t0 + span <= T0)) ++k;
                    if (k >= ne) break;
                    const PxEntry ea = E[k++];
                    while (k < ne && (E[k].t0 >= T0 + PXW_CHUNK || E[k].t0 + span <= T0)) ++k;
                    float4 va[4], vb[4];
                    px_load(out, ea.off, ea.t0, T0, lane, span, va);
                    if (k < ne) {
                        const PxEntry eb = E[k++];
                        px_load(out, eb.off, eb.t0, T0, lane, span, vb);
                        px_add(acc, va);
                        px_add(acc, vb);
                    } else {
                        px_add(acc, va);
                    }
                }
            } else {
                const int bt_lo = max(0, floordiv(T0 - span, c.bt) + 1);
                const int bt_hi = min(c.nbt - 1, floordiv(T0 + PXW_CHUNK - 1, c.bt));
                for (int by = by_lo; by <= by_hi; ++by)
                    for (int bx = bx_lo; bx <= bx_hi; ++bx) {
                        const int uy = y - by * c.bp + c.R, ux = x - bx * c.bp + c.R;
                        for (int bt = bt_lo; bt <= bt_hi; ++bt) {
                            const int slot = slot_of[((int64_t)by * c.nbx + bx) * c.nbt + bt];
                            if (slot < 0) continue;
                            px_accumulate(out, (((long long)slot * LP + uy) * LP + ux) * c.lt, bt * c.bt, T0, lane,
                                          span, acc);
                        }
                    }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int t = T0 + 128 * i + 4 * lane;
                if (t < c.nt) {
                    const float4 o = make_float4((float)acc[i][0], (float)acc[i][1], (float)acc[i][2], (float)acc[i][3]);
                    *reinterpret_cast<float4 *>(dst + t) = o;
                    pos += fmaxf(o.x, 0.f) + fmaxf(o.y, 0.f) + fmaxf(o.z, 0.f) + fmaxf(o.w, 0.f);
                }
            }
        }
        if (possum) {
#pragma unroll
            for (int o = 16; o; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
            if (lane == 0) possum[row] = pos;
        }
    }
}

// block -> slot map of the listed active blocks (the rest -1)
__global__ void k_slot_map(const int32_t *__restrict__ block_ids, const int32_t *__restrict__ n_blocks_dev,
                           int32_t *__restrict__ slot_of) {
    const int nb = n_blocks_dev[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x)
        slot_of[block_ids[k]] = k;
}

static GatherConst gather_const_of(const tred_handle *h) {
    return GatherConst{h->g.npx_x, h->d.npy, h->g.nt, h->g.bp, h->g.bt, h->g.nr, h->g.lt, h->d.R,
                       h->d.nbx, h->d.nby, h->d.nbt, h->p.compensated_gather, h->d.npy_e, h->d.nby_e};
}

int launch_pixel_list(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev, int32_t *pixel_ids,
                      int32_t *n_pixels_dev, cudaStream_t s, int32_t **queue) {
    const GatherConst c = gather_const_of(h);
    const int64_t npx = (int64_t)h->g.npx_x * h->d.npy;
    int rc = check_cuda(h, cudaMemsetAsync(h->pix_flag, 0, sizeof(int32_t) * npx, s), "clear pixel flags");
    if (rc) return rc;
    const int sms = num_sms(h);
    rc = check_cuda(h, cudaMemsetAsync(h->blk_slot, 0xff, sizeof(int32_t) * h->d.nblk, s), "clear slots");
    if (rc) return rc;
    k_slot_map<<<sms * 2, 256, 0, s>>>(block_ids, n_blocks_dev, h->blk_slot);
    k_px_mark<<<sms * 8, 256, 0, s>>>(block_ids, n_blocks_dev, c, h->pix_flag);
    k_px_chunk<<<(unsigned)h->pix_chunks, 1024, 0, s>>>(npx, h->pix_flag, h->pix_part);
    k_scan_small<<<1, 1024, 0, s>>>(h->pix_chunks, h->pix_part, h->max_pixels, n_pixels_dev, h->status,
                                    TRED_ST_PIXEL_OVERFLOW, 4);
    k_px_emit<<<(unsigned)h->pix_chunks, 1024, 0, s>>>(npx, h->pix_flag, h->pix_part, h->max_pixels, pixel_ids);
    h->launches += 5;
    *queue = h->pix_part + h->pix_chunks + 4;   // past the scan's total
    return check_cuda(h, cudaGetLastError(), "pixel list launch");
}

int launch_gather(tred_handle *h, const int32_t *block_ids, const int32_t *n_blocks_dev,
                  const float *out, int32_t *pixel_ids, float *wave, int32_t *n_pixels_dev,
                  cudaStream_t s, float *possum) {
    const GatherConst c = gather_const_of(h);
    int32_t *queue = nullptr;
    int rc = launch_pixel_list(h, block_ids, n_blocks_dev, pixel_ids, n_pixels_dev, s, &queue);
    if (rc) return rc;
    const int sms = num_sms(h);
    const int pxw_grid = min(sms * 8, (h->max_pixels + PXW_WARPS - 1) / PXW_WARPS);   // a warp per pixel
    rc = check_cuda(h, cudaMemsetAsync(queue, 0, sizeof(int32_t), s), "gather queue reset");
    if (rc) return rc;
    if (c.comp)
        k_px_wave<true><<<pxw_grid, PXW_THREADS, 0, s>>>(pixel_ids, n_pixels_dev, h->blk_slot, out, c, wave, possum,
                                                        queue);
    else
        k_px_wave<false><<<pxw_grid, PXW_THREADS, 0, s>>>(pixel_ids, n_pixels_dev, h->blk_slot, out, c, wave, possum,
                                                         queue);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "gather launch");
}

// the indices of the set flags among flags[0..n), ascending, into ids[] and their count to
// *count_dev (flags rewritten to the index's position or -1, as in the pixel list); part:
// [n / 1024 + 8] scratch
int launch_flag_list(tred_handle *h, int64_t n, int32_t *flags, int32_t *part, int32_t *ids, int32_t *count_dev,
                     cudaStream_t s) {
    const unsigned nch = (unsigned)((n + 1023) / 1024);
    k_px_chunk<<<nch, 1024, 0, s>>>(n, flags, part);
    k_scan_small<<<1, 1024, 0, s>>>(nch, part, (int32_t)n, count_dev, h->status, 0, -1);
    k_px_emit<<<nch, 1024, 0, s>>>(n, flags, part, (int32_t)n, ids);
    h->launches += 3;
    return check_cuda(h, cudaGetLastError(), "flag list launch");
}

// exported for the readout
int launch_scan_small(tred_handle *h, int64_t n, int32_t *part, int32_t cap, int32_t *count_dev,
                      int flag, int word, cudaStream_t s) {
    k_scan_small<<<1, 1024, 0, s>>>(n, part, cap, count_dev, h->status, flag, word);
    h->launches += 1;
    return check_cuda(h, cudaGetLastError(), "scan launch");
}

// Exclusive scan of a long array in three passes: the sum of every 1024-entry chunk (one
// CTA each), the single-CTA scan of those sums (total, cap and overflow flag as
// k_scan_small), then each chunk's own scan plus its offset.
__device__ __forceinline__ int block_incl_scan1024(int v, int *s) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = s[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s[lane] = w;
    }
    __syncthreads();
    return x + (warp ? s[warp - 1] : 0);
}
__global__ void __launch_bounds__(1024) k_chunk_sum(int64_t n, const int32_t *__restrict__ part,
                                                    int32_t *__restrict__ sums) {
    __shared__ int s[32];
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const int x = block_incl_scan1024(i < n ? part[i] : 0, s);
    if (threadIdx.x == 1023) sums[blockIdx.x] = x;
}
__global__ void __launch_bounds__(1024) k_chunk_apply(int64_t n, int32_t *__restrict__ part,
                                                      const int32_t *__restrict__ sums, int nchunks) {
    __shared__ int s[32];
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const int v = i < n ? part[i] : 0;
    const int x = block_incl_scan1024(v, s);
    if (i < n) part[i] = sums[blockIdx.x] + x - v;
    if (blockIdx.x == 0 && threadIdx.x == 0) part[n] = sums[nchunks];
}
int launch_scan_large(tred_handle *h, int64_t n, int32_t *part, int32_t *sums, int32_t cap, int32_t *count_dev,
                      int flag, int word, cudaStream_t s) {
    const int nchunks = (int)((n + 1023) / 1024);
    if (nchunks < 1) return launch_scan_small(h, n, part, cap, count_dev, flag, word, s);
    k_chunk_sum<<<nchunks, 1024, 0, s>>>(n, part, sums);
    k_scan_small<<<1, 1024, 0, s>>>(nchunks, sums, cap, count_dev, h->status, flag, word);
    k_chunk_apply<<<nchunks, 1024, 0, s>>>(n, part, sums, nchunks);
    h->launches += 3;
    return check_cuda(h, cudaGetLastError(), "scan launch");
}

}  // namespace tred
