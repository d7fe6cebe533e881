// sort.cu -- uniform-grid binning: stable sorts of particles by cell key.
//
// Neighbour search (the paper uses compact hashing, Sec. 5.1) is replaced by
// a dense grid whose cell ids follow a fixed float32 quantization contract
// (gs.h), so that cell ids, counts and the sorted order are bit-exact
// reproducible.  Every sort here is stable by (key, index), so the two
// methods below give the same order:
//  - counting sort (LR cells; HR fine cells when the key space is not much
//    larger than the HR set): atomic counts per key, an exclusive scan into
//    cell starts, a scatter by arrival rank, then each cell's entries put in
//    index order;
//  - LSD radix sort (HR fine cells in sparse grids, the static-scratch
//    binning): each 8-bit pass ranks equal digits in index order within a
//    tile (warp match + per-warp counts), and tiles are laid out in order by
//    an exclusive scan over (digit, tile).
#include <cuda_runtime.h>

#include <algorithm>

#include "grid.cuh"
#include "gs_internal.cuh"

namespace {

constexpr int kBins = 256;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kTargetBlocks = 152;   // one tile per SM; the scan grows with the tile count
constexpr int kMaxItems = 32;

int items_for(int64_t n)
{
    int64_t it = (n + (int64_t)kThreads * kTargetBlocks - 1) / ((int64_t)kThreads * kTargetBlocks);
    return (int)std::min<int64_t>(std::max<int64_t>(it, 1), kMaxItems);
}

int64_t blocks_for(int64_t n, int items) { return (n + (int64_t)kThreads * items - 1) / ((int64_t)kThreads * items); }

__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                      int items, uint32_t* __restrict__ hist, int64_t nblocks)
{
    __shared__ uint32_t h[kBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * items * kThreads;
    for (int r = 0; r < items; ++r) {
        int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of total words in place, one block.  The data is walked in
// coalesced tiles of kScanThreads x 8 words (two 16-byte loads per thread),
// each tile scanned with warp shuffles and carried into the next.  total is
// a multiple of 256 (digits x tiles), so the vector accesses stay in bounds.
__global__ void __launch_bounds__(kScanThreads) k_rs_scan(uint32_t* __restrict__ data, int64_t total)
{
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    __shared__ uint32_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    constexpr int kPer = 8;
    for (int64_t base = 0; base < total; base += (int64_t)kScanThreads * kPer) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kPer;
        uint32_t v[kPer];
        if (i0 + kPer <= total) {
            uint4 a = *reinterpret_cast<const uint4*>(data + i0);
            uint4 b = *reinterpret_cast<const uint4*>(data + i0 + 4);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < kPer; ++k) v[k] = i0 + k < total ? data[i0 + k] : 0u;
        }
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) s += v[k];
        uint32_t x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const uint32_t carry = carry_s;
        uint32_t run = carry + x - s + (warp > 0 ? warp_sums[warp - 1] : 0u);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            uint32_t t = v[k];
            v[k] = run;
            run += t;
        }
        if (i0 + kPer <= total) {
            *reinterpret_cast<uint4*>(data + i0) = make_uint4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<uint4*>(data + i0 + 4) = make_uint4(v[4], v[5], v[6], v[7]);
        } else {
            for (int k = 0; k < kPer; ++k)
                if (i0 + k < total) data[i0 + k] = v[k];
        }
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry_s = run;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         int64_t n, int shift, int items,
                                                         const uint32_t* __restrict__ offsets, int64_t nblocks)
{
    __shared__ uint32_t run[kBins];
    __shared__ uint32_t wcnt[kWarps][kBins];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offsets[(int64_t)tid * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * items * kThreads;
    for (int r = 0; r < items; ++r) {
        int64_t i = base + (int64_t)r * kThreads + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((key >> shift) & (kBins - 1)) : (uint32_t)kBins;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            tot += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += tot;
        __syncthreads();
    }
}


__global__ void k_cell_keys(const float4* __restrict__ pos, int64_t n, GridDev g, int fine,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos[i];
    int sx = grid_sub_coord(p.x, g.ox, g.inv_h, g.dx);
    int sy = grid_sub_coord(p.y, g.oy, g.inv_h, g.dy);
    int sz = grid_sub_coord(p.z, g.oz, g.inv_h, g.dz);
    uint32_t cell = ((uint32_t)(sz >> 1) * (uint32_t)g.dy + (uint32_t)(sy >> 1)) * (uint32_t)g.dx + (uint32_t)(sx >> 1);
    keys[i] = fine ? cell * 8u + (uint32_t)((sz & 1) * 4 + (sy & 1) * 2 + (sx & 1)) : cell;
    vals[i] = (uint32_t)i;
}

__device__ __forceinline__ uint32_t scene_key(const float4* __restrict__ pos, int64_t i,
                                              const SceneDev* __restrict__ scenes, const uint32_t* __restrict__ tag,
                                              int fine)
{
    const uint32_t t = tag[i];
    const SceneDev& sc = scenes[t & ~kPadBit];
    if (t & kPadBit) return fine ? (sc.cell_off + sc.n_cell) * 8u : sc.cell_off + sc.n_cell;
    const GridDev& g = sc.g;
    float4 p = pos[i];
    int sx = grid_sub_coord(p.x, g.ox, g.inv_h, g.dx);
    int sy = grid_sub_coord(p.y, g.oy, g.inv_h, g.dy);
    int sz = grid_sub_coord(p.z, g.oz, g.inv_h, g.dz);
    uint32_t cell = sc.cell_off +
                    ((uint32_t)(sz >> 1) * (uint32_t)g.dy + (uint32_t)(sy >> 1)) * (uint32_t)g.dx + (uint32_t)(sx >> 1);
    return fine ? cell * 8u + (uint32_t)((sz & 1) * 4 + (sy & 1) * 2 + (sx & 1)) : cell;
}

// Global key of a slot that belongs to scene tag & ~kPadBit: the scene's
// cell offset plus its cell id (times 8 plus the octant when fine); padding
// slots take the scene's padding cell so they sort to the end of its range.
__global__ void k_scene_keys(const float4* __restrict__ pos, int64_t n, const SceneDev* __restrict__ scenes,
                             const uint32_t* __restrict__ tag, int fine, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals, uint32_t* __restrict__ count)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (count) {
        // counting sort: the lanes of a warp that share a key take
        // consecutive ranks from one atomic (a reordered set arrives sorted)
        const bool ok = i < n;
        const uint32_t key = ok ? scene_key(pos, i, scenes, tag, fine) : 0xffffffffu;   // above every key
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (ok && lane == leader) base = atomicAdd(count + key, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (ok) {
            keys[i] = key;
            vals[i] = base + __popc(peers & ((1u << lane) - 1u));
        }
        return;
    }
    if (i >= n) return;
    keys[i] = scene_key(pos, i, scenes, tag, fine);
    vals[i] = (uint32_t)i;
}

// ---- stable counting sort by cell (the LR set) ------------------------
// Items are counted per cell with atomics, each keeping its arrival rank
// within its cell; the exclusive scan of the counts is the cell start table;
// items go to start + rank; finally every cell's entries are put in
// ascending item order, which makes the result that of a stable sort.

__global__ void k_cs_keys(const float4* __restrict__ pos, int64_t n, const SceneDev* __restrict__ scenes,
                          const uint32_t* __restrict__ tag, uint32_t* __restrict__ keys, uint32_t* __restrict__ rank,
                          uint32_t* __restrict__ cnt, unsigned* solid_flag, const uint32_t* __restrict__ body)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SceneDev& sc = scenes[tag[i] & ~kPadBit];
    const float4 p = pos[i];
    // a particle of infinite mass or of a rigid body
    if (solid_flag && (p.w == 0.0f || (body && body[i] != 0u))) atomicOr(solid_flag, 1u);
    const uint32_t cell = grid_cell_of(sc, p.x, p.y, p.z);
    keys[i] = cell;
    rank[i] = atomicAdd(cnt + cell, 1u);
}

constexpr int kScanBlock = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanBlock * kScanPer;

// Block-wide inclusive scan of one value per thread; returns the inclusive
// sum, *total receives the block total.
__device__ __forceinline__ uint32_t block_scan(uint32_t x, uint32_t* warp_sums, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    const uint32_t r = x + (warp > 0 ? warp_sums[warp - 1] : 0u);
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void load_tile(const uint32_t* data, int64_t total, int64_t i0, uint32_t v[kScanPer])
{
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) v[k] = i0 + k < total ? data[i0 + k] : 0u;
}

// tile_sums[b] = sum of tile b
__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(const uint32_t* __restrict__ data, int64_t total,
                                                           uint32_t* __restrict__ tile_sums)
{
    __shared__ uint32_t ws[32];
    const int64_t i0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    load_tile(data, total, i0, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) s += v[k];
    uint32_t tot;
    block_scan(s, ws, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// exclusive scan of the nt tile sums in place (one block, chunks with carry)
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(uint32_t* __restrict__ sums, int64_t nt)
{
    __shared__ uint32_t ws[32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < nt; b += kScanBlock) {
        const int64_t i = b + threadIdx.x;
        const uint32_t x = i < nt ? sums[i] : 0u;
        uint32_t tot;
        const uint32_t inc = block_scan(x, ws, &tot);
        if (i < nt) sums[i] = carry + inc - x;
        carry += tot;
    }
}

// exclusive scan of every tile plus its tile offset, in place
// raw_sums: tile_sums holds each tile's own total (k_scan_sums skipped) and
// every block adds up the totals of the tiles before it (few tiles).
__global__ void __launch_bounds__(kScanBlock) k_scan_apply(uint32_t* __restrict__ data, int64_t total,
                                                           const uint32_t* __restrict__ tile_sums, int raw_sums)
{
    __shared__ uint32_t ws[32];
    uint32_t tot;
    uint32_t base;
    if (raw_sums) {
        uint32_t part = 0;
        for (int64_t t = threadIdx.x; t < (int64_t)blockIdx.x; t += kScanBlock) part += tile_sums[t];
        block_scan(part, ws, &tot);
        base = tot;
    } else {
        base = tile_sums[blockIdx.x];
    }
    const int64_t i0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    load_tile(data, total, i0, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) s += v[k];
    const uint32_t inc = block_scan(s, ws, &tot);
    uint32_t run = base + inc - s;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const uint32_t t = v[k];
        if (i0 + k < total) data[i0 + k] = run;
        run += t;
    }
}

__global__ void k_cs_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rank, int64_t n,
                             const uint32_t* __restrict__ start, uint32_t* __restrict__ out_keys,
                             uint32_t* __restrict__ out_idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = keys[i];
    const uint32_t pos = start[k] + rank[i];
    out_keys[pos] = k;
    out_idx[pos] = (uint32_t)i;
}

// every cell's entries in ascending item order.  A cell holds a handful of
// LR particles (HR fine cells a few dozen): its entries are loaded at once
// into registers (padded with the largest key) and ordered by a fixed
// compare-exchange network; larger cells are ordered cooperatively (see
// k_cs_order), so no cell costs quadratic work.
template <int K>
__device__ __forceinline__ void order_small(uint32_t* __restrict__ idx, uint32_t b, uint32_t n)
{
    uint32_t v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (uint32_t)k < n ? idx[b + k] : 0xffffffffu;
#pragma unroll
    for (int i = 0; i < K - 1; ++i) {
#pragma unroll
        for (int j = 0; j < K - 1 - i; ++j) {
            const uint32_t lo = min(v[j], v[j + 1]), hi = max(v[j], v[j + 1]);
            v[j] = lo;
            v[j + 1] = hi;
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
        if ((uint32_t)k < n) idx[b + k] = v[k];
}

// 32 entries: Batcher's odd-even merge sort network (191 compare-exchanges
// against 496 for the transposition network above).
__device__ __forceinline__ void order_32(uint32_t* __restrict__ idx, uint32_t b, uint32_t n)
{
    constexpr int K = 32;
    uint32_t v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (uint32_t)k < n ? idx[b + k] : 0xffffffffu;
    // stage (p, k): entry i meets i + k when i lies in the lower half of its
    // 2k-block counted from k mod p and both lie in the same 2p-block
#pragma unroll
    for (int p = 1; p < K; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int j0 = k % p;
                if (i >= j0 && ((i - j0) / k) % 2 == 0 && i + k < K && i / (2 * p) == (i + k) / (2 * p)) {
                    const uint32_t lo = min(v[i], v[i + k]), hi = max(v[i], v[i + k]);
                    v[i] = lo;
                    v[i + k] = hi;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
        if ((uint32_t)k < n) idx[b + k] = v[k];
}

// One warp orders a cell of up to 32 R distinct entries: lane l holds
// entries l, l + 32, ... (coalesced), every entry's place is the number of
// entries below it, counted against all of them broadcast by shuffles.
template <int R>
__device__ __forceinline__ void order_warp(uint32_t* __restrict__ idx, uint32_t b, uint32_t n, int lane)
{
    uint32_t v[R], rk[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t t = (uint32_t)(r * 32 + lane);
        v[r] = t < n ? idx[b + t] : 0xffffffffu;   // above every entry: never counted
        rk[r] = 0;
    }
#pragma unroll
    for (int r2 = 0; r2 < R; ++r2) {
        if ((uint32_t)(r2 * 32) >= n) break;   // warp-uniform
#pragma unroll
        for (int s = 0; s < 32; ++s) {
            const uint32_t u = __shfl_sync(0xffffffffu, v[r2], s);
#pragma unroll
            for (int r = 0; r < R; ++r) rk[r] += u < v[r] ? 1u : 0u;
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r)
        if ((uint32_t)(r * 32 + lane) < n) idx[b + rk[r]] = v[r];
    __syncwarp();
}

// One warp orders a cell of any size (entries below 2^bits) by stable
// 4-bit LSD passes, ping-ponging between idx and scratch over the cell's
// range: per pass a digit histogram (lane d counts digit d), its exclusive
// scan, then chunks of 32 in order, each entry placed after the earlier
// lanes of its chunk with the same digit.  Linear work per pass; no shared
// memory.
__device__ void warp_lsd(uint32_t* __restrict__ idx, uint32_t* __restrict__ scratch, uint32_t b, uint32_t n,
                         int bits, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* src = idx + b;
    uint32_t* dst = scratch + b;
    for (int shift = 0; shift < bits; shift += 4) {
        uint32_t cnt = 0;
        for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t t = base + (uint32_t)lane;
            const uint32_t d = t < n ? (src[t] >> shift) & 15u : 16u;
#pragma unroll
            for (uint32_t q = 0; q < 16; ++q) {
                const unsigned m = __ballot_sync(0xffffffffu, d == q);
                if ((uint32_t)lane == q) cnt += (uint32_t)__popc(m);
            }
        }
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t off = inc - cnt;   // lane d < 16: where digit d starts
        for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t t = base + (uint32_t)lane;
            const bool valid = t < n;
            const uint32_t v = valid ? src[t] : 0u;
            const uint32_t d = valid ? (v >> shift) & 15u : 16u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t o = __shfl_sync(0xffffffffu, off, (int)d);
            if (valid) dst[o + (uint32_t)__popc(peers & lt)] = v;
#pragma unroll
            for (uint32_t q = 0; q < 16; ++q) {
                const unsigned m = __ballot_sync(0xffffffffu, d == q);
                if ((uint32_t)lane == q) off += (uint32_t)__popc(m);
            }
        }
        __syncwarp();
        uint32_t* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != idx + b)
        for (uint32_t t = (uint32_t)lane; t < n; t += 32) idx[b + t] = src[t];
    __syncwarp();
}

// Entries [b + first, e) step `step` of one ordered cell: two arrays copied
// into cell order with the extras, and each particle's slot.
__device__ __forceinline__ void copy_cell(const uint32_t* __restrict__ idx, uint32_t b, uint32_t e, uint32_t first,
                                          uint32_t step, const float4* __restrict__ ga, const float4* __restrict__ gb,
                                          float4* __restrict__ ga_out, float4* __restrict__ gb_out,
                                          const CsExtras& ex)
{
    if (ga) {
        for (uint32_t j = b + first; j < e; j += step) {
            const uint32_t i = idx[j];
            float4 u = ga[i];
            if (ex.ga_solid && ex.ga_solid[i] != 0u) u.w = 0.0f;
            ga_out[j] = u;
            if (gb) {
                float4 v = gb[i];
                if (ex.gb_w) v.w = __uint_as_float(ex.gb_w[i]);
                gb_out[j] = v;
            }
        }
    }
    if (ex.slot_of)
        for (uint32_t j = b + first; j < e; j += step) ex.slot_of[idx[j]] = j;
}

// One thread per cell.  Cells of more than 32 entries go to ex.big_list
// when there is one (ordered by k_cs_order_big, which balances them over
// the whole grid); otherwise the warp that met them orders them one after
// another (order_warp up to 256 entries, warp_lsd beyond, scratch: n words
// of which those cells' ranges are overwritten).
__global__ void __launch_bounds__(256, 4) k_cs_order(const uint32_t* __restrict__ start, int64_t n_cell,
                                                     uint32_t* __restrict__ idx, const float4* __restrict__ ga,
                                                     const float4* __restrict__ gb, float4* __restrict__ ga_out,
                                                     float4* __restrict__ gb_out, uint32_t* __restrict__ scratch,
                                                     int bits, const CsExtras ex)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(threadIdx.x & 31u);
    uint32_t b = 0, e = 0;
    bool big = false;   // every lane reaches the ballot below: no early return
    if (c < n_cell) {
        b = start[c];
        e = start[c + 1];
        const uint32_t n = e - b;
        if (n > 32) {
            if (ex.big_list) ex.big_list[atomicAdd(ex.big_count, 1u)] = (uint32_t)c;
            else big = true;
        } else if (n > 0) {
            if (n == 1) {
            } else if (n <= 4) {
                order_small<4>(idx, b, n);
            } else if (n <= 8) {
                order_small<8>(idx, b, n);
            } else if (n <= 16) {
                order_small<16>(idx, b, n);
            } else {
                order_32(idx, b, n);
            }
            copy_cell(idx, b, e, 0, 1, ga, gb, ga_out, gb_out, ex);
        }
    }
    unsigned pend = __ballot_sync(0xffffffffu, big);
    while (pend) {   // warp-uniform
        const int j = __ffs(pend) - 1;
        pend &= pend - 1u;
        const uint32_t cb = __shfl_sync(0xffffffffu, b, j), ce = __shfl_sync(0xffffffffu, e, j);
        const uint32_t n = ce - cb;
        if (n <= 64) order_warp<2>(idx, cb, n, lane);
        else if (n <= 256) order_warp<8>(idx, cb, n, lane);
        else warp_lsd(idx, scratch, cb, n, bits, lane);
        copy_cell(idx, cb, ce, (uint32_t)lane, 32u, ga, gb, ga_out, gb_out, ex);
        __syncwarp();
    }
}

// Cells of more than 32 entries, listed by k_cs_order.  Cells of up to 256
// entries are ordered by one warp each (order_warp).  Larger ones, one block
// each, by stable 8-bit LSD passes over the cell's item indices (the tile
// ranking of k_rs_scatter over the cell's range, tiles in order),
// ping-ponging between idx and scratch over the same range: work linear in
// the cell's size per pass, so a degenerate cell (every particle at one
// point) costs a few passes over the set, not a quadratic sort.
__global__ void __launch_bounds__(kThreads) k_cs_order_big(const uint32_t* __restrict__ start,
                                                           const uint32_t* __restrict__ list,
                                                           const uint32_t* __restrict__ count,
                                                           uint32_t* __restrict__ idx, uint32_t* __restrict__ scratch,
                                                           int bits)
{
    __shared__ uint32_t run[kBins];
    __shared__ uint32_t wcnt[kWarps][kBins];
    __shared__ uint32_t wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t n_big = *count;
    const uint32_t n_warps = gridDim.x * kWarps;
    for (uint32_t q = blockIdx.x * kWarps + warp; q < n_big; q += n_warps) {
        const uint32_t cell = list[q];
        const uint32_t b = start[cell], n = start[cell + 1] - b;
        if (n <= 64) order_warp<2>(idx, b, n, lane);
        else if (n <= 256) order_warp<8>(idx, b, n, lane);
    }
    for (uint32_t q = blockIdx.x; q < n_big; q += gridDim.x) {
        const uint32_t cell = list[q];
        const uint32_t b = start[cell], n = start[cell + 1] - b;
        if (n <= 256) continue;   // the same cell for the whole block: uniform
        uint32_t* src = idx + b;
        uint32_t* dst = scratch + b;
        for (int shift = 0; shift < bits; shift += 8) {
            run[tid] = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
            __syncthreads();
            for (uint32_t t = tid; t < n; t += kThreads) atomicAdd(&run[(src[t] >> shift) & (kBins - 1)], 1u);
            __syncthreads();
            // exclusive scan of the 256 digit counts, one per thread
            const uint32_t h = run[tid];
            uint32_t inc = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) wsum[warp] = inc;
            __syncthreads();
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += wsum[w];
            run[tid] = before + inc - h;
            __syncthreads();
            for (uint32_t base = 0; base < n; base += kThreads) {
                const uint32_t t = base + tid;
                const bool valid = t < n;
                const uint32_t v = valid ? src[t] : 0u;
                const uint32_t d = valid ? ((v >> shift) & (kBins - 1)) : (uint32_t)kBins;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                const unsigned rank = __popc(peers & lt);
                if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
                __syncthreads();
                if (valid) {
                    uint32_t pos = run[d] + rank;
                    for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
                    dst[pos] = v;
                }
                __syncthreads();
                uint32_t tot = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    tot += wcnt[w][tid];
                    wcnt[w][tid] = 0;
                }
                run[tid] += tot;
                __syncthreads();
            }
            uint32_t* t = src;
            src = dst;
            dst = t;
        }
        if (src != idx + b)
            for (uint32_t t = tid; t < n; t += kThreads) idx[b + t] = src[t];
        __syncthreads();
    }
}

__global__ void k_cell_start(const uint32_t* __restrict__ sk, int64_t n, int64_t n_cell, uint32_t* __restrict__ start)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n_cell) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)sk[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    start[c] = (uint32_t)lo;
}

__global__ void k_gather2(const uint32_t* __restrict__ idx, const float4* __restrict__ a, const float4* __restrict__ b,
                          float4* __restrict__ ao, float4* __restrict__ bo, int64_t n)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t i = idx[p];
    ao[p] = a[i];
    if (b) bo[p] = b[i];
}

// HR exchange in original-id order: slot p (a real particle, not padding)
// holds the particle whose id is in pos.w.
__global__ void k_unpermute(const float4* __restrict__ pos, const float4* __restrict__ f,
                            const uint32_t* __restrict__ tag, float4* __restrict__ out, int64_t n_slots,
                            int64_t n_real, int* err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_slots || (tag[p] & kPadBit)) return;
    uint32_t id = __float_as_uint(pos[p].w);
    if ((int64_t)id >= n_real) {
        atomicOr(err, GS_DEVERR_BAD_ID);
        return;
    }
    out[id] = f[p];
}

// Both HR fields at once: position and velocity of slot p to their ids.
__global__ void k_unpermute2(const float4* __restrict__ pos, const float4* __restrict__ vel,
                             const uint32_t* __restrict__ tag, float4* __restrict__ out_pos,
                             float4* __restrict__ out_vel, int64_t n_slots, int64_t n_real, int* err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_slots || (tag[p] & kPadBit)) return;
    const float4 x = pos[p];
    uint32_t id = __float_as_uint(x.w);
    if ((int64_t)id >= n_real) {
        atomicOr(err, GS_DEVERR_BAD_ID);
        return;
    }
    out_pos[id] = x;
    out_vel[id] = vel[p];
}

__global__ void k_permute_in(const float4* __restrict__ pos, const float4* __restrict__ f,
                             const uint32_t* __restrict__ tag, float4* __restrict__ out, int64_t n_slots,
                             int64_t n_real, int* err)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_slots || (tag[p] & kPadBit)) return;
    uint32_t id = __float_as_uint(pos[p].w);
    if ((int64_t)id >= n_real) {
        atomicOr(err, GS_DEVERR_BAD_ID);
        return;
    }
    out[p] = f[id];
}

__global__ void k_check_finite(const float4* __restrict__ a, int64_t n, int* flag, int bit)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float4 v = a[p];
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) atomicOr(flag, bit);
}

}  // namespace

size_t gs_sort_hist_words(int64_t n)
{
    int items = items_for(n);
    int64_t nb = blocks_for(n, items);
    return (size_t)kBins * (size_t)std::max<int64_t>(nb, 1);
}

int gs_key_bits(int64_t n_keys)
{
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) < n_keys) ++b;
    return b;
}

cudaError_t gs_radix_sort(cudaStream_t s, uint32_t* keys[2], uint32_t* vals[2], int* which, uint32_t* hist,
                          int64_t n, int key_bits, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    int items = items_for(n);
    int64_t nb = blocks_for(n, items);
    for (int shift = 0; shift < key_bits; shift += 8) {
        int a = *which, b = a ^ 1;
        k_rs_hist<<<(unsigned)nb, kThreads, 0, s>>>(keys[a], n, shift, items, hist, nb);
        k_rs_scan<<<1, kScanThreads, 0, s>>>(hist, (int64_t)kBins * nb);
        k_rs_scatter<<<(unsigned)nb, kThreads, 0, s>>>(keys[a], vals[a], keys[b], vals[b], n, shift, items, hist, nb);
        *launches += 3;
        *which = b;
    }
    return cudaGetLastError();
}

size_t gs_scan_aux_words(int64_t total) { return (size_t)std::max<int64_t>(1, (total + kScanTile - 1) / kScanTile); }

cudaError_t gs_cs_clear(cudaStream_t s, uint32_t* cell_start, int64_t n_cell, int extra)
{
    return cudaMemsetAsync(cell_start, 0, (size_t)(n_cell + 1 + extra) * sizeof(uint32_t), s);
}

cudaError_t gs_cs_keys(cudaStream_t s, const float4* pos, int64_t n, const SceneDev* scenes, const uint32_t* tag,
                       uint32_t* keys, uint32_t* rank, uint32_t* cell_start, int64_t* launches,
                       unsigned* solid_flag, const uint32_t* body)
{
    if (n <= 0) return cudaSuccess;
    k_cs_keys<<<gs_blocks(n, 256), 256, 0, s>>>(pos, n, scenes, tag, keys, rank, cell_start, solid_flag, body);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_cs_finish(cudaStream_t s, int64_t n, int64_t n_cell, const uint32_t* keys, uint32_t* rank,
                         uint32_t* out_keys, uint32_t* out_idx, uint32_t* cell_start, uint32_t* aux, const float4* ga,
                         const float4* gb, float4* ga_out, float4* gb_out, int64_t* launches, const CsExtras& ex)
{
    const int64_t total = n_cell + 1;
    const int64_t nt = (total + kScanTile - 1) / kScanTile;
    // up to kScanBlock tiles the apply blocks add up the tile totals before
    // them themselves (at most one word per thread), saving the tile-sum scan
    const int raw = nt <= kScanBlock;
    k_scan_tiles<<<(unsigned)nt, kScanBlock, 0, s>>>(cell_start, total, aux);
    if (!raw) k_scan_sums<<<1, kScanBlock, 0, s>>>(aux, nt);
    k_scan_apply<<<(unsigned)nt, kScanBlock, 0, s>>>(cell_start, total, aux, raw);
    *launches += raw ? 2 : 3;
    if (n > 0) {
        if (ex.big_list && (ga || ex.slot_of || ex.big_blocks <= 0 || !ex.big_count || !ex.big_scratch))
            return cudaErrorInvalidValue;   // listed cells are ordered without copies
        k_cs_scatter<<<gs_blocks(n, 256), 256, 0, s>>>(keys, rank, n, cell_start, out_keys, out_idx);
        // the ranks are dead once scattered: scratch for large cells
        k_cs_order<<<gs_blocks(n_cell, 256), 256, 0, s>>>(cell_start, n_cell, out_idx, ga, gb, ga_out, gb_out, rank,
                                                          gs_key_bits(n), ex);
        *launches += 2;
        if (ex.big_list) {
            k_cs_order_big<<<(unsigned)ex.big_blocks, kThreads, 0, s>>>(cell_start, ex.big_list, ex.big_count, out_idx,
                                                                       ex.big_scratch, ex.big_bits);
            *launches += 1;
        }
    }
    return cudaGetLastError();
}

cudaError_t gs_count_sort_cells(cudaStream_t s, const float4* pos, int64_t n, const SceneDev* scenes,
                                const uint32_t* tag, int64_t n_cell, uint32_t* keys, uint32_t* rank,
                                uint32_t* out_keys, uint32_t* out_idx, uint32_t* cell_start, uint32_t* aux,
                                int64_t* launches)
{
    cudaError_t e = gs_cs_clear(s, cell_start, n_cell);
    if (e == cudaSuccess) e = gs_cs_keys(s, pos, n, scenes, tag, keys, rank, cell_start, launches);
    if (e == cudaSuccess)
        e = gs_cs_finish(s, n, n_cell, keys, rank, out_keys, out_idx, cell_start, aux, nullptr, nullptr, nullptr,
                         nullptr, launches);
    return e;
}

cudaError_t gs_launch_cell_keys(cudaStream_t s, const float4* pos, int64_t n, GridDev g, int fine, uint32_t* keys,
                                uint32_t* vals, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    k_cell_keys<<<gs_blocks(n, 256), 256, 0, s>>>(pos, n, g, fine, keys, vals);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_cell_start(cudaStream_t s, const uint32_t* sorted_keys, int64_t n, int64_t n_cell,
                                 uint32_t* start, int64_t* launches)
{
    k_cell_start<<<gs_blocks(n_cell + 1, 256), 256, 0, s>>>(sorted_keys, n, n_cell, start);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_gather2(cudaStream_t s, const uint32_t* idx, const float4* a, const float4* b, float4* a_out,
                              float4* b_out, int64_t n, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    k_gather2<<<gs_blocks(n, 256), 256, 0, s>>>(idx, a, b, a_out, b_out, n);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_unpermute(cudaStream_t s, const float4* pos_internal, const float4* field_internal,
                                const uint32_t* hr_tag, float4* out, int64_t n_slots, int64_t n_real, int* err,
                                int64_t* launches)
{
    if (n_slots <= 0) return cudaSuccess;
    k_unpermute<<<gs_blocks(n_slots, 256), 256, 0, s>>>(pos_internal, field_internal, hr_tag, out, n_slots, n_real,
                                                        err);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_unpermute2(cudaStream_t s, const float4* pos_internal, const float4* vel_internal,
                                 const uint32_t* hr_tag, float4* out_pos, float4* out_vel, int64_t n_slots,
                                 int64_t n_real, int* err, int64_t* launches)
{
    if (n_slots <= 0) return cudaSuccess;
    k_unpermute2<<<gs_blocks(n_slots, 256), 256, 0, s>>>(pos_internal, vel_internal, hr_tag, out_pos, out_vel,
                                                         n_slots, n_real, err);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_permute_in(cudaStream_t s, const float4* pos_internal, const float4* field_original,
                                 const uint32_t* hr_tag, float4* out, int64_t n_slots, int64_t n_real, int* err,
                                 int64_t* launches)
{
    if (n_slots <= 0) return cudaSuccess;
    k_permute_in<<<gs_blocks(n_slots, 256), 256, 0, s>>>(pos_internal, field_original, hr_tag, out, n_slots,
                                                         n_real, err);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_scene_keys(cudaStream_t s, const float4* pos, int64_t n, const SceneDev* scenes,
                                 const uint32_t* tag, int fine, uint32_t* keys, uint32_t* vals, int64_t* launches,
                                 uint32_t* count)
{
    if (n <= 0) return cudaSuccess;
    k_scene_keys<<<gs_blocks(n, 256), 256, 0, s>>>(pos, n, scenes, tag, fine, keys, vals, count);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t gs_launch_check_finite(cudaStream_t s, const float4* a, int64_t n, int* flag, int64_t* launches, int bit)
{
    if (n <= 0) return cudaSuccess;
    k_check_finite<<<gs_blocks(n, 256), 256, 0, s>>>(a, n, flag, bit);
    *launches += 1;
    return cudaGetLastError();
}
