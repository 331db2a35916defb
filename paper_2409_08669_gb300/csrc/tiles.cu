// Stages 3-5 of the rasterization pipeline (Sec. 3.2.1): DuplicateWithKeys,
// SortPairs by tile and IdentifyTileRanges.  The result is the paper's: for
// every tile, the Gaussians overlapping it in view-depth order (the order of
// the 64-bit (tile | depth) keys), and each tile's [start, end).
//
// Every Gaussian overlaps a rectangle of tiles, so its pairs are w column runs
// (one per tile column tx, covering rows y0 .. y0+h-1).  The sort works on
// that structure in two stable counting passes:
//   pass 1 (columns): the column runs, generated on chip from the
//          depth-ordered Gaussians, are grouped by tx -- C = sum of w items,
//          a few times fewer than the P = sum of w*h pairs;
//   pass 2 (rows):    every run is expanded into its h pairs on chip and the
//          pairs are grouped by ty; only the Gaussian ids are written.
// Grouping by tx and then stably by ty orders the pairs by (ty, tx) = tile id,
// and by depth within a tile, since both passes keep the input order.  Each
// tile's range comes from its pair count (the runs of column tx that cover
// row ty) by one scan, with no boundary search.
//
// Each pass is range-partitioned (count, scan, scatter): CTA b of a grid of G
// owns a contiguous run of 4096-item chunks,
//   1. counts its items per digit (pass 1 straight from the Gaussians'
//      rectangles, pass 2 from the runs' row intervals, as difference arrays),
//   2. the G x 256 counts become the global start of every (digit, CTA) run
//      (per-digit totals are summed with atomics while counting),
//   3. CTA b walks its chunks in order, ranks each chunk's items stably,
//      groups them by digit in shared memory and writes every digit's run
//      contiguously from its running offset.  Pass 1 ranks with a warp
//      ballot per digit bit; pass 2 from per-warp row counts and a walk over
//      the runs (see k_scatter_rows).
// No CTA ever waits for another one: the passes need no co-residency and no
// spin-waits.
#include <cstddef>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kMaxChunkGauss = kSortChunk + 1;          // every listed Gaussian has >= 1 run
constexpr int kStageLen = (kMaxChunkGauss + 3) & ~3;    // keeps the arrays after it 16-byte aligned
constexpr int kRunStage = 512;                          // runs staged at a time in pass 2
constexpr int kColSlots = 8;                            // tile-count columns a CTA keeps on chip

// Column run record: x = Gaussian id, y = y0 | (h - 1) << 8 | tx << 16.
__device__ __forceinline__ uint32_t run_y0(uint32_t y) { return y & 0xFFu; }
__device__ __forceinline__ uint32_t run_h(uint32_t y) { return ((y >> 8) & 0xFFu) + 1u; }
__device__ __forceinline__ uint32_t run_tx(uint32_t y) { return y >> 16; }

struct alignas(16) ColumnShared {
    union {
        struct {
            uint32_t keys[kSortChunk];   // run record y (digit tx = key >> 16)
            uint32_t vals[kSortChunk];   // Gaussian id
        } kv;
        struct {                         // Gaussians overlapping one run chunk
            uint32_t off[kStageLen];
            uint32_t gid[kStageLen];
            uint32_t box[kStageLen];     // x0 | y0 << 8 | (w-1) << 16 | (h-1) << 24
            alignas(16) uint16_t map[kSortChunk];   // chunk slot -> staged Gaussian holding it
        } stage;
    } u;
    uint32_t warp_cnt[kWarps][kRadix + 1];   // +1: out-of-range items of the tail chunk
    uint32_t run[kRadix];                    // next global position of each digit
    uint32_t local[kRadix + 1];              // exclusive prefix of this chunk's digit counts
    uint32_t dst[kRadix];                    // global position of local slot 0, per digit
    uint32_t wsum[kWarps];
};

constexpr int kBands = 16;                   // horizontal bands of tile rows in pass 2
constexpr int kMaxBandRows = kRadix / kBands;   // rows per band at most (256 tile rows)

struct alignas(16) RowShared {
    uint32_t rows[kRunStage];                // staged runs: y0 | y1 << 16 (rows [y0, y1))
    uint32_t gid[kRunStage];                 // their Gaussians
    uint16_t band[kBands][kRunStage];        // staged runs meeting each band, in run order
    uint32_t band_len[kBands];
    uint32_t next_band;                      // next band to sweep
    uint32_t pos[kRadix];                    // next global position of each tile row
};
static_assert(offsetof(ColumnShared, u) % 16 == 0, "staging must be 16-byte aligned");
static_assert((3 * kStageLen * sizeof(uint32_t)) % 16 == 0, "map must be 16-byte aligned");
constexpr size_t kColumnSmem = sizeof(ColumnShared);

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The item count of a pass and the chunks [c0, c1) of CTA blockIdx.x.
struct Span {
    int64_t n;
    uint32_t nchunks, c0, c1;
};
__device__ __forceinline__ Span cta_span(int64_t n, int grid) {
    Span s;
    s.n = n;
    s.nchunks = (uint32_t)((n + kSortChunk - 1) / kSortChunk);
    const uint32_t per = (s.nchunks + (uint32_t)grid - 1u) / (uint32_t)grid;
    s.c0 = min(s.nchunks, per * blockIdx.x);
    s.c1 = min(s.nchunks, s.c0 + per);
    return s;
}

// Items of the two passes: the column runs C, or none when the pairs
// overflowed the capacity (the frame then reports ADR_ERR_CAPACITY).
__device__ __forceinline__ int64_t run_count(const uint32_t* counters, int64_t capacity) {
    if ((int64_t)counters[kCntPairs] > capacity) return 0;
    return min((int64_t)counters[kCntRuns], capacity);
}

// Exclusive block scan over the 256 threads (one value each); returns the
// thread's exclusive prefix, `total` the sum.  Uses wsum; ends synchronised.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* wsum, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t base = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t s = wsum[w];
        base += w < warp ? s : 0u;
        total += s;
    }
    __syncthreads();
    return base + x - v;
}

// In-place running maximum over map[0 .. kSortChunk) (u16 entries, 16 per
// thread), so that every slot names the staged item holding it.
__device__ __forceinline__ void map_running_max(uint16_t* map, uint32_t* wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint4* m4 = reinterpret_cast<uint4*>(map) + 2 * tid;
    const uint4 a = m4[0], b = m4[1];
    const uint32_t w32[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t tmax = 0;
#pragma unroll
    for (int x = 0; x < 8; ++x) tmax = max(tmax, max(w32[x] & 0xFFFFu, w32[x] >> 16));
    uint32_t incl = tmax;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = max(incl, y);
    }
    uint32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    for (int w = 0; w < warp; ++w) excl = max(excl, wsum[w]);
    uint32_t run = excl, out[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const uint32_t lo = run = max(run, w32[x] & 0xFFFFu);
        const uint32_t hi = run = max(run, w32[x] >> 16);
        out[x] = lo | (hi << 16);
    }
    m4[0] = make_uint4(out[0], out[1], out[2], out[3]);
    m4[1] = make_uint4(out[4], out[5], out[6], out[7]);
    __syncthreads();
}

// Stable ranking of one chunk by digit (kRadix = out of range) and the
// per-digit bookkeeping shared by both scatters.  On return: rank[q] = the
// item's position among the items of its digit in its warp; sm.local,
// sm.warp_cnt (exclusive prefix over warps) and sm.dst are set and sm.run
// advanced past the chunk.
template <class Shared>
__device__ __forceinline__ void rank_chunk(Shared& sm, const uint32_t (&dig)[kSortItems],
                                           uint32_t (&rank)[kSortItems]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        const uint32_t d = dig[q];
        // The lanes with the same digit (0..kRadix): one ballot per bit of the
        // 9-bit value, every bit agreeing (match_any's result, without its
        // cost growing with the number of distinct digits).
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b <= kRadixBits; ++b) {
            const uint32_t ones = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? ones : ~ones;
        }
        const uint32_t before = sm.warp_cnt[warp][d];
        rank[q] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (lane == 31 - __clz(peers)) sm.warp_cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // Per digit (thread = digit): prefix over warps and this chunk's count.
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = sm.warp_cnt[w][tid];
        sm.warp_cnt[w][tid] = cnt;
        cnt += c;
    }
    uint32_t total;
    const uint32_t loc = block_exclusive_scan(cnt, sm.wsum, total);
    sm.local[tid] = loc;
    if (tid == kSortThreads - 1) sm.local[kRadix] = loc + cnt;
    const uint32_t r = sm.run[tid];
    sm.dst[tid] = r - loc;
    sm.run[tid] = r + cnt;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Pass 1: column runs grouped by tx.
// ---------------------------------------------------------------------------

// Depth-order positions [i0, i1] of the Gaussians holding runs of chunks
// [c0, c1); false (and kErrRange) if the scan output is inconsistent.
__device__ __forceinline__ bool gauss_span(const PairSource& src, const Span& sp, uint32_t c0,
                                           uint32_t c1, uint32_t* status, uint32_t& i0,
                                           uint32_t& i1) {
    const uint32_t visible = src.counters[kCntVisible];
    i0 = src.chunk_first[c0];
    i1 = c1 < sp.nchunks ? src.chunk_first[c1] : visible - 1u;
    if (visible == 0 || i0 >= visible || i1 < i0 || i1 >= visible) {
        if (threadIdx.x == 0) atomicOr(status, kErrRange);
        return false;
    }
    return true;
}

// Counts of tx over the column runs of this CTA's chunks.  Gaussian i owns
// runs offsets[i] .. offsets[i] + w - 1 for columns x0 .. x0 + w - 1; the part
// inside the CTA's range is one tx interval, added to a difference array.
__global__ void __launch_bounds__(kSortThreads)
k_count_columns(PairSource src, int grid, uint32_t* __restrict__ counts, uint32_t* __restrict__ totals,
                uint32_t* __restrict__ status) {
    pdl_prologue();
    __shared__ int s_diff[kRadix + 1];
    __shared__ uint32_t s_wsum[kWarps];
    const int tid = threadIdx.x;
    for (int d = tid; d <= kRadix; d += kSortThreads) s_diff[d] = 0;
    __syncthreads();
    const Span sp = cta_span(run_count(src.counters, src.capacity), grid);
    uint32_t i0, i1;
    if (sp.c0 < sp.c1 && gauss_span(src, sp, sp.c0, sp.c1, status, i0, i1)) {
        const int64_t A = (int64_t)sp.c0 * kSortChunk;
        const int64_t B = min((int64_t)sp.c1 * kSortChunk, sp.n);
        for (uint32_t i = i0 + tid; i <= i1; i += kSortThreads) {
            const int64_t off = src.offsets[i];
            const uint32_t box = src.sorted_box[i];
            const int w = (int)((box >> 16) & 0xFFu) + 1;
            const int x0 = (int)(box & 0xFFu);
            const int64_t k0 = max(A - off, (int64_t)0), k1 = min(B - off, (int64_t)w);
            if (k0 >= k1) continue;
            if (x0 + w > kRadix) { atomicOr(status, kErrRange); continue; }   // not a scan box
            atomicAdd(&s_diff[x0 + k0], 1);
            atomicAdd(&s_diff[x0 + k1], -1);
        }
    }
    __syncthreads();
    // Inclusive prefix of the difference array = the count of each tx.
    uint32_t total;
    const int v = s_diff[tid];
    const uint32_t c = block_exclusive_scan((uint32_t)v, s_wsum, total) + (uint32_t)v;
    counts[(size_t)tid * grid + blockIdx.x] = c;
    if (c) atomicAdd(totals + tid, c);
}

// Generate the column runs of chunk `chunk` (items base .. base+count-1 of
// the depth-ordered emission) into key (run record y) / val (Gaussian id) in
// warp-striped order.
__device__ __forceinline__ void generate_runs(const PairSource& src, const Span& sp,
                                              ColumnShared& sm, uint32_t chunk, int64_t base,
                                              int count, uint32_t* status,
                                              uint32_t (&key)[kSortItems],
                                              uint32_t (&val)[kSortItems]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t visible = src.counters[kCntVisible];
    uint32_t i0 = src.chunk_first[chunk];
    // Gaussians [i0, i1] hold this chunk's runs; the one holding the next
    // chunk's first run closes the range (the last chunk: at most 4097 on).
    uint32_t i1 = chunk + 1 < sp.nchunks ? src.chunk_first[chunk + 1]
                                         : min(visible - 1u, i0 + (uint32_t)kMaxChunkGauss - 1u);
    if (visible == 0 || i0 >= visible || i1 < i0 || i1 >= visible ||
        i1 - i0 + 1 > (uint32_t)kMaxChunkGauss) {
        if (tid == 0) atomicOr(status, kErrRange);   // inconsistent scan output: stay in bounds
        i0 = visible == 0 ? 0u : min(i0, visible - 1u);
        i1 = visible == 0 ? i0 : min(visible - 1u, i0 + (uint32_t)kMaxChunkGauss - 1u);
    }
    const int G = (int)(i1 - i0 + 1);
    uint32_t* map32 = reinterpret_cast<uint32_t*>(sm.u.stage.map);
    for (int x = tid; x < kSortChunk / 2; x += kSortThreads) map32[x] = 0u;
    for (int j = tid; j < G; j += kSortThreads) {   // coalesced staging
        const uint32_t i = i0 + j;
        sm.u.stage.off[j] = src.offsets[i];
        sm.u.stage.gid[j] = src.order[i];
        sm.u.stage.box[j] = src.sorted_box[i];
    }
    __syncthreads();
    // Mark the slot where each staged Gaussian's first run falls (slot 0
    // belongs to staged Gaussian 0, the holder of the chunk's first run).
    for (int j = tid; j < G; j += kSortThreads) {
        const int64_t slot = (int64_t)sm.u.stage.off[j] - base;
        if (slot > 0 && slot < count) sm.u.stage.map[slot] = (uint16_t)j;
    }
    __syncthreads();
    map_running_max(sm.u.stage.map, sm.wsum);
    const int wfirst = warp * (kSortItems * 32);
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        const int s = wfirst + q * 32 + lane;
        if (s < count) {
            const int jj = sm.u.stage.map[s];
            const uint32_t box = sm.u.stage.box[jj];
            const uint32_t k = (uint32_t)(base + s) - sm.u.stage.off[jj];   // column offset
            const uint32_t tx = (box & 0xFFu) + k;
            key[q] = ((box >> 8) & 0xFFu) | ((box >> 24) << 8) | (tx << 16);
            val[q] = sm.u.stage.gid[jj];
        } else {
            key[q] = 0u;
            val[q] = 0u;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads, 3)
k_scatter_columns(PairSource src, const uint32_t* __restrict__ starts, uint2* __restrict__ runs_out,
                  uint16_t* __restrict__ rows_out,
                  int grid, uint32_t* __restrict__ status) {
    pdl_prologue();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColumnShared& sm = *reinterpret_cast<ColumnShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Span sp = cta_span(run_count(src.counters, src.capacity), grid);
    if (sp.c0 >= sp.c1) return;
    const int64_t n = sp.n;
    sm.run[tid] = starts[(size_t)tid * grid + blockIdx.x];
    for (uint32_t chunk = sp.c0; chunk < sp.c1; ++chunk) {
        for (int d = lane; d <= kRadix; d += 32) sm.warp_cnt[warp][d] = 0;
        const int64_t base = (int64_t)chunk * kSortChunk;
        const int count = (int)min((int64_t)kSortChunk, n - base);
        uint32_t key[kSortItems], val[kSortItems], dig[kSortItems], rank[kSortItems];
        generate_runs(src, sp, sm, chunk, base, count, status, key, val);
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            dig[q] = s < count ? min(run_tx(key[q]), (uint32_t)kRadix - 1u) : (uint32_t)kRadix;
        }
        __syncthreads();   // staging no longer read
        rank_chunk(sm, dig, rank);
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            if (dig[q] < (uint32_t)kRadix) {
                const uint32_t d = dig[q];
                const uint32_t pos = sm.local[d] + sm.warp_cnt[warp][d] + rank[q];
                sm.u.kv.keys[pos] = key[q];
                sm.u.kv.vals[pos] = val[q];
            }
        }
        __syncthreads();
        // Coalesced write-out: each digit's run goes to consecutive addresses.
        for (int s = tid; s < count; s += kSortThreads) {
            const uint32_t k = sm.u.kv.keys[s];
            const uint32_t g = sm.dst[min(run_tx(k), (uint32_t)kRadix - 1u)] + (uint32_t)s;
            if ((int64_t)g < n) {
                runs_out[g] = make_uint2(sm.u.kv.vals[s], k);
                rows_out[g] = (uint16_t)(k & 0xFFFFu);   // y0 | (h - 1) << 8, what Render filters on
            }
            else atomicOr(status, kErrRange);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Pass 2: pairs grouped by ty.
// ---------------------------------------------------------------------------

// Counts of ty over the pairs of this CTA's runs (each run adds its row
// interval to a difference array), and the pairs of every tile: runs of
// column tx covering row ty.  Runs arrive grouped by tx, so the CTA's first
// kColSlots columns are counted on chip; runs beyond them (only in columns
// with few runs) add to tile_counts directly.
__global__ void __launch_bounds__(kSortThreads)
k_count_rows(const uint2* __restrict__ runs, const uint32_t* __restrict__ counters, int64_t capacity,
             int grid, int tiles_x, int num_tiles, uint32_t* __restrict__ counts,
             uint32_t* __restrict__ totals, uint32_t* __restrict__ tile_counts,
             uint32_t* __restrict__ status) {
    pdl_prologue();
    __shared__ int s_diff[kRadix + 1];
    __shared__ int s_col[kColSlots][kRadix + 1];
    __shared__ uint32_t s_wsum[kWarps];
    const int tid = threadIdx.x;
    for (int d = tid; d <= kRadix; d += kSortThreads) s_diff[d] = 0;
    for (int d = tid; d < kColSlots * (kRadix + 1); d += kSortThreads) (&s_col[0][0])[d] = 0;
    __syncthreads();
    const Span sp = cta_span(run_count(counters, capacity), grid);
    uint32_t tx0 = 0;
    if (sp.c0 < sp.c1) {
        const int64_t A = (int64_t)sp.c0 * kSortChunk;
        const int64_t B = min((int64_t)sp.c1 * kSortChunk, sp.n);
        tx0 = run_tx(runs[A].y);
        for (int64_t i = A + tid; i < B; i += kSortThreads) {
            const uint32_t y = runs[i].y;
            const uint32_t y0 = run_y0(y), h = run_h(y), tx = run_tx(y);
            if (y0 + h > (uint32_t)kRadix || tx >= (uint32_t)tiles_x) {   // not a pass-1 record
                atomicOr(status, kErrRange);
                continue;
            }
            atomicAdd(&s_diff[y0], 1);
            atomicAdd(&s_diff[y0 + h], -1);
            const uint32_t c = tx - tx0;
            if (c < (uint32_t)kColSlots) {
                atomicAdd(&s_col[c][y0], 1);
                atomicAdd(&s_col[c][y0 + h], -1);
            } else {
                for (uint32_t ty = y0; ty < y0 + h; ++ty) {
                    const uint32_t t = ty * (uint32_t)tiles_x + tx;
                    if (t < (uint32_t)num_tiles) atomicAdd(tile_counts + t, 1u);
                    else atomicOr(status, kErrRange);
                }
            }
        }
    }
    __syncthreads();
    uint32_t total;
    const int v = s_diff[tid];
    const uint32_t c = block_exclusive_scan((uint32_t)v, s_wsum, total) + (uint32_t)v;
    counts[(size_t)tid * grid + blockIdx.x] = c;
    if (c) atomicAdd(totals + tid, c);
    // Tile counts of the on-chip columns: prefix over rows, one warp per column.
    if (sp.c0 < sp.c1) {
        const int lane = tid & 31, warp = tid >> 5;
        const uint32_t tx = tx0 + (uint32_t)warp;
        if (warp < kColSlots && tx < (uint32_t)tiles_x) {
            int run = 0;
            for (int ty0 = 0; ty0 < kRadix; ty0 += 32) {
                int x = s_col[warp][ty0 + lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const int cnt = run + x;
                const uint32_t t = (uint32_t)(ty0 + lane) * (uint32_t)tiles_x + tx;
                if (cnt > 0 && t < (uint32_t)num_tiles) atomicAdd(tile_counts + t, (uint32_t)cnt);
                run += __shfl_sync(0xffffffffu, x, 31);
            }
        }
    }
}

// Tile ranges: exclusive scan of the tile pair counts in tile order.  One CTA.
constexpr int kRangeThreads = 1024;
__global__ void __launch_bounds__(kRangeThreads)
k_tile_ranges(const uint32_t* __restrict__ tile_counts, int num_tiles,
              const uint32_t* __restrict__ counters, int64_t capacity, uint2* __restrict__ ranges) {
    pdl_prologue();
    __shared__ uint32_t s_w[kRangeThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool overflow = (int64_t)counters[kCntPairs] > capacity;
    const int per = (num_tiles + kRangeThreads - 1) / kRangeThreads;
    const int t0 = tid * per, t1 = min(t0 + per, num_tiles);
    uint32_t sum = 0;
    for (int t = t0; t < t1; ++t) sum += overflow ? 0u : tile_counts[t];
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t run = x - sum;
    for (int w = 0; w < warp; ++w) run += s_w[w];
    for (int t = t0; t < t1; ++t) {
        const uint32_t c = overflow ? 0u : tile_counts[t];
        ranges[t] = make_uint2(run, run + c);
        run += c;
    }
}

// Expand the runs of this CTA's chunks into pairs and scatter their Gaussian
// ids by tile row.  The runs are staged kRunStage at a time and listed per
// band of rows (the tile rows split into kBands bands; a run is listed in
// every band it meets, in run order).  The warps then take the bands one by
// one and sweep each band's list 32 runs at a time: for every row ty of the band,
// the lanes whose run covers ty (ballot) write their Gaussians to consecutive
// positions of the row, in run order.  Each row's output is thus written front
// to back with coalesced stores, and no pair is staged on chip.
__global__ void __launch_bounds__(kSortThreads, 8)   // 8 CTAs per SM: 32 registers, 22 KB shared
k_scatter_rows(const uint2* __restrict__ runs, const uint32_t* __restrict__ counters,
               int64_t capacity, const uint32_t* __restrict__ starts, uint32_t* __restrict__ gauss_out,
               int grid, int tiles_y, uint32_t* __restrict__ status) {
    pdl_prologue();
    __shared__ RowShared sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Span sp = cta_span(run_count(counters, capacity), grid);
    if (sp.c0 >= sp.c1) return;
    const int64_t n_pairs = min((int64_t)counters[kCntPairs], capacity);
    sm.pos[tid] = starts[(size_t)tid * grid + blockIdx.x];
    const int64_t B = min((int64_t)sp.c1 * kSortChunk, sp.n);
    const uint32_t lt = lanemask_lt();
    const int band_h = (tiles_y + kBands - 1) / kBands;   // rows per band
    for (int64_t r = (int64_t)sp.c0 * kSortChunk; r < B; r += kRunStage) {
        const int avail = (int)min((int64_t)kRunStage, B - r);
        __syncthreads();   // the previous staging is no longer read
        for (int j = tid; j < kRunStage; j += kSortThreads) {
            uint32_t rows = 0u, gid = 0u;   // rows [0, 0): covers nothing
            if (j < avail) {
                const uint2 rec = runs[r + j];
                rows = run_y0(rec.y) | ((run_y0(rec.y) + run_h(rec.y)) << 16);
                gid = rec.x;
            }
            sm.rows[j] = rows;
            sm.gid[j] = gid;
        }
        __syncthreads();
        // Warp w lists, in run order, the staged runs meeting band w of the rows.
        const int nblk = (avail + 31) >> 5;
        for (int k = warp; k < kBands; k += kWarps) {
            const uint32_t b0 = (uint32_t)(k * band_h), b1 = min(b0 + (uint32_t)band_h, (uint32_t)tiles_y);
            uint32_t n = 0;
            for (int blk = 0; blk < nblk; ++blk) {
                const int j = blk * 32 + lane;
                const uint32_t rows = sm.rows[j];
                const bool meets = (rows & 0xFFFFu) < b1 && (rows >> 16) > b0;
                const uint32_t m = __ballot_sync(0xffffffffu, meets);
                if (meets) sm.band[k][n + __popc(m & lt)] = (uint16_t)j;
                n += __popc(m);
            }
            if (lane == 0) sm.band_len[k] = n;
        }
        if (tid == 0) sm.next_band = 0u;
        __syncthreads();
        // The warps take bands dynamically (their lists differ in length):
        // each batch of 32 listed runs is tested against every row of the band.
        for (int k = 0;;) {
            if (lane == 0) k = (int)atomicAdd(&sm.next_band, 1u);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= kBands) break;
            const int y0b = k * band_h, nr = min(band_h, tiles_y - y0b);
            if (nr <= 0) continue;
            const uint32_t len = sm.band_len[k];
            const uint16_t* list = sm.band[k];
            uint32_t p[kMaxBandRows];
#pragma unroll
            for (int q = 0; q < kMaxBandRows; ++q) p[q] = q < nr ? sm.pos[y0b + q] : 0u;
            for (uint32_t i0 = 0; i0 < len; i0 += 32) {
                const uint32_t i = i0 + (uint32_t)lane;
                const uint32_t j = i < len ? list[i] : 0u;
                const uint32_t rows = i < len ? sm.rows[j] : 0u;   // rows [0, 0): covers nothing
                const uint32_t gid = sm.gid[j];
#pragma unroll
                for (int q = 0; q < kMaxBandRows; ++q) {
                    if (q >= nr) break;
                    const uint32_t ty = (uint32_t)(y0b + q);
                    const bool cover = (rows & 0xFFFFu) <= ty && ty < (rows >> 16);
                    const uint32_t m = __ballot_sync(0xffffffffu, cover);
                    if (cover) {
                        const uint32_t g = p[q] + __popc(m & lt);
                        if ((int64_t)g < n_pairs) gauss_out[g] = gid;
                        else atomicOr(status, kErrRange);
                    }
                    p[q] += __popc(m);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < kMaxBandRows; ++q)
                    if (q < nr) sm.pos[y0b + q] = p[q];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Global start of every (digit, CTA) run: counts [256][grid] in place.
// CTA d: start of digit d = sum of the totals of the digits below it, then an
// exclusive scan of its grid counts.
// ---------------------------------------------------------------------------
constexpr int kScanCtaThreads = 512;
constexpr int kScanPerThread = kMaxTileGrid / kScanCtaThreads;
static_assert(kScanPerThread * kScanCtaThreads == kMaxTileGrid, "scan covers the largest grid");

__global__ void __launch_bounds__(kScanCtaThreads)
k_count_scan(uint32_t* __restrict__ counts, const uint32_t* __restrict__ totals, int grid) {
    pdl_prologue();
    __shared__ uint32_t s_w[kScanCtaThreads / 32];
    __shared__ uint32_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int d = blockIdx.x;
    if (warp == 0) {
        uint32_t b = 0;
        for (int e = lane; e < d; e += 32) b += totals[e];
        b = __reduce_add_sync(0xffffffffu, b);
        if (lane == 0) s_base = b;
    }
    uint32_t* row = counts + (size_t)d * grid;
    uint32_t v[kScanPerThread], t = 0;
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u) {
        const int b = tid * kScanPerThread + u;
        v[u] = b < grid ? row[b] : 0u;
        t += v[u];
    }
    uint32_t x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t run = s_base + x - t;
    for (int w = 0; w < warp; ++w) run += s_w[w];
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u) {
        const int b = tid * kScanPerThread + u;
        if (b < grid) row[b] = run;
        run += v[u];
    }
}

}  // namespace

int tile_scatter_blocks_per_sm() {
    cudaFuncSetAttribute(k_scatter_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColumnSmem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scatter_columns, kSortThreads,
                                                      kColumnSmem) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_tile_count_columns(const PairSource& src, uint32_t* counts, uint32_t* totals,
                               uint32_t* status, int grid, cudaStream_t stream) {
    launch_pdl(k_count_columns, grid, kSortThreads, 0, stream, src, grid, counts, totals, status);
}

void launch_tile_scatter_columns(const PairSource& src, const uint32_t* starts, uint2* runs_out,
                                 uint16_t* rows_out, uint32_t* status, int grid, cudaStream_t stream) {
    launch_pdl(k_scatter_columns, grid, kSortThreads, kColumnSmem, stream, src, starts, runs_out, rows_out, grid,
                                                                  status);
}

void launch_tile_count_rows(const uint2* runs, const uint32_t* counters, int64_t capacity,
                            int tiles_x, int num_tiles, uint32_t* counts, uint32_t* totals,
                            uint32_t* tile_counts, uint32_t* status, int grid, cudaStream_t stream) {
    launch_pdl(k_count_rows, grid, kSortThreads, 0, stream, runs, counters, capacity, grid, tiles_x, num_tiles,
                                                    counts, totals, tile_counts, status);
}

void launch_tile_ranges(const uint32_t* tile_counts, int num_tiles, const uint32_t* counters,
                        int64_t capacity, uint2* ranges, cudaStream_t stream) {
    if (num_tiles <= 0) return;
    launch_pdl(k_tile_ranges, 1, kRangeThreads, 0, stream, tile_counts, num_tiles, counters, capacity, ranges);
}

void launch_tile_scatter_rows(const uint2* runs, const uint32_t* counters, int64_t capacity,
                              const uint32_t* starts, uint32_t* gauss_out, uint32_t* status,
                              int grid, int tiles_y, cudaStream_t stream) {
    launch_pdl(k_scatter_rows, grid, kSortThreads, 0, stream, runs, counters, capacity, starts, gauss_out,
                                                      grid, tiles_y, status);
}

void launch_tile_count_scan(uint32_t* counts, const uint32_t* totals, int grid, cudaStream_t stream) {
    launch_pdl(k_count_scan, kRadix, kScanCtaThreads, 0, stream, counts, totals, grid);
}

}  // namespace adr
