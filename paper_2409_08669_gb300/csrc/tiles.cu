// Stages 3-5 of the rasterization pipeline (Sec. 3.2.1): DuplicateWithKeys,
// SortPairs by tile and IdentifyTileRanges, as two stable counting-sort
// passes over the Gaussian-tile pairs, first by the tile column tx, then by
// the tile row ty.  The pairs of each Gaussian are listed in depth order
// (the Gaussians were sorted by view depth before), so the result is ordered
// by (tile, depth), as the paper's 64-bit (tile | depth) key orders them.
//
// Each pass is range-partitioned (reduce, scan, scatter): CTA b of a grid of
// G owns a contiguous run of 4096-pair chunks,
//   1. counts its pairs per digit (pass 1 straight from the Gaussians'
//      tile rectangles, without generating the pairs; pass 2 from the keys),
//   2. one CTA turns the G x 256 counts into the global start of every
//      (digit, CTA) run,
//   3. CTA b walks its chunks in order, ranks each chunk's keys stably
//      (warp match_any), groups them by digit in shared memory and writes
//      every digit's run contiguously from its running offset.
// No CTA ever waits for another one, so the passes need no co-residency and
// no spin-waits.  Pass 1 generates the pairs on chip from the depth-ordered
// Gaussians (the unsorted pair list never exists in memory) and writes a
// 16-bit key (ty << 8 | tx) and the Gaussian id; pass 2 writes only the
// Gaussian ids and each tile's [start, end) (atomicMin / atomicMax per run of
// equal keys).
#include <cstddef>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kMaxChunkGauss = kSortChunk + 1;          // every listed Gaussian has >= 1 pair
constexpr int kStageLen = (kMaxChunkGauss + 3) & ~3;    // keeps the arrays after it 16-byte aligned

struct alignas(16) TileShared {
    union {
        struct {
            uint32_t keys[kSortChunk];
            uint32_t vals[kSortChunk];
        } kv;
        struct {                      // Gaussians overlapping one pair chunk
            uint32_t off[kStageLen];
            uint32_t gid[kStageLen];
            uint32_t box[kStageLen];        // x0 | y0 << 8 | (w-1) << 16 | (h-1) << 24
            alignas(16) uint16_t map[kSortChunk];   // chunk slot -> staged Gaussian holding it
        } stage;
    } u;
    uint32_t warp_cnt[kWarps][kRadix + 1];   // +1: out-of-range items of the tail chunk
    uint32_t run[kRadix];                    // next global position of each digit
    uint32_t local[kRadix + 1];              // exclusive prefix of this chunk's digit counts
    uint32_t dst[kRadix];                    // global position of local slot 0, per digit
    uint32_t wsum[kWarps];
};
constexpr size_t kTileSmem = sizeof(TileShared);
static_assert(offsetof(TileShared, u) % 16 == 0, "staging must be 16-byte aligned");
static_assert((3 * kStageLen * sizeof(uint32_t)) % 16 == 0, "map must be 16-byte aligned");

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The chunks [c0, c1) of CTA b and the pair count n of the frame.
struct Span {
    int64_t n;
    uint32_t nchunks, c0, c1;
};
__device__ __forceinline__ Span cta_span(const uint32_t* counters, int64_t capacity, int grid) {
    Span s;
    s.n = min((int64_t)counters[kCntPairs], capacity);
    s.nchunks = (uint32_t)((s.n + kSortChunk - 1) / kSortChunk);
    const uint32_t per = (s.nchunks + (uint32_t)grid - 1u) / (uint32_t)grid;
    s.c0 = min(s.nchunks, per * blockIdx.x);
    s.c1 = min(s.nchunks, s.c0 + per);
    return s;
}

// Depth-order positions [i0, i1] of the Gaussians holding pairs of chunks
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

// ---------------------------------------------------------------------------
// 1. Per-CTA digit counts.
// ---------------------------------------------------------------------------

// Pass 1: counts of tx over the pairs of this CTA's chunks, from the packed
// rectangles.  A Gaussian's pairs k = 0 .. w*h-1 run over its rectangle row
// by row (ty = y0 + k / w, tx = x0 + k % w); the part of them inside the
// CTA's pair range is a partial row, whole rows and a partial row, each a
// contiguous tx interval, added to a difference array.
__global__ void __launch_bounds__(kSortThreads)
k_count_columns(PairSource src, int grid, uint32_t* __restrict__ counts, uint32_t* __restrict__ status) {
    __shared__ int s_diff[kRadix + 1];
    __shared__ uint32_t s_wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = tid; d <= kRadix; d += kSortThreads) s_diff[d] = 0;
    __syncthreads();
    const Span sp = cta_span(src.counters, src.capacity, grid);
    uint32_t i0, i1;
    if (sp.c0 < sp.c1 && gauss_span(src, sp, sp.c0, sp.c1, status, i0, i1)) {
        const int64_t A = (int64_t)sp.c0 * kSortChunk;
        const int64_t B = min((int64_t)sp.c1 * kSortChunk, sp.n);
        for (uint32_t i = i0 + tid; i <= i1; i += kSortThreads) {
            const int64_t off = src.offsets[i];
            const uint32_t box = src.sorted_box[i];
            const int w = (int)((box >> 16) & 0xFFu) + 1, h = (int)(box >> 24) + 1;
            const int x0 = (int)(box & 0xFFu);
            const int64_t k0 = max(A - off, (int64_t)0), k1 = min(B - off, (int64_t)w * h);
            if (k0 >= k1) continue;
            if (x0 + w > kRadix) { atomicOr(status, kErrRange); continue; }   // not a scan box
            const int r0 = (int)(k0 / w), q0 = (int)(k0 - (int64_t)r0 * w);
            const int r1 = (int)((k1 - 1) / w), q1 = (int)(k1 - 1 - (int64_t)r1 * w);
            auto add = [&](int lo, int hi, int v) {
                atomicAdd(&s_diff[lo], v);
                atomicAdd(&s_diff[hi + 1], -v);
            };
            if (r0 == r1) {
                add(x0 + q0, x0 + q1, 1);
            } else {
                add(x0 + q0, x0 + w - 1, 1);
                if (r1 - r0 > 1) add(x0, x0 + w - 1, r1 - r0 - 1);
                add(x0, x0 + q1, 1);
            }
        }
    }
    __syncthreads();
    // Inclusive prefix of the difference array = the count of each tx.
    const int v = s_diff[tid];
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = (uint32_t)x;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += (int)s_wsum[w];
    counts[(size_t)tid * grid + blockIdx.x] = (uint32_t)(wbase + x);
}

// Pass 2: counts of ty (key >> 8) over this CTA's chunks of pass-1 keys.
__global__ void __launch_bounds__(kSortThreads)
k_count_rows(const uint16_t* __restrict__ keys, const uint32_t* __restrict__ counters,
             int64_t capacity, int grid, uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_cnt[kRadix];
    const int tid = threadIdx.x;
    s_cnt[tid] = 0;
    __syncthreads();
    const Span sp = cta_span(counters, capacity, grid);
    if (sp.c0 < sp.c1) {
        const int64_t A = (int64_t)sp.c0 * kSortChunk;
        const int64_t B = min((int64_t)sp.c1 * kSortChunk, sp.n);   // > A
        // A is a multiple of 4096 keys; read 8 keys per 16-byte load up to the
        // last whole group, then the tail one by one.
        const int64_t Bv = A + ((B - A) & ~(int64_t)7);
        const uint4* k4 = reinterpret_cast<const uint4*>(keys + A);
        for (int64_t j = tid; A + 8 * j < Bv; j += kSortThreads) {
            const uint4 q = k4[j];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                atomicAdd(&s_cnt[(w[u] >> 8) & 0xFFu], 1u);
                atomicAdd(&s_cnt[w[u] >> 24], 1u);
            }
        }
        for (int64_t i = Bv + tid; i < B; i += kSortThreads) atomicAdd(&s_cnt[keys[i] >> 8], 1u);
    }
    __syncthreads();
    counts[(size_t)tid * grid + blockIdx.x] = s_cnt[tid];
}

// ---------------------------------------------------------------------------
// 2. Global start of every (digit, CTA) run: counts [256][grid] in place.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_count_scan(uint32_t* __restrict__ counts, int grid) {
    __shared__ uint32_t s_tot[kRadix], s_base[kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = warp; d < kRadix; d += 32) {
        uint32_t s = 0;
        for (int b = lane; b < grid; b += 32) s += counts[(size_t)d * grid + b];
        s = __reduce_add_sync(0xffffffffu, s);
        if (lane == 0) s_tot[d] = s;
    }
    __syncthreads();
    if (warp == 0) {   // exclusive prefix over the 256 digits, 8 per lane
        uint32_t v[8], t = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) { v[u] = s_tot[lane * 8 + u]; t += v[u]; }
        uint32_t x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t run = x - t;
#pragma unroll
        for (int u = 0; u < 8; ++u) { s_base[lane * 8 + u] = run; run += v[u]; }
    }
    __syncthreads();
    for (int d = warp; d < kRadix; d += 32) {
        uint32_t run = s_base[d];
        for (int b0 = 0; b0 < grid; b0 += 32) {
            const int b = b0 + lane;
            const uint32_t v = b < grid ? counts[(size_t)d * grid + b] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (b < grid) counts[(size_t)d * grid + b] = run + x - v;
            run += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// ---------------------------------------------------------------------------
// 3. Scatter.
// ---------------------------------------------------------------------------

// Generate the pairs of chunk `chunk` (items base .. base+count-1 of the
// depth-ordered emission) into key/val in warp-striped order:
// key = ty << 8 | tx, val = Gaussian id.
__device__ __forceinline__ void generate_pairs(const PairSource& src, const Span& sp,
                                               TileShared& sm, uint32_t chunk, int64_t base,
                                               int count, uint32_t* status,
                                               uint32_t (&key)[kSortItems],
                                               uint32_t (&val)[kSortItems]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t visible = src.counters[kCntVisible];
    uint32_t i0 = src.chunk_first[chunk];
    // Gaussians [i0, i1] hold this chunk's pairs; the one holding the next
    // chunk's first pair closes the range (the last chunk: at most 4097 on).
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
    // Mark the slot where each staged Gaussian's first pair falls (slot 0
    // belongs to staged Gaussian 0, the holder of the chunk's first pair).
    for (int j = tid; j < G; j += kSortThreads) {
        const int64_t slot = (int64_t)sm.u.stage.off[j] - base;
        if (slot > 0 && slot < count) sm.u.stage.map[slot] = (uint16_t)j;
    }
    __syncthreads();
    // Running maximum over the slots: thread t owns slots 16t .. 16t+15, then
    // a block-wide exclusive max-scan of the thread maxima.
    {
        uint4* m4 = reinterpret_cast<uint4*>(sm.u.stage.map) + 2 * tid;
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
        if (lane == 31) sm.wsum[warp] = incl;
        __syncthreads();
        for (int w = 0; w < warp; ++w) excl = max(excl, sm.wsum[w]);
        uint32_t run = excl, out[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const uint32_t lo = run = max(run, w32[x] & 0xFFFFu);
            const uint32_t hi = run = max(run, w32[x] >> 16);
            out[x] = lo | (hi << 16);
        }
        m4[0] = make_uint4(out[0], out[1], out[2], out[3]);
        m4[1] = make_uint4(out[4], out[5], out[6], out[7]);
    }
    __syncthreads();
    // Warp w produces items w*512 + q*32 + lane, the warp-striped order the
    // ranking needs.  k / w is exact through a reciprocal biased up by 2^-20:
    // k < 2^16 and w <= 256 keep the product within (q, q + 1).
    const int wfirst = warp * (kSortItems * 32);
#pragma unroll
    for (int q = 0; q < kSortItems; ++q) {
        const int s = wfirst + q * 32 + lane;
        if (s < count) {
            const int jj = sm.u.stage.map[s];
            const uint32_t box = sm.u.stage.box[jj];
            const uint32_t w = ((box >> 16) & 0xFFu) + 1u;
            const uint32_t k = (uint32_t)(base + s) - sm.u.stage.off[jj];
            const float r = __frcp_rn((float)w) * 1.00000095367431640625f;   // (1 + 2^-20) / w
            const uint32_t dy = (uint32_t)((float)k * r);
            const uint32_t dx = k - dy * w;
            key[q] = ((((box >> 8) & 0xFFu) + dy) << 8) | ((box & 0xFFu) + dx);
            val[q] = sm.u.stage.gid[jj];
        } else {
            key[q] = 0xFFFFu;
            val[q] = 0u;
        }
    }
}

struct ScatterArgs {
    PairSource src;                  // pass 1: pairs generated from the Gaussians
    const uint16_t* keys_in;         // pass 2
    const uint32_t* vals_in;         // pass 2
    uint16_t* keys_out;              // pass 1
    uint32_t* vals_out;
    const uint32_t* starts;          // [256][grid] global start of each (digit, CTA) run
    uint2* ranges;                   // pass 2
    const uint32_t* counters;
    int64_t capacity;
    int grid;
    int tiles_x, num_tiles;
    uint32_t* status;
};

template <bool kFirst>
__global__ void __launch_bounds__(kSortThreads, 3) k_tile_scatter(ScatterArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileShared& sm = *reinterpret_cast<TileShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Span sp = cta_span(a.counters, a.capacity, a.grid);
    if (sp.c0 >= sp.c1) return;
    const int64_t n = sp.n;
    sm.run[tid] = a.starts[(size_t)tid * a.grid + blockIdx.x];
    // digit of a key: tx in pass 1, ty in pass 2
    auto digit = [](uint32_t k) { return kFirst ? (k & 0xFFu) : (k >> 8); };

    for (uint32_t chunk = sp.c0; chunk < sp.c1; ++chunk) {
        for (int d = lane; d <= kRadix; d += 32) sm.warp_cnt[warp][d] = 0;
        const int64_t base = (int64_t)chunk * kSortChunk;
        const int count = (int)min((int64_t)kSortChunk, n - base);
        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        if constexpr (kFirst) {
            generate_pairs(a.src, sp, sm, chunk, base, count, a.status, key, val);
        } else {
#pragma unroll
            for (int q = 0; q < kSortItems; ++q) {
                const int s = warp * (kSortItems * 32) + q * 32 + lane;
                const bool ok = s < count;
                key[q] = ok ? (uint32_t)a.keys_in[base + s] : 0xFFFFu;
                val[q] = ok ? a.vals_in[base + s] : 0u;
            }
        }
        __syncthreads();   // warp_cnt cleared; staging (pass 1) no longer read
        // Stable warp-level ranking with match_any (digit kRadix = out of range).
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            const uint32_t d = s < count ? digit(key[q]) : (uint32_t)kRadix;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
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
        uint32_t loc;
        {
            uint32_t x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) sm.wsum[warp] = x;
            __syncthreads();
            uint32_t wbase = 0;
            for (int w = 0; w < warp; ++w) wbase += sm.wsum[w];
            loc = wbase + x - cnt;
            sm.local[tid] = loc;
            if (tid == kSortThreads - 1) sm.local[kRadix] = loc + cnt;
        }
        const uint32_t r = sm.run[tid];
        sm.dst[tid] = r - loc;
        sm.run[tid] = r + cnt;
        __syncthreads();
        // Group by digit in shared memory.
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            if (s < count) {
                const uint32_t d = digit(key[q]);
                const uint32_t pos = sm.local[d] + sm.warp_cnt[warp][d] + rank[q];
                sm.u.kv.keys[pos] = key[q];
                sm.u.kv.vals[pos] = val[q];
            }
        }
        __syncthreads();
        // Coalesced write-out: each digit's run goes to consecutive addresses.
        for (int s = tid; s < count; s += kSortThreads) {
            const uint32_t k = sm.u.kv.keys[s];
            const uint32_t d = digit(k);
            const uint32_t g = sm.dst[d] + (uint32_t)s;   // exact modulo 2^32; true value < 2^30
            if ((int64_t)g >= n) { atomicOr(a.status, kErrRange); continue; }
            a.vals_out[g] = sm.u.kv.vals[s];
            if constexpr (kFirst) {
                a.keys_out[g] = (uint16_t)k;
            } else {
                // Within a digit's run the keys ascend, so each tile's pairs
                // form one segment; record its first and last global slot.
                const bool first = (s == (int)sm.local[d]) || sm.u.kv.keys[s - 1] != k;
                const bool lastp = (s + 1 == (int)sm.local[d + 1]) || sm.u.kv.keys[s + 1] != k;
                const uint32_t tile = (k >> 8) * (uint32_t)a.tiles_x + (k & 0xFFu);
                if ((k & 0xFFu) >= (uint32_t)a.tiles_x || tile >= (uint32_t)a.num_tiles) {
                    atomicOr(a.status, kErrRange);   // not a pass-1 key: skip
                    continue;
                }
                unsigned int* rr = reinterpret_cast<unsigned int*>(a.ranges + tile);
                if (first) atomicMin(rr, g);
                if (lastp) atomicMax(rr + 1, g + 1u);
            }
        }
        __syncthreads();
    }
}

}  // namespace

int tile_scatter_blocks_per_sm() {
    cudaFuncSetAttribute(k_tile_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    cudaFuncSetAttribute(k_tile_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tile_scatter<true>, kSortThreads,
                                                      kTileSmem) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_tile_count_columns(const PairSource& src, uint32_t* counts, uint32_t* status, int grid,
                               cudaStream_t stream) {
    k_count_columns<<<grid, kSortThreads, 0, stream>>>(src, grid, counts, status);
}

void launch_tile_count_rows(const uint16_t* keys, const uint32_t* counters, int64_t capacity,
                            uint32_t* counts, int grid, cudaStream_t stream) {
    k_count_rows<<<grid, kSortThreads, 0, stream>>>(keys, counters, capacity, grid, counts);
}

void launch_tile_count_scan(uint32_t* counts, int grid, cudaStream_t stream) {
    k_count_scan<<<1, 1024, 0, stream>>>(counts, grid);
}

void launch_tile_scatter_columns(const PairSource& src, const uint32_t* starts, uint16_t* keys_out,
                                 uint32_t* gauss_out, uint32_t* status, int grid,
                                 cudaStream_t stream) {
    ScatterArgs a{};
    a.src = src;
    a.keys_out = keys_out;
    a.vals_out = gauss_out;
    a.starts = starts;
    a.counters = src.counters;
    a.capacity = src.capacity;
    a.grid = grid;
    a.tiles_x = src.tiles_x;
    a.status = status;
    k_tile_scatter<true><<<grid, kSortThreads, kTileSmem, stream>>>(a);
}

void launch_tile_scatter_rows(const uint16_t* keys_in, const uint32_t* gauss_in,
                              const uint32_t* starts, uint32_t* gauss_out, uint2* ranges,
                              const uint32_t* counters, int64_t capacity, int tiles_x,
                              int num_tiles, uint32_t* status, int grid, cudaStream_t stream) {
    ScatterArgs a{};
    a.keys_in = keys_in;
    a.vals_in = gauss_in;
    a.vals_out = gauss_out;
    a.starts = starts;
    a.ranges = ranges;
    a.counters = counters;
    a.capacity = capacity;
    a.grid = grid;
    a.tiles_x = tiles_x;
    a.num_tiles = num_tiles;
    a.status = status;
    k_tile_scatter<false><<<grid, kSortThreads, kTileSmem, stream>>>(a);
}

}  // namespace adr
