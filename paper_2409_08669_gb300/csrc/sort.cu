// The view-depth sort of the Gaussians (the depth half of the paper's
// (tile | depth) sort key, Sec. 3.2.1) as stable least-significant-digit radix
// passes of 8 bits.  Each pass is range-partitioned (count, scan, scatter):
// CTA b of the grid owns a contiguous run of 4096-key chunks,
//   1. k_digit_counts counts its keys per digit,
//   2. the tile sort's count scan turns the 256 x grid counts into the global
//      start of every (digit, CTA) run,
//   3. k_digit_scatter walks its chunks in order: each chunk ranks its keys
//      stably (a warp ballot per digit bit), groups them by digit in shared memory and
//      writes every digit's run contiguously from the CTA's running offset.
// No CTA waits for another one, so a pass has no lookback chain.
// The first pass drops the Gaussians without tiles (key 0xFFFFFFFF, which
// would sort last anyway) and counts the others; the later passes sort only
// those, reading their number from device memory.
#include <cstddef>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kWarps = kSortThreads / 32;

struct alignas(16) SortShared {
    uint32_t keys[kSortChunk];
    uint32_t vals[kSortChunk];
    uint32_t warp_cnt[kWarps][kRadix + 1];   // +1: out-of-range items of the tail chunk
    uint32_t run[kRadix];                    // next global position of each digit
    uint32_t local[kRadix + 1];              // exclusive prefix of this chunk's digit counts
    uint32_t dst[kRadix];                    // global position of local slot 0, per digit
    uint32_t wsum[kWarps];
    uint32_t kept;                           // items of the chunk that are written
};
constexpr size_t kSortSmem = sizeof(SortShared);

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr uint32_t kNoTiles = 0xFFFFFFFFu;   // depth key of a Gaussian without tiles

// Items of a pass: the host count, or the device count of the kept keys.
__device__ __forceinline__ int64_t pass_items(int64_t n, const uint32_t* n_dev) {
    return n_dev ? min(n, (int64_t)*n_dev) : n;
}

// The chunks [c0, c1) of CTA blockIdx.x.
__device__ __forceinline__ void chunk_span(int64_t n, int grid, uint32_t& c0, uint32_t& c1) {
    const uint32_t nchunks = (uint32_t)((n + kSortChunk - 1) / kSortChunk);
    const uint32_t per = (nchunks + (uint32_t)grid - 1u) / (uint32_t)grid;
    c0 = min(nchunks, per * blockIdx.x);
    c1 = min(nchunks, c0 + per);
}

__global__ void __launch_bounds__(kSortThreads)
k_digit_counts(const uint32_t* __restrict__ keys, int64_t n_host, const uint32_t* __restrict__ n_dev,
               bool drop, int shift, int grid, uint32_t* __restrict__ counts,
               uint32_t* __restrict__ totals, uint32_t* __restrict__ kept_total) {
    pdl_prologue();
    __shared__ uint32_t s_cnt[kRadix + 1];   // + the dropped keys
    const int tid = threadIdx.x;
    const int64_t n = pass_items(n_host, n_dev);
    s_cnt[tid] = 0;
    if (tid == 0) s_cnt[kRadix] = 0;
    __syncthreads();
    uint32_t c0, c1;
    chunk_span(n, grid, c0, c1);
    if (c0 < c1) {
        const int64_t A = (int64_t)c0 * kSortChunk;
        const int64_t B = min((int64_t)c1 * kSortChunk, n);   // > A
        const int64_t Bv = A + ((B - A) & ~(int64_t)3);         // A is 16-byte aligned
        const uint4* k4 = reinterpret_cast<const uint4*>(keys + A);
        auto digit = [&](uint32_t k) { return (drop && k == kNoTiles) ? (uint32_t)kRadix : (k >> shift) & 0xFFu; };
        for (int64_t j = tid; A + 4 * j < Bv; j += kSortThreads) {
            const uint4 q = k4[j];
            atomicAdd(&s_cnt[digit(q.x)], 1u);
            atomicAdd(&s_cnt[digit(q.y)], 1u);
            atomicAdd(&s_cnt[digit(q.z)], 1u);
            atomicAdd(&s_cnt[digit(q.w)], 1u);
        }
        for (int64_t i = Bv + tid; i < B; i += kSortThreads) atomicAdd(&s_cnt[digit(keys[i])], 1u);
    }
    __syncthreads();
    const uint32_t c = s_cnt[tid];
    counts[(size_t)tid * grid + blockIdx.x] = c;
    if (c) atomicAdd(totals + tid, c);
    if (kept_total && c0 < c1) {   // the kept keys of this CTA: its range minus the dropped ones
        if (tid == 0) {
            const int64_t A = (int64_t)c0 * kSortChunk, B = min((int64_t)c1 * kSortChunk, n);
            atomicAdd(kept_total, (uint32_t)(B - A) - s_cnt[kRadix]);
        }
    }
}

__global__ void __launch_bounds__(kSortThreads, 3)
k_digit_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n_host,
                const uint32_t* __restrict__ n_dev, bool drop, int shift,
                const uint32_t* __restrict__ starts, int grid,
                const uint32_t* __restrict__ pay_in, uint32_t* __restrict__ pay_out,
                uint32_t* __restrict__ status) {
    pdl_prologue();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortShared& sm = *reinterpret_cast<SortShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = pass_items(n_host, n_dev);
    // Output positions are bounded by the kept keys (all of them if nothing is dropped).
    const int64_t n_out = drop ? n_host : n;
    uint32_t c0, c1;
    chunk_span(n, grid, c0, c1);
    if (c0 >= c1) return;
    sm.run[tid] = starts[(size_t)tid * grid + blockIdx.x];
    for (uint32_t chunk = c0; chunk < c1; ++chunk) {
        for (int d = lane; d <= kRadix; d += 32) sm.warp_cnt[warp][d] = 0;
        const int64_t base = (int64_t)chunk * kSortChunk;
        const int count = (int)min((int64_t)kSortChunk, n - base);
        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        // Warp-striped load: item q of lane l in warp w is base + w*512 + q*32 + l.
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            const bool ok = s < count;
            key[q] = ok ? keys_in[base + s] : 0xFFFFFFFFu;
            val[q] = ok ? (vals_in ? vals_in[base + s] : (uint32_t)(base + s)) : 0u;
        }
        __syncwarp();
        // Stable warp-level ranking.  The lanes holding the same digit
        // (peers) come from one ballot per digit bit: the in-range lanes
        // whose every bit agrees with this lane's.  A lane's rank is the
        // warp's running count of its digit plus its peers in lower lanes;
        // the highest peer advances the count.  (match_any gives the same
        // peers, but its cost grows with the number of distinct digits in
        // the warp, ~10x slower on the key's low bytes.)  Out-of-range or
        // dropped items take no rank.
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            const bool in = s < count && !(drop && key[q] == kNoTiles);
            const uint32_t d = (key[q] >> shift) & 0xFFu;
            uint32_t peers = __ballot_sync(0xffffffffu, in);
#pragma unroll
            for (int b = 0; b < kRadixBits; ++b) {
                const uint32_t ones = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? ones : ~ones;
            }
            const uint32_t before = in ? sm.warp_cnt[warp][d] : 0u;
            rank[q] = before + __popc(peers & lanemask_lt());
            __syncwarp();
            if (in && lane == 31 - __clz(peers)) sm.warp_cnt[warp][d] = before + __popc(peers);
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
            if (tid == kSortThreads - 1) sm.kept = wbase + x;   // all digits' items
        }
        const uint32_t r = sm.run[tid];
        sm.dst[tid] = r - loc;
        sm.run[tid] = r + cnt;
        __syncthreads();
        // Scatter into shared memory in digit order.
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            if (s < count && !(drop && key[q] == kNoTiles)) {
                const uint32_t d = (key[q] >> shift) & 0xFFu;
                const uint32_t pos = sm.local[d] + sm.warp_cnt[warp][d] + rank[q];
                sm.keys[pos] = key[q];
                sm.vals[pos] = val[q];
            }
        }
        __syncthreads();
        // Coalesced write-out: each digit's run goes to consecutive addresses.
        const int kept = (int)sm.kept;
        for (int s = tid; s < kept; s += kSortThreads) {
            const uint32_t k = sm.keys[s];
            const uint32_t g = sm.dst[(k >> shift) & 0xFFu] + (uint32_t)s;   // exact modulo 2^32
            if ((int64_t)g >= n_out) { atomicOr(status, kErrRange); continue; }
            const uint32_t v = sm.vals[s];
            keys_out[g] = k;
            vals_out[g] = v;
            if (pay_out) pay_out[g] = pay_in[v];   // the value's payload, in sorted order
        }
        __syncthreads();
    }
}

}  // namespace

int onesweep_blocks_per_sm() {
    // Opt the scatter into more than 48 KB of dynamic shared memory (per device).
    cudaFuncSetAttribute(k_digit_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_digit_scatter, kSortThreads, kSortSmem) !=
        cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_depth_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                       uint32_t* vals_out, int64_t n, uint32_t* kept, bool first, int shift,
                       uint32_t* counts, uint32_t* totals, const uint32_t* pay_in,
                       uint32_t* pay_out, uint32_t* status, int grid, cudaStream_t stream) {
    if (n <= 0) return;
    // First pass: all n keys in, the kept ones counted into *kept.  Later
    // passes: the *kept keys.
    const uint32_t* n_dev = first ? nullptr : kept;
    launch_pdl(k_digit_counts, grid, kSortThreads, 0, stream, keys_in, n, n_dev, first, shift, grid, counts,
                                                      totals, first ? kept : nullptr);
    launch_tile_count_scan(counts, totals, grid, stream);
    launch_pdl(k_digit_scatter, grid, kSortThreads, kSortSmem, stream, keys_in, vals_in, keys_out, vals_out, n,
                                                              n_dev, first, shift, counts, grid,
                                                              pay_in, pay_out, status);
}

}  // namespace adr
