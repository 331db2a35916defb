// Stage 4, SortPairs (Sec. 3.2.1), as stable least-significant-digit radix
// passes in the "onesweep" form: each chunk of 4096 items ranks its keys
// locally (warp match_any), obtains the running per-digit offsets of all
// earlier chunks by decoupled lookback, and scatters through shared memory so
// that each digit's run is written contiguously.
//
// Three uses:
//   * the Gaussians by view depth (4 passes of 8 bits over N keys in memory);
//   * the first tile pass: the (tile, Gaussian) pairs are generated on chip
//     from the depth-ordered Gaussians (a load-balanced search over the
//     scan offsets), so the unsorted pair list never exists in memory;
//   * the last tile pass: writes only the Gaussian ids and derives every
//     tile's [start, end) from its digit runs (atomicMin/atomicMax per run
//     segment), replacing a separate IdentifyTileRanges pass.
//
// Persistent grid: CTAs take chunk tickets in increasing order from an atomic
// counter, so any chunk a CTA waits on is already held by a running CTA.
// Every wait is bounded; on expiry the kernel raises kErrLookback and goes on
// with a wrong but in-bounds placement instead of hanging.
#include <cstddef>

#include "adr_internal.cuh"

namespace adr {
namespace {

// Lookback word: [63:32] epoch of the pass, [31:30] state (1 = aggregate of
// this chunk only, 2 = inclusive prefix), [29:0] count.  A word from another
// epoch reads as "not ready".
constexpr unsigned long long kStateAgg = 1ull << 30;
constexpr unsigned long long kStateInc = 2ull << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kSpinLimit = 1 << 22;
constexpr int kWarps = kSortThreads / 32;
constexpr int kMaxChunkGauss = kSortChunk + 1;   // every listed Gaussian has >= 1 pair
constexpr int kStageLen = (kMaxChunkGauss + 3) & ~3;   // keeps the arrays after it 16-byte aligned

struct alignas(16) SortShared {
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
    uint32_t gbase[kRadix];                  // exclusive prefix of the global digit histogram
    uint32_t local[kRadix + 1];              // exclusive prefix of this chunk's digit counts
    uint32_t dst[kRadix];                    // global position of local slot 0, per digit
    uint32_t wsum[kWarps];
    uint32_t chunk;
};
constexpr size_t kSortSmem = sizeof(SortShared);
static_assert(offsetof(SortShared, u) % 16 == 0, "staging must be 16-byte aligned");
static_assert((3 * kStageLen * sizeof(uint32_t)) % 16 == 0, "map must be 16-byte aligned");

struct SweepArgs {
    const uint32_t* keys_in;
    const uint32_t* vals_in;
    uint32_t* keys_out;
    uint32_t* vals_out;
    int64_t n_host;              // item count, or the capacity bound when counters != null
    const uint32_t* counters;    // tile passes: item count = min(counters[kCntPairs], n_host)
    int shift, digit_bits;
    const uint32_t* hist;        // 256 counts of this pass's digit
    unsigned long long* lookback;
    EpochRef epoch;
    uint32_t* ticket;
    uint32_t* status;
    uint2* ranges;               // last tile pass
    PairSource src;              // first tile pass
};

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(256)
k_digit_hist(const uint32_t* __restrict__ keys, int64_t n, int shift0, int passes,
             uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (shift0 + 8 * p)) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
        const uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(hist + i, v);
    }
}

// Generate the pairs of chunk `chunk` (items base .. base+count-1 of the
// depth-ordered emission) into key/val in warp-striped order.
__device__ __forceinline__ void generate_pairs(const SweepArgs& a, SortShared& sm, uint32_t chunk,
                                               int64_t base, int count, int64_t n,
                                               uint32_t (&key)[kSortItems],
                                               uint32_t (&val)[kSortItems]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PairSource& src = a.src;
    const uint32_t visible = src.counters[kCntVisible];
    const uint32_t i0 = src.chunk_first[chunk];
    // Gaussians [i0, i1] hold this chunk's pairs; the one holding the next
    // chunk's first pair closes the range.
    uint32_t i1 = (base + kSortChunk >= n) ? min(visible - 1u, i0 + (uint32_t)kMaxChunkGauss - 1u)
                                           : src.chunk_first[chunk + 1];
    if (visible == 0 || i1 < i0 || i1 >= visible || i1 - i0 + 1 > (uint32_t)kMaxChunkGauss) {
        if (tid == 0) atomicOr(a.status, kErrRange);   // inconsistent scan output: stay in bounds
        i1 = visible == 0 ? i0 : min(visible - 1u, i0 + (uint32_t)kMaxChunkGauss - 1u);
        if (i1 < i0) i1 = i0;
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
            key[q] = (((box >> 8) & 0xFFu) + dy) * (uint32_t)src.tiles_x + (box & 0xFFu) + dx;
            val[q] = sm.u.stage.gid[jj];
        } else {
            key[q] = 0xFFFFFFFFu;
            val[q] = 0u;
        }
    }
}

template <bool kGen, bool kFinal>
__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortShared& sm = *reinterpret_cast<SortShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t mask = (1u << a.digit_bits) - 1u;
    const int64_t n = a.counters ? min((int64_t)a.counters[kCntPairs], a.n_host) : a.n_host;
    const uint32_t epoch = (*a.epoch.stage) * 8u + a.epoch.pass;
    const unsigned long long tag = (unsigned long long)epoch << 32;

    // Exclusive prefix of the global histogram of this digit (one digit per thread).
    {
        const uint32_t h = a.hist[tid];
        uint32_t x = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm.wsum[warp] = x;
        __syncthreads();
        uint32_t wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += sm.wsum[w];
        sm.gbase[tid] = wbase + x - h;
    }

    for (;;) {
        if (tid == 0) sm.chunk = atomicAdd(a.ticket, 1u);
        for (int d = lane; d <= kRadix; d += 32) sm.warp_cnt[warp][d] = 0;
        __syncthreads();
        const uint32_t chunk = sm.chunk;
        const int64_t base = (int64_t)chunk * kSortChunk;
        if (base >= n) break;
        const int count = (int)min((int64_t)kSortChunk, n - base);

        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        if constexpr (kGen) {
            generate_pairs(a, sm, chunk, base, count, n, key, val);
        } else {
            // Warp-striped load: item q of lane l in warp w is base + w*512 + q*32 + l.
#pragma unroll
            for (int q = 0; q < kSortItems; ++q) {
                const int s = warp * (kSortItems * 32) + q * 32 + lane;
                const bool ok = s < count;
                key[q] = ok ? a.keys_in[base + s] : 0xFFFFFFFFu;
                val[q] = ok ? (a.vals_in ? a.vals_in[base + s] : (uint32_t)(base + s)) : 0u;
            }
        }
        // Stable warp-level ranking with match_any (digit kRadix = out of range).
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            const uint32_t d = s < count ? ((key[q] >> a.shift) & mask) : (uint32_t)kRadix;
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
        // Publish this chunk's per-digit count right away; the lookback waits
        // until the local placement is done, giving predecessors time to post
        // their inclusive prefixes.
        unsigned long long* my = a.lookback + (size_t)chunk * kRadix + tid;
        st_volatile(my, tag | (chunk == 0 ? kStateInc : kStateAgg) | cnt);
        // Exclusive prefix of this chunk's digit counts (local placement).
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
        __syncthreads();
        // Scatter into shared memory in digit order.
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            if (s < count) {
                const uint32_t d = (key[q] >> a.shift) & mask;
                const uint32_t pos = sm.local[d] + sm.warp_cnt[warp][d] + rank[q];
                sm.u.kv.keys[pos] = key[q];
                sm.u.kv.vals[pos] = val[q];
            }
        }
        // Decoupled lookback: sum the earlier chunks' counts of this digit,
        // reading 8 predecessors per round trip, until an inclusive prefix.
        uint32_t excl = 0;
        if (chunk > 0) {
            int64_t j = (int64_t)chunk - 1;
            int spins = 0;
            bool done = false;
            while (!done && j >= 0) {
                unsigned long long wv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    wv[u] = j - u >= 0 ? ld_volatile(a.lookback + (size_t)(j - u) * kRadix + tid) : 0ull;
                int used = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (done || used < u || j - u < 0) continue;
                    const unsigned long long w = wv[u];
                    if ((uint32_t)(w >> 32) != epoch || (w & (3ull << 30)) == 0) continue;
                    excl += (uint32_t)w & kCountMask;
                    used = u + 1;
                    if (w & kStateInc) done = true;
                }
                j -= used;
                if (!done && used < 8 && j >= 0) {   // the next word is not ready yet
                    if (++spins > kSpinLimit) { atomicOr(a.status, kErrLookback); break; }
                    __nanosleep(32);
                }
            }
            st_volatile(my, tag | kStateInc | ((excl + cnt) & kCountMask));
        }
        sm.dst[tid] = sm.gbase[tid] + excl - loc;
        __syncthreads();
        // Coalesced write-out: each digit's run goes to consecutive addresses.
        for (int s = tid; s < count; s += kSortThreads) {
            const uint32_t k = sm.u.kv.keys[s];
            const uint32_t d = (k >> a.shift) & mask;
            const uint32_t g = sm.dst[d] + (uint32_t)s;   // exact modulo 2^32; true value < 2^30
            if ((int64_t)g >= n) { atomicOr(a.status, kErrRange); continue; }
            a.vals_out[g] = sm.u.kv.vals[s];
            if constexpr (kFinal) {
                // Within a digit's run the keys ascend, so each tile's pairs
                // form one segment; record its first and last global slot.
                const bool first = (s == (int)sm.local[d]) || sm.u.kv.keys[s - 1] != k;
                const bool lastp = (s + 1 == (int)sm.local[d + 1]) || sm.u.kv.keys[s + 1] != k;
                unsigned int* r = reinterpret_cast<unsigned int*>(a.ranges + k);
                if (first) atomicMin(r, g);
                if (lastp) atomicMax(r + 1, g + 1u);
            } else {
                a.keys_out[g] = k;
            }
        }
        __syncthreads();
    }
}

template <bool kGen, bool kFinal>
void launch_sweep(const SweepArgs& a, int grid, cudaStream_t stream) {
    k_onesweep<kGen, kFinal><<<grid, kSortThreads, kSortSmem, stream>>>(a);
}

SweepArgs base_args(const uint32_t* hist, unsigned long long* lookback, EpochRef epoch,
                    uint32_t* ticket, uint32_t* status) {
    SweepArgs a{};
    a.hist = hist;
    a.lookback = lookback;
    a.epoch = epoch;
    a.ticket = ticket;
    a.status = status;
    return a;
}

}  // namespace

int onesweep_blocks_per_sm() {
    // Opt the kernels into more than 48 KB of dynamic shared memory (per device).
    cudaFuncSetAttribute(k_onesweep<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
    cudaFuncSetAttribute(k_onesweep<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
    cudaFuncSetAttribute(k_onesweep<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
    cudaFuncSetAttribute(k_onesweep<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_onesweep<true, false>, kSortThreads,
                                                      kSortSmem) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_digit_hist(const uint32_t* keys, int64_t n, int shift0, int passes, uint32_t* hist,
                       int grid, cudaStream_t stream) {
    if (n <= 0) return;
    k_digit_hist<<<grid, 256, 0, stream>>>(keys, n, shift0, passes, hist);
}

void launch_onesweep(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                     uint32_t* vals_out, int64_t n, int shift, int digit_bits,
                     const uint32_t* hist, unsigned long long* lookback, EpochRef epoch,
                     uint32_t* ticket, uint32_t* status, int grid, cudaStream_t stream) {
    if (n <= 0) return;
    SweepArgs a = base_args(hist, lookback, epoch, ticket, status);
    a.keys_in = keys_in;
    a.vals_in = vals_in;
    a.keys_out = keys_out;
    a.vals_out = vals_out;
    a.n_host = n;
    a.shift = shift;
    a.digit_bits = digit_bits;
    launch_sweep<false, false>(a, grid, stream);
}

void launch_tile_pass_first(const PairSource& src, uint32_t* tile_out, uint32_t* gauss_out,
                            int digit_bits, bool final, uint2* ranges, const uint32_t* hist,
                            unsigned long long* lookback, EpochRef epoch, uint32_t* ticket,
                            uint32_t* status, int grid, cudaStream_t stream) {
    SweepArgs a = base_args(hist, lookback, epoch, ticket, status);
    a.keys_out = tile_out;
    a.vals_out = gauss_out;
    a.n_host = src.capacity;
    a.counters = src.counters;
    a.shift = 0;
    a.digit_bits = digit_bits;
    a.ranges = ranges;
    a.src = src;
    if (final) launch_sweep<true, true>(a, grid, stream);
    else launch_sweep<true, false>(a, grid, stream);
}

void launch_tile_pass_last(const uint32_t* tile_in, const uint32_t* gauss_in, uint32_t* gauss_out,
                           const uint32_t* counters, int64_t capacity, int shift, int digit_bits,
                           uint2* ranges, const uint32_t* hist, unsigned long long* lookback,
                           EpochRef epoch, uint32_t* ticket, uint32_t* status, int grid,
                           cudaStream_t stream) {
    SweepArgs a = base_args(hist, lookback, epoch, ticket, status);
    a.keys_in = tile_in;
    a.vals_in = gauss_in;
    a.vals_out = gauss_out;
    a.n_host = capacity;
    a.counters = counters;
    a.shift = shift;
    a.digit_bits = digit_bits;
    a.ranges = ranges;
    launch_sweep<false, true>(a, grid, stream);
}

}  // namespace adr
