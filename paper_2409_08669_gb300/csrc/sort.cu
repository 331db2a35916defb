// The view-depth sort of the Gaussians (the depth half of the paper's
// (tile | depth) sort key, Sec. 3.2.1) as stable least-significant-digit radix
// passes in the "onesweep" form: each chunk of 4096 keys ranks its keys
// locally (warp match_any), obtains the running per-digit offsets of all
// earlier chunks by decoupled lookback, and scatters through shared memory so
// that each digit's run is written contiguously.
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
struct alignas(16) SortShared {
    union {
        struct {
            uint32_t keys[kSortChunk];
            uint32_t vals[kSortChunk];
        } kv;
    } u;
    uint32_t warp_cnt[kWarps][kRadix + 1];   // +1: out-of-range items of the tail chunk
    uint32_t gbase[kRadix];                  // exclusive prefix of the global digit histogram
    uint32_t local[kRadix + 1];              // exclusive prefix of this chunk's digit counts
    uint32_t dst[kRadix];                    // global position of local slot 0, per digit
    uint32_t wsum[kWarps];
    uint32_t chunk;
};
constexpr size_t kSortSmem = sizeof(SortShared);

struct SweepArgs {
    const uint32_t* keys_in;
    const uint32_t* vals_in;
    uint32_t* keys_out;
    uint32_t* vals_out;
    int64_t n;                   // item count
    int shift, digit_bits;
    const uint32_t* hist;        // 256 counts of this pass's digit
    unsigned long long* lookback;
    EpochRef epoch;
    uint32_t* ticket;
    uint32_t* status;
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

__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortShared& sm = *reinterpret_cast<SortShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t mask = (1u << a.digit_bits) - 1u;
    const int64_t n = a.n;
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
        // Warp-striped load: item q of lane l in warp w is base + w*512 + q*32 + l.
#pragma unroll
        for (int q = 0; q < kSortItems; ++q) {
            const int s = warp * (kSortItems * 32) + q * 32 + lane;
            const bool ok = s < count;
            key[q] = ok ? a.keys_in[base + s] : 0xFFFFFFFFu;
            val[q] = ok ? (a.vals_in ? a.vals_in[base + s] : (uint32_t)(base + s)) : 0u;
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
            a.keys_out[g] = k;
        }
        __syncthreads();
    }
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
    cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_onesweep, kSortThreads,
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
    a.n = n;
    a.shift = shift;
    a.digit_bits = digit_bits;
    k_onesweep<<<grid, kSortThreads, kSortSmem, stream>>>(a);
}

}  // namespace adr
