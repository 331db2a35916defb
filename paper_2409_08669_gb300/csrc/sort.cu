// Stage 4, SortPairs (Sec. 3.2.1): a stable least-significant-digit radix
// sort of 32-bit keys with 32-bit values, one kernel per 8-bit digit
// ("onesweep": each chunk ranks its keys locally, obtains the running digit
// offsets of all earlier chunks by decoupled lookback, and scatters).
//
// The same kernel sorts the Gaussians by view depth (4 digits) and the
// depth-ordered pairs by tile (ceil(tile_bits / 8) digits).
//
// Persistent grid: every CTA takes chunk tickets in increasing order from an
// atomic counter, so any chunk a CTA waits on is already held by a running
// CTA.  Each wait is bounded; on expiry the kernel raises kErrLookback and
// continues with a wrong (but in-bounds) placement rather than hanging.
#include "adr_internal.cuh"

namespace adr {
namespace {

// Lookback word: [63:32] epoch of the pass, [31:30] state (1 = aggregate of
// this chunk only, 2 = inclusive prefix), [29:0] count.  A word whose epoch is
// not the current pass's is "not ready yet".
constexpr unsigned long long kStateAgg = 1ull << 30;
constexpr unsigned long long kStateInc = 2ull << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kSpinLimit = 1 << 22;

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
k_digit_hist(const uint32_t* __restrict__ keys, int64_t n_host, const uint32_t* __restrict__ d_n,
             int shift0, int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = d_n ? (int64_t)min((uint64_t)*d_n, (uint64_t)n_host) : n_host;
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

struct SortSmem {
    uint32_t keys[kSortChunk];
    uint32_t vals[kSortChunk];
    uint32_t warp_cnt[kSortThreads / 32][kRadix + 1];   // +1: out-of-range items
    uint32_t gbase[kRadix];      // exclusive prefix of the global digit histogram
    uint32_t local[kRadix + 1];  // exclusive prefix of this chunk's digit counts
    uint32_t dst[kRadix];        // global position of local slot 0 of each digit
    uint32_t chunk;
};

__global__ void __launch_bounds__(kSortThreads)
k_onesweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
           uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n_host,
           const uint32_t* __restrict__ d_n, int shift, int digit_bits,
           const uint32_t* __restrict__ hist, unsigned long long* __restrict__ lookback,
           uint32_t epoch, uint32_t* __restrict__ ticket, uint32_t* __restrict__ status) {
    __shared__ SortSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t mask = (1u << digit_bits) - 1u;
    const int64_t n = d_n ? (int64_t)min((uint64_t)*d_n, (uint64_t)n_host) : n_host;
    const unsigned long long tag = (unsigned long long)epoch << 32;

    // Exclusive prefix of the global histogram of this digit (one digit per thread).
    {
        const uint32_t h = hist[tid];
        uint32_t x = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm.local[warp] = x;
        __syncthreads();
        uint32_t wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += sm.local[w];
        sm.gbase[tid] = wbase + x - h;
        __syncthreads();
    }

    for (;;) {
        if (tid == 0) sm.chunk = atomicAdd(ticket, 1u);
        for (int d = lane; d <= kRadix; d += 32) sm.warp_cnt[warp][d] = 0;
        __syncthreads();
        const uint32_t chunk = sm.chunk;
        const int64_t base = (int64_t)chunk * kSortChunk;
        if (base >= n) break;

        // Warp-striped load: warp w owns 512 consecutive keys, item k of lane l
        // is key w*512 + k*32 + l, so (k, lane) order is the input order.
        uint32_t key[kSortItems], val[kSortItems], dig[kSortItems], rank[kSortItems];
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const int64_t idx = base + warp * (kSortItems * 32) + k * 32 + lane;
            const bool ok = idx < n;
            key[k] = ok ? keys_in[idx] : 0xFFFFFFFFu;
            val[k] = ok ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
            dig[k] = ok ? ((key[k] >> shift) & mask) : (uint32_t)kRadix;
        }
        // Stable warp-level ranking with match_any.
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t peers = __match_any_sync(0xffffffffu, dig[k]);
            const uint32_t before = sm.warp_cnt[warp][dig[k]];
            rank[k] = before + __popc(peers & lanemask_lt());
            __syncwarp();
            if (lane == 31 - __clz(peers)) sm.warp_cnt[warp][dig[k]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();

        // Per digit (thread tid = digit): prefix over warps and chunk count.
        uint32_t cnt = 0;
        {
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = sm.warp_cnt[w][tid];
                sm.warp_cnt[w][tid] = cnt;
                cnt += c;
            }
        }
        // Publish this chunk's count, then look back for the earlier chunks'.
        unsigned long long* my = lookback + (size_t)chunk * kRadix + tid;
        uint32_t excl = 0;
        if (chunk == 0) {
            st_volatile(my, tag | kStateInc | cnt);
        } else {
            st_volatile(my, tag | kStateAgg | cnt);
            int64_t j = (int64_t)chunk - 1;
            int spins = 0;
            while (j >= 0) {
                const unsigned long long w = ld_volatile(lookback + (size_t)j * kRadix + tid);
                if ((w >> 32) != epoch || (w & (3ull << 30)) == 0) {
                    if (++spins > kSpinLimit) { atomicOr(status, kErrLookback); break; }
                    __nanosleep(32);
                    continue;
                }
                excl += (uint32_t)w & kCountMask;
                if (w & kStateInc) break;
                --j;
            }
            st_volatile(my, tag | kStateInc | ((excl + cnt) & kCountMask));
        }
        // Exclusive prefix of this chunk's digit counts (local placement).
        {
            uint32_t x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            __shared__ uint32_t s_wsum[kSortThreads / 32];
            if (lane == 31) s_wsum[warp] = x;
            __syncthreads();
            uint32_t wbase = 0;
            for (int w = 0; w < warp; ++w) wbase += s_wsum[w];
            const uint32_t loc = wbase + x - cnt;
            sm.local[tid] = loc;
            if (tid == kSortThreads - 1) sm.local[kRadix] = loc + cnt;
            sm.dst[tid] = sm.gbase[tid] + excl - loc;
        }
        __syncthreads();
        // Scatter into shared memory in digit order; out-of-range items (tail
        // chunk only) are dropped.
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t d = dig[k];
            if (d < (uint32_t)kRadix) {
                const uint32_t pos = sm.local[d] + sm.warp_cnt[warp][d] + rank[k];
                sm.keys[pos] = key[k];
                sm.vals[pos] = val[k];
            }
        }
        __syncthreads();
        // Coalesced write-out: consecutive slots of one digit go to consecutive addresses.
        const uint32_t valid = sm.local[kRadix];
        for (uint32_t s = tid; s < valid; s += kSortThreads) {
            const uint32_t k = sm.keys[s];
            const uint32_t d = (k >> shift) & mask;
            const uint32_t g = sm.dst[d] + s;   // exact modulo 2^32; true value < 2^30
            if ((int64_t)g < n) {
                keys_out[g] = k;
                vals_out[g] = sm.vals[s];
            } else {
                atomicOr(status, kErrRange);
            }
        }
        __syncthreads();
    }
}

}  // namespace

int onesweep_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_onesweep, kSortThreads, 0) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_digit_hist(const uint32_t* keys, int64_t n, const uint32_t* d_n, int shift0, int passes,
                       uint32_t* hist, int grid, cudaStream_t stream) {
    if (n <= 0) return;
    k_digit_hist<<<grid, 256, 0, stream>>>(keys, n, d_n, shift0, passes, hist);
}

void launch_onesweep(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                     uint32_t* vals_out, int64_t n, const uint32_t* d_n, int shift, int digit_bits,
                     const uint32_t* hist, unsigned long long* lookback, uint32_t epoch,
                     uint32_t* ticket, uint32_t* status, int grid, cudaStream_t stream) {
    if (n <= 0) return;
    k_onesweep<<<grid, kSortThreads, 0, stream>>>(keys_in, vals_in, keys_out, vals_out, n, d_n,
                                                   shift, digit_bits, hist, lookback, epoch,
                                                   ticket, status);
}

}  // namespace adr
