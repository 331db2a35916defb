// Stages 2-3 of the rasterization pipeline (Sec. 3.2.1), InclusiveSum and the
// bookkeeping DuplicateWithKeys needs, over the Gaussians in view-depth order.
// A Gaussian's pairs form w x h tiles, i.e. w column runs (one per tile
// column); the tile sort works on the runs, so the scan is over w:
//   * offsets[i] = exclusive prefix sum of the run counts (decoupled lookback,
//     32 predecessor words per round trip), the run total C and the number
//     of Gaussians with tiles;
//   * the pair total P = sum of w h (64-bit atomics, published by a one-thread
//     kernel after the scan) and the capacity check;
//   * chunk_first[c] = depth-order position of the Gaussian that holds run
//     c * 4096, so the tile sort can generate each chunk's runs on chip;
// It reads the packed rectangles in depth order, which the last depth-sort
// pass carries along.  Plus small helpers for the tile ranges.
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kScanThreads = 256;
#ifndef ADR_SCAN_ITEMS
#define ADR_SCAN_ITEMS 16
#endif
constexpr int kScanItems = ADR_SCAN_ITEMS;   // a multiple of 4
static_assert(kScanItems % 4 == 0, "16-byte loads and stores");
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr uint32_t kSat = 0x7FFFFFFFu;   // running sums saturate here (> any capacity)
constexpr unsigned long long kScanInc = 1ull << 31;

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return (s < a || s > kSat) ? kSat : s;
}

// Exclusive prefix of chunk `chunk` by decoupled lookback, run by one warp:
// lane l reads the word of chunk j - l, so each round trip covers 32
// predecessors; the words up to the nearest inclusive prefix are summed.
// Lane 0 publishes this chunk's aggregate first and its inclusive prefix last
// (except the chunk the testing hook withholds).  A wait that makes no
// progress for lt.spin_limit polls gives up: it flags the status word and the
// frame's counters and returns the partial prefix.
__device__ uint32_t warp_lookback(unsigned long long* lookback, uint32_t chunk, uint32_t total,
                                  uint32_t epoch, uint32_t* status, uint32_t* counters,
                                  LookbackTest lt) {
    const int lane = threadIdx.x & 31;
    const unsigned long long tag = (unsigned long long)epoch << 32;
    volatile unsigned long long* lb = lookback;
    const bool publish = chunk != lt.withhold;
    if (chunk == 0) {
        if (lane == 0 && publish) lb[0] = tag | kScanInc | min(total, kSat);
        return 0;
    }
    if (lane == 0 && publish) lb[chunk] = tag | min(total, kSat);
    uint64_t excl = 0;
    int64_t j = (int64_t)chunk - 1;   // the nearest predecessor not yet summed
    int spins = 0;
    for (;;) {
        const int64_t idx = j - lane;
        // Before chunk 0 reads as an inclusive prefix of 0 (never reached:
        // chunk 0 always publishes one).
        const unsigned long long w = idx >= 0 ? lb[idx] : (tag | kScanInc);
        const bool ready = (uint32_t)(w >> 32) == epoch;
        const uint32_t not_ready = __ballot_sync(0xffffffffu, !ready);
        const uint32_t inc = __ballot_sync(0xffffffffu, ready && (w & kScanInc));
        const int first_nr = not_ready ? __ffs(not_ready) - 1 : 32;
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        const int take = first_inc < first_nr ? first_inc + 1 : first_nr;   // summed lanes
        uint64_t v = lane < take ? (uint64_t)((uint32_t)w & kSat) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (first_inc < first_nr) break;
        j -= take;
        if (take == 0) {
            if (++spins > lt.spin_limit) {
                if (lane == 0) {
                    atomicOr(status, kErrLookback);
                    atomicExch(counters + kCntScanFailed, 1u);
                }
                break;
            }
            __nanosleep(32);
        }
    }
    const uint32_t e = (uint32_t)min(excl, (uint64_t)kSat);
    __threadfence();
    if (lane == 0 && publish) lb[chunk] = tag | kScanInc | sat_add(e, total);
    return e;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const uint32_t* __restrict__ sorted_box, int64_t n_host, int64_t capacity,
             uint32_t* __restrict__ offsets, uint32_t* __restrict__ chunk_first,
             unsigned long long* __restrict__ lookback, EpochRef eref,
             uint32_t* __restrict__ counters, uint32_t* __restrict__ status, LookbackTest lt) {
    pdl_prologue();
    const uint32_t epoch = (*eref.stage) * 8u + eref.pass;
    // The depth sort kept only the Gaussians with tiles: scan those.
    const int64_t n = min(n_host, (int64_t)counters[kCntDepthKept]);
    __shared__ uint32_t s_warp[kScanThreads / 32], s_pairs[kScanThreads / 32];
    __shared__ uint32_t s_chunk, s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long* pairs64 = reinterpret_cast<unsigned long long*>(counters + kCntPairs64);

    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(counters + kCntScanTicket, 1u);
        __syncthreads();
        const uint32_t chunk = s_chunk;
        const int64_t base = (int64_t)chunk * kScanChunk;
        if (base >= n) break;
        // Blocked arrangement: thread t owns items base + t*kScanItems and the
        // kScanItems after it, read with 16-byte loads where all are in range.
        const int64_t i0 = base + (int64_t)tid * kScanItems;
        const bool full = i0 + kScanItems <= n;
        uint32_t w[kScanItems];
        if (full) {
            const uint4* b4 = reinterpret_cast<const uint4*>(sorted_box + i0);
#pragma unroll
            for (int k = 0; k < kScanItems / 4; ++k) {
                const uint4 q = b4[k];
                w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k) w[k] = i0 + k < n ? sorted_box[i0 + k] : 0xFFFFFFFFu;
        }
        uint32_t tsum = 0, psum = 0, nonzero = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const uint32_t box = w[k];   // all ones: no tiles
            const bool has = box != 0xFFFFFFFFu;
            w[k] = has ? ((box >> 16) & 0xFFu) + 1u : 0u;
            const uint32_t t = has ? w[k] * ((box >> 24) + 1u) : 0u;
            tsum += w[k];   // <= 16 * 256 per thread
            psum += t;      // <= 16 * 2^16 per thread
            nonzero += has;
        }
        // Block exclusive scan of the thread run sums, block sum of the pairs.
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t wp = __reduce_add_sync(0xffffffffu, psum);
        if (lane == 31) s_warp[warp] = x;
        if (lane == 0) s_pairs[warp] = wp;
        __syncthreads();
        uint32_t wbase = 0, total = 0, pairs = 0;
        for (int q = 0; q < kScanThreads / 32; ++q) {
            if (q < warp) wbase += s_warp[q];
            total += s_warp[q];
            pairs += s_pairs[q];   // <= 4096 * 2^16
        }
        const uint32_t texcl = wbase + x - tsum;
        if (warp == 0) {
            if (lane == 0 && pairs) atomicAdd(pairs64, (unsigned long long)pairs);
            const uint32_t excl = warp_lookback(lookback, chunk, total, epoch, status, counters, lt);
            if (lane == 0) {
                s_prefix = excl;
                if (base + kScanChunk >= n) counters[kCntRuns] = sat_add(excl, total);
            }
        }
        const uint32_t nz = __reduce_add_sync(0xffffffffu, nonzero);
        if (lane == 0 && nz) atomicAdd(counters + kCntVisible, nz);
        __syncthreads();
        uint32_t run = sat_add(s_prefix, texcl);
        uint32_t quad[4];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = i0 + k;
            const uint32_t t = w[k];
            quad[k & 3] = run;
            if (full) {
                if ((k & 3) == 3)
                    reinterpret_cast<uint4*>(offsets + i0)[k >> 2] = make_uint4(quad[0], quad[1], quad[2], quad[3]);
            } else if (i < n) {
                offsets[i] = run;
            }
            if (t != 0 && (int64_t)run < capacity) {
                // run chunks start inside [run, run + t)
                const uint64_t c_lo = ((uint64_t)run + kSortChunk - 1) / kSortChunk;
                uint64_t c_hi = ((uint64_t)run + t - 1) / kSortChunk;
                const uint64_t c_max = ((uint64_t)capacity - 1) / kSortChunk;
                if (c_hi > c_max) c_hi = c_max;
                for (uint64_t c = c_lo; c <= c_hi; ++c) chunk_first[c] = (uint32_t)i;
            }
            run = sat_add(run, t);
        }
        __syncthreads();
    }
}

// After the scan: the pair total P (saturated to 31 bits) and the capacity
// flag.  If a lookback wait gave up, the run offsets are not a valid scan:
// P reads as saturated (above any capacity), so every later stage skips its
// work as after an overflow, and only kErrLookback reports it.
__global__ void k_finish_pairs(uint32_t* __restrict__ counters, int64_t capacity,
                               uint32_t* __restrict__ status) {
    pdl_prologue();
    const unsigned long long p = *reinterpret_cast<const unsigned long long*>(counters + kCntPairs64);
    if (counters[kCntScanFailed] != 0u) {
        counters[kCntPairs] = kSat;
        return;
    }
    counters[kCntPairs] = (uint32_t)min(p, (unsigned long long)kSat);
    if (p > (unsigned long long)capacity) atomicOr(status, kErrCapacity);
}

__global__ void k_copy_ranges(const uint2* __restrict__ ranges, int num_tiles, uint2* __restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < num_tiles; t += gridDim.x * blockDim.x) {
        const uint2 r = ranges[t];
        out[t] = r.x < r.y ? r : make_uint2(0u, 0u);
    }
}

// One CTA per tile writes that tile's slice of the inspection output.
__global__ void __launch_bounds__(256)
k_pair_keys(const uint2* __restrict__ ranges, const uint32_t* __restrict__ sorted_gauss,
            const uint32_t* __restrict__ depth_key, int64_t count,
            unsigned long long* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    const uint32_t t = blockIdx.x;
    const uint2 r = ranges[t];
    if (!(r.x < r.y)) return;
    for (uint32_t i = r.x + threadIdx.x; i < r.y && (int64_t)i < count; i += blockDim.x) {
        const uint32_t g = sorted_gauss[i];
        keys_out[i] = ((unsigned long long)t << 32) | depth_key[g];
        vals_out[i] = g;
    }
}

__global__ void __launch_bounds__(256)
k_read_gaussians(const float4* __restrict__ rec, const float4* __restrict__ aux,
                 const uint32_t* __restrict__ gbox, int n, float* __restrict__ geom,
                 int32_t* __restrict__ rect_out, int32_t* __restrict__ tiles_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t box = gbox[i];
    const bool has = box != 0xFFFFFFFFu;
    // Preprocess writes the records of Gaussians with tiles only: the others
    // report zeros except their radii and depth.
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 r0 = has ? rec[3 * i + 0] : z4, r2 = has ? rec[3 * i + 2] : z4;
    const float4 a0 = has ? aux[2 * i + 0] : z4, a1 = aux[2 * i + 1];
    if (geom) {
        float* o = geom + (size_t)i * ADR_GEOM_FLOATS;
        o[0] = r0.x; o[1] = r0.y; o[2] = a0.x; o[3] = a0.y; o[4] = a0.z; o[5] = a0.w;
        o[6] = a1.x; o[7] = a1.y; o[8] = r2.x; o[9] = r2.y; o[10] = r2.z; o[11] = a1.z;
    }
    const int32_t x0 = has ? (int32_t)(box & 0xFFu) : 0, y0 = has ? (int32_t)((box >> 8) & 0xFFu) : 0;
    const int32_t w = has ? (int32_t)((box >> 16) & 0xFFu) + 1 : 0, h = has ? (int32_t)(box >> 24) + 1 : 0;
    if (rect_out) {
        rect_out[4 * i + 0] = x0; rect_out[4 * i + 1] = y0;
        rect_out[4 * i + 2] = x0 + w; rect_out[4 * i + 3] = y0 + h;
    }
    if (tiles_out) tiles_out[i] = w * h;
}

}  // namespace

int scan_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scan_tiles, kScanThreads, 0) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_scan_tiles(const uint32_t* sorted_box, int64_t n, int64_t capacity, uint32_t* offsets,
                       uint32_t* chunk_first, unsigned long long* lookback, EpochRef epoch,
                       uint32_t* counters, uint32_t* status, int grid, cudaStream_t stream) {
    if (n > 0)
        launch_pdl(k_scan_tiles, grid, kScanThreads, 0, stream, sorted_box, n, capacity, offsets, chunk_first,
                                                        lookback, epoch, counters, status,
                                                        lookback_test());
    launch_pdl(k_finish_pairs, 1, 1, 0, stream, counters, capacity, status);
}

void launch_copy_ranges(const uint2* ranges, int num_tiles, uint2* out, cudaStream_t stream) {
    if (num_tiles <= 0) return;
    k_copy_ranges<<<(num_tiles + 255) / 256, 256, 0, stream>>>(ranges, num_tiles, out);
}

void launch_pair_keys(const uint2* ranges, int num_tiles, const uint32_t* sorted_gauss,
                      const uint32_t* depth_key_by_gauss, int64_t count,
                      unsigned long long* keys_out, uint32_t* vals_out, cudaStream_t stream) {
    if (count <= 0 || num_tiles <= 0) return;
    k_pair_keys<<<num_tiles, 256, 0, stream>>>(ranges, sorted_gauss, depth_key_by_gauss, count,
                                               keys_out, vals_out);
}

void launch_read_gaussians(const float4* rec, const float4* aux, const uint32_t* gbox, int n,
                           float* geom, int32_t* rect_out, int32_t* tiles_out, cudaStream_t stream) {
    if (n <= 0) return;
    k_read_gaussians<<<(n + 255) / 256, 256, 0, stream>>>(rec, aux, gbox, n, geom, rect_out,
                                                          tiles_out);
}

}  // namespace adr
