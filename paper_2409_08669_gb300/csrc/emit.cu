// Stages 2-3 and 5 of the rasterization pipeline (Sec. 3.2.1):
//   InclusiveSum      scan of per-Gaussian tile counts (decoupled lookback)
//   DuplicateWithKeys one (tile, Gaussian) pair per overlapped tile, emitted
//                     cooperatively by a warp (warp-aggregated emission)
//   IdentifyTileRanges [start, end) of each tile in the sorted pair list
// The Gaussians are visited in view-depth order, so the pair list is already
// depth-ordered and only needs a stable sort by tile.
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr uint32_t kSat = 0x7FFFFFFFu;   // running sums saturate here (> any capacity)
constexpr unsigned long long kScanInc = 1ull << 31;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return (s < a || s > kSat) ? kSat : s;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const uint32_t* __restrict__ order, const uint32_t* __restrict__ tiles, int64_t n,
             uint32_t* __restrict__ offsets, unsigned long long* __restrict__ lookback,
             uint32_t epoch, uint32_t* __restrict__ counters, uint32_t* __restrict__ status) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_chunk, s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long tag = (unsigned long long)epoch << 32;
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(counters + kCntScanTicket, 1u);
        __syncthreads();
        const uint32_t chunk = s_chunk;
        const int64_t base = (int64_t)chunk * kScanChunk;
        if (base >= n) break;
        // Blocked arrangement: thread t owns items base + t*16 .. +15.
        uint32_t v[kScanItems];
        uint32_t tsum = 0, nonzero = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + tid * kScanItems + k;
            v[k] = i < n ? tiles[order[i]] : 0u;
            tsum += v[k];   // <= 16 * 2^16 per thread, no overflow
            nonzero += v[k] != 0;
        }
        // Block exclusive scan of the thread sums (chunk total < 2^31).
        uint32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t wbase = 0, total = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) {
            if (w < warp) wbase += s_warp[w];
            total += s_warp[w];
        }
        const uint32_t texcl = wbase + x - tsum;
        // Chunk prefix by decoupled lookback (one thread).
        if (tid == 0) {
            unsigned long long* my = lookback + chunk;
            uint32_t excl = 0;
            if (chunk == 0) {
                *reinterpret_cast<volatile unsigned long long*>(my) = tag | kScanInc | min(total, kSat);
            } else {
                *reinterpret_cast<volatile unsigned long long*>(my) = tag | min(total, kSat);
                int64_t j = (int64_t)chunk - 1;
                int spins = 0;
                while (j >= 0) {
                    const unsigned long long w =
                        *reinterpret_cast<volatile unsigned long long*>(lookback + j);
                    if ((w >> 32) != epoch) {
                        if (++spins > kSpinLimit) { atomicOr(status, kErrLookback); break; }
                        __nanosleep(32);
                        continue;
                    }
                    excl = sat_add(excl, (uint32_t)w & kSat);
                    if (w & kScanInc) break;
                    --j;
                }
                *reinterpret_cast<volatile unsigned long long*>(my) =
                    tag | kScanInc | sat_add(excl, total);
            }
            s_prefix = excl;
            if (base + kScanChunk >= n) counters[kCntPairs] = sat_add(excl, total);
        }
        // Visible (non-empty) count.
        uint32_t nz = __reduce_add_sync(0xffffffffu, nonzero);
        if (lane == 0 && nz) atomicAdd(counters + kCntVisible, nz);
        __syncthreads();
        uint32_t run = sat_add(s_prefix, texcl);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + tid * kScanItems + k;
            if (i < n) offsets[i] = run;
            run = sat_add(run, v[k]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_emit(const uint32_t* __restrict__ order, const uint32_t* __restrict__ tiles,
       const uint32_t* __restrict__ offsets, const ushort4* __restrict__ rect, int64_t n,
       int tiles_x, int64_t capacity, uint32_t* __restrict__ pair_tile,
       uint32_t* __restrict__ pair_gauss, uint32_t* __restrict__ tile_hist, int hist_passes,
       uint32_t* __restrict__ status) {
    __shared__ uint32_t s_hist[2][kRadix];
    for (int i = threadIdx.x; i < 2 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x / 32);
    bool overflow = false;
    for (int64_t wbase = ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32;
         wbase < n; wbase += warps_total * 32) {
        const int64_t pos = wbase + lane;
        uint32_t g = 0, t = 0, off = 0;
        ushort4 r = make_ushort4(0, 0, 1, 1);
        if (pos < n) {
            g = order[pos];
            t = tiles[g];
            if (t) {
                off = offsets[pos];
                r = rect[g];
            }
        }
        // Inclusive warp scan of the tile counts.
        uint32_t incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - t;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t rx0 = r.x, ry0 = r.y, rw = (uint32_t)(r.z - r.x);
        for (uint32_t j = 0; j < total; j += 32) {
            const uint32_t p = j + lane;
            // Source lane: the largest s with excl[s] <= p.
            int s = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, excl, s + step);
                if (e <= p) s += step;
            }
            const uint32_t e_s = __shfl_sync(0xffffffffu, excl, s);
            const uint32_t off_s = __shfl_sync(0xffffffffu, off, s);
            const uint32_t g_s = __shfl_sync(0xffffffffu, g, s);
            const uint32_t x0 = __shfl_sync(0xffffffffu, rx0, s);
            const uint32_t y0 = __shfl_sync(0xffffffffu, ry0, s);
            const uint32_t w = __shfl_sync(0xffffffffu, rw, s);
            if (p < total) {
                const uint32_t k = p - e_s;
                const uint32_t dy = k / w, dx = k - dy * w;
                const uint32_t tile = (y0 + dy) * (uint32_t)tiles_x + (x0 + dx);
                const uint64_t gp = (uint64_t)off_s + k;
                if (gp < (uint64_t)capacity) {
                    pair_tile[gp] = tile;
                    pair_gauss[gp] = g_s;
                    atomicAdd(&s_hist[0][tile & 0xFF], 1u);
                    if (hist_passes > 1) atomicAdd(&s_hist[1][(tile >> 8) & 0xFF], 1u);
                } else {
                    overflow = true;
                }
            }
        }
    }
    if (overflow) atomicOr(status, kErrCapacity);
    __syncthreads();
    for (int i = threadIdx.x; i < hist_passes * kRadix; i += blockDim.x) {
        const uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(tile_hist + i, v);
    }
}

__global__ void __launch_bounds__(256)
k_ranges(const uint32_t* __restrict__ sorted_tile, const uint32_t* __restrict__ d_n,
         int64_t capacity, uint32_t num_tiles, uint2* __restrict__ ranges) {
    const int64_t n = (int64_t)min((uint64_t)*d_n, (uint64_t)capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = sorted_tile[i];
        if (t >= num_tiles) continue;   // only after a failed (flagged) sort
        if (i == 0 || sorted_tile[i - 1] != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || sorted_tile[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

__global__ void __launch_bounds__(256)
k_pair_keys(const uint32_t* __restrict__ sorted_tile, const uint32_t* __restrict__ sorted_gauss,
            const uint32_t* __restrict__ depth_key, const uint32_t* __restrict__ d_n,
            int64_t count, unsigned long long* __restrict__ keys_out,
            uint32_t* __restrict__ vals_out) {
    const int64_t n = (int64_t)min((uint64_t)*d_n, (uint64_t)count);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = sorted_gauss[i];
        keys_out[i] = ((unsigned long long)sorted_tile[i] << 32) | depth_key[g];
        vals_out[i] = g;
    }
}

__global__ void __launch_bounds__(256)
k_read_gaussians(const float4* __restrict__ rec, const float4* __restrict__ aux,
                 const ushort4* __restrict__ rect, const uint32_t* __restrict__ tiles, int n,
                 float* __restrict__ geom, int32_t* __restrict__ rect_out,
                 int32_t* __restrict__ tiles_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 r0 = rec[3 * i + 0], r2 = rec[3 * i + 2];
    const float4 a0 = aux[2 * i + 0], a1 = aux[2 * i + 1];
    if (geom) {
        float* o = geom + (size_t)i * ADR_GEOM_FLOATS;
        o[0] = r0.x; o[1] = r0.y; o[2] = a0.x; o[3] = a0.y; o[4] = a0.z; o[5] = a0.w;
        o[6] = a1.x; o[7] = a1.y; o[8] = r2.x; o[9] = r2.y; o[10] = r2.z; o[11] = a1.z;
    }
    if (rect_out) {
        const ushort4 r = rect[i];
        rect_out[4 * i + 0] = r.x; rect_out[4 * i + 1] = r.y;
        rect_out[4 * i + 2] = r.z; rect_out[4 * i + 3] = r.w;
    }
    if (tiles_out) tiles_out[i] = (int32_t)tiles[i];
}

}  // namespace

int scan_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scan_tiles, kScanThreads, 0) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

void launch_scan_tiles(const uint32_t* order, const uint32_t* tiles, int64_t n, uint32_t* offsets,
                       unsigned long long* lookback, uint32_t epoch, uint32_t* counters,
                       uint32_t* status, int grid, cudaStream_t stream) {
    if (n <= 0) return;
    k_scan_tiles<<<grid, kScanThreads, 0, stream>>>(order, tiles, n, offsets, lookback, epoch,
                                                    counters, status);
}

void launch_emit(const uint32_t* order, const uint32_t* tiles, const uint32_t* offsets,
                 const ushort4* rect, int64_t n, const CamDev& cam, int64_t capacity,
                 uint32_t* pair_tile, uint32_t* pair_gauss, uint32_t* tile_hist, int hist_passes,
                 int hist_bits, uint32_t* status, cudaStream_t stream) {
    (void)hist_bits;
    if (n <= 0) return;
    const int64_t warps = (n + 31) / 32;
    const int64_t blocks = (warps + 7) / 8;
    const int grid = (int)(blocks < 152 * 16 ? blocks : 152 * 16);
    k_emit<<<grid, 256, 0, stream>>>(order, tiles, offsets, rect, n, cam.tiles_x, capacity,
                                     pair_tile, pair_gauss, tile_hist, hist_passes, status);
}

void launch_ranges(const uint32_t* sorted_tile, const uint32_t* d_n, int64_t capacity,
                   uint32_t num_tiles, uint2* ranges, int grid, cudaStream_t stream) {
    k_ranges<<<grid, 256, 0, stream>>>(sorted_tile, d_n, capacity, num_tiles, ranges);
}

void launch_pair_keys(const uint32_t* sorted_tile, const uint32_t* sorted_gauss,
                      const uint32_t* depth_key_by_gauss, const uint32_t* d_n, int64_t count,
                      unsigned long long* keys_out, uint32_t* vals_out, cudaStream_t stream) {
    if (count <= 0) return;
    k_pair_keys<<<152 * 4, 256, 0, stream>>>(sorted_tile, sorted_gauss, depth_key_by_gauss, d_n,
                                             count, keys_out, vals_out);
}

void launch_read_gaussians(const float4* rec, const float4* aux, const ushort4* rect,
                           const uint32_t* tiles, int n, float* geom, int32_t* rect_out,
                           int32_t* tiles_out, cudaStream_t stream) {
    if (n <= 0) return;
    k_read_gaussians<<<(n + 255) / 256, 256, 0, stream>>>(rec, aux, rect, tiles, n, geom,
                                                          rect_out, tiles_out);
}

}  // namespace adr
