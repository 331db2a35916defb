// Depth slices of the forward frame.  A pixel stops once its transmittance
// falls below t_min, and at the benchmark workloads a tile's slowest pixel
// stops within the first ~1-3% of its depth-ordered list, so most column runs
// are never read.  The frame therefore builds the column runs in two slices
// of the depth order:
//   slice 0: the nearest V/16 Gaussians with tiles (all their runs);
//   slice 1: the other Gaussians that touch a tile with a pixel still going
//            after slice 0 (a stable compaction of the depth order).
// Render blends slice 0, keeps the state of the unfinished tiles, and blends
// slice 1 into them.  A tile's list is the concatenation of its slice-0 and
// slice-1 lists, which is its full list with only Gaussians behind its last
// pixel's stop left out, so every pixel is the same as from the full list.
//
//   k_slice0_setup   counters of slice 0 (its Gaussians, runs, the pair flag)
//   k_sat_rows / k_sat_cols
//                    summed-area table of the unfinished tiles
//   k_surv_count / k_surv_scan / k_surv_scatter
//                    stable compaction of the Gaussians [K0, V) whose tile
//                    rectangle holds an unfinished tile, with their run
//                    offsets and chunk starts and slice 1's counters
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kSurvThreads = 256;

// Gaussians of slice 0: ceil(V / kSliceDiv), at least one when V > 0.
__device__ __forceinline__ uint32_t slice0_count(uint32_t visible) {
    const uint32_t div = kSliceDiv > 0 ? (uint32_t)kSliceDiv : 1u;
    return visible == 0 ? 0u : max(1u, (visible + div - 1u) / div);
}

__global__ void k_slice0_setup(const uint32_t* __restrict__ counters,
                               const uint32_t* __restrict__ offsets, uint32_t* __restrict__ c0) {
    pdl_prologue();
    const uint32_t V = counters[kCntVisible];
    const uint32_t K0 = slice0_count(V);
    c0[kCntPairs] = counters[kCntPairs];
    c0[kCntVisible] = K0;
    c0[kCntRuns] = K0 < V ? offsets[K0] : counters[kCntRuns];
    c0[kCntDepthKept] = K0;
}

// Inclusive prefix over the 32 lanes of a warp.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Summed-area table of the unfinished tiles: sat[y * (tiles_x + 1) + x] =
// unfinished tiles in [0, x) x [0, y), x <= tiles_x, y <= tiles_y (<= 257
// entries per row or column: 9 chunks of 32).  Row pass: one warp per row.
constexpr int kSatChunks = (kRadix + 1 + 31) / 32;
__global__ void __launch_bounds__(kSurvThreads)
k_sat_rows(const uint32_t* __restrict__ tile_done, int tiles_x, int tiles_y, uint32_t* __restrict__ sat) {
    pdl_prologue();
    const int lane = threadIdx.x & 31;
    const int y = (int)(blockIdx.x * (kSurvThreads / 32) + (threadIdx.x >> 5));
    const int W = tiles_x + 1;
    if (y > tiles_y) return;
    uint32_t v[kSatChunks];
#pragma unroll
    for (int c = 0; c < kSatChunks; ++c) {   // all loads first
        const int x = c * 32 + lane;
        v[c] = (y > 0 && x > 0 && x < W && tile_done[(size_t)(y - 1) * tiles_x + (x - 1)] == 0u) ? 1u : 0u;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int c = 0; c < kSatChunks; ++c) {
        const int x = c * 32 + lane;
        const uint32_t t = warp_incl_scan(v[c], lane) + carry;
        if (x < W) sat[(size_t)y * W + x] = t;
        carry = __shfl_sync(0xffffffffu, t, 31);
    }
}

// Column pass: one warp per column.
__global__ void __launch_bounds__(kSurvThreads)
k_sat_cols(int tiles_x, int tiles_y, uint32_t* __restrict__ sat) {
    pdl_prologue();
    const int lane = threadIdx.x & 31;
    const int x = (int)(blockIdx.x * (kSurvThreads / 32) + (threadIdx.x >> 5));
    const int W = tiles_x + 1, H = tiles_y + 1;
    if (x >= W) return;
    uint32_t v[kSatChunks];
#pragma unroll
    for (int c = 0; c < kSatChunks; ++c) {
        const int y = c * 32 + lane;
        v[c] = y < H ? sat[(size_t)y * W + x] : 0u;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int c = 0; c < kSatChunks; ++c) {
        const int y = c * 32 + lane;
        const uint32_t t = warp_incl_scan(v[c], lane) + carry;
        if (y < H) sat[(size_t)y * W + x] = t;
        carry = __shfl_sync(0xffffffffu, t, 31);
    }
}

// Does the packed rectangle (x0 | y0 << 8 | (w-1) << 16 | (h-1) << 24) hold
// an unfinished tile?
__device__ __forceinline__ bool survives(uint32_t box, const uint32_t* __restrict__ sat, int W) {
    if (box == 0xFFFFFFFFu) return false;
    const int x0 = (int)(box & 0xFFu), y0 = (int)((box >> 8) & 0xFFu);
    const int x1 = x0 + (int)((box >> 16) & 0xFFu) + 1, y1 = y0 + (int)(box >> 24) + 1;
    const uint32_t s = __ldg(sat + (size_t)y1 * W + x1) - __ldg(sat + (size_t)y0 * W + x1) -
                       __ldg(sat + (size_t)y1 * W + x0) + __ldg(sat + (size_t)y0 * W + x0);
    return s != 0u;
}

// Positions [K0 + b * per, K0 + (b + 1) * per) of the depth order for CTA b.
__device__ __forceinline__ void surv_span(const uint32_t* counters, int grid, uint32_t& a,
                                          uint32_t& e) {
    const uint32_t V = counters[kCntVisible];
    const uint32_t K0 = slice0_count(V);
    const uint32_t per = (V - K0 + (uint32_t)grid - 1u) / (uint32_t)grid;
    a = min(V, K0 + per * blockIdx.x);
    e = min(V, a + per);
}

__device__ __forceinline__ uint32_t box_runs(uint32_t box) { return ((box >> 16) & 0xFFu) + 1u; }

// Per CTA: the kept Gaussians and their column runs (cnt[b], cnt[grid + b]).
__global__ void __launch_bounds__(kSurvThreads)
k_surv_count(const uint32_t* __restrict__ sorted_box, const uint32_t* __restrict__ counters,
             const uint32_t* __restrict__ sat, int tiles_x, int grid, uint32_t* __restrict__ cnt,
             uint8_t* __restrict__ keep_flag) {
    pdl_prologue();
    __shared__ uint32_t s_w[2][kSurvThreads / 32];
    uint32_t a, e;
    surv_span(counters, grid, a, e);
    uint32_t c = 0, r = 0;
    for (uint32_t i = a + threadIdx.x; i < e; i += kSurvThreads) {
        const uint32_t box = sorted_box[i];
        const bool keep = survives(box, sat, tiles_x + 1);
        keep_flag[i] = keep ? 1 : 0;
        if (keep) {
            ++c;
            r += box_runs(box);
        }
    }
    c = __reduce_add_sync(0xffffffffu, c);
    r = __reduce_add_sync(0xffffffffu, r);
    if ((threadIdx.x & 31) == 0) {
        s_w[0][threadIdx.x >> 5] = c;
        s_w[1][threadIdx.x >> 5] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tc = 0, tr = 0;
        for (int w = 0; w < kSurvThreads / 32; ++w) {
            tc += s_w[0][w];
            tr += s_w[1][w];
        }
        cnt[blockIdx.x] = tc;
        cnt[grid + blockIdx.x] = tr;
    }
}

// Exclusive scans of the grid's kept counts and runs (grid <= kMaxTileGrid,
// one CTA of kMaxTileGrid / 8 threads); the totals are slice 1's Gaussians
// and runs.  Slice 1's counters: kept = visible = Gaussians, runs, and the
// frame's pair count (its capacity flag).
__global__ void __launch_bounds__(kMaxTileGrid / 8)
k_surv_scan(uint32_t* __restrict__ cnt, int grid, const uint32_t* __restrict__ counters,
            uint32_t* __restrict__ c1) {
    pdl_prologue();
    constexpr int kT = kMaxTileGrid / 8, kPer = 8;
    __shared__ uint32_t s_w[kT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int which = 0; which < 2; ++which) {
        uint32_t* arr = cnt + which * grid;
        uint32_t v[kPer], t = 0;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int b = tid * kPer + u;
            v[u] = b < grid ? arr[b] : 0u;
            t += v[u];
        }
        const uint32_t x = warp_incl_scan(t, lane);
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        uint32_t base = 0, total = 0;
        for (int w = 0; w < kT / 32; ++w) {
            base += w < warp ? s_w[w] : 0u;
            total += s_w[w];
        }
        uint32_t run = base + x - t;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int b = tid * kPer + u;
            if (b < grid) arr[b] = run;
            run += v[u];
        }
        if (tid == 0) {
            if (which == 0) {
                c1[kCntDepthKept] = total;
                c1[kCntVisible] = total;
            } else {
                c1[kCntRuns] = total;
                c1[kCntPairs] = counters[kCntPairs];
            }
        }
        __syncthreads();
    }
}

// Writes the kept Gaussians in depth order with their packed rectangles, run
// offsets (exclusive prefix of their widths) and, for every 4096-run chunk
// that starts inside a Gaussian's runs, that Gaussian's position.
__global__ void __launch_bounds__(kSurvThreads)
k_surv_scatter(const uint32_t* __restrict__ sorted_box, const uint32_t* __restrict__ order,
               const uint32_t* __restrict__ counters, const uint8_t* __restrict__ keep_flag,
               int grid, const uint32_t* __restrict__ starts, int64_t n_max, int64_t chunk_max,
               uint32_t* __restrict__ s_order, uint32_t* __restrict__ s_box,
               uint32_t* __restrict__ s_offsets, uint32_t* __restrict__ s_chunk_first,
               uint32_t* __restrict__ status) {
    pdl_prologue();
    __shared__ uint32_t s_w[2][kSurvThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t a, e;
    surv_span(counters, grid, a, e);
    uint32_t out = starts[blockIdx.x], roff = starts[grid + blockIdx.x];
    for (uint32_t b0 = a; b0 < e; b0 += kSurvThreads) {
        const uint32_t i = b0 + tid;
        const bool keep = i < e && keep_flag[i] != 0;
        const uint32_t box = keep ? sorted_box[i] : 0xFFFFFFFFu;
        const uint32_t w = keep ? box_runs(box) : 0u;
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        const uint32_t wr = warp_incl_scan(w, lane);
        if (lane == 31) {
            s_w[0][warp] = __popc(m);
            s_w[1][warp] = wr;
        }
        __syncthreads();
        uint32_t before = 0, total = 0, rbefore = 0, rtotal = 0;
#pragma unroll
        for (int q = 0; q < kSurvThreads / 32; ++q) {
            const uint32_t c = s_w[0][q], r = s_w[1][q];
            before += q < warp ? c : 0u;
            rbefore += q < warp ? r : 0u;
            total += c;
            rtotal += r;
        }
        if (keep) {
            const uint32_t j = out + before + __popc(m & ((1u << lane) - 1u));
            const uint32_t o = roff + rbefore + wr - w;   // first run of this Gaussian
            if ((int64_t)j < n_max) {
                s_order[j] = order[i];
                s_box[j] = box;
                s_offsets[j] = o;
                for (uint32_t c = (o + (uint32_t)kSortChunk - 1u) / (uint32_t)kSortChunk;
                     (int64_t)c < chunk_max && c * (uint32_t)kSortChunk < o + w; ++c)
                    s_chunk_first[c] = j;
            } else {
                atomicOr(status, kErrRange);
            }
        }
        out += total;
        roff += rtotal;
        __syncthreads();
    }
}

}  // namespace

void launch_slice0_setup(const uint32_t* counters, const uint32_t* offsets, uint32_t* c0,
                         cudaStream_t stream) {
    launch_pdl(k_slice0_setup, 1, 1, 0, stream, counters, offsets, c0);
}

void launch_survivors(const uint32_t* tile_done, int tiles_x, int tiles_y, uint32_t* sat,
                      const uint32_t* sorted_box, const uint32_t* order, const uint32_t* counters,
                      int grid, uint32_t* cnt, uint8_t* keep_flag, int64_t n_max, int64_t chunk_max,
                      uint32_t* s_order, uint32_t* s_box, uint32_t* s_offsets,
                      uint32_t* s_chunk_first, uint32_t* c1, uint32_t* status, cudaStream_t stream) {
    const int warps = kSurvThreads / 32;
    launch_pdl(k_sat_rows, (tiles_y + 1 + warps - 1) / warps, kSurvThreads, 0, stream, tile_done, tiles_x,
                                                                               tiles_y, sat);
    launch_pdl(k_sat_cols, (tiles_x + 1 + warps - 1) / warps, kSurvThreads, 0, stream, tiles_x, tiles_y, sat);
    launch_pdl(k_surv_count, grid, kSurvThreads, 0, stream, sorted_box, counters, sat, tiles_x, grid, cnt,
                                                    keep_flag);
    launch_pdl(k_surv_scan, 1, kMaxTileGrid / 8, 0, stream, cnt, grid, counters, c1);
    launch_pdl(k_surv_scatter, grid, kSurvThreads, 0, stream, sorted_box, order, counters, keep_flag, grid,
                                                      cnt, n_max, chunk_max, s_order, s_box,
                                                      s_offsets, s_chunk_first, status);
}

}  // namespace adr
