// Stage 6, Render (Sec. 3.2.1): pixel-parallel, Gaussian-serial front-to-back
// alpha blending (Eq. 2-3) over each tile's depth-sorted list, with the
// alpha < alpha_low skip, early termination and the per-pixel load l_i
// (Sec. 4.4, Eq. 12).
//
// One CTA of 256 threads per 16x16 tile.  The tile reads a depth-ordered list
// that holds its own list as a subsequence -- the column runs of its column of
// tiles (kRuns) -- or its own list.  Each batch reads up to 2048 runs (8 per
// thread), keeps those whose rows hold the tile's row, compacts the first 256
// kept ones stably into shared memory with their records, and every pixel
// blends them.  Pixels stop early (transmittance below t_min), so a tile
// usually reads only the front of its list; the CTA leaves as soon as every
// pixel has terminated (__syncthreads_count).  Pixel offsets are taken
// relative to the tile origin so the float-float centre collapses to one
// well-conditioned float per Gaussian per tile.
//
// With depth slices (slices.cu) the kernel runs twice per frame: phase 1 over
// slice 0's runs finishes the tiles whose pixels all stopped and saves the
// state of the others; phase 2 resumes those over slice 1's runs.
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kRenderThreads = kTilePixels;

constexpr int kRunFill = 8;   // list entries each thread reads per batch (column runs)

template <bool kRuns>
__global__ void __launch_bounds__(kRenderThreads, 4)   // 4 CTAs per SM: <= 64 registers
k_render(const uint2* __restrict__ ranges, const uint32_t* __restrict__ sorted_gauss,
         const uint2* __restrict__ runs, const float4* __restrict__ rec,
         const FrameParams* __restrict__ fp, float* __restrict__ img,
         float* __restrict__ t_final, int32_t* __restrict__ load, int32_t* __restrict__ last_out,
         int32_t* __restrict__ trav_out, float* __restrict__ tfin, int32_t* __restrict__ lstat,
         SliceState ss) {
    __shared__ float2 s_xy[kRenderThreads];
    __shared__ float4 s_w[kRenderThreads];
    __shared__ float4 s_c[kRenderThreads];
    __shared__ uint32_t s_gid[kRenderThreads];
    __shared__ uint32_t s_wcnt[kRunFill][kRenderThreads / 32];   // kept per (k, warp)
    __shared__ uint32_t s_off[kRunFill * (kRenderThreads / 32)];  // their exclusive prefix
    __shared__ uint32_t s_total;
    __shared__ uint32_t s_next;
    __shared__ uint2 s_range;

    const CamDev cam = fp->cam;
    const SetDev st = fp->st;
    // CTAs walk the tiles column by column: the tiles in flight at once share
    // a few columns' run lists and Gaussian records in L2.
    const int ty = (int)(blockIdx.x % cam.tiles_y), tx = (int)(blockIdx.x / cam.tiles_y);
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool inside = x < cam.width && y < cam.height;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    const float fx = (float)lx, fy = (float)ly;

    // The tile's own list; for column runs, see below.
    uint2 range = kRuns ? make_uint2(0u, 0u) : ranges[ty * cam.tiles_x + tx];
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int32_t count = 0, last = 0, trav = 0;
    bool done = !inside, stopped = false;
    const float alpha_low = st.alpha_low, t_min = st.t_min;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t fbase = 0;   // position in the tile's own list of this batch's first entry
    const int tile_rm = ty * cam.tiles_x + tx;
    const size_t pix = inside ? (size_t)y * cam.width + x : 0;
    if (ss.phase == 2) {   // last slice: resume the tiles the first slice left unfinished
        if (ss.tile_done[tile_rm]) return;
        if (inside) {
            const float4 a = ss.pst[pix];
            const int4 b = ss.pis[pix];
            T = a.x; C0 = a.y; C1 = a.z; C2 = a.w;
            count = b.x; last = b.y; trav = b.z; stopped = b.w != 0;
            done = stopped;
        }
        fbase = ss.tile_fbase[tile_rm];
    }
    if (kRuns) {   // column tx's runs start after the runs of the columns before it
        if (warp == 0) {
            uint32_t before = 0;
            for (int c = lane; c < tx; c += 32) before += ss.col_totals[c];
            before = __reduce_add_sync(0xffffffffu, before);
            if (lane == 0) {
                const bool overflow = (int64_t)ss.col_counters[kCntPairs] > ss.capacity;
                s_range = overflow ? make_uint2(0u, 0u)
                                   : make_uint2(before, before + ss.col_totals[tx]);
            }
        }
        __syncthreads();
        range = s_range;
    }

    // Each batch reads kFill list entries per thread (list order: entry
    // base + k * 256 + thread) and stages the first 256 kept ones; the list
    // resumes at the first kept entry not staged.
    constexpr int kFill = kRuns ? kRunFill : 1;
    uint32_t base = range.x;
    while (base < range.y) {
        if (__syncthreads_count(done) == kRenderThreads) break;
        uint32_t g[kFill], kept[kFill];
        bool keep[kFill];
#pragma unroll
        for (int k = 0; k < kFill; ++k) {
            const uint32_t idx = base + (uint32_t)(k * kRenderThreads) + threadIdx.x;
            g[k] = 0;
            keep[k] = idx < range.y;
            if (keep[k]) {
                if (kRuns) {   // run record: Gaussian, y0 | (h - 1) << 8 | tx << 16
                    const uint2 r = runs[idx];
                    g[k] = r.x;
                    keep[k] = (uint32_t)ty - (r.y & 0xFFu) <= ((r.y >> 8) & 0xFFu);
                } else {
                    g[k] = sorted_gauss[idx];
                }
            }
        }
        // Stable compaction: ballots per (k, warp); warp 0 scans their counts
        // in list order (k-major).
#pragma unroll
        for (int k = 0; k < kFill; ++k) {
            kept[k] = __ballot_sync(0xffffffffu, keep[k]);
            if (lane == 0) s_wcnt[k][warp] = __popc(kept[k]);
        }
        __syncthreads();
        if (warp == 0) {
            constexpr int kN = kFill * (kRenderThreads / 32);
            constexpr int kPer = (kN + 31) / 32;                 // counts per lane
            uint32_t v[kPer], t = 0;
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
                const int i = lane * kPer + e;
                v[e] = i < kN ? (&s_wcnt[0][0])[i] : 0u;
                t += v[e];
            }
            uint32_t x = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t run = x - t;
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
                const int i = lane * kPer + e;
                if (i < kN) s_off[i] = run;
                run += v[e];
            }
            if (lane == 31) s_total = x;
        }
        __syncthreads();
        const uint32_t total = s_total;
        uint32_t before[kFill];
#pragma unroll
        for (int k = 0; k < kFill; ++k) before[k] = s_off[k * (kRenderThreads / 32) + warp];
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < kFill; ++k) {
            if (keep[k]) {
                const uint32_t slot = before[k] + __popc(kept[k] & lt);
                if (slot < (uint32_t)kRenderThreads) s_gid[slot] = g[k];
                else if (slot == (uint32_t)kRenderThreads)
                    s_next = base + (uint32_t)(k * kRenderThreads) + threadIdx.x;
            }
        }
        const int m = (int)min(total, (uint32_t)kRenderThreads);
        __syncthreads();
        const uint32_t next = total > (uint32_t)kRenderThreads
                                  ? s_next
                                  : min(range.y, base + (uint32_t)(kFill * kRenderThreads));
        if ((int)threadIdx.x < m) {
            const uint32_t gi = s_gid[threadIdx.x];
            const float4 r0 = rec[3 * (size_t)gi + 0];
            const float4 w = rec[3 * (size_t)gi + 1];
            // centre relative to the tile origin: (hi - origin) is exact, one rounding for lo
            const float2 c = make_float2(__fadd_rn(__fsub_rn(r0.x, ox), r0.z),
                                         __fadd_rn(__fsub_rn(r0.y, oy), r0.w));
            s_xy[threadIdx.x] = quad_k(c, w);
            s_w[threadIdx.x] = w;
            s_c[threadIdx.x] = rec[3 * (size_t)gi + 2];
        }
        __syncthreads();
        if (!done) {
            int j = 0;
            for (; j < m; ++j) {
                const float4 col = s_c[j];
                const float e = quad_exponent(s_xy[j], s_w[j], col.w, fx, fy);   // log2(sigma) - q log2(e)/2
                const float alpha = fminf(0.99f, ex2_approx(e));
                if (alpha < alpha_low) continue;
                const float test_T = T * (1.f - alpha);
                if (test_T < t_min) { done = stopped = true; ++j; break; }
                const float wgt = alpha * T;
                C0 = fmaf(col.x, wgt, C0);
                C1 = fmaf(col.y, wgt, C1);
                C2 = fmaf(col.z, wgt, C2);
                T = test_T;
                ++count;
                last = fbase + j + 1;
            }
            trav += j;
        }
        fbase += m;
        base = next;
    }
    if (ss.phase == 1) {   // first slice: finish the tile, or keep its state for the last one
        const bool all_done = __syncthreads_count(done) == kRenderThreads;
        if (threadIdx.x == 0) {
            ss.tile_done[tile_rm] = all_done ? 1u : 0u;
            if (!all_done) ss.tile_fbase[tile_rm] = fbase;
        }
        if (!all_done) {
            if (inside) {
                ss.pst[pix] = make_float4(T, C0, C1, C2);
                ss.pis[pix] = make_int4(count, last, trav, stopped ? 1 : 0);
            }
            return;
        }
    }
    if (inside) {
        const size_t hw = (size_t)cam.width * cam.height;
        img[pix] = C0 + T * st.bg[0];
        img[hw + pix] = C1 + T * st.bg[1];
        img[2 * hw + pix] = C2 + T * st.bg[2];
        if (t_final) t_final[pix] = T;
        if (load) load[pix] = count;
        if (last_out) last_out[pix] = last;
        if (trav_out) trav_out[pix] = trav;
        if (tfin) tfin[pix] = T;
        if (lstat) lstat[pix] = count | (stopped ? (int32_t)0x80000000u : 0);
    }
}

}  // namespace

void launch_render(const uint2* ranges, const uint32_t* sorted_gauss, const uint2* runs,
                   const float4* rec, int lists, const FrameParams* fp, int num_tiles, float* img,
                   float* t_final, int32_t* load, int32_t* last, int32_t* trav, float* tfin,
                   int32_t* lstat, const SliceState& ss, cudaStream_t stream) {
    const int tiles = num_tiles;
    if (tiles <= 0) return;
    if (lists == kListsColumns)
        k_render<true><<<tiles, kRenderThreads, 0, stream>>>(ranges, sorted_gauss, runs, rec, fp, img,
                                                             t_final, load, last, trav, tfin, lstat,
                                                             ss);
    else
        k_render<false><<<tiles, kRenderThreads, 0, stream>>>(ranges, sorted_gauss, runs, rec, fp,
                                                              img, t_final, load, last, trav, tfin,
                                                              lstat, ss);
}

}  // namespace adr
