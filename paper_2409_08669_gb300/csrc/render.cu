// Stage 6, Render (Sec. 3.2.1): pixel-parallel, Gaussian-serial front-to-back
// alpha blending (Eq. 2-3) over each tile's depth-sorted list, with the
// alpha < alpha_low skip, early termination and the per-pixel load l_i
// (Sec. 4.4, Eq. 12).
//
// One CTA of 128 threads per 16x16 tile, two pixels per thread.  The tile
// reads a depth-ordered list that holds its own list as a subsequence -- the
// column runs of its column of tiles (kRuns) -- or its own list.  Each batch
// reads up to 2048 runs (16 per thread), keeps those whose rows hold the
// tile's row, compacts the first 256 kept ones stably into shared memory with
// their records, and every pixel blends them.  Pixels stop early (transmittance below t_min), so a tile
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

// One CTA of 128 threads per 16x16 tile.  Warp w renders the 8x8 quadrant
// (w mod 2, w div 2) of the tile; lane l owns the two vertically adjacent
// pixels (l mod 8, 2 (l div 8)) and (l mod 8, 2 (l div 8) + 1) of it, so
// both share fx.  Each pixel's two eigen components u_i = (k_i - w_ix fx) -
// w_iy fy advance together in one paired FP32 FMA (fma.rn.f32x2, each lane
// rounding as the scalar fmaf does), the fx-term is formed once for both
// pixels, and the blend of the two pixels is one paired sequence without
// branches (weight alpha T, then T - alpha T, which is T (1 - alpha) of Eq. 3
// with one rounding fewer): every pixel takes exactly the decisions of
// quad_exponent's scalar evaluation, which the backward uses too.  The loop
// is unrolled by four.
constexpr int kRenderThreads = kTilePixels / 2;
constexpr int kStage = kTilePixels;          // Gaussians staged per batch
constexpr int kRenderWarps = kRenderThreads / 32;
constexpr float kInf = __builtin_huge_valf();


__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Column tx's run range [start, end) in its pass's column lists (empty after
// a pair overflow); warp 0 writes it to *out, the caller synchronises.
__device__ __forceinline__ void column_range(const SliceState& ss, int tx, int lane, int warp,
                                             uint2* out) {
    if (warp != 0) return;
    uint32_t before = 0;
    for (int c = lane; c < tx; c += 32) before += ss.col_totals[c];
    before = __reduce_add_sync(0xffffffffu, before);
    if (lane == 0) {
        const bool overflow = (int64_t)ss.col_counters[kCntPairs] > ss.capacity;
        *out = overflow ? make_uint2(0u, 0u) : make_uint2(before, before + ss.col_totals[tx]);
    }
}

// One batch of a tile's list from its column's runs [base, end): thread t
// reads the packed row intervals of the 16 consecutive runs from a0 + 16 t
// (a0 = base rounded down to a 16-byte boundary: two 16-byte loads), keeps
// those covering row ty, and a block scan of the per-thread counts places
// the first kStage kept ones' Gaussian ids stably in s_gid.  Returns the
// kept count; *next is where the list resumes (the first kept run not
// staged).  Ends with a block barrier.
__device__ __forceinline__ uint32_t stage_column_batch(uint32_t base, uint32_t end, int ty,
                                                       const uint16_t* __restrict__ rows,
                                                       const uint2* __restrict__ runs,
                                                       uint32_t* s_gid, uint32_t* s_wsum,
                                                       uint32_t* s_next, int lane, int warp,
                                                       uint32_t* next) {
    const uint32_t a0 = base & ~7u;
    const uint32_t first = a0 + 16u * threadIdx.x;
    // the thread's runs inside [base, end) as bits 0..15 (first > base only
    // for thread 0, by at most 7)
    const uint32_t lo = base > first ? base - first : 0u;
    const uint32_t hi = end > first ? min(16u, end - first) : 0u;
    const uint32_t in_range = hi > lo ? (0xFFFFu >> (16u - hi)) & (0xFFFFu << lo) : 0u;
    // Row test of two runs per 32-bit word, one per 16-bit lane holding
    // y0 | (h - 1) << 8: a run covers row ty iff y0 <= ty and ty - y0 <= h - 1.
    // Per lane x = ty + 256 - y0 and then (256 + h - 1) - (x mod 256) stay in
    // 1..511, so no lane borrows from the next; bit 8 of x is set iff
    // y0 <= ty, and bit 8 of the second iff ty - y0 <= h - 1.
    const uint32_t t2 = (uint32_t)ty * 0x00010001u + 0x01000100u;
    uint32_t mask = 0;
    const uint4* r4 = reinterpret_cast<const uint4*>(rows + first);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t g0 = first + 8u * (uint32_t)h;
        if (g0 < end) {
            const uint4 q = r4[h];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t x = t2 - (w[j] & 0x00FF00FFu);                   // ty + 256 - y0
                const uint32_t z = ((w[j] >> 8) & 0x00FF00FFu) | 0x01000100u;   // 256 + h - 1
                const uint32_t b = (z - (x & 0x00FF00FFu)) & x & 0x01000100u;  // bits 8, 24
                mask |= (((b >> 8) | (b >> 23)) & 3u) << (8 * h + 2 * j);
            }
        }
    }
    mask &= in_range;
    // block exclusive scan of the kept counts, in thread (= list) order
    const uint32_t cnt = __popc(mask);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yv = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += yv;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t before = incl - cnt, total = 0;
#pragma unroll
    for (int q = 0; q < kRenderWarps; ++q) {
        const uint32_t v = s_wsum[q];
        before += q < warp ? v : 0u;
        total += v;
    }
    uint32_t slot = before;
    while (mask) {
        const int e = __ffs(mask) - 1;
        mask &= mask - 1u;
        if (slot < (uint32_t)kStage) s_gid[slot] = runs[first + (uint32_t)e].x;
        else if (slot == (uint32_t)kStage) *s_next = first + (uint32_t)e;
        ++slot;
    }
    __syncthreads();
    *next = total > (uint32_t)kStage ? *s_next : min(end, a0 + 16u * kRenderThreads);
    return total;
}

// The m staged Gaussians' terms, the centre taken relative to the tile origin
// (ox, oy): (hi - origin) is exact, one rounding for lo.  Ends with a barrier.
__device__ __forceinline__ void stage_records(int m, const uint32_t* s_gid, const float4* __restrict__ rec,
                                              float ox, float oy, float4* s_kl, float4* s_nw,
                                              float4* s_rg, float2* s_bb) {
    for (int sl = threadIdx.x; sl < m; sl += kRenderThreads) {
        const uint32_t gi = s_gid[sl];
        const float4 r0 = rec[3 * (size_t)gi + 0];
        const float4 w = rec[3 * (size_t)gi + 1];
        const float4 col = rec[3 * (size_t)gi + 2];
        const float2 c = make_float2(__fadd_rn(__fsub_rn(r0.x, ox), r0.z),
                                     __fadd_rn(__fsub_rn(r0.y, oy), r0.w));
        const float2 k = quad_k(c, w);
        s_kl[sl] = make_float4(k.x, k.y, col.w, 0.f);   // k1, k2, log2(sigma), -
        s_nw[sl] = make_float4(-w.x, -w.z, -w.y, -w.w);  // -w1x, -w2x, -w1y, -w2y
        s_rg[sl] = make_float4(col.x, col.x, col.y, col.y);
        s_bb[sl] = make_float2(col.z, col.z);
    }
    __syncthreads();
}

// A launch renders a batch of cameras (the serving scheduler's batched
// frames; one camera otherwise): blocks [tile_begin[b], tile_begin[b + 1])
// are camera b's tiles.
// The tile's constants, kept in shared memory so that the blend loop holds
// only its own state in registers: with them, and the pixels' stop positions,
// out of the registers and the single-camera launch indexing no camera array,
// the column-run kernel of one camera fits 56 registers without spilling,
// i.e. 9 CTAs (36 warps) per SM.
struct TileInfo {
    int width, height, tiles_x, tiles_y, tx, ty;
};

#ifndef ADR_RENDER_CTAS
#define ADR_RENDER_CTAS 9   // CTAs per SM: 56 registers, no spills (10: 48 with spills)
#endif
// kBatched: blocks of several cameras (the serving scheduler's batched frames).
template <bool kRuns, bool kBatched>
__global__ void __launch_bounds__(kRenderThreads, ADR_RENDER_CTAS)
k_render(const RenderBatch batch) {
    pdl_prologue();
    int cb = 0;
    if (kBatched) {
#pragma unroll
        for (int q = 1; q < kMaxBatch; ++q) cb += (q < batch.count && (int)blockIdx.x >= batch.tile_begin[q]) ? 1 : 0;
    }
    __shared__ uint32_t s_tstart;
    __shared__ TileInfo s_ti;
    __shared__ float4 s_kl[kStage];    // k1, k2, log2(sigma), -
    __shared__ float4 s_nw[kStage];    // -w1x, -w2x, -w1y, -w2y
    __shared__ float4 s_rg[kStage];    // red, red, green, green
    __shared__ float2 s_bb[kStage];    // blue, blue
    __shared__ uint32_t s_gid[kStage];
    __shared__ int2 s_stop[kRenderThreads];             // each thread's stop positions (0: none)
    __shared__ uint32_t s_wsum[kRenderWarps];           // kept runs per warp
    __shared__ uint32_t s_next;
    __shared__ uint2 s_range;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Warp w renders the 8x8 quadrant (w mod 2, w div 2); lane l the pixels
    // (l mod 8, 2 (l div 8)) and (l mod 8, 2 (l div 8) + 1) of it.
    const int lx = (warp & 1) * 8 + (lane & 7), ly = (warp >> 1) * 8 + 2 * (lane >> 3);
    // Values used before the blend loop only; after it they are read back
    // from s_ti.
    const int tile_index = (int)blockIdx.x - (kBatched ? batch.tile_begin[cb] : 0);
    const CamDev cam = batch.cam[cb].fp->cam;
    // CTAs walk the tiles column by column: the tiles in flight at once share
    // a few columns' run lists and Gaussian records in L2.
    const int ty0 = tile_index % cam.tiles_y, tx0 = tile_index / cam.tiles_y;
    if (threadIdx.x == 0) {
        s_ti = TileInfo{cam.width, cam.height, cam.tiles_x, cam.tiles_y, tx0, ty0};
        if (batch.cam[cb].trace) {
            uint32_t t;
            asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t));
            s_tstart = t;
        }
    }
    const int x0 = tx0 * kTile + lx, ya0 = ty0 * kTile + ly;
    // Each pixel's limit on the exponent: a Gaussian reaches it iff e >= limit.
    // e_low while the pixel blends; +inf for a pixel outside the image or
    // one that stopped (done), so the skip test needs no separate flag.
    const float e_low = batch.cam[cb].fp->st.e_low, t_min = batch.cam[cb].fp->st.t_min;
    float2 elim = make_float2((x0 < cam.width && ya0 < cam.height) ? e_low : kInf,
                              (x0 < cam.width && ya0 + 1 < cam.height) ? e_low : kInf);
    const int tile_rm0 = ty0 * cam.tiles_x + tx0;
    uint2 range = kRuns ? make_uint2(0u, 0u) : batch.cam[cb].ranges[tile_rm0];
    const float2 fx2 = make_float2((float)lx, (float)lx);
    const float2 fya2 = make_float2((float)ly, (float)ly), fyb2 = make_float2((float)(ly + 1), (float)(ly + 1));
    // Per-pixel blend state: pixel a in .x, pixel b in .y.  A pixel's stop
    // position (0 while it blends) lives in s_stop.
    float2 T = make_float2(1.f, 1.f), C0 = make_float2(0.f, 0.f), C1 = C0, C2 = C0;
    int32_t cnt_a = 0, cnt_b = 0, last_a = 0, last_b = 0;
    int2 stop = make_int2(0, 0);
    int32_t fbase = 0;   // position in the tile's own list of this batch's first entry
    if (batch.cam[cb].ss.phase == 2) {   // last slice: resume the tiles the first slice left unfinished
        const SliceState& ss = batch.cam[cb].ss;
        if (ss.tile_done[tile_rm0]) return;
        const size_t pixa = (size_t)ya0 * cam.width + x0;
        // a pixel that stopped keeps its traversal as its stop position
        if (elim.x != kInf) {
            const float4 a = ss.pst[pixa];
            const int4 b = ss.pis[pixa];
            T.x = a.x; C0.x = a.y; C1.x = a.z; C2.x = a.w;
            cnt_a = b.x; last_a = b.y;
            if (b.w != 0) { elim.x = kInf; stop.x = b.z; }
        }
        if (elim.y != kInf) {
            const size_t pixb = pixa + (size_t)cam.width;
            const float4 a = ss.pst[pixb];
            const int4 b = ss.pis[pixb];
            T.y = a.x; C0.y = a.y; C1.y = a.z; C2.y = a.w;
            cnt_b = b.x; last_b = b.y;
            if (b.w != 0) { elim.y = kInf; stop.y = b.z; }
        }
        fbase = ss.tile_fbase[tile_rm0];
    }
    s_stop[threadIdx.x] = stop;
    if (kRuns) {   // column tx's runs start after the runs of the columns before it
        column_range(batch.cam[cb].ss, tx0, lane, warp, &s_range);
    }
    __syncthreads();
    if (kRuns) range = s_range;

    // Each batch stages the first 256 kept entries of the next stretch of the
    // list.  Column runs: thread t reads the packed row intervals of the 16
    // consecutive runs from a0 + 16 t (a0 = the batch start rounded down to a
    // 16-byte boundary: two 16-byte loads), keeps those covering the tile's
    // row, and a block scan of the per-thread counts places them stably;
    // only kept runs' Gaussian ids are fetched.  The list resumes at the
    // first kept entry not staged.  Per-tile lists: every entry is kept.
    uint32_t base = range.x;
    const uint32_t end = range.y;
    while (base < end) {
        if (__syncthreads_count(fminf(elim.x, elim.y) == kInf) == kRenderThreads) break;
        const int tx = s_ti.tx, ty = s_ti.ty;
        uint32_t total, next;
        if (kRuns) {
            total = stage_column_batch(base, end, ty, batch.cam[cb].rows, batch.cam[cb].runs, s_gid,
                                       s_wsum, &s_next, lane, warp, &next);
        } else {
            const uint32_t* __restrict__ sorted_gauss = batch.cam[cb].sorted_gauss;
            total = min(end - base, (uint32_t)kStage);
            for (uint32_t e = threadIdx.x; e < total; e += kRenderThreads) s_gid[e] = sorted_gauss[base + e];
            __syncthreads();
            next = base + total;
        }
        const int m = (int)min(total, (uint32_t)kStage);
        stage_records(m, s_gid, batch.cam[cb].rec, (float)(tx * kTile), (float)(ty * kTile), s_kl, s_nw,
                      s_rg, s_bb);
        if (!__all_sync(0xffffffffu, fminf(elim.x, elim.y) == kInf)) {   // warp-uniform: the loop votes
            // A pixel becomes done only where it stops (its exponent limit
            // then becomes +inf, so no later Gaussian reaches it), and the
            // loop leaves there once every pixel of the warp is done.  The batch goes in
            // windows of 32 positions: bit k of bits_a / bits_b records that
            // pixel a / b blended position j0 + k, and each window's bits are
            // folded into l_i (their count) and the last blended position
            // (their highest bit) when the window ends.
            bool warp_done = false;
#pragma unroll 1
            for (int j0 = 0; j0 < m && !warp_done; j0 += 32) {
                const int len = min(32, m - j0);
                uint32_t bits_a = 0u, bits_b = 0u;
#pragma unroll 4
                for (int k = 0; k < len; ++k) {
                    const int j = j0 + k;
                    const float4 kl = s_kl[j];
                    const float4 nw = s_nw[j];
                    // u = (k - w_x fx) - w_y fy, the fx-term shared, as quad_exponent
                    const float2 in = ffma2(make_float2(nw.x, nw.y), fx2, make_float2(kl.x, kl.y));
                    const float2 ua = ffma2(make_float2(nw.z, nw.w), fya2, in);
                    const float2 ub = ffma2(make_float2(nw.z, nw.w), fyb2, in);
                    // e = log2(sigma) - q log2(e) / 2; alpha = min(0.99, 2^e) (Eq. 2)
                    // reaches alpha_low iff e >= e_low
                    const float ea = fmaf(-ua.x, ua.x, fmaf(-ua.y, ua.y, kl.z));
                    const float eb = fmaf(-ub.x, ub.x, fmaf(-ub.y, ub.y, kl.z));
                    const bool la = ea >= elim.x, lb = eb >= elim.y;
                    if (!__any_sync(0xffffffffu, la || lb)) continue;   // no pixel of the warp reaches alpha_low
                    // Front-to-back step (Eq. 3), both pixels at once: a pixel
                    // that skips has alpha 0 here, so T and C stay as they are.
                    float2 alpha = make_float2(la ? fminf(0.99f, ex2_approx(ea)) : 0.f,
                                               lb ? fminf(0.99f, ex2_approx(eb)) : 0.f);
                    // T (1 - alpha) = T - alpha T
                    float2 wgt = fmul2(alpha, T);
                    float2 test_T = fsub2(T, wgt);
                    // a done pixel keeps T >= t_min, so only a pixel stopping here can vote
                    if (__any_sync(0xffffffffu, fminf(test_T.x, test_T.y) < t_min)) {
                        // rare: a pixel stops before this Gaussian, which it does not blend
                        const int32_t pos = fbase + j + 1;
                        if (test_T.x < t_min) { alpha.x = wgt.x = 0.f; test_T.x = T.x; s_stop[threadIdx.x].x = pos; elim.x = kInf; }
                        if (test_T.y < t_min) { alpha.y = wgt.y = 0.f; test_T.y = T.y; s_stop[threadIdx.x].y = pos; elim.y = kInf; }
                        if (__all_sync(0xffffffffu, fminf(elim.x, elim.y) == kInf)) {   // nothing blends this Gaussian
                            warp_done = true;
                            break;
                        }
                    }
                    const float4 rg = s_rg[j];
                    C0 = ffma2(make_float2(rg.x, rg.y), wgt, C0);
                    C1 = ffma2(make_float2(rg.z, rg.w), wgt, C1);
                    C2 = ffma2(s_bb[j], wgt, C2);
                    T = test_T;
                    const uint32_t bit = 1u << k;
                    // blended: alpha >= alpha_low (> 0) and the pixel did not stop here
                    if (alpha.x > 0.f) bits_a |= bit;
                    if (alpha.y > 0.f) bits_b |= bit;
                }
                cnt_a += __popc(bits_a);
                cnt_b += __popc(bits_b);
                if (bits_a) last_a = fbase + j0 + 32 - __clz(bits_a);   // 1-based position of the highest bit
                if (bits_b) last_b = fbase + j0 + 32 - __clz(bits_b);
            }
        }
        fbase += m;
        base = next;
    }
    stop = s_stop[threadIdx.x];
    const TileInfo ti = s_ti;
    const int x = ti.tx * kTile + lx, ya = ti.ty * kTile + ly;
    const bool in_a = x < ti.width && ya < ti.height, in_b = x < ti.width && ya + 1 < ti.height;
    const int tile_rm = ti.ty * ti.tiles_x + ti.tx;
    const bool stopped_a = stop.x != 0, stopped_b = stop.y != 0;
    // Traversal (positions evaluated): up to the stop, else the whole list seen.
    const int32_t trav_a = stopped_a ? stop.x : fbase, trav_b = stopped_b ? stop.y : fbase;
    const RenderCam& rc = batch.cam[cb];
    if (rc.trace && threadIdx.x == 0) {   // tracing: this tile's CTA
        uint32_t t_end, smid;
        asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t_end));
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        const int ntiles = ti.tiles_x * ti.tiles_y;
        rc.trace[(rc.ss.phase == 2 ? ntiles : 0) + tile_rm] = make_uint4(s_tstart, t_end, smid, (uint32_t)fbase);
    }
    const size_t pixa = (size_t)ya * ti.width + x, pixb = pixa + (size_t)ti.width;
    if (rc.ss.phase == 1) {   // first slice: finish the tile, or keep its state for the last one
        const SliceState& ss = rc.ss;
        const bool all_done = __syncthreads_count(fminf(elim.x, elim.y) == kInf) == kRenderThreads;
        if (threadIdx.x == 0) {
            ss.tile_done[tile_rm] = all_done ? 1u : 0u;
            if (!all_done) ss.tile_fbase[tile_rm] = fbase;
        }
        if (!all_done) {
            if (in_a) {
                ss.pst[pixa] = make_float4(T.x, C0.x, C1.x, C2.x);
                ss.pis[pixa] = make_int4(cnt_a, last_a, trav_a, stopped_a ? 1 : 0);
            }
            if (in_b) {
                ss.pst[pixb] = make_float4(T.y, C0.y, C1.y, C2.y);
                ss.pis[pixb] = make_int4(cnt_b, last_b, trav_b, stopped_b ? 1 : 0);
            }
            return;
        }
    }
    const float bg0 = rc.fp->st.bg[0], bg1 = rc.fp->st.bg[1], bg2 = rc.fp->st.bg[2];
    const size_t hw = (size_t)ti.width * ti.height;
    if (in_a) {
        rc.img[pixa] = C0.x + T.x * bg0;
        rc.img[hw + pixa] = C1.x + T.x * bg1;
        rc.img[2 * hw + pixa] = C2.x + T.x * bg2;
        if (rc.t_final) rc.t_final[pixa] = T.x;
        if (rc.load) rc.load[pixa] = cnt_a;
        if (rc.last) rc.last[pixa] = last_a;
        if (rc.trav) rc.trav[pixa] = trav_a;
        if (rc.tfin) rc.tfin[pixa] = T.x;
        if (rc.lstat) rc.lstat[pixa] = cnt_a | (stopped_a ? (int32_t)0x80000000u : 0);
    }
    if (in_b) {
        rc.img[pixb] = C0.y + T.y * bg0;
        rc.img[hw + pixb] = C1.y + T.y * bg1;
        rc.img[2 * hw + pixb] = C2.y + T.y * bg2;
        if (rc.t_final) rc.t_final[pixb] = T.y;
        if (rc.load) rc.load[pixb] = cnt_b;
        if (rc.last) rc.last[pixb] = last_b;
        if (rc.trav) rc.trav[pixb] = trav_b;
        if (rc.tfin) rc.tfin[pixb] = T.y;
        if (rc.lstat) rc.lstat[pixb] = cnt_b | (stopped_b ? (int32_t)0x80000000u : 0);
    }
}


// f2, heavy tiles across CTAs: the last depth slice with every unfinished
// tile split by pixel halves, two CTAs of 128 threads per tile, CTA h
// rendering rows 8h..8h+7 with one pixel per thread, so each tile runs on
// twice the warps (phase 2, column runs; selected with adr_set_tile_split).
// Each pixel takes exactly the operations of k_render's paired lanes, so the
// image, l_i and every per-pixel output are bit-identical to k_render's.
__global__ void __launch_bounds__(kRenderThreads, 8)
k_render_half(const RenderBatch batch) {
    pdl_prologue();
    const int blk = (int)(blockIdx.x >> 1), half = (int)(blockIdx.x & 1u);
    int cb = 0;
#pragma unroll
    for (int q = 1; q < kMaxBatch; ++q) cb += (q < batch.count && blk >= batch.tile_begin[q]) ? 1 : 0;
    const RenderCam& rc = batch.cam[cb];
    const int tile_index = blk - batch.tile_begin[cb];
    const SliceState& ss = rc.ss;
    __shared__ uint32_t s_tstart;
    if (rc.trace && threadIdx.x == 0) {
        uint32_t t;
        asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t));
        s_tstart = t;
    }
    __shared__ float4 s_kl[kStage];
    __shared__ float4 s_nw[kStage];
    __shared__ float4 s_rg[kStage];
    __shared__ float2 s_bb[kStage];
    __shared__ uint32_t s_gid[kStage];
    __shared__ uint32_t s_wsum[kRenderWarps];
    __shared__ uint32_t s_next;
    __shared__ uint2 s_range;

    const CamDev cam = rc.fp->cam;
    const SetDev st = rc.fp->st;
    const int ty = tile_index % cam.tiles_y, tx = tile_index / cam.tiles_y;
    const int tile_rm = ty * cam.tiles_x + tx;
    if (ss.tile_done[tile_rm]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp w: the 8x4 block (w mod 2, w div 2) of the half; lane l: (l mod 8, l div 8)
    const int lx = (warp & 1) * 8 + (lane & 7), ly = half * 8 + (warp >> 1) * 4 + (lane >> 3);
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool in_p = x < cam.width && y < cam.height;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    const float fx = (float)lx, fy = (float)ly;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int32_t cnt = 0, last = 0, stop = 0;
    bool done = !in_p;
    const float e_low = st.e_low, t_min = st.t_min;
    const size_t pix = in_p ? (size_t)y * cam.width + x : 0;
    if (in_p) {   // resume the state slice 0 left
        const float4 a = ss.pst[pix];
        const int4 b = ss.pis[pix];
        T = a.x; C0 = a.y; C1 = a.z; C2 = a.w;
        cnt = b.x; last = b.y; done = b.w != 0; stop = done ? b.z : 0;
    }
    int32_t fbase = ss.tile_fbase[tile_rm];
    column_range(ss, tx, lane, warp, &s_range);
    __syncthreads();
    const uint2 range = s_range;
    uint32_t base = range.x;
    while (base < range.y) {
        if (__syncthreads_count(done) == kRenderThreads) break;
        uint32_t next;
        const uint32_t total = stage_column_batch(base, range.y, ty, rc.rows, rc.runs, s_gid, s_wsum,
                                                  &s_next, lane, warp, &next);
        const int m = (int)min(total, (uint32_t)kStage);
        stage_records(m, s_gid, rc.rec, ox, oy, s_kl, s_nw, s_rg, s_bb);
        if (!__all_sync(0xffffffffu, done)) {
#pragma unroll 1
            for (int j = 0; j < m; ++j) {
                const float4 kl = s_kl[j];
                const float4 nw = s_nw[j];
                const float u1 = fmaf(nw.z, fy, fmaf(nw.x, fx, kl.x));
                const float u2 = fmaf(nw.w, fy, fmaf(nw.y, fx, kl.y));
                const float e = fmaf(-u1, u1, fmaf(-u2, u2, kl.z));
                bool l = !done && e >= e_low;
                if (!__any_sync(0xffffffffu, l)) continue;
                const float alpha = l ? fminf(0.99f, ex2_approx(e)) : 0.f;
                float wgt = __fmul_rn(alpha, T);
                float test_T = __fsub_rn(T, wgt);
                if (__any_sync(0xffffffffu, test_T < t_min)) {
                    if (test_T < t_min) { wgt = 0.f; test_T = T; l = false; stop = fbase + j + 1; done = true; }
                    if (__all_sync(0xffffffffu, done)) break;
                }
                const float4 rg = s_rg[j];
                C0 = fmaf(rg.x, wgt, C0);
                C1 = fmaf(rg.z, wgt, C1);
                C2 = fmaf(s_bb[j].x, wgt, C2);
                T = test_T;
                if (l) { ++cnt; last = fbase + j + 1; }
            }
        }
        fbase += m;
        base = next;
    }
    const bool stopped = stop != 0;
    const int32_t trav = stopped ? stop : fbase;
    if (rc.trace && threadIdx.x == 0 && half == 0) {   // tracing: the tile's first half
        uint32_t t_end, smid;
        asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t_end));
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        rc.trace[cam.tiles_x * cam.tiles_y + tile_rm] = make_uint4(s_tstart, t_end, smid, (uint32_t)fbase);
    }
    if (in_p) {
        const size_t hw = (size_t)cam.width * cam.height;
        rc.img[pix] = C0 + T * st.bg[0];
        rc.img[hw + pix] = C1 + T * st.bg[1];
        rc.img[2 * hw + pix] = C2 + T * st.bg[2];
        if (rc.t_final) rc.t_final[pix] = T;
        if (rc.load) rc.load[pix] = cnt;
        if (rc.last) rc.last[pix] = last;
        if (rc.trav) rc.trav[pix] = trav;
        if (rc.tfin) rc.tfin[pix] = T;
        if (rc.lstat) rc.lstat[pix] = cnt | (stopped ? (int32_t)0x80000000u : 0);
    }
}

}  // namespace

void launch_render(const RenderBatch& batch, cudaStream_t stream) {
    if (batch.count < 1 || batch.count > kMaxBatch) return;
    const int tiles = batch.tile_begin[batch.count];
    if (tiles <= 0) return;
    if (batch.lists == kListsColumns && batch.split && batch.cam[0].ss.phase == 2)
        launch_pdl(k_render_half, 2 * tiles, kRenderThreads, 0, stream, batch);
    else if (batch.lists == kListsColumns)
        launch_pdl(batch.count > 1 ? k_render<true, true> : k_render<true, false>, tiles, kRenderThreads, 0,
                   stream, batch);
    else
        launch_pdl(batch.count > 1 ? k_render<false, true> : k_render<false, false>, tiles, kRenderThreads,
                   0, stream, batch);
}

}  // namespace adr
