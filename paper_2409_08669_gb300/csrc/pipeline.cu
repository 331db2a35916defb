// Stage orchestration shared by every entry point: enqueues the kernels of
// the six-stage rasterizer (Sec. 3.2.1) on one stream for a Workspace,
// wherever its buffers come from.
#include <algorithm>

#include "adr_internal.cuh"

namespace adr {

const char* kernel_name(int id) {
    static const char* names[kKernelCount] = {
        "preprocess", "depth_pass", "scan_tiles", "tile_ranges",
        "tile_count_columns", "tile_scatter_columns", "tile_count_rows", "tile_scatter_rows",
        "tile_count_scan", "render", "render_backward", "preprocess_backward", "slice", "colors"};
    return (id >= 0 && id < kKernelCount) ? names[id] : "?";
}

void Profiler::begin(int kernel, cudaStream_t s) {
    if (used >= kMaxEntries) return;
    while (created < 2 * (used + 1)) {
        if (cudaEventCreate(&ev[created]) != cudaSuccess) return;
        ++created;
    }
    id[used] = kernel;
    cudaEventRecord(ev[2 * used], s);
}

void Profiler::end(cudaStream_t s) {
    if (used >= kMaxEntries || created < 2 * (used + 1)) return;
    cudaEventRecord(ev[2 * used + 1], s);
    ++used;
}

// Times one launch when the workspace has a profiler.
#define TIMED(ws, kid, stream, launch)                      \
    do {                                                    \
        if ((ws).prof) (ws).prof->begin((kid), (stream));   \
        launch;                                             \
        if ((ws).prof) (ws).prof->end(stream);              \
    } while (0)

namespace {
__global__ void k_set_frame_params(FrameParams p, FrameParams* __restrict__ out) {
    pdl_prologue(); *out = p; }
}  // namespace

void launch_set_frame_params(const FrameParams& p, FrameParams* d_fp, cudaStream_t stream) {
    launch_pdl(k_set_frame_params, 1, 1, 0, stream, p, d_fp);
}

const void* set_frame_params_kernel() { return reinterpret_cast<const void*>(&k_set_frame_params); }

void count_stage(std::atomic<uint32_t>& calls, const Workspace& ws, cudaStream_t stream) {
    // The device tag is (stage count) * 8 + pass in 32 bits; clear the lookback
    // words well before it wraps so no stale word can match a new pass.
    const uint32_t c = calls.fetch_add(1) + 1;
    if ((c & ((1u << 28) - 1u)) == 0)
        cudaMemsetAsync(ws.lookback, 0, ws.lookback_words * sizeof(unsigned long long), stream);
}

void fill_frame_state(FrameState& fs, int64_t n, const CamDev& cam, const SetDev& st) {
    fs.n = n;
    fs.cam = cam;
    fs.st = st;
    fs.num_tiles = cam.tiles_x * cam.tiles_y;
    fs.order = nullptr;
    fs.sorted_gauss = nullptr;
}

// Before Preprocess: the stage tag, the frame parameters and the counters.
static void preprocess_head(const Workspace& ws, FrameState& fs, std::atomic<uint32_t>& epoch,
                            cudaStream_t stream, bool set_params) {
    count_stage(epoch, ws, stream);
    if (set_params) launch_set_frame_params(FrameParams{fs.cam, fs.st}, ws.d_fp, stream);
    cudaMemsetAsync(ws.counters, 0, kCntSlots * sizeof(uint32_t), stream);
    cudaMemsetAsync(ws.hist, 0, kHistWords * sizeof(uint32_t), stream);
}

static PreprocessOut preprocess_out(const Workspace& ws) {
    return PreprocessOut{ws.d_fp, ws.d_stage, ws.rec, ws.aux, ws.depth_key, ws.gbox};
}

// After Preprocess: the Gaussians by view depth, then the run scan.
static void preprocess_tail(const Workspace& ws, FrameState& fs, cudaStream_t stream) {
    const int64_t n = fs.n;
    // Gaussians by view depth: 4 stable 8-bit passes over the V Gaussians with
    // tiles (the first pass drops the others, key 0xFFFFFFFF, and counts the
    // V).  The last pass carries the packed rectangles into depth order.
    const uint32_t* kin = ws.depth_key;
    const uint32_t* vin = nullptr;
    for (int p = 0; p < kMaxPasses; ++p) {
        TIMED(ws, kKDepthPass, stream,
              launch_depth_pass(kin, vin, ws.gkeys[p & 1], ws.gvals[p & 1], n,
                                ws.counters + kCntDepthKept, p == 0, 8 * p, ws.tcounts,
                                ws.hist + p * kRadix, p + 1 == kMaxPasses ? ws.gbox : nullptr,
                                p + 1 == kMaxPasses ? ws.sorted_box : nullptr, ws.status,
                                ws.sort_grid, stream));
        kin = ws.gkeys[p & 1];
        vin = ws.gvals[p & 1];
    }
    fs.order = vin;
    // Stage 2 (+ bookkeeping for stage 3): scan of tile counts in depth order
    // over the V Gaussians with tiles.
    const EpochRef ep{ws.d_stage, (uint32_t)kMaxPasses};
    TIMED(ws, kKScanTiles, stream,
          launch_scan_tiles(ws.sorted_box, n, ws.capacity, ws.offsets, ws.chunk_first, ws.lookback,
                            ep, ws.counters, ws.status, ws.scan_grid, stream));
}

void enqueue_preprocess(const Workspace& ws, FrameState& fs, std::atomic<uint32_t>& epoch,
                        const float* means, const float* scales, const float* rots,
                        const float* opac, const float* sh, cudaStream_t stream,
                        bool set_params, bool defer_colors) {
    preprocess_head(ws, fs, epoch, stream, set_params);
    fs.defer_colors = defer_colors;
    fs.means = means;
    fs.sh = sh;
    // Stage 1: per-Gaussian projection, covariance, early cull and (unless
    // deferred to Render) the SH colour.
    PreprocessBatch pb;
    pb.count = 1;
    pb.cam[0] = preprocess_out(ws);
    TIMED(ws, kKPreprocess, stream,
          launch_preprocess((int)fs.n, means, scales, rots, opac, defer_colors ? nullptr : sh, pb,
                            stream));
    preprocess_tail(ws, fs, stream);
}

// Stage 4, pass 2 and stage 5: the pairs of the column runs grouped by tile
// row (per-tile lists), then every tile's [start, end).
static void enqueue_tile_pass2(const Workspace& ws, FrameState& fs, cudaStream_t stream) {
    cudaMemsetAsync(ws.ttotals + kRadix, 0, kRadix * sizeof(uint32_t), stream);
    cudaMemsetAsync(ws.tile_counts, 0, (size_t)fs.num_tiles * sizeof(uint32_t), stream);
    if (fs.n > 0 && fs.order) {
        // The runs' pair counts vary, so the pass uses many small run ranges
        // (kMaxTileGrid CTAs) that the hardware schedules as CTAs finish.
        const int G2 = kMaxTileGrid;
        TIMED(ws, kKTileCountRows, stream,
              launch_tile_count_rows(ws.pruns, ws.counters, ws.capacity, fs.cam.tiles_x, fs.num_tiles,
                                     ws.tcounts, ws.ttotals + kRadix, ws.tile_counts, ws.status, G2,
                                     stream));
        TIMED(ws, kKTileCountScan, stream,
              launch_tile_count_scan(ws.tcounts, ws.ttotals + kRadix, G2, stream));
        TIMED(ws, kKTileScatterRows, stream,
              launch_tile_scatter_rows(ws.pruns, ws.counters, ws.capacity, ws.tcounts, ws.pgauss,
                                       ws.status, G2, fs.cam.tiles_y, stream));
    }
    TIMED(ws, kKTileRanges, stream,
          launch_tile_ranges(ws.tile_counts, fs.num_tiles, ws.counters, ws.capacity, ws.ranges,
                             stream));
    fs.sorted_gauss = ws.pgauss;
    fs.lists = kListsTiles;
}

// Stage 3-4, pass 1: the column runs of `src`'s Gaussians, generated on chip
// and grouped by tile column (stage 5, each column's [start, end), is the
// prefix of the per-column totals, which Render takes itself).
static void enqueue_pass1(const Workspace& ws, const FrameState& fs, const PairSource& src,
                          cudaStream_t stream) {
    const int G = ws.tile_grid;
    cudaMemsetAsync(ws.ttotals, 0, kRadix * sizeof(uint32_t), stream);
    if (fs.n > 0 && fs.order) {
        TIMED(ws, kKTileCountColumns, stream,
              launch_tile_count_columns(src, ws.tcounts, ws.ttotals, ws.status, G, stream));
        TIMED(ws, kKTileCountScan, stream, launch_tile_count_scan(ws.tcounts, ws.ttotals, G, stream));
        TIMED(ws, kKTileScatterColumns, stream,
              launch_tile_scatter_columns(src, ws.tcounts, ws.pruns, ws.prows, ws.status, G, stream));
    }
}

// The Gaussians with tiles in depth order (all of them, or a slice's).
static PairSource pair_source(const Workspace& ws, const FrameState& fs, int which) {
    PairSource src;
    src.capacity = ws.capacity;
    src.tiles_x = fs.cam.tiles_x;
    if (which == 1) {   // slice 1: the compacted Gaussians behind slice 0
        src.order = ws.s_order;
        src.offsets = ws.s_offsets;
        src.sorted_box = ws.s_box;
        src.chunk_first = ws.s_chunk_first;
        src.counters = ws.slice_counters + kCntSlots;
    } else {            // all Gaussians, or (which == 0) the nearest ones of slice 0
        src.order = fs.order;
        src.offsets = ws.offsets;
        src.sorted_box = ws.sorted_box;
        src.chunk_first = ws.chunk_first;
        src.counters = which == 0 ? ws.slice_counters : ws.counters;
    }
    return src;
}

void enqueue_sort(const Workspace& ws, FrameState& fs, std::atomic<uint32_t>& epoch,
                  cudaStream_t stream) {
    (void)epoch;   // the tile sort has no lookback words
    fs.runs = ws.pruns;
    fs.rows = ws.prows;
    fs.sorted_gauss = nullptr;
    fs.lists = kListsColumns;
    fs.sliced = fs.allow_slices && ws.pst != nullptr && kSliceDiv > 0;
    if (fs.sliced) {
        // Slice 0: the nearest Gaussians' runs; Render builds slice 1 from what
        // its pixels still need.
        cudaMemsetAsync(ws.slice_counters, 0, 2 * kCntSlots * sizeof(uint32_t), stream);
        launch_slice0_setup(ws.counters, ws.offsets, ws.slice_counters, stream);
        enqueue_pass1(ws, fs, pair_source(ws, fs, 0), stream);
        fs.runs_held = kRunsSlice0;
    } else {
        enqueue_pass1(ws, fs, pair_source(ws, fs, -1), stream);
        fs.runs_held = kRunsAll;
    }
}

void enqueue_tile_lists(const Workspace& ws, FrameState& fs, cudaStream_t stream) {
    if (fs.lists == kListsTiles) return;
    if (fs.runs_held != kRunsAll) {   // the column runs of every Gaussian first
        enqueue_pass1(ws, fs, pair_source(ws, fs, -1), stream);
        fs.runs_held = kRunsAll;
    }
    enqueue_tile_pass2(ws, fs, stream);
}

// Render's inputs and outputs for one camera, in phase 0 (the whole list),
// 1 (slice 0) or 2 (slice 1).
static RenderCam render_cam(const Workspace& ws, const FrameState& fs, float* img, float* t_final,
                            int32_t* load, int phase) {
    RenderCam rc;
    rc.ranges = ws.ranges;
    rc.sorted_gauss = fs.sorted_gauss;
    rc.runs = fs.runs;
    rc.rows = fs.rows;
    rc.rec = ws.rec;
    rc.fp = ws.d_fp;
    rc.img = img;
    rc.t_final = t_final;
    rc.load = load;
    rc.last = ws.last;
    rc.trav = ws.trav;
    rc.tfin = ws.tfin;
    rc.lstat = ws.lstat;
    rc.trace = ws.tile_trace;
    rc.ss.col_totals = ws.ttotals;
    rc.ss.capacity = ws.capacity;
    rc.ss.phase = phase;
    rc.ss.col_counters = phase == 0 ? ws.counters
                                    : ws.slice_counters + (phase == 2 ? kCntSlots : 0);
    if (phase != 0) {
        rc.ss.pst = ws.pst;
        rc.ss.pis = ws.pis;
        rc.ss.tile_done = ws.tile_done;
        rc.ss.tile_fbase = ws.tile_fbase;
    }
    return rc;
}

// The SH colours of the Gaussians a Render phase blends: phase 0 every
// Gaussian with tiles, phase 1 the nearest K0 (slice 0), phase 2 slice 1's.
static void enqueue_colors(const Workspace& ws, const FrameState& fs, int phase, cudaStream_t stream) {
    if (!fs.defer_colors || fs.n <= 0 || !fs.order || !fs.sh) return;
    const uint32_t* ids = phase == 2 ? ws.s_order : fs.order;
    const uint32_t* count = phase == 0   ? ws.counters + kCntVisible
                            : phase == 1 ? ws.slice_counters + kCntVisible
                                         : ws.slice_counters + kCntSlots + kCntVisible;
    TIMED(ws, kKColors, stream,
          launch_colors(ids, count, fs.means, fs.sh, ws.d_fp, ws.rec, ws.sm_count, stream));
}

// One Render launch over the items' cameras (all of the same list kind).
static void render_launch(const BatchItem* items, int count, int phase, cudaStream_t stream) {
    RenderBatch rb;
    rb.count = count;
    rb.lists = phase == 0 ? items[0].fs->lists : kListsColumns;
    rb.split = phase == 2 && items[0].fs->split_last_slice ? 1 : 0;
    for (int b = 0; b < count; ++b) {
        const BatchItem& it = items[b];
        rb.cam[b] = render_cam(*it.ws, *it.fs, it.img, it.t_final, it.load, phase);
        rb.tile_begin[b + 1] = rb.tile_begin[b] + it.fs->num_tiles;
    }
    TIMED(*items[0].ws, kKRender, stream, launch_render(rb, stream));
}

// Slice 1 of a sliced frame: the Gaussians behind slice 0 that touch an
// unfinished tile, with their run offsets, then their column runs.
static void slice1_runs(const Workspace& ws, FrameState& fs, cudaStream_t stream) {
    uint32_t* c1 = ws.slice_counters + kCntSlots;
    // The survivor selection walks the Gaussians behind slice 0 in 256-item steps,
    // each CTA its own range: ~1024 Gaussians per CTA keeps each CTA's chain of
    // steps short (2048 CTAs at 3M Gaussians: 1.49 -> 1.52 k frames/s).
    const int surv_grid = (int)std::min<int64_t>(kMaxTileGrid, std::max<int64_t>(ws.sort_grid, fs.n / 1024));
    TIMED(ws, kKSlice, stream,
          launch_survivors(ws.tile_done, fs.cam.tiles_x, fs.cam.tiles_y, ws.sat, ws.sorted_box,
                           fs.order, ws.counters, surv_grid, ws.surv_cnt, ws.surv_flag, ws.max_n,
                           ws.capacity / kSortChunk + 2, ws.s_order, ws.s_box, ws.s_offsets,
                           ws.s_chunk_first, c1, ws.status, stream));
    enqueue_pass1(ws, fs, pair_source(ws, fs, 1), stream);
    fs.runs_held = kRunsSlice1;
}

// Runs fn(b, stream_b) for every item, on the item's own stream when a batch
// has them (forked from and joined back into `stream` by events), else on
// `stream`.
template <class Fn>
static void per_item(const BatchItem* items, int count, cudaStream_t stream, const BatchStreams* bs,
                     Fn fn) {
    if (!bs || count == 1) {
        for (int b = 0; b < count; ++b) fn(b, stream);
        return;
    }
    cudaEventRecord(bs->fork, stream);
    for (int b = 0; b < count; ++b) {
        cudaStreamWaitEvent(bs->side[b], bs->fork, 0);
        fn(b, bs->side[b]);
        cudaEventRecord(bs->join[b], bs->side[b]);
    }
    for (int b = 0; b < count; ++b) cudaStreamWaitEvent(stream, bs->join[b], 0);
}

static void render_items(const BatchItem* items, int count, cudaStream_t stream,
                         const BatchStreams* bs) {
    for (int b = 0; b < count; ++b)   // tracing: this frame's tiles only
        if (items[b].ws->tile_trace)
            cudaMemsetAsync(items[b].ws->tile_trace, 0, (size_t)2 * items[b].fs->num_tiles * sizeof(uint4),
                            stream);
    // Stage 6.
    if (!items[0].fs->sliced) {
        per_item(items, count, stream, bs,
                 [&](int b, cudaStream_t s) { enqueue_colors(*items[b].ws, *items[b].fs, 0, s); });
        render_launch(items, count, 0, stream);
        return;
    }
    per_item(items, count, stream, bs, [&](int b, cudaStream_t s) {
        const BatchItem& it = items[b];
        if (it.fs->runs_held != kRunsSlice0) enqueue_pass1(*it.ws, *it.fs, pair_source(*it.ws, *it.fs, 0), s);
        it.fs->runs_held = kRunsSlice0;
        enqueue_colors(*it.ws, *it.fs, 1, s);
    });
    render_launch(items, count, 1, stream);
    per_item(items, count, stream, bs, [&](int b, cudaStream_t s) {
        slice1_runs(*items[b].ws, *items[b].fs, s);
        enqueue_colors(*items[b].ws, *items[b].fs, 2, s);
    });
    render_launch(items, count, 2, stream);
}

void enqueue_render(const Workspace& ws, FrameState& fs, float* img, float* t_final,
                    int32_t* load, cudaStream_t stream) {
    const BatchItem it{&ws, &fs, nullptr, img, t_final, load};
    render_items(&it, 1, stream, nullptr);
}

void enqueue_frame_batch(const BatchItem* items, int count, const float* means, const float* scales,
                         const float* rots, const float* opac, const float* sh, cudaStream_t stream,
                         const BatchStreams* bs, bool set_params) {
    if (count < 1 || count > kMaxBatch) return;
    PreprocessBatch pb;
    pb.count = count;
    for (int b = 0; b < count; ++b) {
        const BatchItem& it = items[b];
        preprocess_head(*it.ws, *it.fs, *it.epoch, stream, set_params);
        it.fs->defer_colors = false;
        it.fs->means = means;
        it.fs->sh = sh;
        pb.cam[b] = preprocess_out(*it.ws);
    }
    // Stage 1 for every camera in one grid: the scene is read once.
    TIMED(*items[0].ws, kKPreprocess, stream,
          launch_preprocess((int)items[0].fs->n, means, scales, rots, opac, sh, pb, stream));
    // Stages 2-5 per camera, side by side.
    per_item(items, count, stream, bs, [&](int b, cudaStream_t s) {
        preprocess_tail(*items[b].ws, *items[b].fs, s);
        enqueue_sort(*items[b].ws, *items[b].fs, *items[b].epoch, s);
    });
    render_items(items, count, stream, bs);
}

void enqueue_backward(const Workspace& ws, const FrameState& fs, const float* means,
                      const float* scales, const float* rots, const float* opac, const float* sh,
                      const float* dl_dimg, const float* dl_dload, float* g_means, float* g_scales,
                      float* g_rots, float* g_opac, float* g_sh, cudaStream_t stream) {
    if (fs.n <= 0) return;
    cudaMemsetAsync(ws.g2d, 0, (size_t)fs.n * 9 * sizeof(float), stream);
    TIMED(ws, kKRenderBackward, stream,
          launch_render_backward(ws.ranges, fs.sorted_gauss, ws.rec, ws.aux, ws.d_fp, fs.num_tiles,
                                 ws.last, ws.tfin, ws.lstat, dl_dimg, dl_dload, ws.g2d, stream));
    TIMED(ws, kKPreprocessBackward, stream,
          launch_preprocess_backward((int)fs.n, means, scales, rots, opac, sh, ws.d_fp, ws.gbox,
                                     ws.aux, ws.g2d, g_means, g_scales, g_rots, g_opac, g_sh,
                                     stream));
}

}  // namespace adr
