// Internal declarations shared by the CUDA translation units of libadr.so.
// Nothing here is part of the public C ABI (see include/adr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include "adr.h"
#include "status_bits.h"   // device-side error word bits and their adr_status

namespace adr {

// Programmatic dependent launch.  The frame's kernels follow one another on
// one stream; each is launched with programmatic stream serialization, so it
// is scheduled as soon as every block of the kernel before it has started
// (pdl_prologue's trigger) instead of after that kernel has drained, and its
// blocks then wait in pdl_prologue until the kernel before has completed and
// its writes are visible.  pdl_prologue() is the first statement of every
// kernel launched this way; on a normal launch both instructions are no-ops.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args&&... args) {
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

constexpr int kTile = ADR_TILE;          // 16x16 pixel tiles (Sec. 3.2)
constexpr int kTilePixels = kTile * kTile;
constexpr int kMaxBatch = 4;             // cameras of one batched frame (serving)

// Camera as the kernels see it.
struct CamDev {
    float v[12];          // rows 0..2 of the world->camera matrix
    float fx, fy, cx, cy;
    float near_z;
    float cam_pos[3];
    float tan_fovx, tan_fovy;
    int width, height;
    int tiles_x, tiles_y;
};

struct SetDev {
    int mode;
    float alpha_low, t_min, lowpass, jac_clamp;
    // log2(alpha_low) rounded once to FP32 on the host: Render and its
    // backward take a pair's alpha < alpha_low skip as e < e_low on the
    // exponent e of alpha = min(0.99, 2^e), so both decide it identically
    // without evaluating 2^e for the pairs they skip.
    float e_low;
    float bg[3];
    int sh_degree;
    int rect_rule;
    int load_grad;
};

// Camera and settings of a frame, read by the kernels from device memory so a
// captured CUDA graph can be replayed for another camera by updating them.
struct FrameParams {
    CamDev cam;
    SetDev st;
};

// Decoupled-lookback pass tag: epoch = (*stage) * 8 + pass, where *stage is a
// device counter bumped by the first kernel of every preprocess call, so every
// pass (also in a replayed graph) gets a tag no stale word carries.
struct EpochRef {
    const uint32_t* stage;
    uint32_t pass;
};

// Bounded waits: a decoupled-lookback wait polls at most kLookbackSpinLimit
// times (about 0.1-0.4 s with its back-off) before it gives up, sets
// kErrLookback and lets the kernel return.
constexpr int kLookbackSpinLimit = 1 << 22;
// Testing hook of that failure path (adr_test_lookback_expiry): chunk
// `withhold` of the run scan never publishes its prefix, and every wait gives
// up after `spin_limit` polls.  withhold = 0xFFFFFFFF: normal operation.
struct LookbackTest {
    uint32_t withhold = 0xFFFFFFFFu;
    int spin_limit = kLookbackSpinLimit;
};
LookbackTest lookback_test();

// Per-Gaussian render record, three float4 per Gaussian:
//   rec[3g+0] = (px_hi, py_hi, px_lo, py_lo)   pixel centre as a float-float pair
//   rec[3g+1] = (w1x, w1y, w2x, w2y)           q(d) = d^T Sigma'^-1 d = 2/log2(e) *
//                                              ((w1.d)^2 + (w2.d)^2), eigen form
//   rec[3g+2] = (red, green, blue, log2(opacity))
// and an auxiliary record (inspection, backward):
//   aux[2g+0] = (conic_a, conic_b, conic_c, opacity)
//   aux[2g+1] = (r_x, r_y, depth, lambda'_max)
constexpr int kRecFloat4 = 3;
constexpr int kAuxFloat4 = 2;

// Radix-sort launch geometry: 256 threads, 16 keys per thread.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortChunk = kSortThreads * kSortItems;   // 4096 keys per chunk
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 4;                           // up to 32 key bits
constexpr int kMaxTiles = 1 << 16;                      // tile ids sort in two 8-bit passes
constexpr int kMaxTileGrid = 2048;                      // CTAs of a tile-sort pass (bounds tcounts)
// Largest scene a context or serving slot accepts: the per-Gaussian kernels
// index their packed arrays as 4 * i + c with a 32-bit thread index i.
constexpr int64_t kMaxGaussians = int64_t(1) << 29;

// Per-call counters kept on the device.
enum Counter : int {
    kCntPairs = 0,        // number of pairs P (sum of tiles over Gaussians), saturating
    kCntVisible = 1,      // Gaussians with at least one tile (they sort first by depth)
    kCntScanTicket = 2,   // chunk ticket of the tile-count scan
    kCntRuns = 3,         // number of column runs C (sum of rectangle widths), saturating
    kCntDepthKept = 4,    // Gaussians with tiles, counted by the first depth pass
    kCntScanFailed = 5,   // non-zero: a lookback wait of the run scan gave up (the frame
                          // is then skipped: its pair count reads as saturated)
                          // words 6-7: unused
    kCntPairs64 = 8,      // words 8-9: P as a 64-bit sum
    kCntSlots = 16
};

// Optional per-launch timing with CUDA events recorded on the launching
// stream (adr_profile_enable / adr_profile_read).
enum KernelId : int {
    kKPreprocess = 0, kKDepthPass, kKScanTiles, kKTileRanges, kKTileCountColumns,
    kKTileScatterColumns, kKTileCountRows, kKTileScatterRows, kKTileCountScan, kKRender,
    kKRenderBackward, kKPreprocessBackward, kKSlice, kKColors, kKernelCount
};
const char* kernel_name(int id);
struct Profiler {
    static constexpr int kMaxEntries = 8192;
    cudaEvent_t ev[2 * kMaxEntries];
    int id[kMaxEntries];
    int used = 0, created = 0;
    void begin(int kernel, cudaStream_t s);
    void end(cudaStream_t s);
};

// Device buffers one frame needs.  The context path allocates them with
// cudaMalloc; the allocation-free path carves them out of a static array.
struct Workspace {
    int64_t max_n = 0, capacity = 0;       // Gaussians, Gaussian-tile pairs
    int max_tiles = 0;
    int sm_count = 0, sort_grid = 0, scan_grid = 0, tile_grid = 0;
    float4* rec = nullptr;                 // [max_n * kRecFloat4]
    float4* aux = nullptr;                 // [max_n * kAuxFloat4]
    uint32_t* depth_key = nullptr;         // [max_n]
    uint32_t* offsets = nullptr;           // [max_n]
    uint32_t* gbox = nullptr;              // [max_n] packed tile rectangle per Gaussian (all ones: none)
    uint32_t* sorted_box = nullptr;        // [max_n] the same per depth-order position
    uint32_t* gkeys[2] = {nullptr, nullptr};   // [max_n] each
    uint32_t* gvals[2] = {nullptr, nullptr};   // [max_n] each
    uint2* pruns = nullptr;                // [capacity] column runs grouped by tile column
    uint16_t* prows = nullptr;             // [capacity] their row intervals y0 | (h - 1) << 8
    uint32_t* pgauss = nullptr;            // [capacity] Gaussian ids of the pairs by (tile, depth)
    uint32_t* tcounts = nullptr;           // [kRadix * kMaxTileGrid] per-(digit, CTA) counts / starts
    uint32_t* ttotals = nullptr;           // [2 * kRadix] per-digit totals of the two tile passes
    uint32_t* tile_counts = nullptr;       // [max_tiles] pairs per tile
    uint32_t* chunk_first = nullptr;       // [capacity / kSortChunk + 2]
    uint2* ranges = nullptr;               // [max_tiles]
    int32_t* last = nullptr;               // [max pixels]
    int32_t* trav = nullptr;               // [max pixels]
    float* tfin = nullptr;                 // [max pixels] final transmittance of the last render
    int32_t* lstat = nullptr;              // [max pixels] l_i | terminated << 31 of the last render
    float* g2d = nullptr;                  // [max_n * 9] backward: dL/d(px, py, conic, sigma, rgb)
    double* load_sums = nullptr;           // [4] load-balancing loss moments
    uint32_t* hist = nullptr;              // [kHistWords]
    uint32_t* counters = nullptr;          // [kCntSlots]
    uint32_t* status = nullptr;            // [4]
    unsigned long long* lookback = nullptr;
    size_t lookback_words = 0;             // (max_n / kSortChunk + 2) * kRadix
    Profiler* prof = nullptr;              // non-null: time every launch
    uint4* tile_trace = nullptr;           // non-null: [2 * max_tiles] Render's per-tile trace
    FrameParams* d_fp = nullptr;           // [1] camera + settings of the current frame
    uint32_t* d_stage = nullptr;           // [1] stage counter (see EpochRef)
    // Depth slices of the forward frame (slices.cu); all null: one slice.
    uint32_t* slice_counters = nullptr;    // [2 * kCntSlots] counter blocks of slices 0 and 1
    uint32_t* s_order = nullptr;           // [max_n] slice-1 Gaussians in depth order
    uint32_t* s_box = nullptr;             // [max_n] their packed rectangles
    uint32_t* s_offsets = nullptr;         // [max_n] their run offsets
    uint32_t* s_chunk_first = nullptr;     // [capacity / kSortChunk + 2]
    uint32_t* surv_cnt = nullptr;          // [2 * kMaxTileGrid] per-CTA kept counts and runs
    uint8_t* surv_flag = nullptr;          // [max_n] kept flag per depth-order position
    float4* pst = nullptr;                 // [max pixels] T, C of unfinished tiles
    int4* pis = nullptr;                   // [max pixels] l_i, last, traversed, stopped
    uint32_t* tile_done = nullptr;         // [max_tiles]
    int32_t* tile_fbase = nullptr;         // [max_tiles]
    uint32_t* sat = nullptr;               // [(tiles_x + 1) * (tiles_y + 1)] at the largest image
};

// hist layout: 4 x 256 per-digit totals of the depth passes.
constexpr int kHistWords = kMaxPasses * kRadix;

// Contents of the column-run buffer: every Gaussian's runs, or a slice's.
enum RunsHeld : int { kRunsAll = 0, kRunsSlice0 = 1, kRunsSlice1 = 2 };

// What one frame's stages hand to the next.
struct FrameState {
    int64_t n = 0;
    CamDev cam{};
    SetDev st{};
    int num_tiles = 0;
    const uint32_t* order = nullptr;         // Gaussians by depth (the first V have tiles)
    // Deferred colours (frames whose parameters sit in host memory): Preprocess
    // skips the SH colour and each Render phase first computes it for the
    // Gaussians it blends, from these arrays (nullptr once they may be gone).
    bool defer_colors = false;
    const float* means = nullptr;
    const float* sh = nullptr;
    const uint32_t* sorted_gauss = nullptr;  // list entries' Gaussians by (cell, depth)
    const uint2* runs = nullptr;             // column runs by (column, depth)
    const uint16_t* rows = nullptr;          // their row intervals
    bool allow_slices = true;                // the caller's choice for the next sort
    bool sliced = false;                     // the frame renders in two depth slices
    bool split_last_slice = false;           // slice 1 renders tiles by pixel halves (f2)
    int runs_held = 0;                       // which Gaussians' column runs ws.pruns holds
    int lists = -1;                          // a ListKind; -1 before the first sort
};

// The lists Render reads: the column runs of the first tile-sort pass (each
// column of tiles reads its runs in depth order; a tile's own list is the
// runs covering its row, and the second pass is not run), or per-tile lists
// (the second pass; built on demand for the backward and the pair inspection).
enum ListKind : int { kListsTiles = 0, kListsColumns = 1 };

// Counts stage calls on the host; every 2^28 calls (before the device tag
// wraps) clears the lookback words.
void count_stage(std::atomic<uint32_t>& calls, const Workspace& ws, cudaStream_t stream);
// One-thread kernel that stores a frame's camera and settings in device
// memory, so the kernels that read them can be captured once in a graph and
// replayed for other cameras.
void launch_set_frame_params(const FrameParams& p, FrameParams* d_fp, cudaStream_t stream);
const void* set_frame_params_kernel();

// Stage orchestration shared by every entry point (pipeline.cu).
// set_params = false leaves the camera/settings in ws.d_fp to the caller (a
// captured graph replayed for other cameras writes them before each replay).
void enqueue_preprocess(const Workspace& ws, FrameState& fs, std::atomic<uint32_t>& epoch,
                        const float* means, const float* scales, const float* rots,
                        const float* opac, const float* sh, cudaStream_t stream,
                        bool set_params = true, bool defer_colors = false);
void enqueue_sort(const Workspace& ws, FrameState& fs, std::atomic<uint32_t>& epoch,
                  cudaStream_t stream);
// Builds per-tile lists (from every Gaussian's column runs) if the last sort
// made column lists; what the backward and the pair inspection read.
void enqueue_tile_lists(const Workspace& ws, FrameState& fs, cudaStream_t stream);
void enqueue_render(const Workspace& ws, FrameState& fs, float* img, float* t_final,
                    int32_t* load, cudaStream_t stream);
// A batched frame: up to kMaxBatch cameras of one scene (same n, same
// settings), each with its own workspace, rendered with one Preprocess and
// one Render launch per phase for all of them; each camera's sort stages run
// on its own stream of `bs` (forked from `stream` and joined back), or all on
// `stream` when bs is null.
struct BatchItem {
    const Workspace* ws;
    FrameState* fs;
    std::atomic<uint32_t>* epoch;
    float* img;
    float* t_final;
    int32_t* load;
};
struct BatchStreams {
    cudaStream_t side[kMaxBatch];
    cudaEvent_t fork;
    cudaEvent_t join[kMaxBatch];
};
void enqueue_frame_batch(const BatchItem* items, int count, const float* means, const float* scales,
                         const float* rots, const float* opac, const float* sh, cudaStream_t stream,
                         const BatchStreams* bs, bool set_params);
void fill_frame_state(FrameState& fs, int64_t n, const CamDev& cam, const SetDev& st);

// Kernel launchers (each enqueues on `stream`; all pointers are device memory).
// Preprocess and Render take a batch of up to kMaxBatch cameras of one scene
// in one grid (the serving scheduler's batched frames; one camera otherwise).
struct PreprocessOut {
    const FrameParams* fp;   // the camera's frame parameters
    uint32_t* stage;         // its workspace's stage counter (EpochRef)
    float4* rec;
    float4* aux;
    uint32_t* depth_key;
    uint32_t* gbox;
};
struct PreprocessBatch {
    int count = 0;
    PreprocessOut cam[kMaxBatch];
};
// grid = chunks of 256 Gaussians x count, the camera index fastest
// sh == nullptr defers the SH colours to launch_colors.
void launch_preprocess(int n, const float* means, const float* scales, const float* rots,
                       const float* opac, const float* sh, const PreprocessBatch& batch,
                       cudaStream_t stream);

// One stable 8-bit pass of the depth sort (sort.cu): keys (>> shift) & 255.
// first: all n keys in, keys 0xFFFFFFFF (no tiles) dropped and the kept ones
// counted into *kept; later passes sort the *kept keys; vals_in == nullptr
// means the values are 0..n-1.  counts: kRadix x grid words; totals: kRadix
// words, zeroed before.  With pay_out, also writes pay_out[i] = pay_in[vals_out[i]].
void launch_depth_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                       uint32_t* vals_out, int64_t n, uint32_t* kept, bool first, int shift,
                       uint32_t* counts, uint32_t* totals, const uint32_t* pay_in,
                       uint32_t* pay_out, uint32_t* status, int grid, cudaStream_t stream);

// SH colours (Sec. 3.2.1, stage 1's view-dependent colour) of the Gaussians
// ids[0 .. *count) into their render records (rec[3 i + 2].xyz), on demand:
// a frame with deferred colours computes them only for the Gaussians a Render
// launch blends.
void launch_colors(const uint32_t* ids, const uint32_t* count, const float* means, const float* sh,
                   const FrameParams* fp, float4* rec, int sm_count, cudaStream_t stream);

// Inputs of the tile passes.
struct PairSource {
    const uint32_t* order = nullptr;       // Gaussians by depth
    const uint32_t* offsets = nullptr;     // exclusive scan of their column-run counts
    const uint32_t* sorted_box = nullptr;  // packed rectangle per depth-order position
    const uint32_t* chunk_first = nullptr; // sorted position holding each chunk's first run
    const uint32_t* counters = nullptr;    // kCntPairs, kCntRuns, kCntVisible
    int64_t capacity = 0;
    int tiles_x = 0;
};

// Tile sort (tiles.cu): two range-partitioned counting passes, over the
// column runs by tx, then over the pairs by ty; `grid` CTAs, each owning a
// contiguous run of 4096-item chunks; counts holds kRadix x grid words, totals
// kRadix words (zeroed before the count kernel that sums into them).
//   count_columns:   per-CTA tx counts of the runs, from the Gaussians' rectangles;
//   scatter_columns: runs generated on chip from the depth-ordered Gaussians,
//                    written grouped by tx (x = Gaussian, y = y0 | (h-1) << 8 | tx << 16);
//   count_rows:      per-CTA ty counts of the pairs and the pairs of every
//                    tile (tile_counts, zeroed before);
//   tile_ranges:     each tile's [start, end) from tile_counts;
//   scatter_rows:    runs expanded into pairs, Gaussian ids grouped by ty;
//   count_scan:      counts -> global start of every (digit, CTA) run, in place.
int tile_scatter_blocks_per_sm();
void launch_tile_count_columns(const PairSource& src, uint32_t* counts, uint32_t* totals,
                               uint32_t* status, int grid, cudaStream_t stream);
void launch_tile_scatter_columns(const PairSource& src, const uint32_t* starts, uint2* runs_out,
                                 uint16_t* rows_out, uint32_t* status, int grid, cudaStream_t stream);
void launch_tile_count_rows(const uint2* runs, const uint32_t* counters, int64_t capacity,
                            int tiles_x, int num_tiles, uint32_t* counts, uint32_t* totals,
                            uint32_t* tile_counts, uint32_t* status, int grid, cudaStream_t stream);
void launch_tile_ranges(const uint32_t* tile_counts, int num_tiles, const uint32_t* counters,
                        int64_t capacity, uint2* ranges, cudaStream_t stream);
void launch_tile_scatter_rows(const uint2* runs, const uint32_t* counters, int64_t capacity,
                              const uint32_t* starts, uint32_t* gauss_out, uint32_t* status,
                              int grid, int tiles_y, cudaStream_t stream);
void launch_tile_count_scan(uint32_t* counts, const uint32_t* totals, int grid, cudaStream_t stream);

// Packed tile rectangle: x0 | y0 << 8 | (w-1) << 16 | (h-1) << 24 (tile
// coordinates and extents fit 8 bits because images are at most 4096 pixels
// per side).
// Exclusive scan of the column-run counts (rectangle widths) over the packed
// rectangles in depth order (sorted_box, all ones = no tiles), with decoupled
// lookback.  Also writes the run total, visible count and pair total to
// counters (with the capacity flag), and chunk_first[c] = position of the
// Gaussian holding run c * kSortChunk.
// A wait that gives up sets kErrLookback and counters[kCntScanFailed]; the
// pair total then reads as saturated, so every later stage of the frame
// skips its work exactly as after a capacity overflow.
void launch_scan_tiles(const uint32_t* sorted_box, int64_t n, int64_t capacity, uint32_t* offsets,
                       uint32_t* chunk_first, unsigned long long* lookback, EpochRef epoch,
                       uint32_t* counters, uint32_t* status, int grid, cudaStream_t stream);

// Render in depth slices (slices.cu): phase 0 renders a whole list; phase 1
// the first slice, finishing the tiles whose pixels all stopped (tile_done =
// 1) and keeping the per-pixel state of the others (pst: T, C; pis: l_i,
// last, traversed, stopped) and their list position (tile_fbase); phase 2
// resumes those tiles and finishes them.
struct SliceState {
    int phase = 0;
    float4* pst = nullptr;
    int4* pis = nullptr;
    uint32_t* tile_done = nullptr;
    int32_t* tile_fbase = nullptr;
    // Column lists: the pass's per-column run totals and the counters whose
    // pair count flags an overflow (the lists are then empty).
    const uint32_t* col_totals = nullptr;
    const uint32_t* col_counters = nullptr;
    int64_t capacity = 0;
};
// Slice 0 = the nearest 1/kSliceDiv of the Gaussians with tiles (0: no slices).
#ifndef ADR_SLICE_DIV
#define ADR_SLICE_DIV 16
#endif
constexpr int kSliceDiv = ADR_SLICE_DIV;
constexpr uint32_t kSliceProbe = 16;   // a context re-measures the slices every 16 frames
// One camera's inputs and outputs of a Render launch.
struct RenderCam {
    const uint2* ranges = nullptr;        // per-tile lists (lists == kListsTiles)
    const uint32_t* sorted_gauss = nullptr;
    const uint2* runs = nullptr;          // column runs (lists == kListsColumns)
    const uint16_t* rows = nullptr;       // their row intervals, 16-byte aligned
    const float4* rec = nullptr;
    const FrameParams* fp = nullptr;
    float* img = nullptr;
    float* t_final = nullptr;
    int32_t* load = nullptr;
    int32_t* last = nullptr;
    int32_t* trav = nullptr;
    float* tfin = nullptr;
    int32_t* lstat = nullptr;
    // Tracing (null: off): per tile, (start, end) of its CTA in %globaltimer
    // nanoseconds (low 32 bits each), the SM it ran on and the positions it
    // staged, at [tile] for phases 0 and 1 and at [num_tiles + tile] for phase 2.
    uint4* trace = nullptr;
    SliceState ss;
};
struct RenderBatch {
    int count = 0;
    int lists = kListsColumns;            // the same kind for every camera of the batch
    int split = 0;                        // phase 2: k_render_half (tiles by pixel halves)
    int tile_begin[kMaxBatch + 1] = {0};  // camera b's tiles are blocks [tile_begin[b], tile_begin[b+1])
    RenderCam cam[kMaxBatch];
};
void launch_render(const RenderBatch& batch, cudaStream_t stream);
void launch_slice0_setup(const uint32_t* counters, const uint32_t* offsets, uint32_t* c0,
                         cudaStream_t stream);
void launch_survivors(const uint32_t* tile_done, int tiles_x, int tiles_y, uint32_t* sat,
                      const uint32_t* sorted_box, const uint32_t* order, const uint32_t* counters,
                      int grid, uint32_t* cnt, uint8_t* keep_flag, int64_t n_max, int64_t chunk_max,
                      uint32_t* s_order, uint32_t* s_box, uint32_t* s_offsets,
                      uint32_t* s_chunk_first, uint32_t* c1, uint32_t* status, cudaStream_t stream);


// Backward (backward.cu).
void launch_render_backward(const uint2* ranges, const uint32_t* sorted_gauss, const float4* rec,
                            const float4* aux, const FrameParams* fp, int num_tiles,
                            const int32_t* last, const float* t_final, const int32_t* lstat,
                            const float* dl_dimg, const float* dl_dload, float* g2d,
                            cudaStream_t stream);
void launch_preprocess_backward(int n, const float* means, const float* scales, const float* rots,
                                const float* opac, const float* sh, const FrameParams* fp,
                                const uint32_t* gbox, const float4* aux,
                                const float* g2d, float* g_means, float* g_scales, float* g_rots,
                                float* g_opac, float* g_sh, cudaStream_t stream);
// 2^x with the hardware's approximate base-2 exponential (PTX ex2.approx.ftz:
// relative error ~2^-22, results below 2^-126 flushed to zero).  Render and its
// backward both evaluate a Gaussian's alpha with it, so they take the same
// alpha < alpha_low skip decisions; a flushed result is below alpha_low anyway.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The eigen-form quadratic of a Gaussian at a pixel, shared by Render and its
// backward so both take identical decisions: with the centre c relative to the
// tile origin, w = (w1, w2) and the pixel offset f from the origin,
// u_i = w_i . (c - f) is evaluated as (k_i - w_ix fx) - w_iy fy with
// k_i = w_i . c formed once per (Gaussian, tile), the fx-term first (Render's
// two pixels of a thread share fx); returns log2(sigma) - (u1^2 + u2^2).
__device__ __forceinline__ float2 quad_k(float2 c, float4 w) {
    return make_float2(fmaf(w.x, c.x, w.y * c.y), fmaf(w.z, c.x, w.w * c.y));
}
__device__ __forceinline__ float quad_exponent(float2 k, float4 w, float log2_sigma, float fx, float fy) {
    const float u1 = fmaf(-w.y, fy, fmaf(-w.x, fx, k.x));
    const float u2 = fmaf(-w.w, fy, fmaf(-w.z, fx, k.y));
    return fmaf(-u1, u1, fmaf(-u2, u2, log2_sigma));
}

// 1-D taps of the SSIM window (the 2-D window is their outer product).
struct LossWindow {
    float w[11];
};
void launch_image_loss(const float* img, const float* ref, int channels, int H, int W,
                       const LossWindow& win, float w_l1, float w_ssim, double* stats,
                       float* dl_dimg, float* scratch, cudaStream_t stream);
void launch_load_loss(const int32_t* load, int64_t hw, double* sums, float weight, float* dl_dload,
                      int sm_count, cudaStream_t stream);
void enqueue_backward(const Workspace& ws, const FrameState& fs, const float* means,
                      const float* scales, const float* rots, const float* opac, const float* sh,
                      const float* dl_dimg, const float* dl_dload, float* g_means, float* g_scales,
                      float* g_rots, float* g_opac, float* g_sh, cudaStream_t stream);

// Inspection: sorted pairs as (tile << 32 | depth bits, Gaussian) from the ranges.
void launch_pair_keys(const uint2* ranges, int num_tiles, const uint32_t* sorted_gauss,
                      const uint32_t* depth_key_by_gauss, int64_t count,
                      unsigned long long* keys_out, uint32_t* vals_out, cudaStream_t stream);
// Inspection: ranges with empty tiles as [0, 0).
void launch_copy_ranges(const uint2* ranges, int num_tiles, uint2* out, cudaStream_t stream);

// Occupancy of the persistent kernels (CTAs per SM), for grid sizing.
int onesweep_blocks_per_sm();
int scan_blocks_per_sm();

void launch_read_gaussians(const float4* rec, const float4* aux, const uint32_t* gbox, int n,
                           float* geom, int32_t* rect_out, int32_t* tiles_out, cudaStream_t stream);

// Workspace allocation with cudaMalloc (context and serving paths).
adr_status alloc_workspace(Workspace& w, int64_t max_gaussians, int64_t pair_capacity,
                           int32_t max_width, int32_t max_height, int device);
void free_workspace(Workspace& w);
size_t workspace_bytes(int64_t max_gaussians, int64_t pair_capacity, int32_t max_width,
                       int32_t max_height);

// Error reporting and argument conversion shared by the entry points.
adr_status report_error(adr_status st, const char* msg);
adr_status report_ok();
adr_status camera_to_dev(const adr_camera* cam, int max_w, int max_h, CamDev& d);
adr_status settings_to_dev(const adr_settings* s, SetDev& d);

}  // namespace adr
