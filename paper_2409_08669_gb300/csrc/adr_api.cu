// C ABI of libadr.so (declared in include/adr.h): the context that owns a
// frame's workspace, argument checking, and the entry points that enqueue the
// six rasterization stages (Sec. 3.2.1) through pipeline.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "adr_internal.cuh"

using namespace adr;

namespace {

thread_local std::string g_last_error;

adr_status fail(adr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

adr_status ok() {
    g_last_error.clear();
    return ADR_OK;
}

#define ADR_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ADR_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

// NVTX range named after the entry point (tracing: visible to nsys / ncu
// range filters; a no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int d) : want(d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != want) cudaSetDevice(want);
    }
    ~DeviceGuard() {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// The device address of HOST memory the current device can access in place
// (pinned memory mapped into its address space), or nullptr for any other
// pointer.
const float* mapped_host(const float* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();   // not an error for this call: clear it
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<const float*>(a.devicePointer) : nullptr;
}

adr_status make_cam(int max_w, int max_h, const adr_camera* cam, CamDev& d) {
    if (!cam) return fail(ADR_ERR_INVALID, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > max_w || cam->height > max_h)
        return fail(ADR_ERR_INVALID, "image %dx%d outside 1..%dx%d", cam->width, cam->height,
                    max_w, max_h);
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy))
        return fail(ADR_ERR_INVALID, "focal lengths must be positive and finite");
    // a Gaussian at depth 0 would project to infinity: the near plane must be in front
    if (!(cam->near_z > 0.f) || !std::isfinite(cam->near_z))
        return fail(ADR_ERR_INVALID, "near_z must be positive and finite");
    for (int i = 0; i < 12; ++i) d.v[i] = cam->view[i];
    d.fx = cam->fx; d.fy = cam->fy; d.cx = cam->cx; d.cy = cam->cy;
    d.near_z = cam->near_z;
    for (int i = 0; i < 3; ++i) d.cam_pos[i] = cam->cam_pos[i];
    d.width = cam->width; d.height = cam->height;
    d.tan_fovx = (float)cam->width / (2.f * cam->fx);
    d.tan_fovy = (float)cam->height / (2.f * cam->fy);
    d.tiles_x = (cam->width + kTile - 1) / kTile;
    d.tiles_y = (cam->height + kTile - 1) / kTile;
    return ADR_OK;
}

adr_status make_settings(const adr_settings* s, SetDev& d) {
    if (!s) return fail(ADR_ERR_INVALID, "settings is NULL");
    if (s->mode < ADR_PLAIN || s->mode > ADR_AABB) return fail(ADR_ERR_INVALID, "bad mode %d", s->mode);
    if (s->sh_degree < 0 || s->sh_degree > 3) return fail(ADR_ERR_INVALID, "sh_degree must be 0..3");
    if (s->rect_rule != ADR_RECT_PIXEL && s->rect_rule != ADR_RECT_3DGS)
        return fail(ADR_ERR_INVALID, "bad rect_rule %d", s->rect_rule);
    if (s->load_grad != ADR_LOAD_GRAD_STRAIGHT && s->load_grad != ADR_LOAD_GRAD_TERMINATION)
        return fail(ADR_ERR_INVALID, "bad load_grad %d", s->load_grad);
    if (!(s->alpha_low > 0.f && s->alpha_low < 1.f)) return fail(ADR_ERR_INVALID, "alpha_low must be in (0,1)");
    if (!(s->t_min >= 0.f && s->t_min < 1.f)) return fail(ADR_ERR_INVALID, "t_min must be in [0,1)");
    if (!(s->lowpass >= 0.f) || !std::isfinite(s->lowpass)) return fail(ADR_ERR_INVALID, "bad lowpass");
    if (!(s->jac_clamp > 0.f)) return fail(ADR_ERR_INVALID, "jac_clamp must be positive");
    d.mode = s->mode;
    d.alpha_low = s->alpha_low; d.t_min = s->t_min; d.lowpass = s->lowpass;
    d.e_low = (float)std::log2((double)s->alpha_low);
    d.jac_clamp = s->jac_clamp;
    for (int i = 0; i < 3; ++i) d.bg[i] = s->bg[i];
    d.sh_degree = s->sh_degree;
    d.rect_rule = s->rect_rule;
    d.load_grad = s->load_grad;
    return ADR_OK;
}

adr_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ADR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ADR_OK;
}

adr_status check_params(const float* means, const float* scales, const float* rots,
                        const float* opac, const float* sh, int64_t n, int64_t max_n) {
    if (n < 0 || n > max_n)
        return fail(ADR_ERR_INVALID, "n=%lld outside 0..%lld", (long long)n, (long long)max_n);
    if (n > 0 && (!means || !scales || !rots || !opac || !sh))
        return fail(ADR_ERR_INVALID, "a Gaussian parameter pointer is NULL");
    if (n > 0 && (!aligned(means, 4) || !aligned(scales, 4) || !aligned(opac, 4) ||
                  !aligned(rots, 16) || !aligned(sh, 16)))
        return fail(ADR_ERR_INVALID, "rots and sh must be 16-byte aligned, the rest 4-byte aligned");
    return ADR_OK;
}

}  // namespace

struct adr_ctx {
    int device = 0;
    int max_w = 0, max_h = 0;
    Workspace ws;
    FrameState fs;
    std::atomic<uint32_t> epoch{0};
    bool have_frame = false, have_sort = false, have_render = false;
    cudaStream_t last_stream = nullptr;
    uint32_t* host_words = nullptr;  // pinned: counters + status readback (words 0-31),
                                     // runs of the last sliced frame (words 40-42)
    // Depth slices pay only when most tiles stop within the nearest Gaussians.
    // After a sliced frame its run counts (all, slice 0, slice 1) come back
    // asynchronously; the next frame slices if the two slices made fewer than
    // half of all runs, and every kSliceProbe-th frame slices to measure again.
    cudaEvent_t slice_ev = nullptr;
    bool slice_probe = false;        // a readback is in flight
    bool slices_pay = true;
    uint32_t frames = 0;
    int32_t slice_mode = ADR_SLICES_ADAPTIVE;
    int32_t host_reads = ADR_HOST_READ_MAPPED;   // adr_render_host: read mapped host buffers in place
    bool defer_colors = false;   // the next adr_preprocess leaves the SH colours to adr_render
    int32_t tile_split = ADR_TILE_SPLIT_OFF;   // adr_set_tile_split
    // host-path staging (adr_render_host), allocated on its first use
    float* stage = nullptr;
    float* stage_img = nullptr;
    int32_t* stage_load = nullptr;
};

namespace {
// Process-wide testing hook of the bounded lookback waits (adr_test_lookback_expiry).
std::atomic<uint32_t> g_lb_withhold{0xFFFFFFFFu};
std::atomic<int> g_lb_spins{kLookbackSpinLimit};
}  // namespace

namespace adr {
// Shared with the other translation units (declared in adr_internal.cuh).
LookbackTest lookback_test() {
    LookbackTest t;
    t.withhold = g_lb_withhold.load();
    t.spin_limit = g_lb_spins.load();
    return t;
}
adr_status report_error(adr_status st, const char* msg) { return fail(st, "%s", msg); }
adr_status report_ok() { return ok(); }
adr_status camera_to_dev(const adr_camera* cam, int max_w, int max_h, CamDev& d) {
    return make_cam(max_w, max_h, cam, d);
}
adr_status settings_to_dev(const adr_settings* s, SetDev& d) { return make_settings(s, d); }

void free_workspace(Workspace& w) {
    if (w.tile_trace) cudaFree(w.tile_trace);
    if (w.prof) {
        for (int i = 0; i < w.prof->created; ++i) cudaEventDestroy(w.prof->ev[i]);
        delete w.prof;
        w.prof = nullptr;
    }
    void* ptrs[] = {w.rec, w.aux, w.depth_key, w.offsets, w.gbox, w.sorted_box, w.gkeys[0],
                    w.gkeys[1], w.gvals[0], w.gvals[1], w.pruns, w.prows, w.pgauss, w.tcounts, w.ttotals, w.tile_counts,
                    w.chunk_first, w.ranges, w.last, w.trav, w.tfin, w.lstat, w.g2d, w.load_sums,
                    w.hist, w.counters, w.status, w.lookback, w.d_fp, w.d_stage,
                    w.slice_counters, w.s_order, w.s_box, w.s_offsets, w.s_chunk_first,
                    w.surv_cnt, w.surv_flag, w.pst, w.pis, w.tile_done, w.tile_fbase, w.sat};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    w = Workspace{};
}

size_t workspace_bytes(int64_t max_gaussians, int64_t pair_capacity, int32_t max_width,
                       int32_t max_height) {
    const size_t N = (size_t)max_gaussians, P = (size_t)pair_capacity;
    const size_t pixels = (size_t)max_width * max_height;
    const size_t tiles = (size_t)((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
    const size_t lb = ((N + kSortChunk - 1) / kSortChunk + 2) * kRadix * 8;
    return N * (kRecFloat4 * 16 + kAuxFloat4 * 16 + 4 * 4 + 8 + 16 + 36 + 12) + P * 14 +
           2 * (P / kSortChunk + 2) * 4 + tiles * 20 + pixels * 48 + lb +
           (size_t)kRadix * (kMaxTileGrid + 2) * 4 + 4096;
}

adr_status alloc_workspace(Workspace& w, int64_t max_gaussians, int64_t pair_capacity,
                           int32_t max_width, int32_t max_height, int device) {
    w = Workspace{};
    w.max_n = max_gaussians;
    w.capacity = pair_capacity;
    w.max_tiles = ((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess || sms <= 0)
        return fail(ADR_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    w.sm_count = sms;
    w.sort_grid = sms * onesweep_blocks_per_sm();
    w.scan_grid = sms * scan_blocks_per_sm();
    w.tile_grid = sms * tile_scatter_blocks_per_sm();
    if (w.tile_grid > kMaxTileGrid) w.tile_grid = kMaxTileGrid;
    const size_t N = (size_t)max_gaussians, P = (size_t)pair_capacity;
    const size_t pixels = (size_t)max_width * max_height;
    w.lookback_words = ((N + kSortChunk - 1) / kSortChunk + 2) * kRadix;
#define ALLOC(ptr, bytes)                                                                   \
    do {                                                                                    \
        e = cudaMalloc((void**)&(ptr), (bytes));                                           \
        if (e != cudaSuccess) {                                                             \
            (void)cudaGetLastError(); /* not sticky: clear it for the next launch check */  \
            free_workspace(w);                                                              \
            return fail(ADR_ERR_CUDA, "cudaMalloc(%zu) for %s: %s", (size_t)(bytes), #ptr,  \
                        cudaGetErrorString(e));                                             \
        }                                                                                   \
    } while (0)
    ALLOC(w.rec, N * kRecFloat4 * sizeof(float4));
    ALLOC(w.aux, N * kAuxFloat4 * sizeof(float4));
    ALLOC(w.depth_key, N * sizeof(uint32_t));
    ALLOC(w.offsets, N * sizeof(uint32_t));
    ALLOC(w.gbox, N * sizeof(uint32_t));
    ALLOC(w.sorted_box, N * sizeof(uint32_t));
    for (int b = 0; b < 2; ++b) {
        ALLOC(w.gkeys[b], N * sizeof(uint32_t));
        ALLOC(w.gvals[b], N * sizeof(uint32_t));
    }
    ALLOC(w.pruns, P * sizeof(uint2));
    ALLOC(w.prows, (P + 8) * sizeof(uint16_t));   // + 16 bytes: Render reads whole 16-byte groups
    ALLOC(w.pgauss, P * sizeof(uint32_t));
    ALLOC(w.tile_counts, (size_t)w.max_tiles * sizeof(uint32_t));
    ALLOC(w.tcounts, (size_t)kRadix * kMaxTileGrid * sizeof(uint32_t));
    ALLOC(w.ttotals, 2 * kRadix * sizeof(uint32_t));
    ALLOC(w.chunk_first, (P / kSortChunk + 2) * sizeof(uint32_t));
    ALLOC(w.ranges, (size_t)w.max_tiles * sizeof(uint2));
    ALLOC(w.last, pixels * sizeof(int32_t));
    ALLOC(w.trav, pixels * sizeof(int32_t));
    ALLOC(w.tfin, pixels * sizeof(float));
    ALLOC(w.lstat, pixels * sizeof(int32_t));
    {
        const size_t tx = (size_t)(max_width + kTile - 1) / kTile, ty = (size_t)(max_height + kTile - 1) / kTile;
        ALLOC(w.slice_counters, 2 * kCntSlots * sizeof(uint32_t));
        ALLOC(w.s_order, N * sizeof(uint32_t));
        ALLOC(w.s_box, N * sizeof(uint32_t));
        ALLOC(w.s_offsets, N * sizeof(uint32_t));
        ALLOC(w.s_chunk_first, (P / kSortChunk + 2) * sizeof(uint32_t));
        ALLOC(w.surv_cnt, 2 * kMaxTileGrid * sizeof(uint32_t));
        ALLOC(w.surv_flag, N);
        ALLOC(w.pst, pixels * sizeof(float4));
        ALLOC(w.pis, pixels * sizeof(int4));
        ALLOC(w.tile_done, (size_t)w.max_tiles * sizeof(uint32_t));
        ALLOC(w.tile_fbase, (size_t)w.max_tiles * sizeof(int32_t));
        ALLOC(w.sat, (tx + 1) * (ty + 1) * sizeof(uint32_t));
    }
    ALLOC(w.g2d, N * 9 * sizeof(float));
    ALLOC(w.load_sums, 4 * sizeof(double));
    ALLOC(w.hist, kHistWords * sizeof(uint32_t));
    ALLOC(w.counters, kCntSlots * sizeof(uint32_t));
    ALLOC(w.status, sizeof(uint32_t) * 4);
    ALLOC(w.lookback, w.lookback_words * sizeof(unsigned long long));
    ALLOC(w.d_fp, sizeof(FrameParams));
    ALLOC(w.d_stage, sizeof(uint32_t));
#undef ALLOC
    if (cudaMemset(w.lookback, 0, w.lookback_words * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(w.status, 0, sizeof(uint32_t) * 4) != cudaSuccess ||
        cudaMemset(w.counters, 0, kCntSlots * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(w.d_stage, 0, sizeof(uint32_t)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        free_workspace(w);
        return fail(ADR_ERR_CUDA, "workspace initialisation failed");
    }
    return ADR_OK;
}
}  // namespace adr

namespace {

void free_ctx(adr_ctx* c) {
    free_workspace(c->ws);
    void* ptrs[] = {c->stage, c->stage_img, c->stage_load};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->host_words) cudaFreeHost(c->host_words);
    if (c->slice_ev) cudaEventDestroy(c->slice_ev);
    delete c;
}

}  // namespace

extern "C" {

const char* adr_last_error(void) { return g_last_error.c_str(); }

const char* adr_version(void) { return "adr-gb300 0.3 (sm_103a)"; }

adr_status adr_test_lookback_expiry(int32_t withheld_chunk, int32_t spin_limit) {
    if (withheld_chunk < 0) {
        g_lb_withhold.store(0xFFFFFFFFu);
        g_lb_spins.store(kLookbackSpinLimit);
        return ok();
    }
    if (spin_limit < 1 || spin_limit > kLookbackSpinLimit)
        return fail(ADR_ERR_INVALID, "spin_limit must be in 1..%d", kLookbackSpinLimit);
    g_lb_spins.store(spin_limit);
    g_lb_withhold.store((uint32_t)withheld_chunk);
    return ok();
}

adr_status adr_create(adr_ctx** out, int64_t max_gaussians, int64_t pair_capacity,
                      int32_t max_width, int32_t max_height, int32_t device) {
    if (!out) return fail(ADR_ERR_INVALID, "ctx out-pointer is NULL");
    *out = nullptr;
    if (max_gaussians <= 0 || max_gaussians > kMaxGaussians)
        return fail(ADR_ERR_INVALID, "max_gaussians must be in 1..2^29");
    if (pair_capacity <= 0 || pair_capacity > (int64_t(1) << 30))
        return fail(ADR_ERR_INVALID, "pair_capacity must be in 1..2^30");
    if (max_width <= 0 || max_height <= 0 || max_width > 4096 || max_height > 4096)
        return fail(ADR_ERR_INVALID, "max image size must be in 1..4096 per side");
    int ndev = 0;
    ADR_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(ADR_ERR_INVALID, "device %d not present", device);
    DeviceGuard guard(device);

    adr_ctx* c = new adr_ctx();
    c->device = device;
    c->max_w = max_width;
    c->max_h = max_height;
    adr_status st = alloc_workspace(c->ws, max_gaussians, pair_capacity, max_width, max_height, device);
    if (st != ADR_OK) {
        delete c;
        return st;
    }
    cudaError_t e = cudaHostAlloc((void**)&c->host_words, 64 * sizeof(uint32_t), cudaHostAllocDefault);
    if (e != cudaSuccess) { free_ctx(c); return fail(ADR_ERR_CUDA, "cudaHostAlloc: %s", cudaGetErrorString(e)); }
    e = cudaEventCreateWithFlags(&c->slice_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { free_ctx(c); return fail(ADR_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e)); }
    *out = c;
    return ok();
}

void adr_destroy(adr_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    cudaDeviceSynchronize();
    free_ctx(ctx);
}

adr_status adr_preprocess(adr_ctx* c, const float* means, const float* scales, const float* rots,
                          const float* opac, const float* sh, int64_t n, const adr_camera* camera,
                          const adr_settings* settings, void* stream) {
    NvtxRange range_("adr_preprocess");
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    adr_status s;
    if ((s = check_params(means, scales, rots, opac, sh, n, c->ws.max_n)) != ADR_OK) return s;
    CamDev cam;
    SetDev st;
    if ((s = make_cam(c->max_w, c->max_h, camera, cam)) != ADR_OK) return s;
    if ((s = make_settings(settings, st)) != ADR_OK) return s;
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    fill_frame_state(c->fs, n, cam, st);
    enqueue_preprocess(c->ws, c->fs, c->epoch, means, scales, rots, opac, sh, strm, true,
                       c->defer_colors);
    if ((s = check_launch("adr_preprocess")) != ADR_OK) return s;
    c->have_frame = true;
    c->have_sort = c->have_render = false;
    return ok();
}

// Whether the context's next adr_sort builds depth slices: always, never, or
// (adaptive) when the last sliced frame's run counts, read back without
// waiting, showed they pay, and every kSliceProbe-th frame to measure again.
static bool next_frame_slices(adr_ctx* c) {
    if (c->slice_probe) {   // the last sliced frame's run counts, if they are back
        const cudaError_t q = cudaEventQuery(c->slice_ev);
        if (q == cudaSuccess) {
            const uint64_t all = c->host_words[40], used = (uint64_t)c->host_words[41] + c->host_words[42];
            c->slices_pay = 2 * used < all;
            c->slice_probe = false;
        } else if (q == cudaErrorNotReady && cudaPeekAtLastError() == cudaErrorNotReady) {
            cudaGetLastError();   // not an error: clear it
        }
    }
    return c->slice_mode == ADR_SLICES_ALWAYS ||
           (c->slice_mode == ADR_SLICES_ADAPTIVE && (c->slices_pay || (c->frames % kSliceProbe) == 0));
}

adr_status adr_sort(adr_ctx* c, void* stream) {
    NvtxRange range_("adr_sort");
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_frame) return fail(ADR_ERR_INVALID, "adr_sort before adr_preprocess");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    c->fs.allow_slices = next_frame_slices(c);
    ++c->frames;
    enqueue_sort(c->ws, c->fs, c->epoch, strm);
    adr_status s;
    if ((s = check_launch("adr_sort")) != ADR_OK) return s;
    c->have_sort = true;
    return ok();
}

adr_status adr_render(adr_ctx* c, float* img, float* t_final, int32_t* load, void* stream) {
    NvtxRange range_("adr_render");
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_sort) return fail(ADR_ERR_INVALID, "adr_render before adr_sort");
    if (!img) return fail(ADR_ERR_INVALID, "img is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    c->fs.split_last_slice = c->tile_split == ADR_TILE_SPLIT_LAST_SLICE;
    enqueue_render(c->ws, c->fs, img, t_final, load, strm);
    if (c->fs.sliced && !c->slice_probe) {
        // Runs of every Gaussian, of slice 0 and of slice 1, back to the host.
        const uint32_t* src[3] = {c->ws.counters + kCntRuns, c->ws.slice_counters + kCntRuns,
                                  c->ws.slice_counters + kCntSlots + kCntRuns};
        for (int k = 0; k < 3; ++k)
            ADR_CUDA(cudaMemcpyAsync(c->host_words + 40 + k, src[k], sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost, strm));
        ADR_CUDA(cudaEventRecord(c->slice_ev, strm));
        c->slice_probe = true;
    }
    adr_status s;
    if ((s = check_launch("adr_render")) != ADR_OK) return s;
    c->have_render = true;
    return ok();
}

adr_status adr_sync_status(adr_ctx* c) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    DeviceGuard guard(c->device);
    ADR_CUDA(cudaStreamSynchronize(c->last_stream));
    ADR_CUDA(cudaMemcpy(c->host_words, c->ws.status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    const uint32_t bits = c->host_words[0];
    ADR_CUDA(cudaMemset(c->ws.status, 0, sizeof(uint32_t)));
    const StatusReport r = status_from_bits(bits, 0, c->ws.capacity);
    if (r.status != ADR_OK) return fail(r.status, "%s", r.message);
    return ok();
}

adr_status adr_num_pairs(adr_ctx* c, int64_t* num_pairs) {
    if (!c || !num_pairs) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->have_frame) return fail(ADR_ERR_INVALID, "adr_num_pairs before adr_preprocess");
    DeviceGuard guard(c->device);
    ADR_CUDA(cudaStreamSynchronize(c->last_stream));
    ADR_CUDA(cudaMemcpy(c->host_words, c->ws.counters, kCntSlots * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost));
    *num_pairs = (int64_t)c->host_words[kCntPairs];
    adr_status s = adr_sync_status(c);
    if (s != ADR_OK) return s;
    if (*num_pairs > c->ws.capacity)
        return fail(ADR_ERR_CAPACITY, "P=%lld exceeds pair_capacity=%lld", (long long)*num_pairs,
                    (long long)c->ws.capacity);
    return ok();
}

adr_status adr_frame_counts(adr_ctx* c, int64_t* out, int32_t n) {
    if (!c || !out || n < 1) return fail(ADR_ERR_INVALID, "bad argument");
    if (!c->have_render) return fail(ADR_ERR_INVALID, "adr_frame_counts before adr_render");
    DeviceGuard guard(c->device);
    ADR_CUDA(cudaStreamSynchronize(c->last_stream));
    uint32_t w[3 * kCntSlots] = {0};
    ADR_CUDA(cudaMemcpy(w, c->ws.counters, kCntSlots * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (c->fs.sliced)
        ADR_CUDA(cudaMemcpy(w + kCntSlots, c->ws.slice_counters, 2 * kCntSlots * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost));
    const uint32_t* s0 = w + kCntSlots;
    const uint32_t* s1 = w + 2 * kCntSlots;
    const int64_t vals[7] = {(int64_t)w[kCntPairs], (int64_t)w[kCntVisible], (int64_t)w[kCntRuns],
                             c->fs.sliced ? 1 : 0, c->fs.sliced ? (int64_t)s0[kCntRuns] : 0,
                             c->fs.sliced ? (int64_t)s1[kCntRuns] : 0,
                             c->fs.sliced ? (int64_t)s1[kCntVisible] : 0};
    for (int i = 0; i < n && i < 7; ++i) out[i] = vals[i];
    return ok();
}

adr_status adr_read_pairs(adr_ctx* c, uint64_t* keys, uint32_t* vals, int64_t capacity,
                          void* stream) {
    if (!c || !keys || !vals) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->have_sort) return fail(ADR_ERR_INVALID, "adr_read_pairs before adr_sort");
    if (capacity < 0) return fail(ADR_ERR_INVALID, "negative capacity");
    DeviceGuard guard(c->device);
    const int64_t cap = capacity < c->ws.capacity ? capacity : c->ws.capacity;
    c->last_stream = (cudaStream_t)stream;
    enqueue_tile_lists(c->ws, c->fs, (cudaStream_t)stream);
    launch_pair_keys(c->ws.ranges, c->fs.num_tiles, c->fs.sorted_gauss, c->ws.depth_key, cap,
                     reinterpret_cast<unsigned long long*>(keys), vals, (cudaStream_t)stream);
    return check_launch("adr_read_pairs") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_read_gaussians(adr_ctx* c, float* geom, int32_t* rect, int32_t* tiles,
                              void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_frame) return fail(ADR_ERR_INVALID, "adr_read_gaussians before adr_preprocess");
    DeviceGuard guard(c->device);
    // A frame computes the SH colours of the Gaussians it blends only; the
    // inspection reports every Gaussian with tiles, from the frame's SH array.
    if (geom && c->fs.defer_colors && c->fs.sh && c->fs.order && c->fs.n > 0)
        launch_colors(c->fs.order, c->ws.counters + kCntVisible, c->fs.means, c->fs.sh, c->ws.d_fp,
                      c->ws.rec, c->ws.sm_count, (cudaStream_t)stream);
    launch_read_gaussians(c->ws.rec, c->ws.aux, c->ws.gbox, (int)c->fs.n, geom, rect,
                          tiles, (cudaStream_t)stream);
    return check_launch("adr_read_gaussians") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_read_ranges(adr_ctx* c, uint32_t* ranges, void* stream) {
    if (!c || !ranges) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->have_sort) return fail(ADR_ERR_INVALID, "adr_read_ranges before adr_sort");
    DeviceGuard guard(c->device);
    c->last_stream = (cudaStream_t)stream;
    enqueue_tile_lists(c->ws, c->fs, (cudaStream_t)stream);
    launch_copy_ranges(c->ws.ranges, c->fs.num_tiles, reinterpret_cast<uint2*>(ranges),
                       (cudaStream_t)stream);
    return check_launch("adr_read_ranges") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_read_pixel_stats(adr_ctx* c, int32_t* last, int32_t* traversed, void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_render) return fail(ADR_ERR_INVALID, "adr_read_pixel_stats before adr_render");
    DeviceGuard guard(c->device);
    const size_t bytes = (size_t)c->fs.cam.width * c->fs.cam.height * sizeof(int32_t);
    if (last) ADR_CUDA(cudaMemcpyAsync(last, c->ws.last, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    if (traversed)
        ADR_CUDA(cudaMemcpyAsync(traversed, c->ws.trav, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ok();
}

adr_status adr_render_backward(adr_ctx* c, const float* means, const float* scales,
                               const float* rots, const float* opac, const float* sh,
                               const float* dl_dimg, const float* dl_dload, float* g_means,
                               float* g_scales, float* g_rots, float* g_opac, float* g_sh,
                               void* stream) {
    NvtxRange range_("adr_render_backward");
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_render) return fail(ADR_ERR_INVALID, "adr_render_backward before adr_render");
    adr_status s;
    if ((s = check_params(means, scales, rots, opac, sh, c->fs.n, c->ws.max_n)) != ADR_OK) return s;
    if (!dl_dimg) return fail(ADR_ERR_INVALID, "dl_dimg is NULL");
    if (c->fs.n > 0 && (!g_means || !g_scales || !g_rots || !g_opac || !g_sh))
        return fail(ADR_ERR_INVALID, "a gradient output pointer is NULL");
    if (c->fs.n > 0 && (!aligned(g_rots, 16) || !aligned(g_sh, 16)))
        return fail(ADR_ERR_INVALID, "g_rots and g_sh must be 16-byte aligned");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    enqueue_tile_lists(c->ws, c->fs, strm);   // the backward walks per-tile lists
    enqueue_backward(c->ws, c->fs, means, scales, rots, opac, sh, dl_dimg, dl_dload, g_means,
                     g_scales, g_rots, g_opac, g_sh, strm);
    return check_launch("adr_render_backward") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_load_loss(adr_ctx* c, const int32_t* load, int64_t hw, float weight,
                         double* stats, float* dl_dload, void* stream) {
    NvtxRange range_("adr_load_loss");
    if (!c || !load || !stats) return fail(ADR_ERR_INVALID, "NULL argument");
    if (hw <= 0) return fail(ADR_ERR_INVALID, "hw must be positive");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    launch_load_loss(load, hw, c->ws.load_sums, weight, dl_dload, c->ws.sm_count, strm);
    ADR_CUDA(cudaMemcpyAsync(stats, c->ws.load_sums + 2, 2 * sizeof(double),
                             cudaMemcpyDeviceToDevice, strm));
    return check_launch("adr_load_loss") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_image_loss(const float* img, const float* ref, int32_t channels, int32_t height,
                          int32_t width, float w_l1, float w_ssim, double* stats, float* dl_dimg,
                          float* scratch, void* stream) {
    NvtxRange range_("adr_image_loss");
    if (!img || !ref || !stats) return fail(ADR_ERR_INVALID, "NULL argument");
    if (channels <= 0 || height <= 0 || width <= 0 || (int64_t)channels * height * width > (1ll << 31))
        return fail(ADR_ERR_INVALID, "image size %d x %d x %d out of range", channels, height, width);
    if (dl_dimg && !scratch) return fail(ADR_ERR_INVALID, "scratch is required with dl_dimg");
    if (!std::isfinite(w_l1) || !std::isfinite(w_ssim)) return fail(ADR_ERR_INVALID, "bad weight");
    // Gaussian window of standard deviation 1.5 over 11 taps, normalised to sum 1.
    LossWindow win;
    double w[11], sum = 0.0;
    for (int k = 0; k < 11; ++k) {
        const double d = k - 5;
        w[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += w[k];
    }
    for (int k = 0; k < 11; ++k) win.w[k] = (float)(w[k] / sum);
    launch_image_loss(img, ref, channels, height, width, win, w_l1, w_ssim, stats, dl_dimg,
                      scratch, (cudaStream_t)stream);
    return check_launch("adr_image_loss") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_set_tile_split(adr_ctx* c, int32_t mode) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (mode != ADR_TILE_SPLIT_OFF && mode != ADR_TILE_SPLIT_LAST_SLICE)
        return fail(ADR_ERR_INVALID, "unknown tile split mode %d", (int)mode);
    c->tile_split = mode;
    return ok();
}

adr_status adr_set_host_reads(adr_ctx* c, int32_t mode) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (mode != ADR_HOST_READ_COPY && mode != ADR_HOST_READ_MAPPED)
        return fail(ADR_ERR_INVALID, "unknown host read mode %d", (int)mode);
    c->host_reads = mode;
    return ok();
}

adr_status adr_set_depth_slices(adr_ctx* c, int32_t mode) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (mode != ADR_SLICES_NEVER && mode != ADR_SLICES_ALWAYS && mode != ADR_SLICES_ADAPTIVE)
        return fail(ADR_ERR_INVALID, "bad depth-slice mode %d", mode);
    c->slice_mode = mode;
    return ok();
}

adr_status adr_profile_enable(adr_ctx* c, int32_t enable) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    DeviceGuard guard(c->device);
    if (enable && !c->ws.prof) c->ws.prof = new Profiler();
    if (!enable && c->ws.prof) {
        ADR_CUDA(cudaDeviceSynchronize());
        for (int i = 0; i < c->ws.prof->created; ++i) cudaEventDestroy(c->ws.prof->ev[i]);
        delete c->ws.prof;
        c->ws.prof = nullptr;
    }
    return ok();
}

adr_status adr_trace_tiles(adr_ctx* c, int32_t enable) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    DeviceGuard guard(c->device);
    if (enable && !c->ws.tile_trace) {
        const size_t bytes = (size_t)2 * c->ws.max_tiles * sizeof(uint4);
        cudaError_t e = cudaMalloc((void**)&c->ws.tile_trace, bytes);
        if (e == cudaSuccess) e = cudaMemset(c->ws.tile_trace, 0, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            if (c->ws.tile_trace) cudaFree(c->ws.tile_trace);
            c->ws.tile_trace = nullptr;
            return fail(ADR_ERR_CUDA, "tile trace allocation: %s", cudaGetErrorString(e));
        }
    }
    if (!enable && c->ws.tile_trace) {
        ADR_CUDA(cudaDeviceSynchronize());
        cudaFree(c->ws.tile_trace);
        c->ws.tile_trace = nullptr;
    }
    return ok();
}

adr_status adr_read_tile_trace(adr_ctx* c, uint32_t* out, void* stream) {
    if (!c || !out) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->ws.tile_trace) return fail(ADR_ERR_INVALID, "tile tracing is not enabled");
    if (!c->have_render) return fail(ADR_ERR_INVALID, "adr_read_tile_trace before adr_render");
    DeviceGuard guard(c->device);
    const size_t nt = (size_t)c->fs.num_tiles;
    cudaStream_t strm = (cudaStream_t)stream;
    ADR_CUDA(cudaMemcpyAsync(out, c->ws.tile_trace, nt * sizeof(uint4), cudaMemcpyDeviceToDevice, strm));
    ADR_CUDA(cudaMemcpyAsync(out + 4 * nt, c->ws.tile_trace + nt, nt * sizeof(uint4),
                             cudaMemcpyDeviceToDevice, strm));
    return ok();
}

adr_status adr_profile_read(adr_ctx* c, int32_t max_kernels, int32_t* kernel_ids, double* total_ms,
                            int32_t* launches, int32_t* num_kernels) {
    if (!c || !kernel_ids || !total_ms || !launches || !num_kernels)
        return fail(ADR_ERR_INVALID, "NULL argument");
    Profiler* p = c->ws.prof;
    *num_kernels = 0;
    if (!p) return fail(ADR_ERR_INVALID, "profiling is not enabled");
    DeviceGuard guard(c->device);
    double ms[kKernelCount] = {0};
    int cnt[kKernelCount] = {0};
    for (int i = 0; i < p->used; ++i) {
        float t = 0.f;
        ADR_CUDA(cudaEventSynchronize(p->ev[2 * i + 1]));
        ADR_CUDA(cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1]));
        ms[p->id[i]] += t;
        cnt[p->id[i]] += 1;
    }
    p->used = 0;
    int k = 0;
    for (int id = 0; id < kKernelCount && k < max_kernels; ++id) {
        if (!cnt[id]) continue;
        kernel_ids[k] = id;
        total_ms[k] = ms[id];
        launches[k] = cnt[id];
        ++k;
    }
    *num_kernels = k;
    return ok();
}

const char* adr_profile_kernel_name(int32_t kernel_id) { return kernel_name(kernel_id); }

adr_status adr_render_host(adr_ctx* c, const float* means, const float* scales, const float* rots,
                           const float* opac, const float* sh, int64_t n, const adr_camera* camera,
                           const adr_settings* settings, float* img, float* t_final, int32_t* load,
                           void* stream) {
    NvtxRange range_("adr_render_host");
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!img) return fail(ADR_ERR_INVALID, "img is NULL");
    if (n < 0 || n > c->ws.max_n) return fail(ADR_ERR_INVALID, "n outside 0..max_gaussians");
    if (n > 0 && (!means || !scales || !rots || !opac || !sh))
        return fail(ADR_ERR_INVALID, "a Gaussian parameter pointer is NULL");
    if (!camera) return fail(ADR_ERR_INVALID, "camera is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    const size_t hw = (size_t)camera->width * camera->height;
    // Pinned host memory mapped into the device's address space is read (and
    // the image written) in place over the host link: Preprocess then moves
    // only what it reads -- 44 bytes of every Gaussian and the 192 bytes of
    // SH of the Gaussians with tiles -- instead of a copy of every array.
    if (c->host_reads == ADR_HOST_READ_MAPPED) {
        const float* dm = mapped_host(means);
        const float* ds = mapped_host(scales);
        const float* dr = mapped_host(rots);
        const float* dop = mapped_host(opac);
        const float* dsh = mapped_host(sh);
        float* di = const_cast<float*>(mapped_host(img));
        float* dt = t_final ? const_cast<float*>(mapped_host(t_final)) : nullptr;
        int32_t* dl = load ? reinterpret_cast<int32_t*>(const_cast<float*>(
                                 mapped_host(reinterpret_cast<const float*>(load))))
                           : nullptr;
        const bool inputs = n == 0 || (dm && ds && dr && dop && dsh && aligned(dr, 16) && aligned(dsh, 16));
        const bool outputs = di && (!t_final || dt) && (!load || dl);
        if (inputs && outputs) {
            // The colours come from host memory too: a sliced frame reads
            // only those of the Gaussians each Render phase blends; an
            // unsliced frame blends every Gaussian with tiles and reads them
            // in Preprocess, in index order.
            c->defer_colors = next_frame_slices(c);
            adr_status s = adr_preprocess(c, dm, ds, dr, dop, dsh, n, camera, settings, stream);
            c->defer_colors = false;
            if (s != ADR_OK) return s;
            if ((s = adr_sort(c, stream)) != ADR_OK) return s;
            if ((s = adr_render(c, di, dt, dl, stream)) != ADR_OK) return s;
            ADR_CUDA(cudaStreamSynchronize(strm));
            c->fs.means = c->fs.sh = nullptr;   // the caller's buffers: not read after the call
            return ok();
        }
    }
    const size_t N = (size_t)c->ws.max_n;
    const size_t per = 3 + 3 + 4 + 1 + 48;   // floats per Gaussian
    if (!c->stage) {   // all three staging buffers, or none (a later call retries)
        float *stage = nullptr, *stage_img = nullptr;
        int32_t* stage_load = nullptr;
        const size_t px = (size_t)c->max_w * c->max_h;
        cudaError_t e = cudaMalloc((void**)&stage, N * per * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&stage_img, px * 4 * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&stage_load, px * sizeof(int32_t));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();   // clear it, or the next launch check would report it
            if (stage) cudaFree(stage);
            if (stage_img) cudaFree(stage_img);
            return fail(ADR_ERR_CUDA, "adr_render_host staging allocation: %s", cudaGetErrorString(e));
        }
        c->stage = stage;
        c->stage_img = stage_img;
        c->stage_load = stage_load;
    }
    // Device layout: sh first (16-byte aligned), then rots, means, scales, opac.
    float* d_sh = c->stage;
    float* d_rots = d_sh + N * 48;
    float* d_means = d_rots + N * 4;
    float* d_scales = d_means + N * 3;
    float* d_opac = d_scales + N * 3;
    const size_t nn = (size_t)n;
    if (n > 0) {
        ADR_CUDA(cudaMemcpyAsync(d_sh, sh, nn * 48 * sizeof(float), cudaMemcpyHostToDevice, strm));
        ADR_CUDA(cudaMemcpyAsync(d_rots, rots, nn * 4 * sizeof(float), cudaMemcpyHostToDevice, strm));
        ADR_CUDA(cudaMemcpyAsync(d_means, means, nn * 3 * sizeof(float), cudaMemcpyHostToDevice, strm));
        ADR_CUDA(cudaMemcpyAsync(d_scales, scales, nn * 3 * sizeof(float), cudaMemcpyHostToDevice, strm));
        ADR_CUDA(cudaMemcpyAsync(d_opac, opac, nn * sizeof(float), cudaMemcpyHostToDevice, strm));
    }
    adr_status s = adr_preprocess(c, d_means, d_scales, d_rots, d_opac, d_sh, n, camera, settings, stream);
    if (s != ADR_OK) return s;
    if ((s = adr_sort(c, stream)) != ADR_OK) return s;
    float* d_img = c->stage_img;
    float* d_t = d_img + 3 * hw;
    if ((s = adr_render(c, d_img, d_t, c->stage_load, stream)) != ADR_OK) return s;
    ADR_CUDA(cudaMemcpyAsync(img, d_img, 3 * hw * sizeof(float), cudaMemcpyDeviceToHost, strm));
    if (t_final) ADR_CUDA(cudaMemcpyAsync(t_final, d_t, hw * sizeof(float), cudaMemcpyDeviceToHost, strm));
    if (load) ADR_CUDA(cudaMemcpyAsync(load, c->stage_load, hw * sizeof(int32_t), cudaMemcpyDeviceToHost, strm));
    ADR_CUDA(cudaStreamSynchronize(strm));
    return ok();
}

}  // extern "C"
