// C ABI of libadr.so (declared in include/adr.h): context workspace and the
// host-side orchestration of the six rasterization stages (Sec. 3.2.1).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

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

int ceil_log2(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) < v) ++b;
    return b;
}

}  // namespace

struct adr_ctx {
    int device = 0;
    int64_t max_n = 0, capacity = 0;
    int max_w = 0, max_h = 0, max_tiles = 0;
    int sm_count = 0, sort_grid = 0, scan_grid = 0;
    uint32_t epoch = 0;

    // per-Gaussian
    float4* rec = nullptr;
    float4* aux = nullptr;
    uint32_t* depth_key = nullptr;
    uint32_t* tiles = nullptr;
    ushort4* rect = nullptr;
    uint32_t* offsets = nullptr;
    uint32_t* gkeys[2] = {nullptr, nullptr};
    uint32_t* gvals[2] = {nullptr, nullptr};
    // per-pair
    uint32_t* ptile[2] = {nullptr, nullptr};
    uint32_t* pgauss[2] = {nullptr, nullptr};
    // per-tile / per-pixel
    uint2* ranges = nullptr;
    int32_t* last = nullptr;         // 1-based list position of the last blended Gaussian
    int32_t* trav = nullptr;         // list positions each pixel evaluated
    // bookkeeping
    uint32_t* hist = nullptr;        // [kMaxPasses][256] depth digits, then [2][256] tile digits
    uint32_t* counters = nullptr;    // kCntSlots
    uint32_t* status = nullptr;      // error bits
    unsigned long long* lookback = nullptr;
    size_t lookback_words = 0;
    uint32_t* host_words = nullptr;  // pinned: counters + status readback

    // last frame
    int64_t n = 0;
    CamDev cam{};
    SetDev st{};
    int tile_passes = 0, tile_bits = 0;
    bool have_frame = false, have_sort = false, have_render = false;
    cudaStream_t last_stream = nullptr;
    const uint32_t* sorted_order = nullptr;   // Gaussians in depth order
    uint32_t* sorted_tile = nullptr;          // pairs after adr_sort
    uint32_t* sorted_gauss = nullptr;

    // host-path staging (adr_render_host), allocated on first use
    float* stage = nullptr;
    float* stage_img = nullptr;
    int32_t* stage_load = nullptr;
};

namespace {

void free_ctx(adr_ctx* c) {
    void* ptrs[] = {c->rec, c->aux, c->depth_key, c->tiles, c->rect, c->offsets,
                    c->gkeys[0], c->gkeys[1], c->gvals[0], c->gvals[1], c->ptile[0],
                    c->ptile[1], c->pgauss[0], c->pgauss[1], c->ranges, c->last, c->trav,
                    c->hist, c->counters, c->status, c->lookback, c->stage,
                    c->stage_img, c->stage_load};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->host_words) cudaFreeHost(c->host_words);
    delete c;
}

uint32_t next_epoch(adr_ctx* c, cudaStream_t s) {
    if (++c->epoch == 0) {
        // All lookback words carry the epoch of their pass; on wrap-around clear
        // them so no stale word can match a new pass.
        cudaMemsetAsync(c->lookback, 0, c->lookback_words * sizeof(unsigned long long), s);
        c->epoch = 1;
    }
    return c->epoch;
}

adr_status make_cam(const adr_ctx* c, const adr_camera* cam, CamDev& d) {
    if (!cam) return fail(ADR_ERR_INVALID, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > c->max_w || cam->height > c->max_h)
        return fail(ADR_ERR_INVALID, "image %dx%d outside 1..%dx%d", cam->width, cam->height,
                    c->max_w, c->max_h);
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy))
        return fail(ADR_ERR_INVALID, "focal lengths must be positive and finite");
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
    if (!(s->alpha_low > 0.f && s->alpha_low < 1.f)) return fail(ADR_ERR_INVALID, "alpha_low must be in (0,1)");
    if (!(s->t_min >= 0.f && s->t_min < 1.f)) return fail(ADR_ERR_INVALID, "t_min must be in [0,1)");
    if (!(s->lowpass >= 0.f) || !std::isfinite(s->lowpass)) return fail(ADR_ERR_INVALID, "bad lowpass");
    if (!(s->jac_clamp > 0.f)) return fail(ADR_ERR_INVALID, "jac_clamp must be positive");
    d.mode = s->mode;
    d.alpha_low = s->alpha_low; d.t_min = s->t_min; d.lowpass = s->lowpass;
    d.jac_clamp = s->jac_clamp;
    for (int i = 0; i < 3; ++i) d.bg[i] = s->bg[i];
    d.sh_degree = s->sh_degree;
    return ADR_OK;
}

adr_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ADR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ADR_OK;
}

}  // namespace

namespace adr {
// Shared with other translation units of the library (declared in adr_internal.cuh).
adr_status report_error(adr_status st, const char* msg) { return fail(st, "%s", msg); }
adr_status report_ok() { return ok(); }
adr_status camera_to_dev(const adr_camera* cam, int max_w, int max_h, CamDev& d) {
    adr_ctx probe;
    probe.max_w = max_w;
    probe.max_h = max_h;
    return make_cam(&probe, cam, d);
}
adr_status settings_to_dev(const adr_settings* s, SetDev& d) { return make_settings(s, d); }
}  // namespace adr

extern "C" {

const char* adr_last_error(void) { return g_last_error.c_str(); }

const char* adr_version(void) { return "adr-gb300 0.1 (sm_103a)"; }

adr_status adr_create(adr_ctx** out, int64_t max_gaussians, int64_t pair_capacity,
                      int32_t max_width, int32_t max_height, int32_t device) {
    if (!out) return fail(ADR_ERR_INVALID, "ctx out-pointer is NULL");
    *out = nullptr;
    if (max_gaussians <= 0 || max_gaussians > (int64_t(1) << 30))
        return fail(ADR_ERR_INVALID, "max_gaussians must be in 1..2^30");
    if (pair_capacity <= 0 || pair_capacity > (int64_t(1) << 30))
        return fail(ADR_ERR_INVALID, "pair_capacity must be in 1..2^30");
    if (max_width <= 0 || max_height <= 0 || max_width > 16384 || max_height > 16384)
        return fail(ADR_ERR_INVALID, "max image size must be in 1..16384");
    if ((int64_t)((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile) > kMaxTiles)
        return fail(ADR_ERR_INVALID, "at most %d tiles of 16x16 pixels (e.g. 4096x4096)", kMaxTiles);
    int ndev = 0;
    ADR_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(ADR_ERR_INVALID, "device %d not present", device);
    DeviceGuard guard(device);

    adr_ctx* c = new adr_ctx();
    c->device = device;
    c->max_n = max_gaussians;
    c->capacity = pair_capacity;
    c->max_w = max_width;
    c->max_h = max_height;
    c->max_tiles = ((max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { free_ctx(c); return fail(ADR_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e)); }
    c->sm_count = prop.multiProcessorCount;
    c->sort_grid = c->sm_count * onesweep_blocks_per_sm();
    c->scan_grid = c->sm_count * scan_blocks_per_sm();

    const size_t N = (size_t)max_gaussians, P = (size_t)pair_capacity;
    const size_t chunks = ((N > P ? N : P) + kSortChunk - 1) / kSortChunk + 1;
    c->lookback_words = chunks * kRadix;
#define ALLOC(ptr, bytes)                                                                   \
    do {                                                                                    \
        e = cudaMalloc((void**)&(ptr), (bytes));                                           \
        if (e != cudaSuccess) {                                                             \
            free_ctx(c);                                                                    \
            return fail(ADR_ERR_CUDA, "cudaMalloc(%zu) for %s: %s", (size_t)(bytes), #ptr,  \
                        cudaGetErrorString(e));                                             \
        }                                                                                   \
    } while (0)
    ALLOC(c->rec, N * kRecFloat4 * sizeof(float4));
    ALLOC(c->aux, N * kAuxFloat4 * sizeof(float4));
    ALLOC(c->depth_key, N * sizeof(uint32_t));
    ALLOC(c->tiles, N * sizeof(uint32_t));
    ALLOC(c->rect, N * sizeof(ushort4));
    ALLOC(c->offsets, N * sizeof(uint32_t));
    for (int b = 0; b < 2; ++b) {
        ALLOC(c->gkeys[b], N * sizeof(uint32_t));
        ALLOC(c->gvals[b], N * sizeof(uint32_t));
        ALLOC(c->ptile[b], P * sizeof(uint32_t));
        ALLOC(c->pgauss[b], P * sizeof(uint32_t));
    }
    ALLOC(c->ranges, (size_t)c->max_tiles * sizeof(uint2));
    ALLOC(c->last, (size_t)max_width * max_height * sizeof(int32_t));
    ALLOC(c->trav, (size_t)max_width * max_height * sizeof(int32_t));
    ALLOC(c->hist, (kMaxPasses + 2) * kRadix * sizeof(uint32_t));
    ALLOC(c->counters, kCntSlots * sizeof(uint32_t));
    ALLOC(c->status, sizeof(uint32_t) * 4);
    ALLOC(c->lookback, c->lookback_words * sizeof(unsigned long long));
#undef ALLOC
    e = cudaHostAlloc((void**)&c->host_words, 64 * sizeof(uint32_t), cudaHostAllocDefault);
    if (e != cudaSuccess) { free_ctx(c); return fail(ADR_ERR_CUDA, "cudaHostAlloc: %s", cudaGetErrorString(e)); }
    if (cudaMemset(c->lookback, 0, c->lookback_words * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->status, 0, sizeof(uint32_t) * 4) != cudaSuccess ||
        cudaMemset(c->counters, 0, kCntSlots * sizeof(uint32_t)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        free_ctx(c);
        return fail(ADR_ERR_CUDA, "workspace initialisation failed");
    }
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
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (n < 0 || n > c->max_n) return fail(ADR_ERR_INVALID, "n=%lld outside 0..%lld", (long long)n, (long long)c->max_n);
    if (n > 0 && (!means || !scales || !rots || !opac || !sh))
        return fail(ADR_ERR_INVALID, "a Gaussian parameter pointer is NULL");
    if (n > 0 && (!aligned(means, 4) || !aligned(scales, 4) || !aligned(opac, 4) ||
                  !aligned(rots, 16) || !aligned(sh, 16)))
        return fail(ADR_ERR_INVALID, "rots and sh must be 16-byte aligned, the rest 4-byte aligned");
    CamDev cam;
    SetDev st;
    adr_status s;
    if ((s = make_cam(c, camera, cam)) != ADR_OK) return s;
    if ((s = make_settings(settings, st)) != ADR_OK) return s;
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->n = n;
    c->cam = cam;
    c->st = st;
    const int64_t num_tiles = (int64_t)cam.tiles_x * cam.tiles_y;
    c->tile_bits = ceil_log2(num_tiles);
    c->tile_passes = (c->tile_bits + kRadixBits - 1) / kRadixBits;
    c->last_stream = strm;

    ADR_CUDA(cudaMemsetAsync(c->counters, 0, kCntSlots * sizeof(uint32_t), strm));
    ADR_CUDA(cudaMemsetAsync(c->hist, 0, (kMaxPasses + 2) * kRadix * sizeof(uint32_t), strm));
    launch_preprocess((int)n, means, scales, rots, opac, sh, cam, st, c->rec, c->aux, c->depth_key,
                      c->tiles, c->rect, strm);
    // Gaussians by view depth: 4 stable 8-bit passes (keys of culled Gaussians
    // are 0xFFFFFFFF and sort last; they carry no tiles).
    launch_digit_hist(c->depth_key, n, nullptr, 0, kMaxPasses, c->hist, c->sm_count * 4, strm);
    const uint32_t* kin = c->depth_key;
    const uint32_t* vin = nullptr;
    for (int p = 0; p < kMaxPasses; ++p) {
        uint32_t* kout = c->gkeys[p & 1];
        uint32_t* vout = c->gvals[p & 1];
        launch_onesweep(kin, vin, kout, vout, n, nullptr, 8 * p, 8, c->hist + p * kRadix,
                        c->lookback, next_epoch(c, strm), c->counters + kCntSortTicket0 + p,
                        c->status, c->sort_grid, strm);
        kin = kout;
        vin = vout;
    }
    c->sorted_order = vin;
    launch_scan_tiles(c->sorted_order, c->tiles, n, c->offsets, c->lookback, next_epoch(c, strm),
                      c->counters, c->status, c->scan_grid, strm);
    launch_emit(c->sorted_order, c->tiles, c->offsets, c->rect, n, cam, c->capacity, c->ptile[0],
                c->pgauss[0], c->hist + kMaxPasses * kRadix, c->tile_passes, c->tile_bits,
                c->status, strm);
    if ((s = check_launch("adr_preprocess")) != ADR_OK) return s;
    c->have_frame = true;
    c->have_sort = false;
    return ok();
}

adr_status adr_sort(adr_ctx* c, void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_frame) return fail(ADR_ERR_INVALID, "adr_sort before adr_preprocess");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    const uint32_t* d_n = c->counters + kCntPairs;
    const int tk = kCntSortTicket0 + kMaxPasses;
    ADR_CUDA(cudaMemsetAsync(c->counters + tk, 0, 2 * sizeof(uint32_t), strm));
    int cur = 0;
    for (int p = 0; p < c->tile_passes; ++p) {
        const int bits = (c->tile_bits - 8 * p) < 8 ? (c->tile_bits - 8 * p) : 8;
        launch_onesweep(c->ptile[cur], c->pgauss[cur], c->ptile[cur ^ 1], c->pgauss[cur ^ 1],
                        c->capacity, d_n, 8 * p, bits, c->hist + (kMaxPasses + p) * kRadix,
                        c->lookback, next_epoch(c, strm), c->counters + tk + p, c->status,
                        c->sort_grid, strm);
        cur ^= 1;
    }
    c->sorted_tile = c->ptile[cur];
    c->sorted_gauss = c->pgauss[cur];
    const int64_t num_tiles = (int64_t)c->cam.tiles_x * c->cam.tiles_y;
    ADR_CUDA(cudaMemsetAsync(c->ranges, 0, num_tiles * sizeof(uint2), strm));
    launch_ranges(c->sorted_tile, d_n, c->capacity, (uint32_t)num_tiles, c->ranges,
                  c->sm_count * 8, strm);
    adr_status s;
    if ((s = check_launch("adr_sort")) != ADR_OK) return s;
    c->have_sort = true;
    return ok();
}

adr_status adr_render(adr_ctx* c, float* img, float* t_final, int32_t* load, void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_sort) return fail(ADR_ERR_INVALID, "adr_render before adr_sort");
    if (!img) return fail(ADR_ERR_INVALID, "img is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    c->last_stream = strm;
    launch_render(c->ranges, c->sorted_gauss, c->rec, c->cam, c->st, img, t_final, load, c->last,
                  c->trav, strm);
    c->have_render = true;
    return check_launch("adr_render") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_sync_status(adr_ctx* c) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    DeviceGuard guard(c->device);
    ADR_CUDA(cudaStreamSynchronize(c->last_stream));
    ADR_CUDA(cudaMemcpy(c->host_words, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    const uint32_t bits = c->host_words[0];
    ADR_CUDA(cudaMemset(c->status, 0, sizeof(uint32_t)));
    if (bits & kErrLookback) return fail(ADR_ERR_TIMEOUT, "a device-side lookback wait gave up");
    if (bits & kErrCapacity) return fail(ADR_ERR_CAPACITY, "pair count exceeded pair_capacity");
    if (bits & kErrRange) return fail(ADR_ERR_TIMEOUT, "a scatter index was out of range (skipped)");
    return ok();
}

adr_status adr_num_pairs(adr_ctx* c, int64_t* num_pairs) {
    if (!c || !num_pairs) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->have_frame) return fail(ADR_ERR_INVALID, "adr_num_pairs before adr_preprocess");
    DeviceGuard guard(c->device);
    ADR_CUDA(cudaStreamSynchronize(c->last_stream));
    ADR_CUDA(cudaMemcpy(c->host_words, c->counters, kCntSlots * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost));
    *num_pairs = (int64_t)c->host_words[kCntPairs];
    adr_status s = adr_sync_status(c);
    if (s != ADR_OK) return s;
    if (*num_pairs > c->capacity) return fail(ADR_ERR_CAPACITY, "P=%lld exceeds pair_capacity=%lld",
                                              (long long)*num_pairs, (long long)c->capacity);
    return ok();
}

adr_status adr_read_pairs(adr_ctx* c, uint64_t* keys, uint32_t* vals, int64_t capacity,
                          void* stream) {
    if (!c || !keys || !vals) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->have_sort) return fail(ADR_ERR_INVALID, "adr_read_pairs before adr_sort");
    if (capacity < 0) return fail(ADR_ERR_INVALID, "negative capacity");
    DeviceGuard guard(c->device);
    const int64_t cap = capacity < c->capacity ? capacity : c->capacity;
    launch_pair_keys(c->sorted_tile, c->sorted_gauss, c->depth_key, c->counters + kCntPairs, cap,
                     reinterpret_cast<unsigned long long*>(keys), vals, (cudaStream_t)stream);
    return check_launch("adr_read_pairs") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_read_gaussians(adr_ctx* c, float* geom, int32_t* rect, int32_t* tiles,
                              void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_frame) return fail(ADR_ERR_INVALID, "adr_read_gaussians before adr_preprocess");
    DeviceGuard guard(c->device);
    launch_read_gaussians(c->rec, c->aux, c->rect, c->tiles, (int)c->n, geom, rect, tiles,
                          (cudaStream_t)stream);
    return check_launch("adr_read_gaussians") == ADR_OK ? ok() : ADR_ERR_CUDA;
}

adr_status adr_read_ranges(adr_ctx* c, uint32_t* ranges, void* stream) {
    if (!c || !ranges) return fail(ADR_ERR_INVALID, "NULL argument");
    if (!c->have_sort) return fail(ADR_ERR_INVALID, "adr_read_ranges before adr_sort");
    DeviceGuard guard(c->device);
    const size_t bytes = (size_t)c->cam.tiles_x * c->cam.tiles_y * sizeof(uint2);
    ADR_CUDA(cudaMemcpyAsync(ranges, c->ranges, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ok();
}

adr_status adr_read_pixel_stats(adr_ctx* c, int32_t* last, int32_t* traversed, void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!c->have_render) return fail(ADR_ERR_INVALID, "adr_read_pixel_stats before adr_render");
    DeviceGuard guard(c->device);
    const size_t bytes = (size_t)c->cam.width * c->cam.height * sizeof(int32_t);
    if (last) ADR_CUDA(cudaMemcpyAsync(last, c->last, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    if (traversed)
        ADR_CUDA(cudaMemcpyAsync(traversed, c->trav, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ok();
}

adr_status adr_render_host(adr_ctx* c, const float* means, const float* scales, const float* rots,
                           const float* opac, const float* sh, int64_t n, const adr_camera* camera,
                           const adr_settings* settings, float* img, float* t_final, int32_t* load,
                           void* stream) {
    if (!c) return fail(ADR_ERR_INVALID, "ctx is NULL");
    if (!img) return fail(ADR_ERR_INVALID, "img is NULL");
    if (n < 0 || n > c->max_n) return fail(ADR_ERR_INVALID, "n outside 0..max_gaussians");
    if (n > 0 && (!means || !scales || !rots || !opac || !sh))
        return fail(ADR_ERR_INVALID, "a Gaussian parameter pointer is NULL");
    if (!camera) return fail(ADR_ERR_INVALID, "camera is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t strm = (cudaStream_t)stream;
    const size_t N = (size_t)c->max_n;
    const size_t per = 3 + 3 + 4 + 1 + 48;   // floats per Gaussian
    if (!c->stage) {
        ADR_CUDA(cudaMalloc((void**)&c->stage, N * per * sizeof(float)));
        ADR_CUDA(cudaMalloc((void**)&c->stage_img, (size_t)c->max_w * c->max_h * 4 * sizeof(float)));
        ADR_CUDA(cudaMalloc((void**)&c->stage_load, (size_t)c->max_w * c->max_h * sizeof(int32_t)));
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
    const size_t hw = (size_t)camera->width * camera->height;
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
