// adr_render_frame_noalloc: the whole forward path (preprocess, depth sort,
// tile-count scan, pair emission, tile sort, ranges, render) for small frames,
// with every intermediate buffer carved out of one file-scope device array
// instead of memory the caller or the library allocates at run time.
//
// Who needs it: callers that cannot call cudaMalloc (or anything that does)
// when they render, e.g. a host application whose GPU memory is owned by
// another allocator and forbids allocations after start-up, a real-time loop
// where an allocation's implicit device synchronisation is unacceptable, or
// a plugin loaded into a process that has no spare device memory budget for
// a library context.  They pass their own input and output buffers; the
// scratch lives in the library image itself.
//
// The array is sized for at most kNaMaxGaussians Gaussians, kNaMaxPairs
// Gaussian-tile pairs and kNaMaxWidth x kNaMaxHeight images (about 20 MB).
// CUDA loads this file's module (the array and its kernels) on a device when
// the module is first used there, by default lazily at the first call on that
// device; from then on that device holds the array until the process exits.
// Callers for whom that first load (a one-time allocation by the driver, and
// possibly a synchronisation) is unacceptable make the first call during
// start-up, or run with CUDA_MODULE_LOADING=EAGER.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int64_t kNaMaxGaussians = 1 << 15;
constexpr int64_t kNaMaxPairs = 1 << 20;
constexpr int kNaMaxWidth = 512;
constexpr int kNaMaxHeight = 512;
constexpr int kNaMaxTiles = (kNaMaxWidth / kTile) * (kNaMaxHeight / kTile);
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte offsets of each buffer inside the array.
constexpr size_t kPixels = (size_t)kNaMaxWidth * kNaMaxHeight;
constexpr size_t kOffRec = 0;
constexpr size_t kOffAux = align256(kOffRec + kNaMaxGaussians * kRecFloat4 * 16);
constexpr size_t kOffDepth = align256(kOffAux + kNaMaxGaussians * kAuxFloat4 * 16);
constexpr size_t kOffOffsets = align256(kOffDepth + kNaMaxGaussians * 4);
constexpr size_t kOffGBox = align256(kOffOffsets + kNaMaxGaussians * 4);
constexpr size_t kOffSortedBox = align256(kOffGBox + kNaMaxGaussians * 4);
constexpr size_t kOffGKeys = align256(kOffSortedBox + kNaMaxGaussians * 4);   // 2 buffers
constexpr size_t kOffGVals = align256(kOffGKeys + 2 * kNaMaxGaussians * 4);   // 2 buffers
constexpr size_t kOffPRuns = align256(kOffGVals + 2 * kNaMaxGaussians * 4);
constexpr size_t kOffPRows = align256(kOffPRuns + kNaMaxPairs * 8);
constexpr size_t kOffPGauss = align256(kOffPRows + (kNaMaxPairs + 8) * 2);
constexpr size_t kOffChunkFirst = align256(kOffPGauss + kNaMaxPairs * 4);
constexpr size_t kOffRanges = align256(kOffChunkFirst + (kNaMaxPairs / kSortChunk + 2) * 4);
constexpr size_t kOffLast = align256(kOffRanges + kNaMaxTiles * 8);
constexpr size_t kOffTrav = align256(kOffLast + kPixels * 4);
constexpr size_t kOffTfin = align256(kOffTrav + kPixels * 4);
constexpr size_t kOffHist = align256(kOffTfin + kPixels * 4);
constexpr size_t kOffCounters = align256(kOffHist + kHistWords * 4);
constexpr size_t kOffStatus = align256(kOffCounters + kCntSlots * 4);
constexpr size_t kLookbackWords = (kNaMaxGaussians / kSortChunk + 2) * kRadix;
constexpr size_t kOffFrameParams = align256(kOffStatus + 16);
constexpr size_t kOffStage = align256(kOffFrameParams + sizeof(FrameParams));
constexpr size_t kOffTCounts = align256(kOffStage + 16);
constexpr size_t kOffTTotals = align256(kOffTCounts + (size_t)kRadix * kMaxTileGrid * 4);
constexpr size_t kOffTileCounts = align256(kOffTTotals + 2 * kRadix * 4);
constexpr size_t kOffLookback = align256(kOffTileCounts + kNaMaxTiles * 4);
constexpr size_t kNaBytes = align256(kOffLookback + kLookbackWords * 8);

// The scratch.  Zero-initialised when the module loads (the lookback words
// rely on that: a zero word never matches a pass's non-zero epoch).
static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

struct DeviceState {
    unsigned char* base = nullptr;   // device address of g_na_scratch on this device
    Workspace ws;                    // buffers inside the array
    std::atomic<uint32_t> epoch{0};
};

std::mutex g_setup_mutex;
DeviceState g_state[kMaxDevices];

// Once per device, with that device current: resolve the array's device
// address (the host-side symbol is only a stand-in) and size the grids.
adr_status setup(int dev, DeviceState*& out) {
    if (dev < 0 || dev >= kMaxDevices) return report_error(ADR_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceState& s = g_state[dev];
    if (!s.base) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || p == nullptr)
            return report_error(ADR_ERR_CUDA, "cudaGetSymbolAddress(g_na_scratch) failed");
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            return report_error(ADR_ERR_CUDA, "cudaDeviceGetAttribute(multiProcessorCount) failed");
        unsigned char* b = static_cast<unsigned char*>(p);
        Workspace& w = s.ws;
        w.max_n = kNaMaxGaussians;
        w.capacity = kNaMaxPairs;
        w.max_tiles = kNaMaxTiles;
        w.sm_count = sms;
        w.sort_grid = sms * onesweep_blocks_per_sm();
        w.scan_grid = sms * scan_blocks_per_sm();
        w.tile_grid = sms * tile_scatter_blocks_per_sm();
        if (w.tile_grid > kMaxTileGrid) w.tile_grid = kMaxTileGrid;
        w.rec = reinterpret_cast<float4*>(b + kOffRec);
        w.aux = reinterpret_cast<float4*>(b + kOffAux);
        w.depth_key = reinterpret_cast<uint32_t*>(b + kOffDepth);
        w.offsets = reinterpret_cast<uint32_t*>(b + kOffOffsets);
        w.gbox = reinterpret_cast<uint32_t*>(b + kOffGBox);
        w.sorted_box = reinterpret_cast<uint32_t*>(b + kOffSortedBox);
        for (int k = 0; k < 2; ++k) {
            w.gkeys[k] = reinterpret_cast<uint32_t*>(b + kOffGKeys) + k * kNaMaxGaussians;
            w.gvals[k] = reinterpret_cast<uint32_t*>(b + kOffGVals) + k * kNaMaxGaussians;
        }
        w.pruns = reinterpret_cast<uint2*>(b + kOffPRuns);
        w.prows = reinterpret_cast<uint16_t*>(b + kOffPRows);
        w.pgauss = reinterpret_cast<uint32_t*>(b + kOffPGauss);
        w.tile_counts = reinterpret_cast<uint32_t*>(b + kOffTileCounts);
        w.tcounts = reinterpret_cast<uint32_t*>(b + kOffTCounts);
        w.ttotals = reinterpret_cast<uint32_t*>(b + kOffTTotals);
        w.chunk_first = reinterpret_cast<uint32_t*>(b + kOffChunkFirst);
        w.ranges = reinterpret_cast<uint2*>(b + kOffRanges);
        w.last = reinterpret_cast<int32_t*>(b + kOffLast);
        w.trav = reinterpret_cast<int32_t*>(b + kOffTrav);
        w.tfin = reinterpret_cast<float*>(b + kOffTfin);
        w.hist = reinterpret_cast<uint32_t*>(b + kOffHist);
        w.counters = reinterpret_cast<uint32_t*>(b + kOffCounters);
        w.status = reinterpret_cast<uint32_t*>(b + kOffStatus);
        w.lookback = reinterpret_cast<unsigned long long*>(b + kOffLookback);
        w.d_fp = reinterpret_cast<FrameParams*>(b + kOffFrameParams);
        w.d_stage = reinterpret_cast<uint32_t*>(b + kOffStage);
        w.lookback_words = kLookbackWords;
        s.base = b;
    }
    out = &s;
    return ADR_OK;
}

}  // namespace
}  // namespace adr

using namespace adr;

extern "C" adr_status adr_render_frame_noalloc(const float* means, const float* scales,
                                               const float* rots, const float* opac,
                                               const float* sh, int64_t n,
                                               const adr_camera* camera,
                                               const adr_settings* settings, float* img,
                                               float* t_final, int32_t* load, void* stream) {
    if (n < 0 || n > kNaMaxGaussians)
        return report_error(ADR_ERR_INVALID,
                            "adr_render_frame_noalloc: n must be in 0..32768 (static scratch limit)");
    if (!img) return report_error(ADR_ERR_INVALID, "adr_render_frame_noalloc: img is NULL");
    if (n > 0 && (!means || !scales || !rots || !opac || !sh))
        return report_error(ADR_ERR_INVALID, "adr_render_frame_noalloc: a parameter pointer is NULL");
    if (n > 0 && ((uintptr_t)rots % 16 || (uintptr_t)sh % 16 || (uintptr_t)means % 4 ||
                  (uintptr_t)scales % 4 || (uintptr_t)opac % 4))
        return report_error(ADR_ERR_INVALID,
                            "adr_render_frame_noalloc: rots and sh must be 16-byte aligned");
    CamDev cam;
    SetDev st;
    adr_status s = camera_to_dev(camera, kNaMaxWidth, kNaMaxHeight, cam);
    if (s != ADR_OK) return s;   // includes images larger than 512 x 512
    if ((s = settings_to_dev(settings, st)) != ADR_OK) return s;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return report_error(ADR_ERR_CUDA, "cudaGetDevice failed");
    DeviceState* ds = nullptr;
    if ((s = setup(dev, ds)) != ADR_OK) return s;

    const Workspace& ws = ds->ws;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: clear what must start at zero.
    if (cudaMemsetAsync(ws.status, 0, 16, strm) != cudaSuccess)
        return report_error(ADR_ERR_CUDA, "adr_render_frame_noalloc: cudaMemsetAsync failed");
    FrameState fs;
    fill_frame_state(fs, n, cam, st);
    enqueue_preprocess(ws, fs, ds->epoch, means, scales, rots, opac, sh, strm);
    enqueue_sort(ws, fs, ds->epoch, strm);
    enqueue_render(ws, fs, img, t_final, load, strm);
    if (cudaGetLastError() != cudaSuccess)
        return report_error(ADR_ERR_CUDA, "adr_render_frame_noalloc: kernel launch failed");

    // Report pair overflow and bounded-wait expiry: read the status word and the
    // pair count back (into host stack memory) and wait for the frame.
    uint32_t words[2] = {0, 0};
    if (cudaMemcpyAsync(&words[0], ws.status, 4, cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
        cudaMemcpyAsync(&words[1], ws.counters + kCntPairs, 4, cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
        cudaStreamSynchronize(strm) != cudaSuccess)
        return report_error(ADR_ERR_CUDA, "adr_render_frame_noalloc: status readback failed");
    // A wait that gave up skips the frame and reads its pair count as
    // saturated, so it is reported before the capacity check.
    const StatusReport r = status_from_bits(words[0], (int64_t)words[1], kNaMaxPairs);
    if (r.status == ADR_ERR_CAPACITY)
        return report_error(ADR_ERR_CAPACITY,
                            "adr_render_frame_noalloc: more than 1048576 Gaussian-tile pairs "
                            "(static scratch limit); the image is incomplete");
    if (r.status != ADR_OK) {
        char msg[256];
        snprintf(msg, sizeof msg, "adr_render_frame_noalloc: %s", r.message);
        return report_error(r.status, msg);
    }
    return report_ok();
}
