// Internal declarations shared by the CUDA translation units of libadr.so.
// Nothing here is part of the public C ABI (see include/adr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adr.h"

namespace adr {

constexpr int kTile = ADR_TILE;          // 16x16 pixel tiles (Sec. 3.2)
constexpr int kTilePixels = kTile * kTile;

// Device-side error word bits (ctx->d_status[0]).
constexpr uint32_t kErrCapacity = 1u;    // more Gaussian-tile pairs than pair_capacity
constexpr uint32_t kErrLookback = 2u;    // a decoupled-lookback wait hit its iteration limit
constexpr uint32_t kErrRange = 4u;       // a scatter index fell outside its buffer (skipped)

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
    float bg[3];
    int sh_degree;
};

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

// Per-call counters kept on the device (ctx->d_counters).
enum Counter : int {
    kCntPairs = 0,        // number of pairs P (sum of tiles over Gaussians)
    kCntVisible = 1,      // Gaussians with at least one tile
    kCntScanTicket = 2,   // chunk ticket of the tile-count scan
    kCntSortTicket0 = 4,  // chunk tickets of the sort passes (kMaxPasses * 2 slots)
    kCntSlots = 16
};

// Launchers (each enqueues on `stream`; all pointers are device memory).
void launch_preprocess(int n, const float* means, const float* scales, const float* rots,
                       const float* opac, const float* sh, const CamDev& cam, const SetDev& st,
                       float4* rec, float4* aux, uint32_t* depth_key, uint32_t* tiles,
                       ushort4* rect, cudaStream_t stream);

// Histogram of `passes` 8-bit digits of u32 keys (count read from *d_n if
// d_n != nullptr, else n).  hist must hold passes*256 zeroed u32.
void launch_digit_hist(const uint32_t* keys, int64_t n, const uint32_t* d_n, int shift0, int passes,
                       uint32_t* hist, int grid, cudaStream_t stream);

// One stable onesweep pass of 8-bit digit at `shift`.  vals_in == nullptr
// means the values are the indices 0..n-1.  lookback holds chunks*256 u64.
void launch_onesweep(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                     uint32_t* vals_out, int64_t n, const uint32_t* d_n, int shift, int digit_bits,
                     const uint32_t* hist, unsigned long long* lookback, uint32_t epoch,
                     uint32_t* ticket, uint32_t* status, int grid, cudaStream_t stream);

// Exclusive scan of tiles[order[i]] with decoupled lookback; writes offsets,
// the total to counters[kCntPairs] and the non-empty count to kCntVisible.
void launch_scan_tiles(const uint32_t* order, const uint32_t* tiles, int64_t n, uint32_t* offsets,
                       unsigned long long* lookback, uint32_t epoch, uint32_t* counters,
                       uint32_t* status, int grid, cudaStream_t stream);

// Emit (tile, Gaussian) pairs in depth order; accumulates the tile-digit
// histogram for the pair sort.
void launch_emit(const uint32_t* order, const uint32_t* tiles, const uint32_t* offsets,
                 const ushort4* rect, int64_t n, const CamDev& cam, int64_t capacity,
                 uint32_t* pair_tile, uint32_t* pair_gauss, uint32_t* tile_hist, int hist_passes,
                 int hist_bits, uint32_t* status, cudaStream_t stream);

void launch_ranges(const uint32_t* sorted_tile, const uint32_t* d_n, int64_t capacity,
                   uint32_t num_tiles, uint2* ranges, int grid, cudaStream_t stream);

void launch_render(const uint2* ranges, const uint32_t* sorted_gauss, const float4* rec,
                   const CamDev& cam, const SetDev& st, float* img, float* t_final, int32_t* load,
                   int32_t* last, int32_t* trav, cudaStream_t stream);

void launch_pair_keys(const uint32_t* sorted_tile, const uint32_t* sorted_gauss,
                      const uint32_t* depth_key_by_gauss, const uint32_t* d_n, int64_t count,
                      unsigned long long* keys_out, uint32_t* vals_out, cudaStream_t stream);

// Occupancy of the persistent kernels (CTAs per SM), for grid sizing.
int onesweep_blocks_per_sm();
int scan_blocks_per_sm();

void launch_read_gaussians(const float4* rec, const float4* aux, const ushort4* rect,
                           const uint32_t* tiles, int n, float* geom, int32_t* rect_out,
                           int32_t* tiles_out, cudaStream_t stream);

// Error reporting and argument conversion shared by the entry points.
adr_status report_error(adr_status st, const char* msg);
adr_status report_ok();
adr_status camera_to_dev(const adr_camera* cam, int max_w, int max_h, CamDev& d);
adr_status settings_to_dev(const adr_settings* s, SetDev& d);

}  // namespace adr
