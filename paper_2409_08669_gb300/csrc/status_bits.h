// The device-side error word of a frame and how every entry point that
// reports it (adr_sync_status, adr_render_frame_noalloc, the serving
// scheduler) turns it into an adr_status.  Host and device code; no CUDA
// calls, so the mapping is testable on a machine without a GPU.
#pragma once

#include <stdint.h>

#include "adr.h"

namespace adr {

// Device-side error word bits (Workspace::status[0]).
constexpr uint32_t kErrCapacity = 1u;    // more Gaussian-tile pairs than pair_capacity
constexpr uint32_t kErrLookback = 2u;    // a decoupled-lookback wait hit its iteration limit
constexpr uint32_t kErrRange = 4u;       // a scatter index fell outside its buffer (skipped)

struct StatusReport {
    adr_status status;
    const char* message;
};

// In order of precedence: a wait that gave up skips the rest of its frame and
// reads its pair count as saturated, so it comes before the capacity check;
// `pairs` is the frame's pair count as read back (or 0 when not read).
inline StatusReport status_from_bits(uint32_t bits, int64_t pairs, int64_t capacity) {
    if (bits & kErrLookback)
        return {ADR_ERR_TIMEOUT, "a device-side lookback wait gave up; the frame was skipped"};
    if ((bits & kErrCapacity) || pairs > capacity)
        return {ADR_ERR_CAPACITY, "the frame has more Gaussian-tile pairs than the pair capacity; "
                                  "the image is incomplete"};
    if (bits & kErrRange)
        return {ADR_ERR_CUDA, "device-side consistency check: a scatter index fell outside its "
                              "buffer (the write was skipped)"};
    return {ADR_OK, ""};
}

}  // namespace adr
