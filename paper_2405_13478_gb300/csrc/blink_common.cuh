// blink_common.cuh -- types shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace blink {

constexpr double kSpeedOfLight = 299792458.0;  // m/s (SI definition)
constexpr int32_t kDropped = INT32_MIN;        // cell of a baseline that is not gridded
constexpr uint32_t kCodeDropped = 0xFFFFFFFFu;  // packed canonical cell of a dropped baseline

// Per-channel geometry.  A "channel" is one distinct (n_px, weighting,
// freq_hz, delta_u) among the layers of a call: every layer of a channel
// shares the same cells, because a coplanar zenith-phased array has
// time-independent (u,v) (Sec. 4.3).
struct ChanGeom {
    double freq_hz;
    double delta_u;
    int32_t n_px;
    int32_t weighting;
};

// Per-channel results of the table kernels.
struct ChanInfo {
    int32_t n_px;
    int32_t weighting;
    int32_t rows;      // support rows R: canonical rows 0..R-1 can be non-zero
    int32_t kmax_u;    // max |k_u| over kept baselines
    int64_t n_kept;    // baselines kept (|k| <= N/2-1)
    float wsum;        // summed weight of all grid entries
    int32_t pad;
    int64_t code_off;  // element offset into the packed-code table ([B] per channel)
    int64_t wgt_off;   // element offset into the weight table ([N/2][N] floats), -1 if natural
};

// Per-layer work item on the device.
struct DevLayer {
    int64_t vis_off;  // complex64 element offset of the layer's visibilities
    int64_t out_off;  // element offset of the layer's output
    int32_t chan;     // channel index
    int32_t layer;    // index in the caller's layer array (for d_wsum)
};

// Canonical half-grid cell of a baseline, packed in 32 bits:
//   bits 0-14  column c = k_u mod N (after the mirror below), N <= 16384
//   bit  15    1 if conj(V) is gridded there (baseline mirrored into the half)
//   bits 16-31 row r = k_v >= 0
// The canonical half is k_v > 0, or k_v == 0 and k_u >= 0.  Every kept
// baseline lands on exactly one canonical cell; the other half of the grid is
// its Hermitian mirror G[-k] = conj(G[k]).
__host__ __device__ inline uint32_t pack_code(uint32_t r, uint32_t c, uint32_t conj) {
    return (r << 16) | (conj << 15) | c;
}
__host__ __device__ inline uint32_t code_row(uint32_t code) { return code >> 16; }
__host__ __device__ inline uint32_t code_col(uint32_t code) { return code & 0x7FFFu; }
__host__ __device__ inline uint32_t code_conj(uint32_t code) { return (code >> 15) & 1u; }

// Status plumbing.
struct Error {
    int status;
    std::string msg;
};

}  // namespace blink

#define BLINK_CUDA_TRY(call)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ::blink::Error{-3, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)
