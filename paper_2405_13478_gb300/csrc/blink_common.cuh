// blink_common.cuh -- types shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

// Supported image sizes (N_px): products of small radices whose four-step
// split N = N1 * N2 has register-sized codelets.  Every per-size dispatch in
// the library expands this list.
#define BLINK_FOR_EACH_SIZE(X) \
    X(16) X(20) X(24) X(32) X(36) X(48) X(64) X(96) X(120) X(128) X(160) X(180) X(192) X(256) \
    X(360) X(384) X(512) X(768) X(1024)

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
    int32_t sched;     // 1 if the register-accumulation gridding schedule is built
    int64_t code_off;  // element offset into the packed-code table ([B] per channel)
    int64_t wgt_off;   // element offset into the count/weight table ([N/2][N]), -1 if none
    int32_t m_slots;   // cell slots per thread used by the schedule
    int32_t n_chunks;  // staging chunks per layer
    int32_t chunk;     // baselines per staging chunk
    int32_t stream_len;  // entries in the schedule stream
    int64_t sched_off;   // byte offset of this channel's schedule block (-1 if none)
    int32_t max_seg;     // longest per-chunk stream segment (entries)
    int32_t sched_large; // 1: the schedule serves the compact gridding of a size > 256
    int64_t csr_off;     // row-bucketed entries of this channel (-1 if none), see CsrLayout
};

// Kept baselines bucketed by canonical row (large images): row_ptr[r] ..
// row_ptr[r + 1] index ents = {baseline, packed code}; bucket N/2 holds the
// dropped baselines.  Inside a row bucket the entries are ordered by column,
// then by baseline; the dropped bucket by baseline.  Both orders come from
// stable counting sorts -- by row over blocks of kCsrBlock baselines (tot[r]
// counts bucket r; blk_off[r][blk] holds block blk's count of bucket r, then
// its first position), into ents_by_b; then by column inside every row --
// so the entries of one cell are contiguous and in a fixed order, and the
// gridding that sums them is deterministic.
//
// The same block also holds the chunk-sorted entries of the compact gridding
// (k_grid_compact): the baselines in chunks of kCgChunk, and inside chunk q
// its kept baselines ordered by compact cell, then baseline, one 32-bit word
// each: cell << 12 | conj << 11 | (baseline - q kCgChunk), where the compact
// cell of row r and column k_u is r (2 kmax + 1) + k_u + kmax (kmax: the
// channel's largest |k_u|).  cg_ents[q][i], i < cg_cnt[q]; the rest of a
// chunk's kCgChunk words are 0xFFFFFFFF.  Filled only for channels whose
// compact grid fits (cg_fits below).
constexpr int kCsrBlock = 256;        // baselines per block of the bucket sort
constexpr int kCsrMaxBuckets = 1024 / 2 + 1;  // largest supported n_px / 2 + 1
constexpr int kCgChunk = 2048;        // baselines per chunk of the compact gridding
struct CsrLayout {
    int64_t row_ptr, tot, blk_off, ents_by_b, ents, cg_ents, cg_cnt, bytes;
    int32_t n_blk, n_bkt;  // baseline blocks, buckets (n_px / 2 rows + dropped)
    int32_t n_cg;          // chunks of the compact gridding
    __host__ __device__ CsrLayout(int n_px, int64_t nb) {
        auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
        n_bkt = n_px / 2 + 1;
        n_blk = int32_t((nb + kCsrBlock - 1) / kCsrBlock);
        n_cg = int32_t((nb + kCgChunk - 1) / kCgChunk);
        int64_t o = 0;
        row_ptr = o; o = up(o + 4 * int64_t(n_bkt + 1));
        tot = o; o = up(o + 4 * int64_t(n_bkt));
        blk_off = o; o = up(o + 4 * int64_t(n_blk) * n_bkt);
        ents_by_b = o; o = up(o + 8 * nb);
        ents = o; o = up(o + 8 * nb);
        cg_ents = o; o = up(o + 4 * int64_t(n_cg) * kCgChunk);
        cg_cnt = o; o = up(o + 4 * int64_t(n_cg));
        bytes = o;
    }
};

// Compact grid of a large-image layer: its support rows r < R and columns
// |k_u| <= kmax only, row-major [R][2 kmax + 1] (complex64), weighted and
// with row 0 Hermitian-complete.  The group's layers take the compact
// gridding when that grid, for the group's largest R and kmax, fits
// kCgGridBytes (it is built in shared memory next to two staging chunks).
constexpr size_t kCgGridBytes = 40 * 1024;
__host__ __device__ inline int64_t cg_cells(int rows, int kmax) { return int64_t(rows) * (2 * kmax + 1); }
__host__ __device__ inline bool cg_fits(int rows, int kmax) { return cg_cells(rows, kmax) * 8 <= int64_t(kCgGridBytes); }

// Host bound of a channel's compact support from the array's extent
// (span_x, span_y: largest coordinate differences in metres): every baseline
// has |u| <= span_x / lambda, so |k_u| <= span_x / (lambda delta_u) + 1/2; two
// cells of margin cover the rounding.  Decides, before the tables are built,
// whether a large-size channel gets a gridding schedule.
inline bool cg_bound_fits(double span_x, double span_y, double freq_hz, double delta_u, int n_px) {
    const double lambda = kSpeedOfLight / freq_hz;
    const double tu = span_x / (lambda * delta_u), tv = span_y / (lambda * delta_u);
    if (!(tu < 1e6 && tv < 1e6)) return false;
    const int kmax = std::min(n_px / 2 - 1, int(tu) + 2);
    const int rows = std::min(n_px / 2, int(tv) + 3);
    return cg_fits(rows, kmax);
}

// Register-accumulation gridding schedule (one block per channel).
//
// A layer's visibilities are staged in shared memory in n_chunks chunks of
// `chunk` baselines.  Thread t of the imaging CTA owns up to kSchedSlots
// occupied canonical cells (slot j of thread t), handed out in order of
// decreasing entry count so the 32 lanes of a warp carry similar loads.  For
// chunk q, slot j and warp w the entries of the 32 lanes are interleaved
// (entry k of lane l at stream[base + 32 k + l]), padded to the longest lane
// with a sentinel that points at a zero staging element.  An entry is the
// baseline's index inside the chunk (15 bits) and a conjugate flag (bit 15).
constexpr int kSchedThreads = 384;
constexpr int kSchedWarps = kSchedThreads / 32;
constexpr int kSchedSlots = 16;
constexpr int kSchedMaxChunk = 8192;        // baselines per staging chunk (64 KB)
constexpr uint32_t kSlotEmpty = 0xFFFFFFFFu;
constexpr uint32_t kSlotOrigin = 1u << 30;  // slot is the origin cell: 2 Re(sum) * w
constexpr uint32_t kSlotMirror = 1u << 31;  // row-0 slot: also write conj at N - c

// The fused single-CTA image kernels (k_image_sched, k_image_small) take a
// group when its support rows plus the pass-2 column-pair buffer (24 pairs,
// 384 threads in 16-lane groups) fit this shared-memory budget.
constexpr int kSmallColPairs = 24;
constexpr size_t kSmallSmemLimit = 200 * 1024;
__host__ __device__ inline bool small_path_fits(int n_px, int rows) {
    return n_px <= 256 && size_t(rows + kSmallColPairs) * size_t(n_px + 1) * 8 <= kSmallSmemLimit;
}

struct SchedLayout {
    int64_t cnt_q, rank, cell_slot, slot_pos, slot_w, meta, stream, bytes;
    int64_t stream_cap;
    __host__ __device__ SchedLayout(int n_px, int64_t nb, int n_chunks) {
        const int64_t cells = int64_t(n_px / 2) * n_px;
        auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
        int64_t o = 0;
        cnt_q = o; o = up(o + 4 * cells * n_chunks);
        rank = o; o = up(o + 4 * nb);
        cell_slot = o; o = up(o + 4 * cells);
        slot_pos = o; o = up(o + 4 * int64_t(kSchedSlots) * kSchedThreads);
        slot_w = o; o = up(o + 4 * int64_t(kSchedSlots) * kSchedThreads);
        meta = o; o = up(o + 8 * int64_t(n_chunks) * kSchedSlots * kSchedWarps);
        stream_cap = 4 * nb + 32 * int64_t(n_chunks) * kSchedSlots * kSchedWarps;
        stream = o; o = up(o + 2 * (stream_cap + 16));
        bytes = o;
    }
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
