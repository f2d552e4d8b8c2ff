// blink_grid_sorted.cuh -- deterministic, atomic-free gridding of a band of
// canonical rows from the sorted row buckets (Sec. 5.2.1 steps 2-3).
//
// In a row bucket the entries of one cell are contiguous (ordered by column,
// then baseline).  Per chunk of NT x kRowGridU entries, thread t takes entries
// [kRowGridU t, kRowGridU (t+1)): it loads their baselines and cells and the
// visibilities (gains applied, conjugated for mirrored baselines), and a
// block-wide segmented scan (in-thread, warp shuffles, then across warps)
// gives each run of equal cells its sum at its last entry, which adds it to
// the cell.  Each cell has one writer per chunk and chunks follow one another,
// so the grid never depends on timing: the image is the same bits on every
// call.  The caller maps a cell key (row - r0) << 16 | column to its address.
//
// Latency: the first chunk's loads are issued before `prologue` (the caller's
// zeroing and copies) and the barrier after it, and every later chunk's
// baselines and cells are loaded while the chunk before it is summed.
#pragma once
#include "blink_common.cuh"
#include "blink_image_small.cuh"

namespace blink {

namespace {

// Segmented-sum operator on (partial sum, "a run starts here") pairs:
// (a, fa) + (b, fb) = (fb ? b : a + b, fa | fb).  Associative, so a scan with a
// fixed tree of these gives every run's sum in an order set by the chunk
// layout alone.
struct SegSum {
    float2 v;
    bool head;
};
__device__ __forceinline__ SegSum seg_add(const SegSum &a, const SegSum &b) {
    return SegSum{b.head ? b.v : make_float2(a.v.x + b.v.x, a.v.y + b.v.y), a.head || b.head};
}

constexpr int kRowGridU = 8;
struct GridChunk {
    uint32_t key[kRowGridU], bl[kRowGridU];
    uint32_t conj;          // bit u: entry u is a mirrored baseline
    uint32_t kprev, knext;  // cell keys of the entries just before and after this thread's
    int n;                  // entries in the chunk (<= 0: none)
};

__device__ __forceinline__ void grid_load_codes(GridChunk &c, const uint2 *__restrict__ ents, int c0, int n, int r0,
                                                int tid) {
    constexpr int U = kRowGridU;
    constexpr uint32_t kPastEnd = 0xFFFFFFFFu, kBeforeStart = 0xFFFFFFFEu;  // never a cell key
    auto key_of = [r0](uint32_t code) { return ((code_row(code) - uint32_t(r0)) << 16) | code_col(code); };
    const int i0 = tid * U;
    c.n = n;
    c.conj = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const bool live = i0 + u < n;
        const uint2 en = live ? __ldg(ents + c0 + i0 + u) : make_uint2(0u, 0u);
        c.bl[u] = en.x;
        c.key[u] = live ? key_of(en.y) : kPastEnd;
        c.conj |= (live && code_conj(en.y)) ? (1u << u) : 0u;
    }
    c.kprev = (i0 > 0 && i0 <= n) ? key_of(__ldg(ents + c0 + i0 - 1).y) : kBeforeStart;
    c.knext = i0 + U < n ? key_of(__ldg(ents + c0 + i0 + U).y) : kPastEnd;
}

__device__ __forceinline__ void grid_load_vis(const GridChunk &c, float2 (&v)[kRowGridU],
                                              const float2 *__restrict__ vis, const LayerGains &gl, int tid) {
    const int i0 = tid * kRowGridU;
#pragma unroll
    for (int u = 0; u < kRowGridU; ++u) v[u] = i0 + u < c.n ? __ldg(vis + c.bl[u]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kRowGridU; ++u) {
        if (i0 + u < c.n) {
            if (gl) v[u] = apply_gain(v[u], gl, c.bl[u]);
            if ((c.conj >> u) & 1u) v[u].y = -v[u].y;
        }
    }
}

// Segmented scan of one chunk and its cell updates (two barriers).  `cell`
// returns the address of a cell key, or null for a cell outside the band's
// storage (its run is not written).
template <int NT, class Cell>
__device__ __forceinline__ void grid_sum_chunk(const GridChunk &c, const float2 (&v)[kRowGridU], int tid,
                                               Cell &&cell) {
    constexpr int U = kRowGridU, NW = NT / 32;
    __shared__ float2 s_wv[NW];
    __shared__ int s_wh[NW];
    const int lane = tid & 31, warp = tid >> 5, i0 = tid * U;
    const unsigned full = 0xFFFFFFFFu;
    SegSum agg{v[0], c.key[0] != c.kprev};
#pragma unroll
    for (int u = 1; u < U; ++u) agg = seg_add(agg, SegSum{v[u], c.key[u] != c.key[u - 1]});
    SegSum inc = agg;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        SegSum up;
        up.v.x = __shfl_up_sync(full, inc.v.x, d);
        up.v.y = __shfl_up_sync(full, inc.v.y, d);
        up.head = __shfl_up_sync(full, int(inc.head), d) != 0;
        if (lane >= d) inc = seg_add(up, inc);
    }
    if (lane == 31) {
        s_wv[warp] = inc.v;
        s_wh[warp] = int(inc.head);
    }
    SegSum ex;  // everything before this thread's entries, inside the warp
    ex.v.x = __shfl_up_sync(full, inc.v.x, 1);
    ex.v.y = __shfl_up_sync(full, inc.v.y, 1);
    ex.head = __shfl_up_sync(full, int(inc.head), 1) != 0;
    __syncthreads();
    SegSum pre{make_float2(0.f, 0.f), false};
    for (int w = 0; w < warp; ++w) pre = seg_add(pre, SegSum{s_wv[w], s_wh[w] != 0});
    SegSum run = lane == 0 ? pre : seg_add(pre, ex);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        run = seg_add(run, SegSum{v[u], c.key[u] != (u == 0 ? c.kprev : c.key[u - 1])});
        const bool last = u + 1 < U ? c.key[u + 1] != c.key[u] : c.knext != c.key[u];
        if (i0 + u < c.n && last) {
            float2 *p = cell(c.key[u]);
            if (p) {
                p->x += run.v.x;
                p->y += run.v.y;
            }
        }
    }
    __syncthreads();  // cells and warp sums are reused by the next chunk
}

// Grids the entries [ptr[r0], ptr[r0 + nrows]) of one layer.  Every thread
// of the NT-thread block calls it; `prologue` runs once all threads have
// issued the first chunk's loads, followed by a barrier.
template <int NT, class Cell, class Prologue>
__device__ __forceinline__ void grid_band_sorted(int r0, int nrows, const int32_t *__restrict__ ptr,
                                                 const uint2 *__restrict__ ents, const float2 *__restrict__ vis,
                                                 const LayerGains &gl, int tid, Cell &&cell, Prologue &&prologue) {
    constexpr int CH = NT * kRowGridU;
    const int e_begin = __ldg(ptr + r0), e_end = __ldg(ptr + r0 + nrows);
    GridChunk cur;
    float2 v[kRowGridU];
    int c0 = e_begin;
    grid_load_codes(cur, ents, c0, min(CH, e_end - c0), r0, tid);
    grid_load_vis(cur, v, vis, gl, tid);
    prologue();
    __syncthreads();
    while (cur.n > 0) {
        GridChunk nxt;
        const int c1 = c0 + CH;
        grid_load_codes(nxt, ents, c1, min(CH, e_end - c1), r0, tid);
        grid_sum_chunk<NT>(cur, v, tid, cell);
        cur = nxt;
        c0 = c1;
        if (cur.n > 0) grid_load_vis(cur, v, vis, gl, tid);
    }
}

}  // namespace

}  // namespace blink
