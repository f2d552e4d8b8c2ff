// blink_compact.cu -- compact gridding of large-image layers (Sec. 5.2.1
// steps 2-3, and the weighting of Sec. 4.4.2).
//
// The support of a large image is often a small part of its grid: a station
// imaged at 512^2 or 1024^2 with the cell size of its all-sky image touches
// only rows r < R and columns |k_u| <= kmax.  Where that compact grid fits in
// shared memory, one CTA per layer grids the whole layer there: the layer's
// visibilities pass through shared memory in chunks of kCgChunk baselines
// (coalesced 16-byte copies, two chunks in flight), and the chunk's entries,
// sorted by cell at plan time (k_cg_sort), are summed run by run, each run
// (cell) by one thread in entry order -- every random read is a shared-memory
// read, every cell gets one add per chunk, chunks in order, so the result
// does not depend on timing.  The CTA then applies the weights,
// completes row 0 with its Hermitian mirror and writes the compact grid; the
// row items of the large-image path expand its rows, so they no longer gather
// visibilities from global memory.
#include "blink_common.cuh"
#include "blink_grid_sorted.cuh"
#include "blink_kernels.cuh"

#include <algorithm>

namespace blink {

namespace {

constexpr int kCgThreads = 256;
static_assert(kCgThreads * kRowGridU == kCgChunk, "eight entries per thread cover a staging chunk");

// Entries [8 tid, 8 tid + 8) of a chunk with n kept entries, as packed words
// (cell << 12 | conj << 11 | index in the chunk), and the cells of the entries
// just before and after them.
struct CgChunk {
    uint32_t w[kRowGridU];
    uint32_t kprev, knext;  // cells of entries 8 tid - 1 and 8 tid + 8 (sentinels outside)
    int n;
};

__device__ __forceinline__ void cg_load_ents(CgChunk &c, const uint32_t *__restrict__ e, int n, int tid) {
    constexpr int U = kRowGridU;
    const int i0 = tid * U;
    c.n = n;
    if (i0 < n) {  // the chunk's words are 16-byte aligned: two vector loads
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(e + i0));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(e + i0 + 4));
        c.w[0] = a.x; c.w[1] = a.y; c.w[2] = a.z; c.w[3] = a.w;
        c.w[4] = b.x; c.w[5] = b.y; c.w[6] = b.z; c.w[7] = b.w;
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) c.w[u] = 0xFFFFFFFFu;
    }
    c.kprev = (i0 > 0 && i0 <= n) ? __ldg(e + i0 - 1) >> 12 : 0xFFFFFFFEu;  // never a cell
    c.knext = i0 + U < n ? __ldg(e + i0 + U) >> 12 : 0xFFFFFFFFu;
}

// cp.async of baselines [b0, b0 + n) of a layer's visibilities into dst
// (16-byte pieces when the source is 16-byte aligned), one commit group.
__device__ __forceinline__ void cg_stage(float2 *dst, const float2 *src, int n, int tid, uint64_t pol) {
    const uint32_t d = uint32_t(__cvta_generic_to_shared(dst));
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        for (int i = tid; i < n / 2; i += kCgThreads)
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(d + 16 * i),
                         "l"(src + 2 * i), "l"(pol)
                         : "memory");
        if ((n & 1) && tid == 0)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d + 8 * (n - 1)), "l"(src + n - 1)
                         : "memory");
    } else {
        for (int i = tid; i < n; i += kCgThreads)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d + 8 * i), "l"(src + i) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Sums of one chunk.  The entries are sorted by cell, so each cell is one run;
// the thread whose window [8 tid, 8 tid + 8) holds a run's first entry adds
// the whole run to the cell, entry by entry in order -- past the window's end
// when the run goes on.  A cell therefore has one writer per chunk and one
// fixed summation order: no scan, no atomics.  buf holds the chunk's staged
// visibilities (baselines b0 ..).
__device__ __forceinline__ void cg_sum_chunk(float2 *G, const CgChunk &c, const uint32_t *__restrict__ e,
                                             const float2 *buf, int64_t b0, const LayerGains &gl, int tid) {
    constexpr int U = kRowGridU;
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    const int i0 = tid * U;
    if (i0 >= c.n) return;
    auto value = [&](uint32_t w) {
        float2 x = buf[w & 0x7FFu];
        if (gl) x = apply_gain(x, gl, b0 + (w & 0x7FFu));
        if ((w >> 11) & 1u) x.y = -x.y;
        return x;
    };
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = i0 + u < c.n ? value(c.w[u]) : make_float2(0.f, 0.f);
    uint32_t last = kNone;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t k = c.w[u] >> 12;
        if (i0 + u < c.n && k != c.kprev) {  // leading entries equal to kprev continue an earlier run
            float2 *p = G + k;
            p->x += v[u].x;
            p->y += v[u].y;
            last = k;
        }
    }
    if (last != kNone && c.knext == last) {  // the last run goes on past the window
        for (int j = i0 + U; j < c.n; ++j) {
            const uint32_t w = __ldg(e + j);
            if ((w >> 12) != last) break;
            const float2 x = value(w);
            G[last].x += x.x;
            G[last].y += x.y;
        }
    }
}

// One CTA per layer l0 + blockIdx.x of a.layers; its compact grid goes to
// a.cg + blockIdx.x * a.cg_stride.  Shared memory: the compact grid of the
// group's largest support, then two staging chunks.
__global__ void __launch_bounds__(kCgThreads, 3) k_grid_compact(ImageArgs a, int l0) {
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x;
    const DevLayer L = a.layers[l0 + blockIdx.x];
    const ChanInfo ci = a.chans[L.chan];
    const int N = ci.n_px, R = ci.rows, km = ci.kmax_u, kc = 2 * km + 1;
    const int ncell = R * kc;
    float2 *G = sm;
    float2 *stg = sm + ((a.cg_stride + 1) & ~int64_t(1));  // 16-byte aligned
    const CsrLayout cl(N, a.nb);
    const uint32_t *ents = reinterpret_cast<const uint32_t *>(a.csr + ci.csr_off + cl.cg_ents);
    const int32_t *cnt = reinterpret_cast<const int32_t *>(a.csr + ci.csr_off + cl.cg_cnt);
    const float2 *vis = a.vis + L.vis_off;
    const LayerGains gl = layer_gains(a, L);
    const uint64_t pol = l2_evict_first();
    const int Q = cl.n_cg;
    auto chunk_n = [&](int q) { return int(a.nb - int64_t(q) * kCgChunk < kCgChunk ? a.nb - int64_t(q) * kCgChunk
                                                                                   : int64_t(kCgChunk)); };
    CgChunk cur;
    if (Q > 0) {
        cg_stage(stg, vis, chunk_n(0), tid, pol);
        cg_load_ents(cur, ents, __ldg(cnt), tid);
    }
    for (int i = tid; i < ncell; i += kCgThreads) G[i] = make_float2(0.f, 0.f);
    for (int q = 0; q < Q; ++q) {
        CgChunk nxt;
        const bool more = q + 1 < Q;
        if (more) {
            // the other buffer was last read in chunk q - 1, before the
            // barrier that ended its sums
            cg_stage(stg + ((q + 1) & 1) * kCgChunk, vis + int64_t(q + 1) * kCgChunk, chunk_n(q + 1), tid, pol);
            cg_load_ents(nxt, ents + int64_t(q + 1) * kCgChunk, __ldg(cnt + q + 1), tid);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();  // chunk q staged by every thread; the grid zeroed
        const float2 *buf = stg + (q & 1) * kCgChunk;
        cg_sum_chunk(G, cur, ents + int64_t(q) * kCgChunk, buf, int64_t(q) * kCgChunk, gl, tid);
        __syncthreads();  // the chunk's adds precede the next chunk's; its buffer is free
        if (more) cur = nxt;
    }
    // weights (rows >= 1), then row 0: weight, origin 2 Re(V) w, mirror
    // G[0][-k_u] = conj G[0][k_u] (row 0 was gridded at k_u >= 0 only)
    const float *w = ci.weighting == 1 ? a.wgt + ci.wgt_off : nullptr;
    if (w)
        for (int i = kc + tid; i < ncell; i += kCgThreads) {
            const int r = i / kc, ku = i % kc - km;
            const float wv = w[r * N + (ku < 0 ? ku + N : ku)];
            G[i].x *= wv;
            G[i].y *= wv;
        }
    for (int ku = tid; ku <= km; ku += kCgThreads) {
        const float wv = w ? w[ku] : 1.f;
        const float2 g = G[km + ku];
        if (ku == 0) {
            G[km] = make_float2(2.f * g.x * wv, 0.f);
        } else {
            G[km + ku] = make_float2(g.x * wv, g.y * wv);
            G[km - ku] = make_float2(g.x * wv, -g.y * wv);
        }
    }
    __syncthreads();
    float2 *dst = a.cg + int64_t(blockIdx.x) * a.cg_stride;
    for (int i = tid; i < ncell; i += kCgThreads) dst[i] = G[i];
}

// Scheduled compact gridding: the register-accumulation schedule of the
// fused small-image kernel, built for the channel's own size (slot positions
// r (N + 1) + c).  Per chunk of the schedule the visibilities, the entry
// stream segment and its metadata are staged with cp.async; each thread sums
// the entries of the <= kSchedSlots cells it owns in registers over all
// chunks (one add per entry, no per-chunk writes), then writes every owned
// cell once, weighted, into the compact grid in shared memory (row 0 with its
// mirror), which goes out coalesced.  The sums follow the schedule's fixed
// entry order: the same bits on every call.
__global__ void __launch_bounds__(kSchedThreads, 2) k_grid_compact_sched(ImageArgs a, int l0) {
    constexpr int NT = kSchedThreads;
    extern __shared__ float2 sm[];
    const DevLayer L = a.layers[l0 + blockIdx.x];
    const ChanInfo ci = a.chans[L.chan];
    const int N = ci.n_px, S = N + 1, R = ci.rows, km = ci.kmax_u, kc = 2 * km + 1, ncell = R * kc;
    const int Q = ci.n_chunks, K = ci.chunk, M = ci.m_slots;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SchedLayout lay(N, a.nb, Q);
    const StageLayout sl(a.max_chunk, a.max_seg, kSchedSlots);
    const unsigned char *blk = a.sched + ci.sched_off;
    const uint2 *meta_g = reinterpret_cast<const uint2 *>(blk + lay.meta);
    const uint16_t *stream_g = reinterpret_cast<const uint16_t *>(blk + lay.stream);
    char *smc = reinterpret_cast<char *>(sm);
    float2 *stage = reinterpret_cast<float2 *>(smc + sl.vis);
    const uint16_t *ent = reinterpret_cast<const uint16_t *>(smc + sl.ent);
    const uint2 *meta = reinterpret_cast<const uint2 *>(smc + sl.meta);
    const float2 *vis = a.vis + L.vis_off;
    const LayerGains gl = layer_gains(a, L);
    const uint64_t pol_vis = l2_evict_first();

    float2 acc[kSchedSlots];
#pragma unroll
    for (int j = 0; j < kSchedSlots; ++j) acc[j] = make_float2(0.f, 0.f);
    if (tid == 0) stage[K] = make_float2(0.f, 0.f);  // sentinel target
    const int per_chunk = M * kSchedWarps;
    auto seg_start = [&](int c) { return c < Q ? int(__ldg(&meta_g[c * per_chunk].x)) : ci.stream_len; };
    int s_beg = seg_start(0), s_end = seg_start(1);
    for (int q = 0; q < Q; ++q) {
        const int64_t rem = a.nb - int64_t(q) * K;
        const int n_q = int(rem < K ? rem : int64_t(K));
        const int s0 = s_beg & ~7;
        stage_async<NT>(stage, vis + int64_t(q) * K, n_q, tid, pol_vis);
        cp16_async<NT>(smc + sl.ent, stream_g + s0, (s_end - s0 + 7) >> 3, tid);
        cp16_async<NT>(smc + sl.meta, meta_g + q * per_chunk, per_chunk >> 1, tid);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const int s_next = seg_start(q + 2);
        stage_wait();
        __syncthreads();
        if (gl) {  // gains on the staged visibilities (fused epilogue)
            const int64_t b0 = int64_t(q) * K;
            for (int e = tid; e < n_q; e += NT) stage[e] = apply_gain(stage[e], gl, b0 + e);
            __syncthreads();
        }
        const int shift = -s0;
#pragma unroll
        for (int j = 0; j < kSchedSlots; ++j) {
            if (j < M) {
                const uint2 m = meta[j * kSchedWarps + warp];
                const uint16_t *e = ent + int(m.x) + shift + lane;
                float2 sum = make_float2(0.f, 0.f);
#pragma unroll 4
                for (uint32_t k = 0; k < m.y; ++k) {
                    const uint32_t code = e[32 * k];
                    const float2 v = stage[code & 0x7FFFu];
                    sum.x += v.x;
                    sum.y += (code & 0x8000u) ? -v.y : v.y;
                }
                acc[j].x += sum.x;
                acc[j].y += sum.y;
            }
        }
        s_beg = s_end;
        s_end = s_next;
        __syncthreads();
    }
    // the staging area becomes the compact grid: zero it, write the slots
    float2 *G = sm;
    const uint32_t *slot_pos = reinterpret_cast<const uint32_t *>(blk + lay.slot_pos);
    const float *slot_w = reinterpret_cast<const float *>(blk + lay.slot_w);
    for (int i = tid; i < ncell; i += NT) G[i] = make_float2(0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSchedSlots; ++j) {
        if (j < M) {
            const uint32_t sp = __ldg(slot_pos + j * NT + tid);
            if (sp != kSlotEmpty) {
                const float wv = __ldg(slot_w + j * NT + tid);
                const int p = int(sp & 0x3FFFFFFFu), r = p / S, c = p % S, ku = c <= N / 2 ? c : c - N;
                if (sp & kSlotOrigin) {
                    G[km] = make_float2(2.f * acc[j].x * wv, 0.f);
                } else {
                    const float2 g = make_float2(acc[j].x * wv, acc[j].y * wv);
                    G[r * kc + ku + km] = g;
                    if (sp & kSlotMirror) G[km - ku] = make_float2(g.x, -g.y);  // row 0
                }
            }
        }
    }
    __syncthreads();
    float2 *dst = a.cg + int64_t(blockIdx.x) * a.cg_stride;
    for (int i = tid; i < ncell; i += NT) dst[i] = G[i];
}

}  // namespace

size_t grid_compact_smem(int64_t cg_stride) {
    return size_t((cg_stride + 1) & ~int64_t(1)) * sizeof(float2) + 2 * size_t(kCgChunk) * sizeof(float2);
}

Error launch_grid_compact(const ImageArgs &a, int l0, int cnt, cudaStream_t st) {
    if (cnt <= 0) return Error{0, ""};
    if (!a.cg || cnt > a.cg_cap) return Error{-3, "compact gridding without its buffer"};
    if (a.sched && a.sched_ok) {  // every channel of the group has its schedule
        const size_t smem = std::max(size_t(StageLayout(a.max_chunk, a.max_seg, kSchedSlots).bytes),
                                     size_t(a.cg_stride) * sizeof(float2));
        BLINK_CUDA_TRY(
            cudaFuncSetAttribute(k_grid_compact_sched, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        for (int k = 0; k < cnt; k += 1 << 30) {
            const int c = std::min(cnt - k, 1 << 30);
            ImageArgs b = a;
            b.cg = a.cg + int64_t(k) * a.cg_stride;
            k_grid_compact_sched<<<unsigned(c), kSchedThreads, smem, st>>>(b, l0 + k);
            BLINK_CUDA_TRY(cudaGetLastError());
        }
        return Error{0, ""};
    }
    if (!a.csr) return Error{-3, "compact gridding without its tables"};
    const size_t smem = grid_compact_smem(a.cg_stride);
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_grid_compact, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    for (int k = 0; k < cnt; k += 1 << 30) {
        const int c = std::min(cnt - k, 1 << 30);
        ImageArgs b = a;
        b.cg = a.cg + int64_t(k) * a.cg_stride;
        k_grid_compact<<<unsigned(c), kCgThreads, smem, st>>>(b, l0 + k);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

}  // namespace blink
