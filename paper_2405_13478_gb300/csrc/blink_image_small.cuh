// blink_image_small.cuh -- the fused single-CTA image kernels (N <= 256).
//
// One CTA per layer grids the whole layer in shared memory and runs both
// passes of the inverse 2-D FFT there, so a layer costs one read of its
// visibilities and one write of its image (Sec. 5.2.1 steps 1-3 and
// Sec. 5.2.2, fused).  Two gridding forms:
//   k_image_sched  atomic-free: a per-channel schedule tells every thread
//                  which staged visibilities belong to the <= 16 canonical
//                  cells it owns; it sums them in registers and writes each
//                  cell once (deterministic, bit-reproducible);
//   k_image_small  shared-memory float atomics (channels without a schedule).
// Layout and transform conventions are those of blink_image_impl.cuh: only
// the canonical half-grid (rows k_v >= 0, columns in FFT order) is built,
// pass 1 transforms the support rows along u, pass 2 pairs two real image
// columns in one complex transform along v, and the output fftshift is folded
// into the store addresses.
#pragma once
#include "blink_common.cuh"
#include "blink_fft.cuh"
#include "blink_kernels.cuh"
#include "blink_pairs.cuh"

#include <algorithm>

namespace blink {

namespace {

constexpr int kNormalize = 1;


// Four-step twiddle W_N^(n2 k1) of the inverse transform (SIGN > 0) or its
// conjugate, read from the transposed global table: the lanes of a warp
// differ in n2, and the constant cache would serialise their distinct
// addresses where this read coalesces.
template <int N, int SIGN>
__device__ __forceinline__ c32 four_step_tw(int k1, int n2) {
    const float2 w = __ldg(reinterpret_cast<const float2 *>(&g_four_step<N>.v[k1 * Plan<N>::N2 + n2]));
    return c32{w.x, SIGN > 0 ? w.y : -w.y};
}

// Fused epilogue, gains: visibility b of a layer becomes g_i conj(g_j) V_b
// (calibration applied after correlation, Sec. 4.2 step ii).  gl is the
// layer's gain row (null: no gains).
// A layer's gains: its row of the gain-product table (gp, when the host built
// one) or its row of antenna gains (gl, products formed per visibility).
struct LayerGains {
    const float2 *gl;
    const float2 *gp;
    int n_ant;
    __device__ __forceinline__ explicit operator bool() const { return gl != nullptr; }
};

__device__ __forceinline__ LayerGains layer_gains(const ImageArgs &a, const DevLayer &L) {
    if (!a.gains) return LayerGains{nullptr, nullptr, a.n_ant};
    const int64_t row = a.gain_stride == 0 ? 0
                        : (a.gain_period > 0 ? int64_t(L.layer) % a.gain_period : int64_t(L.layer));
    return LayerGains{a.gains + row * a.gain_stride, a.gprod ? a.gprod + row * a.nb : nullptr, a.n_ant};
}

__device__ __forceinline__ float2 cmul(float2 p, float2 v) {
    return make_float2(p.x * v.x - p.y * v.y, p.x * v.y + p.y * v.x);
}

__device__ __forceinline__ float2 apply_gain(float2 v, const LayerGains &g, int64_t b) {
    if (g.gp) return cmul(__ldg(g.gp + b), v);
    int i, j;
    baseline_pair(b, g.n_ant, i, j);
    const float2 gi = __ldg(g.gl + i), gj = __ldg(g.gl + j);
    return cmul(make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y), v);  // g_i conj(g_j) V
}


// ------------------------------------------------------------- small path
// One CTA per layer; every step after the tables happens in shared
// memory.  Thread layout: 16-lane groups.  In the four-step A steps a lane is
// n2 (its twiddles W_N^(n2 k1) live in registers for the whole kernel) and a
// group is a row (pass 1) or a column pair (pass 2); in pass-1 step B a lane
// is k1; in pass-2 step B a lane is a column pair so image stores coalesce.
template <int N>
struct SmallCfg {
    static constexpr int NT = 384;
    static constexpr int GROUPS = NT / 16;  // 16-lane groups per CTA
    static constexpr int P = GROUPS;        // column pairs per pass-2 chunk
    static_assert(N > 256 || (Plan<N>::N1 <= 16 && Plan<N>::N2 <= 16), "small path needs N1, N2 <= 16");
};

// Grid one layer into G (stride S) with shared-memory float atomics.  Four
// baselines per 16-byte code load and two 16-byte visibility loads; two quads
// in flight per thread before any atomic.
template <int NT>
__device__ __forceinline__ void grid_layer_vec(float2 *G, int S, const uint32_t *code,
                                               const float2 *vis, int64_t nb, int tid,
                                               const LayerGains gl) {
    auto put = [&](uint32_t cd, float re, float im, int64_t b) {
        if (cd == kCodeDropped) return;
        if (gl) {
            const float2 v = apply_gain(make_float2(re, im), gl, b);
            re = v.x;
            im = v.y;
        }
        float2 *cell = G + code_row(cd) * S + code_col(cd);
        atomicAdd(&cell->x, re);
        atomicAdd(&cell->y, code_conj(cd) ? -im : im);
    };
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(code) | reinterpret_cast<uintptr_t>(vis)) & 15) == 0) {
        const int64_t nq = nb >> 2;
        const uint4 *c4 = reinterpret_cast<const uint4 *>(code);
        const float4 *v4 = reinterpret_cast<const float4 *>(vis);
        for (int64_t q = tid; q < nq; q += 2 * NT) {
            const bool two = q + NT < nq;
            const uint4 ca = __ldg(c4 + q);
            const float4 va = __ldcs(v4 + 2 * q), vb = __ldcs(v4 + 2 * q + 1);
            uint4 cb = make_uint4(kCodeDropped, kCodeDropped, kCodeDropped, kCodeDropped);
            float4 vc = make_float4(0.f, 0.f, 0.f, 0.f), vd = vc;
            if (two) {
                cb = __ldg(c4 + q + NT);
                vc = __ldcs(v4 + 2 * (q + NT));
                vd = __ldcs(v4 + 2 * (q + NT) + 1);
            }
            const int64_t b0 = 4 * q, b1 = 4 * (q + NT);
            put(ca.x, va.x, va.y, b0);
            put(ca.y, va.z, va.w, b0 + 1);
            put(ca.z, vb.x, vb.y, b0 + 2);
            put(ca.w, vb.z, vb.w, b0 + 3);
            put(cb.x, vc.x, vc.y, b1);
            put(cb.y, vc.z, vc.w, b1 + 1);
            put(cb.z, vd.x, vd.y, b1 + 2);
            put(cb.w, vd.z, vd.w, b1 + 3);
        }
        done = nq << 2;
    }
    for (int64_t b = done + tid; b < nb; b += NT) {
        const float2 v = __ldcs(vis + b);
        put(__ldg(code + b), v.x, v.y, b);
    }
}

// Both passes of the transform for one layer whose canonical rows [0, R) are
// in G (stride N + 1), Hermitian-complete in row 0.  Rows >= 1 are multiplied
// by w_rows (uniform weights, [N/2][N]) on the way in when it is not null.
// Sum of one double per thread over the CTA, in a fixed order (a shuffle
// tree per warp, then the warps' sums in warp order), so the result has the
// same bits on every run; valid in thread 0.  Every thread calls it.
template <int NT>
__device__ __forceinline__ double block_sum_f64(double v, int tid) {
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // the previous call's reads of red are done
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

// Sum of squares of a layer's output (the fused epilogue's per-layer norm):
// slot `slot` of the layer's row of partial sums gets `s`; with slot 0 the
// caller also zeroes slots [used, stride), which its size never writes, so
// that the per-layer total can add a fixed number of slots.
template <int NT>
__device__ __forceinline__ void store_sq_slot(double *row, int slot, int used, int stride, double s, int tid) {
    if (tid == 0) row[slot] = s;
    if (slot == 0)
        for (int i = used + tid; i < stride; i += NT) row[i] = 0.0;
}

// With want_sq, the sum of the squares of the stored values is returned
// (valid in thread 0): each task's squares (2 N2 values) added in FP32, the
// tasks' sums in FP64, in a fixed order.
template <int N>
__device__ __forceinline__ double small_transform(float2 *G, float2 *Z, int R, const float *w_rows,
                                                  float *img, float scale, int tid, const float *ref,
                                                  bool want_sq = false) {
    constexpr int NT = SmallCfg<N>::NT, GR = SmallCfg<N>::GROUPS, P = SmallCfg<N>::P;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, S = N + 1, H = N / 2;
    const int ln = tid & 15, grp = tid >> 4;
    // four-step twiddles W_N^(n2 k1) for n2 = ln (kept in registers), from
    // the transposed table: coalesced loads instead of constant-cache reads,
    // which would serialise over the 16 distinct lanes
    c32 tw[N1];
    {
        const int n2c = ln < N2 ? ln : N2 - 1;  // lanes >= N2 idle in the A steps
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) tw[k1] = four_step_tw<N, +1>(k1, n2c);
    }
    double acc = 0.0;  // squares of the stored values (want_sq)

    // pass 1, step A
    for (int r = grp; r < R; r += GR) {
        if (ln < N2) {
            float2 *row = G + r * S + ln;
            float2 x[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                float2 g = row[N2 * n1];
                if (w_rows && r > 0) {
                    const float wv = __ldg(w_rows + r * N + N2 * n1 + ln);
                    g.x *= wv;
                    g.y *= wv;
                }
                x[n1] = g;
            }
            dft<N1, +1>(x);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) row[N2 * k1] = k1 == 0 ? x[0] : cmulc(x[k1], tw[k1]);
        }
    }
    __syncthreads();
    // pass 1, step B: lanes are k1; result stays in place (transposed order)
    for (int r = grp; r < R; r += GR) {
        if (ln < N1) {
            float2 *run = G + r * S + N2 * ln;
            float2 y[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) y[n2] = run[n2];
            dft<N2, +1>(y);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) run[k2] = y[k2];
        }
    }
    __syncthreads();

    for (int j0 = 0; j0 < H; j0 += P) {
        // pass 2, step A: group = column pair, lane = n2
        {
            const int ja = j0 + grp;
            if (ja < H && ln < N2) {
                const int jb = ja + H;
                const int pa = N2 * (ja % N1) + ja / N1, pb = N2 * (jb % N1) + jb / N1;
                float2 x[N1];
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) {
                    const int k = N2 * n1 + ln;
                    float2 z = make_float2(0.f, 0.f);
                    if (k < H) {
                        if (k < R) {
                            const float2 u = G[k * S + pa], v = G[k * S + pb];
                            z = make_float2(u.x - v.y, u.y + v.x);  // H_a + i H_b
                        }
                    } else if (k > H) {
                        const int m = N - k;
                        if (m < R) {
                            const float2 u = G[m * S + pa], v = G[m * S + pb];
                            z = make_float2(u.x + v.y, v.x - u.y);  // conj(H_a) + i conj(H_b)
                        }
                    }
                    x[n1] = z;
                }
                dft<N1, +1>(x);
                float2 *zp = Z + grp * S + ln;
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) zp[N2 * k1] = k1 == 0 ? x[0] : cmulc(x[k1], tw[k1]);
            }
        }
        __syncthreads();
        // pass 2, step B: lane = column pair (coalesced stores), warp = k1
        {
            const int jj = tid & 31, ja = j0 + jj;
            if (jj < P && ja < H) {
                for (int k1 = tid >> 5; k1 < N1; k1 += NT / 32) {
                    const float2 *zp = Z + jj * S + N2 * k1;
                    // fused epilogue: every reference value this thread needs is
                    // requested before the transform, so the loads overlap it
                    float2 rf[N2];
                    if (ref) {
#pragma unroll
                        for (int k2 = 0; k2 < N2; ++k2) {
                            const int q = k1 + N1 * k2;
                            const float *rp = ref + (q < H ? q + H : q - H) * N;  // 32-bit: N * N < 2^31
                            rf[k2] = make_float2(__ldcs(rp + ja + H), __ldcs(rp + ja));
                        }
                    }
                    float2 y[N2];
#pragma unroll
                    for (int n2 = 0; n2 < N2; ++n2) y[n2] = zp[n2];
                    dft<N2, +1>(y);
                    float sq = 0.f;
#pragma unroll
                    for (int k2 = 0; k2 < N2; ++k2) {
                        const int q = k1 + N1 * k2;
                        const int row = q < H ? q + H : q - H;
                        const int o = row * N;  // offsets inside one image fit 32 bits
                        float va = y[k2].x * scale, vb = y[k2].y * scale;
                        if (ref) {
                            va -= rf[k2].x;
                            vb -= rf[k2].y;
                        }
                        __stcs(img + o + ja + H, va);
                        __stcs(img + o + ja, vb);
                        if (want_sq) sq = fmaf(va, va, fmaf(vb, vb, sq));
                    }
                    if (want_sq) acc += double(sq);
                }
            }
        }
        __syncthreads();
    }
    return want_sq ? block_sum_f64<NT>(acc, tid) : 0.0;
}

// L2 eviction policies (createpolicy): visibilities are read once, so they
// leave L2 first; a prefetched reference image should stay until it is used.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Fused epilogue: ask the TMA unit to pull a layer's reference image into L2
// at kernel start (cp.async.bulk.prefetch.L2), so the store phase reads it
// from L2 in whole lines instead of waiting on DRAM fragment by fragment.
// Only the 16-byte aligned interior is prefetched (the hint never touches
// bytes outside the image).
__device__ __forceinline__ void prefetch_l2(const float *p, int64_t n_floats, int tid, int nt) {
    const uintptr_t a0 = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t a1 = (reinterpret_cast<uintptr_t>(p + n_floats)) & ~uintptr_t(15);
    constexpr uintptr_t kPiece = 16384;
    const uint64_t pol = l2_evict_last();
    for (uintptr_t s0 = a0 + uintptr_t(tid) * kPiece; s0 < a1; s0 += uintptr_t(nt) * kPiece) {
        const uint32_t bytes = uint32_t(a1 - s0 < kPiece ? a1 - s0 : kPiece);
        asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(s0), "r"(bytes),
                     "l"(pol)
                     : "memory");
    }
}

// L2 prefetch of [p, p + bytes) with the default eviction priority (the
// 16-byte aligned interior; a hint, never a fault outside the range).
__device__ __forceinline__ void prefetch_l2_bytes(const void *p, int64_t bytes, int tid, int nt) {
    const uintptr_t a0 = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t a1 = (reinterpret_cast<uintptr_t>(p) + uintptr_t(bytes)) & ~uintptr_t(15);
    constexpr uintptr_t kPiece = 16384;
    for (uintptr_t s0 = a0 + uintptr_t(tid) * kPiece; s0 < a1; s0 += uintptr_t(nt) * kPiece) {
        const uint32_t n = uint32_t(a1 - s0 < kPiece ? a1 - s0 : kPiece);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s0), "r"(n) : "memory");
    }
}

// Fused layer with shared-memory float atomics for the gridding (used when a
// channel has no register-accumulation schedule).
template <int N, bool EPI>
__global__ void __launch_bounds__(SmallCfg<N>::NT, 2) k_image_small(ImageArgs a, float *__restrict__ out,
                                                                     const float *__restrict__ ref) {
    constexpr int NT = SmallCfg<N>::NT, S = N + 1, H = N / 2;
    extern __shared__ float2 sm[];
    const DevLayer L = a.layers[blockIdx.x];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows;
    float2 *G = sm;
    float2 *Z = sm + size_t(a.r_alloc) * S;
    const int tid = threadIdx.x;
    const float *w = ci.weighting == 1 ? a.wgt + ci.wgt_off : nullptr;
    if (EPI && ref) prefetch_l2(ref + L.out_off, int64_t(N) * N, tid, NT);
    {
        float4 *g4 = reinterpret_cast<float4 *>(G);
        const int n4 = (R * S) >> 1;
        for (int i = tid; i < n4; i += NT) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (((R * S) & 1) && tid == 0) G[R * S - 1] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    grid_layer_vec<NT>(G, S, a.codes + ci.code_off, a.vis + L.vis_off, a.nb, tid,
                       EPI ? layer_gains(a, L) : LayerGains{nullptr, nullptr, 0});
    __syncthreads();
    // row 0: weights, origin doubling and Hermitian completion
    for (int c = tid; c < H; c += NT) {
        const float wv = w ? w[c] : 1.f;
        const float2 g = G[c];
        if (c == 0) {
            G[0] = make_float2(2.f * g.x * wv, 0.f);
        } else {
            G[c] = make_float2(g.x * wv, g.y * wv);
            G[N - c] = make_float2(g.x * wv, -g.y * wv);
        }
    }
    __syncthreads();
    const float scale = ((a.flags & kNormalize) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f;
    const bool want_sq = EPI && a.sq_part;
    const double sq = small_transform<N>(G, Z, R, w, out + L.out_off, scale, tid,
                                         EPI && ref ? ref + L.out_off : nullptr, want_sq);
    if (want_sq) store_sq_slot<NT>(a.sq_part + int64_t(L.layer) * a.sq_stride, 0, 1, a.sq_stride, sq, tid);
    if (tid == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return uint32_t(__cvta_generic_to_shared(p));
}

// Copy n complex64 values global -> shared with cp.async (16-byte pieces
// when the source is 16-byte aligned, else 8-byte pieces).  The 16-byte
// copies carry the L2 policy `pol`; the 8-byte ones (ragged or unaligned
// layers only) are plain: with the cache-hint qualifier they raised an
// illegal-instruction error on this GPU.  No wait here.
template <int NT>
__device__ __forceinline__ void stage_async(float2 *dst, const float2 *src, int n, int tid, uint64_t pol) {
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int n2 = n >> 1;
        for (int i = tid; i < n2; i += NT)
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst + 2 * i)),
                         "l"(src + 2 * i), "l"(pol)
                         : "memory");
        if ((n & 1) && tid == 0)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst + n - 1)), "l"(src + n - 1)
                         : "memory");
    } else {
        for (int i = tid; i < n; i += NT)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst + i)), "l"(src + i)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared-memory layout of the staging phase of k_image_sched: the chunk's
// visibilities (plus one zero element, the sentinel target), the chunk's
// stream segment (16-byte aligned copy) and its (slot, warp) metadata.
struct StageLayout {
    int vis, ent, meta, bytes;
    __host__ __device__ StageLayout(int chunk, int max_seg, int m_slots) {
        auto up16 = [](int x) { return (x + 15) / 16 * 16; };
        vis = 0;
        ent = up16((chunk + 1) * 8);
        meta = up16(ent + (max_seg + 16) * 2);
        bytes = meta + m_slots * kSchedWarps * 8;
    }
};

template <int NT>
__device__ __forceinline__ void cp16_async(void *dst, const void *src, int n16, int tid) {
    for (int i = tid; i < n16; i += NT)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(static_cast<char *>(dst) + 16 * i)),
                     "l"(static_cast<const char *>(src) + 16 * i)
                     : "memory");
}

// Fused layer with atomic-free gridding: for every chunk the visibilities,
// the chunk's entry stream and its metadata go to shared memory with
// cp.async; each thread gathers the entries of the cells it owns into
// registers (schedule in ChanInfo / SchedLayout), then writes every owned cell
// once, weighted, with row 0 completed.  Results do not depend on the plan.
template <int N, bool EPI>
__global__ void __launch_bounds__(SmallCfg<N>::NT, 2) k_image_sched(ImageArgs a, float *__restrict__ out,
                                                                     const float *__restrict__ ref) {
    constexpr int NT = SmallCfg<N>::NT, S = N + 1;
    static_assert(NT == kSchedThreads, "schedule built for a different CTA size");
    extern __shared__ float2 sm[];
    const DevLayer L = a.layers[blockIdx.x];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows, Q = ci.n_chunks, K = ci.chunk, M = ci.m_slots;
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
    const LayerGains gl = EPI ? layer_gains(a, L) : LayerGains{nullptr, nullptr, 0};
    const uint64_t pol_vis = l2_evict_first();
    if (EPI && ref) prefetch_l2(ref + L.out_off, int64_t(N) * N, tid, NT);

    float2 acc[kSchedSlots];
#pragma unroll
    for (int j = 0; j < kSchedSlots; ++j) acc[j] = make_float2(0.f, 0.f);
    if (tid == 0) stage[K] = make_float2(0.f, 0.f);  // sentinel target
    const int per_chunk = M * kSchedWarps;
    // stream segment bounds of chunk q: [s_beg, s_end); the end of the next
    // chunk is requested one chunk ahead so its latency hides behind a gather
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
        if (EPI && gl) {
            // fused epilogue: gains on the staged visibilities.  The chunk
            // covers antenna rows i_first..i_last of the upper triangle; warp w
            // takes rows i_first + w, i_first + w + 12, ... with g_i in a
            // register and its lanes striding over j (coalesced gain loads,
            // conflict-free shared memory, no per-entry pair arithmetic).
            const int64_t b0 = int64_t(q) * K;
            if (gl.gp) {  // products from the table: one coalesced load per entry
                for (int e = tid; e < n_q; e += NT) stage[e] = cmul(__ldg(gl.gp + b0 + e), stage[e]);
            } else {
            int i_first, j_first, i_last, j_last;
            baseline_pair(b0, a.n_ant, i_first, j_first);
            baseline_pair(b0 + n_q - 1, a.n_ant, i_last, j_last);
            for (int i = i_first + warp; i <= i_last; i += kSchedWarps) {
                const int e_row = int(pair_row_start(i, a.n_ant) - b0) - i - 1;  // entry of (i, j) = e_row + j
                const int jlo = i == i_first ? j_first : i + 1;
                const int jhi = i == i_last ? j_last : a.n_ant - 1;
                const float2 gi = __ldg(gl.gl + i);
                for (int j = jlo + lane; j <= jhi; j += 32) {
                    const float2 gj = __ldg(gl.gl + j);
                    const float pr = gi.x * gj.x + gi.y * gj.y, pim = gi.y * gj.x - gi.x * gj.y;
                    const float2 v = stage[e_row + j];
                    stage[e_row + j] = make_float2(pr * v.x - pim * v.y, pr * v.y + pim * v.x);
                }
            }
            }
            __syncthreads();
        }
        const int shift = -s0;
#pragma unroll
        for (int j = 0; j < kSchedSlots; ++j) {
            if (j < M) {
                const uint2 m = meta[j * kSchedWarps + warp];
                const uint16_t *e = ent + int(m.x) + shift + lane;
                float2 s = make_float2(0.f, 0.f);
#pragma unroll 4
                for (uint32_t k = 0; k < m.y; ++k) {
                    const uint32_t code = e[32 * k];
                    const float2 v = stage[code & 0x7FFFu];
                    s.x += v.x;
                    s.y += (code & 0x8000u) ? -v.y : v.y;
                }
                acc[j].x += s.x;
                acc[j].y += s.y;
            }
        }
        s_beg = s_end;
        s_end = s_next;
        __syncthreads();
    }
    // the staging area becomes the grid: zero the support rows, write the
    // slots.  The first kSlotBatch slot positions and weights are requested
    // before the zeroing so their latency overlaps it.
    float2 *G = sm;
    float2 *Z = sm + size_t(a.r_alloc) * S;
    const uint32_t *slot_pos = reinterpret_cast<const uint32_t *>(blk + lay.slot_pos);
    const float *slot_w = reinterpret_cast<const float *>(blk + lay.slot_w);
    constexpr int kSlotBatch = 8;
    uint32_t sp_b[kSlotBatch];
    float w_b[kSlotBatch];
#pragma unroll
    for (int j = 0; j < kSlotBatch; ++j) {
        sp_b[j] = j < M ? __ldg(slot_pos + j * NT + tid) : kSlotEmpty;
        w_b[j] = j < M ? __ldg(slot_w + j * NT + tid) : 0.f;
    }
    {
        float4 *g4 = reinterpret_cast<float4 *>(G);
        const int n4 = (R * S) >> 1;
        for (int i = tid; i < n4; i += NT) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (((R * S) & 1) && tid == 0) G[R * S - 1] = make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSchedSlots; ++j) {
        if (j < M) {
            const uint32_t sp = j < kSlotBatch ? sp_b[j] : __ldg(slot_pos + j * NT + tid);
            if (sp != kSlotEmpty) {
                const float wv = j < kSlotBatch ? w_b[j] : __ldg(slot_w + j * NT + tid);
                const int p = int(sp & 0x3FFFFFFFu);
                if (sp & kSlotOrigin) {
                    G[p] = make_float2(2.f * acc[j].x * wv, 0.f);
                } else {
                    const float2 g = make_float2(acc[j].x * wv, acc[j].y * wv);
                    G[p] = g;
                    if (sp & kSlotMirror) G[N - p] = make_float2(g.x, -g.y);
                }
            }
        }
    }
    __syncthreads();
    const float scale = ((a.flags & kNormalize) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f;
    const bool want_sq = EPI && a.sq_part;
    const double sq = small_transform<N>(G, Z, R, nullptr, out + L.out_off, scale, tid,
                                         EPI && ref ? ref + L.out_off : nullptr, want_sq);
    if (want_sq) store_sq_slot<NT>(a.sq_part + int64_t(L.layer) * a.sq_stride, 0, 1, a.sq_stride, sq, tid);
    if (tid == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
}

template <int N>
size_t small_smem(int r_alloc) {
    return size_t(r_alloc + SmallCfg<N>::P) * (N + 1) * sizeof(float2);
}

// Launches the fused kernel for a size group when the fused path takes it
// (sizes <= 256 whose support fits the shared-memory budget, and not forced
// to the two-kernel path); returns false when the group needs another path.
template <int N>
bool launch_fused_n(const ImageArgs &a, cudaStream_t st, Error &err) {
    err = Error{0, ""};
    if constexpr (N <= 256) {
        static_assert(SmallCfg<N>::P == kSmallColPairs, "column-pair buffer of the fused kernels");
        if (a.force_path >= 3 || !small_path_fits(N, a.r_alloc)) return false;
        size_t smem = small_smem<N>(a.r_alloc);
        const bool sched = a.sched && a.sched_ok && a.force_path != 2;
        if (sched) smem = std::max(smem, size_t(StageLayout(a.max_chunk, a.max_seg, kSchedSlots).bytes));
        const bool epi = a.gains || a.ref || a.sq_part;
        auto kern = sched ? (epi ? k_image_sched<N, true> : k_image_sched<N, false>)
                          : (epi ? k_image_small<N, true> : k_image_small<N, false>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) {
            err = Error{-3, std::string("fused kernel attribute: ") + cudaGetErrorString(e)};
            return true;
        }
        for (int l0 = 0; l0 < a.n_layers; l0 += 1 << 30) {
            ImageArgs b = a;
            b.layers = a.layers + l0;
            const int cnt = std::min(a.n_layers - l0, 1 << 30);
            kern<<<cnt, SmallCfg<N>::NT, smem, st>>>(b, static_cast<float *>(b.out), b.ref);
            e = cudaGetLastError();
            if (e != cudaSuccess) {
                err = Error{-3, std::string("fused kernel launch: ") + cudaGetErrorString(e)};
                return true;
            }
        }
        return true;
    } else {
        (void)a;
        (void)st;
        return false;
    }
}

}  // namespace

}  // namespace blink
