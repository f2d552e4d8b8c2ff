// blink_image_impl.cuh -- gridding and the shifted inverse 2-D FFT: kernel
// templates, included by the per-size translation units blink_image_<sizes>.cu.
//
// Layout of the gridded data.  Only the canonical half of each grid is ever
// built: rows r = k_v in [0, R) (R = support rows of the channel), columns
// c = k_u mod N (FFT order, so the ifftshift of Sec. 5.2.1 step 1 costs
// nothing).  Row 0 holds k_u >= 0 after gridding and is completed with its
// Hermitian mirror G[0][N-c] = conj(G[0][c]) before the transform; the other
// half-plane is never stored because G[-k] = conj(G[k]) (Sec. 5.2.1: the
// correlation matrix holds V_ij and V_ji = conj V_ij).
//
// Transform.  Pass 1: an N-point inverse DFT along u on every support row
// (four-step, N = N1 * N2).  Pass 2: along v the image is real, so two output
// columns (j and j + N/2) share one N-point complex transform,
// Z = H_a + i H_b with H[N-k] = conj(H[k]) and H = 0 for R <= k <= N-R;
// the real and imaginary parts of the result are the two image columns.  The
// output fftshift (Sec. 5.2.2) is folded into the store addresses.
//
// Paths.  Small images (blink_image_small.cuh): one CTA grids a whole layer
// in shared memory -- by default with the atomic-free register schedule --
// and runs both passes there.  Large images (this file): k_rows grids a band
// of rows per CTA and writes transformed rows to a scratch buffer; k_cols
// runs pass 2 from it.
#pragma once
#include "blink_common.cuh"
#include "blink_fft.cuh"
#include "blink_kernels.cuh"
#include "blink_pairs.cuh"
#include "blink_image_small.cuh"
#include "blink_grid_sorted.cuh"
#include "blink_sync.cuh"

#include <algorithm>

namespace blink {

namespace {


// Layers per wave of the two-kernel paths: the row-transform scratch of a
// wave stays within a budget that fits in L2 (so the second kernel reads it
// from L2), within the scratch buffer and within a grid dimension.
constexpr size_t kL2WaveBytes = size_t(48) << 20;
inline int wave_size(int n_layers, size_t scratch_bytes, size_t per_layer, size_t budget = 0) {
    const size_t b = budget ? budget : kL2WaveBytes;
    size_t w = std::min(scratch_bytes / per_layer, std::max<size_t>(1, b / per_layer));
    w = std::min<size_t>(w, 65535);
    return int(std::min<size_t>(size_t(n_layers), std::max<size_t>(w, 1)));
}

__device__ __forceinline__ float2 ld_stream(const float2 *p) { return __ldcs(p); }

// Row layout of the two-kernel (large image) path in shared memory.  When
// the four-step split has N2 a multiple of 32, consecutive frequencies of a
// transformed row sit 32 elements apart (N2 (p mod N1) + p / N1) and would hit
// one bank; one padding element per 32 (phys(q) = q + q / 32) spreads them.
template <int N>
struct RowLayout {
    static constexpr bool pad = Plan<N>::N2 % 32 == 0;
    static constexpr int S = pad ? N + N / 32 + 1 : N + 1;  // odd row stride
    __device__ __forceinline__ static int phys(int q) { return pad ? q + (q >> 5) : q; }
};

// Weight the canonical cells and complete row 0.  G has row stride S.
// Cells outside the canonical half are zero on entry.
template <int N, bool PAD = false>
__device__ __forceinline__ void weight_and_complete(float2 *G, int S, int r_begin, int r_end,
                                                    const ChanInfo &ci, const float *wgt, int tid,
                                                    int nt) {
    auto ph = [](int q) { return PAD ? RowLayout<N>::phys(q) : q; };
    constexpr int H = N / 2;
    const float *w = ci.weighting == 1 ? wgt + ci.wgt_off : nullptr;
    if (w) {
        const int first = max(r_begin, 1);
        for (int idx = tid; idx < (r_end - first) * N; idx += nt) {
            const int r = first + idx / N, c = idx % N;
            float2 &g = G[(r - r_begin) * S + ph(c)];
            const float wv = w[r * N + c];
            g.x *= wv;
            g.y *= wv;
        }
    }
    if (r_begin == 0) {
        for (int c = tid; c < H; c += nt) {
            const float wv = w ? w[c] : 1.f;
            float2 g = G[ph(c)];
            if (c == 0) {
                // origin: V and conj(V) of every baseline there
                G[ph(0)] = make_float2(2.f * g.x * wv, 0.f);
            } else {
                g.x *= wv;
                g.y *= wv;
                G[ph(c)] = g;
                G[ph(N - c)] = make_float2(g.x, -g.y);
            }
        }
    }
}

// Pass 1 on rows [0, nrows) of G (row stride S): N-point DFT (direction
// SIGN) of each row in place.  Output frequency p ends at position
// N2 * (p % N1) + p / N1.  `tw` holds the transposed four-step twiddles in
// shared memory; lanes run along a row (n2 in step A, k1 in step B), so with
// the padded layout (PAD) and the table's order every shared access of a
// warp is conflict-free.
template <int N, int SIGN = +1, bool PAD = false, bool NARROW = false>
__device__ __forceinline__ void rows_fft(float2 *G, int S, int nrows, int tid, int nt, const float2 *tw,
                                         int kmax = N, float2 *__restrict__ dst = nullptr) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    auto ph = [](int q) { return PAD ? RowLayout<N>::phys(q) : q; };
    // rows that are zero outside |k_u| <= kmax < 2 N2: only n1 = 0, 1 and
    // N1 - 2, N1 - 1 of step A hold data (the other inputs are constant zeros)
    bool narrow = false;
    if constexpr (NARROW && N > 4 * N2 && N1 >= 4) narrow = kmax < 2 * N2;
    // step A: N1-point transforms along stride N2, then twiddle W_N^(n2 k1)
    for (int t = tid; t < nrows * N2; t += nt) {
        const int r = t / N2, n2 = t % N2;
        float2 *row = G + r * S;
        float2 x[N1];
        if constexpr (NARROW && N > 4 * N2 && N1 >= 4) {
            if (narrow) {
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) x[n1] = make_float2(0.f, 0.f);
                x[0] = row[ph(n2)];
                x[1] = row[ph(N2 + n2)];
                x[N1 - 2] = row[ph(N - 2 * N2 + n2)];
                x[N1 - 1] = row[ph(N - N2 + n2)];
            } else {
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) x[n1] = row[ph(N2 * n1 + n2)];
            }
        } else {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) x[n1] = row[ph(N2 * n1 + n2)];
        }
        dft<N1, SIGN>(x);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
            const float2 w = tw[k1 * N2 + n2];
            x[k1] = cmulc(x[k1], c32{w.x, SIGN > 0 ? w.y : -w.y});
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) row[ph(N2 * k1 + n2)] = x[k1];
    }
    __syncthreads();
    // step B: N2-point transforms on contiguous runs; the result stays in
    // place (transposed order), or with dst goes straight to dst[r][p] in
    // natural order p = k1 + N1 k2 (consecutive k1 of a warp: coalesced)
    for (int t = tid; t < nrows * N1; t += nt) {
        const int r = t / N1, k1 = t % N1;
        float2 *run = G + r * S;
        float2 y[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) y[n2] = run[ph(N2 * k1 + n2)];
        dft<N2, SIGN>(y);
        if (dst) {
            float2 *o = dst + int64_t(r) * N + k1;
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) o[N1 * k2] = y[k2];
        } else {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) run[ph(N2 * k1 + k2)] = y[k2];
        }
    }
    __syncthreads();
}

template <int N>
__device__ __forceinline__ int pos_after_rows(int p) {
    return Plan<N>::N2 * (p % Plan<N>::N1) + p / Plan<N>::N1;
}

// Shared-memory layout of the pass-2 intermediate Z of P column pairs: the
// element q of pair jj sits at jj * ZS + phys(q).  When N2 is a multiple of
// 32, one padding element per 32 (phys(q) = q + q / 32) separates the k1
// runs read by the lanes of pass-2 step B, and the pair stride ZS = 16 / P
// (mod 16, in 8-byte bank pairs) spreads the P pairs of a half-warp over
// distinct banks in both steps.
template <int N, int P>
struct ZLayout {
    static constexpr bool pad = Plan<N>::N2 % 32 == 0;
    static constexpr int len = pad ? N + N / 32 : N;
    static constexpr int want = P >= 16 ? 1 : 16 / P;  // stride mod 16
    static constexpr int S = len + ((want - len % 16) % 16 + 16) % 16;
    __device__ __forceinline__ static int phys(int q) { return pad ? q + (q >> 5) : q; }
};

// Pass 2 of the two-kernel path pairs adjacent frequency columns: pair q
// (< N/2) is the FFT-order columns 2q and 2q + 1, whose real transforms are
// image columns (2q + N/2) mod N and the next one (N/2 is even for every
// supported size, so the two never wrap apart).  A CTA's P pairs are thus 2P
// adjacent columns: one contiguous piece of every pass-1 row read, and of
// every image row written.
//
// Pass 2, step A for pairs j0 + jj, jj < P.  `hrow2(k, c)` returns row k (< R)
// of the pass-1 output at the frequency columns c and c + 1.  Writes the
// four-step intermediate of pair jj to Z + jj * S.
template <int N, int P, class ZL, int NT, bool NARROW, class HRow2>
__device__ __forceinline__ void cols_step_a(float2 *Z, int R, int j0, HRow2 hrow2, int tid) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H = N / 2;
    // (the narrow layout needs 2 N2 < N / 2 and four distinct n1; kernels
    // that never see a narrow support leave it out of their code)
    if constexpr (NARROW && N > 4 * N2 && N1 >= 4) {
    if (R <= 2 * N2) {
        // narrow support (a compact station grid): only n1 = 0, 1 (rows
        // k < R) and n1 = N1 - 2, N1 - 1 (mirrored rows N - k < R) hold data.
        // Every task's four loads are issued before any transform, and the
        // other inputs are constant zeros.
        constexpr int TPT = (P * N2 + NT - 1) / NT;
        float4 ld[TPT][4];
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            const int t = tid + u * NT, jj = t % P, n2 = t / P, q = j0 + jj;
            const bool ok = t < P * N2 && q < H;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            ld[u][0] = ok && n2 < R ? hrow2(n2, 2 * q) : z4;                    // k = n2
            ld[u][1] = ok && N2 + n2 < R ? hrow2(N2 + n2, 2 * q) : z4;          // k = N2 + n2
            ld[u][2] = ok && 2 * N2 - n2 < R ? hrow2(2 * N2 - n2, 2 * q) : z4;  // N - k, n1 = N1 - 2
            ld[u][3] = ok && N2 - n2 < R ? hrow2(N2 - n2, 2 * q) : z4;          // N - k, n1 = N1 - 1
        }
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            const int t = tid + u * NT, jj = t % P, n2 = t / P, q = j0 + jj;
            if (t >= P * N2 || q >= H) continue;
            float2 x[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) x[n1] = make_float2(0.f, 0.f);
            x[0] = make_float2(ld[u][0].x - ld[u][0].w, ld[u][0].y + ld[u][0].z);            // H_a + i H_b
            x[1] = make_float2(ld[u][1].x - ld[u][1].w, ld[u][1].y + ld[u][1].z);
            x[N1 - 2] = make_float2(ld[u][2].x + ld[u][2].w, ld[u][2].z - ld[u][2].y);       // conj(H_a) + i conj(H_b)
            x[N1 - 1] = make_float2(ld[u][3].x + ld[u][3].w, ld[u][3].z - ld[u][3].y);
            dft<N1, +1>(x);
            float2 *zp = Z + jj * ZL::S;
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1)
                zp[ZL::phys(N2 * k1 + n2)] = k1 == 0 ? x[0] : cmulc(x[k1], four_step_tw<N, +1>(k1, n2));
        }
        return;
    }
    }
    for (int t = tid; t < P * N2; t += NT) {
        const int jj = t % P, n2 = t / P;
        const int q = j0 + jj;
        if (q >= H) continue;
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int k = N2 * n1 + n2;
            float2 z = make_float2(0.f, 0.f);
            if (k < H) {
                if (k < R) {
                    const float4 ab = hrow2(k, 2 * q);
                    z = make_float2(ab.x - ab.w, ab.y + ab.z);  // H_a + i H_b
                }
            } else if (k > H) {
                const int m = N - k;
                if (m < R) {
                    const float4 ab = hrow2(m, 2 * q);
                    z = make_float2(ab.x + ab.w, ab.z - ab.y);  // conj(H_a) + i conj(H_b)
                }
            }
            x[n1] = z;
        }
        dft<N1, +1>(x);
        float2 *zp = Z + jj * ZL::S;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1)
            zp[ZL::phys(N2 * k1 + n2)] = k1 == 0 ? x[0] : cmulc(x[k1], four_step_tw<N, +1>(k1, n2));
    }
}

template <int N>
struct DegridCfg;
template <int N>
struct AdjFusable;
template <int N>
__device__ __forceinline__ void degrid_cols_strip(float2 *sm, int R, int x0, float2 *__restrict__ out, int tid);

// The N2 results y of one pass-2 step-B task (pair jj, FFT-order rows
// k1 + N1 k2) as image values: scaled, the reference subtracted, stored at
// image column xa and xa + 1 (when img is set) and at strip[row][2 jj] (when
// strip is set: FFT-order rows of 16 floats).  Returns the sum of their
// squares in FP32 when want_sq.
template <int N, bool EPI>
__device__ __forceinline__ float store_task(const float2 (&y)[Plan<N>::N2], int k1, int xa, int jj, float *img,
                                            float scale, const float *ref, bool pair_store, bool want_sq,
                                            float *strip) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H = N / 2;
    // with N2 even, FFT-order row k1 + N1 k2 (k1 < N1) is below H exactly
    // when k2 < N2 / 2: the fftshift is then fixed per k2 at compile time
    constexpr bool split = N2 % 2 == 0;
    auto image_row = [&](int k2) {
        const int qq = k1 + N1 * k2;
        if constexpr (split) return k2 < N2 / 2 ? qq + H : qq - H;
        return qq < H ? qq + H : qq - H;
    };
    float sq = 0.f;
    // stores in batches of KB rows; with the fused epilogue each batch's
    // reference values are requested together before its stores
    constexpr int KB = N2 % 4 == 0 ? 4 : 1;
#pragma unroll
    for (int kb = 0; kb < N2; kb += KB) {
        float2 rf[KB];
        if (ref) {
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                const float *rp = ref + image_row(kb + u) * N + xa;  // 32-bit: N * N < 2^31
                rf[u] = pair_store ? __ldcs(reinterpret_cast<const float2 *>(rp))
                                   : make_float2(__ldcs(rp), __ldcs(rp + 1));
            }
        }
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int k2 = kb + u;
            const int qq = k1 + N1 * k2;              // FFT-order row
            const int row = image_row(k2);            // fftshift
            float2 v = make_float2(y[k2].x * scale, y[k2].y * scale);
            if (ref) {
                v.x -= rf[u].x;
                v.y -= rf[u].y;
            }
            if (!EPI || img) {  // (only the epilogue may store no image)
                float *o = img + row * N + xa;        // offsets inside one image fit 32 bits
                if (pair_store) {
                    __stcs(reinterpret_cast<float2 *>(o), v);
                } else {
                    __stcs(o, v.x);
                    __stcs(o + 1, v.y);
                }
            }
            if (strip) *reinterpret_cast<float2 *>(strip + qq * 16 + 2 * jj) = v;
            if (want_sq) sq = fmaf(v.x, v.x, fmaf(v.y, v.y, sq));
        }
    }
    return sq;
}

// Pass 2, step B: N2-point transforms, then the two real image columns of
// each pair (adjacent) with the fftshift folded into the addresses.  With
// want_sq the sum of the squares of the stored values is returned (valid in
// thread 0; each task's 2 N2 squares in FP32, the tasks' sums in FP64, in a
// fixed order).  With adj (sizes whose column item is one 16-column strip of
// the image: AdjFusable), the CTA's values also go to a strip in Z's buffer
// and the adjoint's column transforms of that strip (rows k < R) go to adj.
template <int N, int P, class ZL, int NT, bool EPI>
__device__ __forceinline__ double cols_step_b(float2 *Z, int j0, float *img, float scale, int tid,
                                              const float *ref, bool want_sq = false, float2 *adj = nullptr,
                                              int R = 0) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H = N / 2;
    const bool pair_store = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(ref)) & 7) == 0;
    double acc = 0.0;
    if constexpr (AdjFusable<N>::value) {
        if (adj) {
            // one task per thread, every pair inside the image: all reads of
            // Z land in registers before the barrier that hands its buffer to
            // the strip
            const int jj = tid % P, k1 = tid / P;
            const int xa = (2 * (j0 + jj) + H) % N;
            const float2 *zp = Z + jj * ZL::S;
            float2 y[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) y[n2] = zp[ZL::phys(N2 * k1 + n2)];
            dft<N2, +1>(y);
            __syncthreads();
            const float sq = store_task<N, EPI>(y, k1, xa, jj, img, scale, ref, pair_store, want_sq,
                                           reinterpret_cast<float *>(Z));
            if (want_sq) acc = double(sq);
            __syncthreads();  // the strip is complete
            degrid_cols_strip<N>(Z, R, (2 * j0 + H) % N, adj, tid);
            return want_sq ? block_sum_f64<NT>(acc, tid) : 0.0;
        }
    }
    for (int t = tid; t < P * N1; t += NT) {
        const int jj = t % P, k1 = t / P;
        const int q = j0 + jj;
        if (q >= H) continue;
        const int xa = (2 * q + H) % N;  // image column of the pair's first column; the second is xa + 1
        const float2 *zp = Z + jj * ZL::S;
        float2 y[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) y[n2] = zp[ZL::phys(N2 * k1 + n2)];
        dft<N2, +1>(y);
        const float sq = store_task<N, EPI>(y, k1, xa, jj, img, scale, ref, pair_store, want_sq, nullptr);
        if (want_sq) acc += double(sq);
    }
    return want_sq ? block_sum_f64<NT>(acc, tid) : 0.0;
}

// Grid the canonical rows [r0, r0 + nrows) of one layer into G (stride S).
template <int NT, int N>
__device__ __forceinline__ void grid_rows(float2 *G, int S, int r0, int nrows, const uint32_t *code,
                                          const float2 *vis, int64_t nb, int tid, const LayerGains gl) {
    for (int64_t b = tid; b < nb; b += NT) {
        const uint32_t cd = __ldg(code + b);
        if (cd == kCodeDropped) continue;
        const int r = int(code_row(cd)) - r0;
        if (r < 0 || r >= nrows) continue;
        float2 v = ld_stream(vis + b);
        if (gl) v = apply_gain(v, gl, b);
        if (code_conj(cd)) v.y = -v.y;
        float2 *cell = G + r * S + RowLayout<N>::phys(int(code_col(cd)));
        atomicAdd(&cell->x, v.x);
        atomicAdd(&cell->y, v.y);
    }
}

// ------------------------------------------------------------- large path
template <int N>
struct LargeCfg {
    static constexpr int NT = 256;
    static constexpr int S = RowLayout<N>::S;
    static constexpr int RB = std::max(1, std::min(32, int(65536 / (S * sizeof(float2)))));
    static constexpr int P = std::max(1, std::min(32, NT / Plan<N>::N1));
};

// Shared-memory offset (in float2) of the four-step twiddle table behind the
// RB rows of the large-image row kernels (16-byte aligned), and its copy.
template <int N>
constexpr int tw_offset() { return (LargeCfg<N>::RB * LargeCfg<N>::S + 1) & ~1; }

template <int N>
constexpr size_t rows_smem() { return (size_t(tw_offset<N>()) + N) * sizeof(float2); }

template <int N>
__device__ __forceinline__ void stage_four_step(float2 *dst, int tid, int nt) {
    const c32 *src = g_four_step<N>.v;
    for (int i = tid; i < N / 2; i += nt)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(uint32_t(__cvta_generic_to_shared(dst + 2 * i))),
                     "l"(src + 2 * i)
                     : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Row items of the image path: a band of RB canonical rows of one layer in
// shared memory (row stride S) and the four-step twiddle table.  RB is the
// largest band (at most 32 rows) that keeps an item within kRowsSmemBudget,
// so three CTAs share an SM.
constexpr size_t kRowsSmemBudget = 72 * 1024;
template <int N>
struct RowsCfg {
    static constexpr int NT = 256;
    static constexpr int S = RowLayout<N>::S;
    static constexpr int RB0 = std::max(1, std::min(32, int((kRowsSmemBudget - size_t(N) * 8) / (size_t(S) * 8))));
    // at 1024^2 (N1 = N2 = 32) a band of 8 rows gives every thread one task
    // in both steps (7 rows left 32 idle) and, at 75.8 KB, still lets three
    // CTAs share an SM
    static constexpr int RB = (Plan<N>::N1 == 32 && Plan<N>::N2 == 32) ? 8 : RB0;
    static constexpr int tw = (RB * S + 1) & ~1;  // float2 offset of the twiddles (16-byte aligned)
    static constexpr size_t smem = (size_t(tw) + N) * sizeof(float2);
};

// Pass 1 for the band of canonical rows [r0, r0 + RB) of one layer (r0 below
// the channel's support R): gridding, weights, Hermitian completion of row 0,
// the row transforms, written in natural column order to dst[r - r0][p].
template <int N, bool NARROW = true>
__device__ __forceinline__ void rows_item(const ImageArgs &a, const DevLayer &L, const ChanInfo &ci, int lidx,
                                          int r0, int nrows, float2 *__restrict__ dst, float2 *sm, int tid) {
    using C = RowsCfg<N>;
    constexpr int NT = C::NT, S = C::S;
    __builtin_assume(nrows >= 1 && nrows <= C::RB);
    float2 *tw = sm + C::tw;
    auto prologue = [&]() {
        stage_four_step<N>(tw, tid, NT);
        // zero the band two elements at a time (sm is 16-byte aligned)
        const int n = nrows * S;
        float4 *z4 = reinterpret_cast<float4 *>(sm);
        for (int i = tid; i < n / 2; i += NT) z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((n & 1) && tid == 0) sm[n - 1] = make_float2(0.f, 0.f);
    };
    if (a.cg) {
        // the layer's compact grid (weighted, row 0 complete): expand the
        // band's rows, columns |k_u| <= kmax, into FFT order
        const int km = ci.kmax_u, kc = 2 * km + 1;
        const float2 *cg = a.cg + int64_t(lidx - a.cg_l0) * a.cg_stride + int64_t(r0) * kc;
        prologue();
        __syncthreads();  // the band is zero before the copies land in it
        for (int i = tid; i < nrows * kc; i += NT) {
            const int r = i / kc, ku = i % kc - km;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(uint32_t(__cvta_generic_to_shared(
                             sm + r * S + RowLayout<N>::phys(ku < 0 ? ku + N : ku)))),
                         "l"(cg + i)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
        const LayerGains gl = layer_gains(a, L);
        if (a.csr && ci.csr_off >= 0) {
            const CsrLayout cl(N, a.nb);
            auto cell = [sm](uint32_t key) { return sm + int(key >> 16) * S + RowLayout<N>::phys(int(key & 0xFFFFu)); };
            grid_band_sorted<NT>(r0, nrows, reinterpret_cast<const int32_t *>(a.csr + ci.csr_off + cl.row_ptr),
                                 reinterpret_cast<const uint2 *>(a.csr + ci.csr_off + cl.ents), a.vis + L.vis_off, gl,
                                 tid, cell, prologue);
        } else {
            // a channel without row buckets (its support always fits the fused
            // kernel; it comes here only when the two-kernel path is forced):
            // shared-memory atomics over the whole code table
            prologue();
            __syncthreads();
            grid_rows<NT, N>(sm, S, r0, nrows, a.codes + ci.code_off, a.vis + L.vis_off, a.nb, tid, gl);
            __syncthreads();
        }
        weight_and_complete<N, true>(sm, S, r0, r0 + nrows, ci, a.wgt, tid, NT);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // twiddle table (and compact rows) in place
    __syncthreads();
    rows_fft<N, +1, true, NARROW>(sm, S, nrows, tid, NT, tw, ci.kmax_u, dst);
}

// Pass 1 of a wave of layers into scratch[layer_in_wave][r][p] (the wave
// path: the tensor-core FP16 modes and callers without a work queue).
// Grid: (bands, layers in wave).
template <int N>
__global__ void __launch_bounds__(RowsCfg<N>::NT, (Plan<N>::N1 == 24 || N >= 1024) ? 2 : 3) k_rows(ImageArgs a, int l0) {
    extern __shared__ float2 sm[];
    const int lw = blockIdx.y;
    const DevLayer L = a.layers[l0 + lw];
    const ChanInfo ci = a.chans[L.chan];
    const int r0 = blockIdx.x * RowsCfg<N>::RB;
    if (r0 >= ci.rows) return;
    rows_item<N>(a, L, ci, l0 + lw, r0, min(RowsCfg<N>::RB, ci.rows - r0),
                 a.scratch + (int64_t(lw) * a.r_alloc + r0) * N, sm, threadIdx.x);
}

// The column pass can stage its scratch columns through shared memory when
// step A has exactly one task per thread (P N2 == NT) and the pairs tile N/2.
template <int N>
struct ColsStaged {
    static constexpr int P = LargeCfg<N>::P, N2 = Plan<N>::N2;
    static constexpr bool value = P * N2 == LargeCfg<N>::NT && (N / 2) % P == 0;
};

// Pass 2, step A from shared memory: the CTA's 2P adjacent scratch columns of
// rows k < R (one contiguous piece of each row) are copied with cp.async at
// once into the buffer Z later holds; each thread reads its N1 inputs into
// registers (one 16-byte load per pair and row), the CTA synchronises, then
// the intermediate overwrites the buffer.
template <int N, int P, class ZL, bool NARROW>
__device__ __forceinline__ void cols_step_a_staged(float2 *Z, int R, int j0, const float2 *Hs, int tid) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H = N / 2, NT = LargeCfg<N>::NT;
    float2 *stg = Z;  // [R][2P]: frequency columns 2 j0 ..
    for (int i = tid; i < R * P; i += NT) {  // P 16-byte pieces per row
        const int k = i / P, pc = i % P;
        const float2 *src = Hs + int64_t(k) * N + 2 * (j0 + pc);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(uint32_t(__cvta_generic_to_shared(
                         stg + k * 2 * P + 2 * pc))),
                     "l"(src)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int jj = tid % P, n2 = tid / P;  // one task per thread
    float2 x[N1];
    bool loaded = false;  // x holds the task's inputs
    if constexpr (NARROW && N > 4 * N2 && N1 >= 4) {
    if (R <= 2 * N2) {
        loaded = true;
        // narrow support: only n1 = 0, 1 and N1 - 2, N1 - 1 hold data (the
        // other inputs are constant zeros)
        auto row = [&](int k) {
            return k < R ? *reinterpret_cast<const float4 *>(stg + k * 2 * P + 2 * jj) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        const float4 a0 = row(n2), a1 = row(N2 + n2), b2 = row(2 * N2 - n2), b1 = row(N2 - n2);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = make_float2(0.f, 0.f);
        x[0] = make_float2(a0.x - a0.w, a0.y + a0.z);  // H_a + i H_b
        x[1] = make_float2(a1.x - a1.w, a1.y + a1.z);
        x[N1 - 2] = make_float2(b2.x + b2.w, b2.z - b2.y);  // conj(H_a) + i conj(H_b)
        x[N1 - 1] = make_float2(b1.x + b1.w, b1.z - b1.y);
    }
    }
    if constexpr (N1 % 2 == 0) {
    if (!loaded && R == H) {
        // full support (rows 0 .. H - 1 all present): n1 < N1 / 2 reads row
        // k = N2 n1 + n2 < H, n1 > N1 / 2 the mirrored row N - k < H; only
        // n1 = N1 / 2 can hit k = H (n2 = 0), whose input is zero
        loaded = true;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int k = N2 * n1 + n2;
            if (n1 < N1 / 2) {
                const float4 ab = *reinterpret_cast<const float4 *>(stg + k * 2 * P + 2 * jj);
                x[n1] = make_float2(ab.x - ab.w, ab.y + ab.z);  // H_a + i H_b
            } else if (n1 > N1 / 2 || n2 > 0) {
                const float4 ab = *reinterpret_cast<const float4 *>(stg + (N - k) * 2 * P + 2 * jj);
                x[n1] = make_float2(ab.x + ab.w, ab.z - ab.y);  // conj(H_a) + i conj(H_b)
            } else {
                x[n1] = make_float2(0.f, 0.f);
            }
        }
    }
    }
    if (!loaded) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int k = N2 * n1 + n2;
            float2 z = make_float2(0.f, 0.f);
            if (k < H) {
                if (k < R) {
                    const float4 ab = *reinterpret_cast<const float4 *>(stg + k * 2 * P + 2 * jj);
                    z = make_float2(ab.x - ab.w, ab.y + ab.z);  // H_a + i H_b
                }
            } else if (k > H) {
                const int m = N - k;
                if (m < R) {
                    const float4 ab = *reinterpret_cast<const float4 *>(stg + m * 2 * P + 2 * jj);
                    z = make_float2(ab.x + ab.w, ab.z - ab.y);  // conj(H_a) + i conj(H_b)
                }
            }
            x[n1] = z;
        }
    }
    __syncthreads();  // every staged value is in registers: the buffer becomes Z
    dft<N1, +1>(x);
    float2 *zp = Z + jj * ZL::S;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
        zp[ZL::phys(N2 * k1 + n2)] = k1 == 0 ? x[0] : cmulc(x[k1], four_step_tw<N, +1>(k1, n2));
}

// Pass 2 for the P column pairs j0.. of one layer from its pass-1 rows Hs
// (scratch written by other CTAs: read through L2, never a stale L1 line).
template <int N, bool EPI, bool NARROW, class Consumed>
__device__ __forceinline__ void cols_item(const ImageArgs &a, const DevLayer &L, const ChanInfo &ci, int j0,
                                          const float2 *Hs, float *__restrict__ out, const float *__restrict__ ref,
                                          float2 *sm, int tid, Consumed &&consumed, int lidx = 0) {
    constexpr int NT = LargeCfg<N>::NT, P = LargeCfg<N>::P;
    using ZL = ZLayout<N, P>;
    const int R = ci.rows;
    if constexpr (ColsStaged<N>::value) {
        cols_step_a_staged<N, P, ZL, NARROW>(sm, R, j0, Hs, tid);
    } else {
        auto hrow2 = [&](int k, int c) { return __ldcg(reinterpret_cast<const float4 *>(Hs + int64_t(k) * N + c)); };
        cols_step_a<N, P, ZL, NT, NARROW>(sm, R, j0, hrow2, tid);
    }
    __syncthreads();
    consumed();  // every read of Hs has landed in registers or shared memory
    const float scale = ((a.flags & kNormalize) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f;
    const bool want_sq = EPI && a.sq_part;
    // fused adjoint columns: layer lidx of the group's slots (r_alloc rows of N)
    float2 *adj = EPI && a.adj ? a.adj + int64_t(lidx) * a.r_alloc * N : nullptr;
    // (no output array: the fused adjoint keeps the columns, no image is stored)
    const double sq = cols_step_b<N, P, ZL, NT, EPI>(sm, j0, out ? out + L.out_off : nullptr, scale, tid,
                                                EPI && ref ? ref + L.out_off : nullptr, want_sq, adj, R);
    if (want_sq)  // one slot per column item
        store_sq_slot<NT>(a.sq_part + int64_t(L.layer) * a.sq_stride, j0 / P, (N / 2 + P - 1) / P, a.sq_stride,
                          sq, tid);
}

template <int N>
constexpr size_t cols_smem(int r_alloc) {
    constexpr int P = LargeCfg<N>::P;
    size_t smem = size_t(P) * ZLayout<N, P>::S * sizeof(float2);
    if (ColsStaged<N>::value)  // the staged columns share the buffer
        smem = std::max(smem, size_t(r_alloc) * 2 * P * sizeof(float2));
    return smem;
}

// Pass 2 of a wave of layers.  Grid: (ceil(N/2 / P), layers in wave).
template <int N, bool EPI>
__global__ void __launch_bounds__(LargeCfg<N>::NT, 3) k_cols(ImageArgs a, int l0, float *__restrict__ out,
                                                          const float *__restrict__ ref) {
    extern __shared__ float2 sm[];
    const int lw = blockIdx.y;
    const DevLayer L = a.layers[l0 + lw];
    const ChanInfo ci = a.chans[L.chan];
    cols_item<N, EPI, true>(a, L, ci, blockIdx.x * LargeCfg<N>::P, a.scratch + int64_t(lw) * a.r_alloc * N, out, ref, sm,
                            threadIdx.x, [] {}, l0 + lw);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
}

// ------------------------------------------------ persistent large-image path
// One launch per image size: a persistent grid pulls work items from a device
// queue.  A layer has nR row items (bands of RB rows: gridding + pass 1 into
// the layer's slot of a ring of `slots` scratch buffers that stays in L2) and
// nC column items (P column pairs each: pass 2 from that slot, image store).
// The queue interleaves the layers with a lag: stage s holds the row items of
// layer s and then the column items of layer s - lag, so a column item's rows
// were handed out lag stages earlier and are normally done when it starts.
// Dependencies, each a bounded wait on a per-layer counter:
//   column item of layer l  needs the nR row items of l   (rows_done[l]),
//   row item of layer l     needs the nC column items of l - slots, whose
//                           slot it overwrites             (cols_done[l - slots]).
// Both point to items earlier in the queue (lag <= slots - 1), and items are
// handed out only to running CTAs, so the earliest unfinished item can always
// run: the waits end.  A wait that runs out of time (a fault elsewhere) sets
// the abort flag and BLINK_ERR_TIMEOUT in the status word; later items then
// skip their work.
struct LargeSched {
    int n;          // layers of the group
    int rb;         // rows per row item (<= RowsCfg<N>::RB)
    int nR, nC;     // row and column items per layer
    int lag;        // stages between a layer's row and column items
    int slots;      // scratch ring slots (layers)
    int ahead;      // layers between a layer and the one whose row buckets it prefetches (0: none)
    int64_t total;  // n (nR + nC)
    unsigned long long wait_ns;
};

// Queue words: a 64-bit item counter, the abort flag, then rows_done[n] and
// cols_done[n] (32-bit counters).
struct QueueView {
    unsigned long long *head;
    int *abort_flag;
    int *rows_done, *cols_done;
    __device__ QueueView(int *q, int n)
        : head(reinterpret_cast<unsigned long long *>(q)), abort_flag(q + 2), rows_done(q + 4),
          cols_done(q + 4 + n) {}
};

__device__ __forceinline__ void decode_item(int64_t i, const LargeSched &q, bool &is_row, int &layer, int &sub) {
    const int64_t per_r = q.nR, per_c = q.nC, lag = q.lag;
    const int64_t p1 = lag * per_r;
    if (i < p1) {
        is_row = true;
        layer = int(i / per_r);
        sub = int(i % per_r);
        return;
    }
    i -= p1;
    const int64_t stage = per_r + per_c, p2 = (int64_t(q.n) - lag) * stage;
    if (i < p2) {
        const int64_t k = i / stage, off = i % stage;
        is_row = off < per_r;
        layer = int(is_row ? lag + k : k);
        sub = int(is_row ? off : off - per_r);
        return;
    }
    i -= p2;
    is_row = false;
    layer = int(int64_t(q.n) - lag + i / per_c);
    sub = int(i % per_c);
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: waits until *ctr >= target (true) or the abort flag is set or the
// limit runs out (false; the timeout also raises the flag and the status).
__device__ __forceinline__ bool wait_count(const int *ctr, int target, int *abort_flag, int *status,
                                           unsigned long long limit_ns) {
    if (ld_acquire_gpu(ctr) >= target) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        __nanosleep(256);
        if (ld_acquire_gpu(ctr) >= target) return true;
        if (ld_acquire_gpu(abort_flag)) return false;
        if (global_ns() - t0 >= limit_ns) {
            atomicExch(abort_flag, 1);
            if (status) atomicExch(status, -4);  // BLINK_ERR_TIMEOUT
            return false;
        }
    }
}

template <int N>
constexpr size_t large_smem(int r_alloc) { return std::max(RowsCfg<N>::smem, cols_smem<N>(r_alloc)); }

template <int N, bool EPI>
__global__ void __launch_bounds__(256, (EPI || Plan<N>::N1 == 24) ? 2 : 3)
    k_large(ImageArgs a, LargeSched q, float *__restrict__ out, const float *__restrict__ ref) {
    static_assert(RowsCfg<N>::NT == 256 && LargeCfg<N>::NT == 256, "one block shape for both item kinds");
    extern __shared__ float2 sm[];
    __shared__ long long s_item[2];
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const QueueView Q(a.queue, q.n);
    if (tid == 0) s_item[0] = (long long)atomicAdd(Q.head, 1ull);
    __syncthreads();
    long long item = s_item[0];
    for (int it = 0; item < q.total; ++it) {
        if (tid == 0) s_item[(it + 1) & 1] = (long long)atomicAdd(Q.head, 1ull);  // next item, fetched early
        bool is_row;
        int layer, sub;
        decode_item(item, q, is_row, layer, sub);
        if (tid == 0) {
            bool ok = ld_acquire_gpu(Q.abort_flag) == 0;
            if (ok && is_row && layer >= q.slots)
                ok = wait_count(Q.cols_done + (layer - q.slots), q.nC, Q.abort_flag, a.status, q.wait_ns);
            else if (ok && !is_row)
                ok = wait_count(Q.rows_done + layer, q.nR, Q.abort_flag, a.status, q.wait_ns);
            s_ok = ok;
        }
        __syncthreads();
        const bool ok = s_ok != 0;
        if (ok) {
            const DevLayer L = a.layers[layer];
            const ChanInfo ci = a.chans[L.chan];
            float2 *Hs = a.scratch + int64_t(layer % q.slots) * a.r_alloc * N;
            if (is_row) {
                // the first row item of a layer pulls the layer's visibilities
                // into L2 for the band gathers of all its row items, and the
                // row buckets of the layer about one grid of items ahead (with
                // many channels the buckets do not stay in L2 between a
                // channel's time steps)
                if (sub == 0 && !a.cg) {
                    prefetch_l2_bytes(a.vis + L.vis_off, 8 * a.nb, tid, 256);
                    const int la = layer + q.ahead;
                    if (q.ahead > 0 && a.csr && la < q.n) {
                        const ChanInfo cp = a.chans[a.layers[la].chan];
                        if (cp.csr_off >= 0) {
                            const CsrLayout cl(N, a.nb);
                            prefetch_l2_bytes(a.csr + cp.csr_off + cl.row_ptr, 4 * int64_t(cl.n_bkt + 1), tid, 256);
                            prefetch_l2_bytes(a.csr + cp.csr_off + cl.ents, 8 * a.nb, tid, 256);
                        }
                    }
                }
                const int r0 = sub * q.rb;
                const int nrows = min(RowsCfg<N>::RB, min(q.rb, ci.rows - r0));
                if (r0 < ci.rows) rows_item<N, false>(a, L, ci, layer, r0, nrows, Hs + int64_t(r0) * N, sm, tid);
                __syncthreads();  // every thread's scratch stores precede the release below
                if (tid == 0) {
                    __threadfence();
                    atomicAdd(Q.rows_done + layer, 1);
                }
            } else {
                // the slot is released as soon as its rows are read: the image
                // stores do not gate its reuse
                cols_item<N, EPI, false>(a, L, ci, sub * LargeCfg<N>::P, Hs, out, ref, sm, tid, [&] {
                    if (tid == 0) atomicAdd(Q.cols_done + layer, 1);
                }, layer);
                if (sub == 0 && tid == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
            }
        }
        __syncthreads();  // shared memory and s_ok are reused by the next item
        item = s_item[(it + 1) & 1];
    }
}

template <int N>
struct DegridCfg {
    static constexpr int NT = 256;
    static constexpr int P = 8;           // column pairs per CTA: 16 adjacent image columns
    // strip row stride in floats: 64-byte rows (16-byte cp.async pieces), and
    // the pair loads of a half-warp (8 pairs x 2 rows) cover all 32 banks once
    static constexpr int W = 2 * P;
    // natural-order result: pair stride N + 2 (2 mod 16 in 8-byte bank pairs),
    // so the 8 pairs of a half-warp store to distinct banks
    static constexpr int ZN = N + 2;
    static constexpr int RB = LargeCfg<N>::RB;
    using ZL = ZLayout<N, P>;
    static_assert(P * Plan<N>::N2 <= NT && P * Plan<N>::N1 <= NT, "one four-step task per thread");
};

// The column item of the forward pass is exactly one strip of the adjoint's
// column kernel (16 adjacent image columns, one task per thread in both).
template <int N>
struct AdjFusable {
    static constexpr bool value = LargeCfg<N>::P == DegridCfg<N>::P && LargeCfg<N>::NT == DegridCfg<N>::NT &&
                                  LargeCfg<N>::P * Plan<N>::N1 == LargeCfg<N>::NT && (N / 2) % LargeCfg<N>::P == 0;
};

template <int N>
size_t degrid_cols_smem() {
    using C = DegridCfg<N>;
    return std::max({size_t(N) * C::W * sizeof(float), size_t(C::P) * C::ZL::S * sizeof(float2),
                     size_t(C::P) * C::ZN * sizeof(float2)});
}

// Forward column transforms of the image gradient (the first half of the
// adjoint's forward 2-D FFT).  CTA x of a layer takes the 16 adjacent image
// columns [16 x, 16 x + 16) -- one 64-byte piece of every image row, read
// once -- as 8 pairs of real columns, each pair one complex N-point transform
// (z = R_a + i R_b).  The strip, the four-step intermediate and the
// natural-order result share one buffer: every task holds its inputs in
// registers across a barrier before the buffer is overwritten.  Rows k < R of
// the two real columns' transforms go to scratch[lw][k][j] (FFT-order column
// j = image column + N/2 mod N), 16 adjacent columns per row.
// Grid: (N / 16, layers in wave).
// The column transforms of one 16-column strip already in shared memory
// (strip[n][c], FFT-order row n = image row (n + N/2) mod N, c < 16, 64-byte
// rows): rows k < R of the two real columns of every pair go to
// out[k][(x0 + c + N/2) mod N] (row stride N).  The strip's buffer is reused:
// it must hold max(N * 16 floats, P * ZL::S, P * ZN complex).  Every thread
// of the CTA calls it (NT = DegridCfg<N>::NT).
template <int N>
__device__ __forceinline__ void degrid_cols_strip(float2 *sm, int R, int x0, float2 *__restrict__ out, int tid) {
    using C = DegridCfg<N>;
    using ZL = typename C::ZL;
    constexpr int P = C::P, W = C::W, H = N / 2;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    const float *strip = reinterpret_cast<const float *>(sm);
    float2 *Z = sm;   // [P][ZL::S] four-step intermediate
    float2 *zn = sm;  // [P][ZN] natural order
    // step A: pair p, n2; z = R_a + i R_b along stride N2, forward twiddles
    const int pa = tid % P, n2 = tid / P;
    const bool task_a = n2 < N2;
    float2 x[N1];
    if (task_a) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = *reinterpret_cast<const float2 *>(strip + (N2 * n1 + n2) * W + 2 * pa);
    }
    __syncthreads();  // the strip is in registers: the buffer becomes Z
    if (task_a) {
        dft<N1, -1>(x);
        float2 *zp = Z + pa * ZL::S;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1)
            zp[ZL::phys(N2 * k1 + n2)] = k1 == 0 ? x[0] : cmulc(x[k1], four_step_tw<N, -1>(k1, n2));
    }
    __syncthreads();
    // step B: pair p, k1; results to natural order (in registers first)
    const int pb = tid % P, k1 = tid / P;
    const bool task_b = k1 < N1;
    float2 y[N2];
    if (task_b) {
        const float2 *zp = Z + pb * ZL::S;
#pragma unroll
        for (int m = 0; m < N2; ++m) y[m] = zp[ZL::phys(N2 * k1 + m)];
        dft<N2, -1>(y);
    }
    __syncthreads();  // Z is in registers: the buffer becomes zn
    if (task_b) {
        // only the frequencies the unpacking below reads: k < R and N - k < R
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int k = k1 + N1 * k2;
            if (k < R || k > N - R) zn[pb * C::ZN + k] = y[k2];
        }
    }
    __syncthreads();
    // unpack the two real columns of each pair and keep rows k < R; image
    // column x goes to FFT-order column (x + N/2) mod N
    for (int i = tid; i < R * P; i += C::NT) {
        const int k = i / P, p = i % P;
        const int xa = x0 + 2 * p;
        if (xa >= N) continue;
        const float2 za = zn[p * C::ZN + k], zb = zn[p * C::ZN + (N - k) % N];
        // C_a = (Z[k] + conj Z[N-k]) / 2, C_b = (Z[k] - conj Z[N-k]) / (2 i)
        out[int64_t(k) * N + (xa + H) % N] = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
        if (xa + 1 < N)
            out[int64_t(k) * N + (xa + 1 + H) % N] = make_float2(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x));
    }
}

// Forward column transforms of the image gradient (the first half of the
// adjoint's forward 2-D FFT).  CTA x of a layer takes the 16 adjacent image
// columns [16 x, 16 x + 16) -- one 64-byte piece of every image row, read
// once -- as 8 pairs of real columns, each pair one complex N-point transform
// (z = R_a + i R_b).  The strip, the four-step intermediate and the
// natural-order result share one buffer: every task holds its inputs in
// registers across a barrier before the buffer is overwritten.  Rows k < R of
// the two real columns' transforms go to scratch[lw][k][j] (FFT-order column
// j = image column + N/2 mod N), 16 adjacent columns per row.
// Grid: (N / 16, layers in wave).
template <int N>
__global__ void __launch_bounds__(DegridCfg<N>::NT, 3) k_degrid_cols(ImageArgs a, const float *resid, int l0) {
    using C = DegridCfg<N>;
    constexpr int NT = C::NT, P = C::P, W = C::W, H = N / 2;
    extern __shared__ float2 sm[];
    float *strip = reinterpret_cast<float *>(sm);  // [N][W]: FFT-order row n = image row (n + H) mod N
    const int lw = blockIdx.y;
    const DevLayer L = a.layers[l0 + lw];
    const ChanInfo ci = a.chans[L.chan];
    const int x0 = blockIdx.x * 2 * P;             // first image column
    const int nc = min(2 * P, N - x0);             // columns of this CTA (the last may be partial)
    const int tid = threadIdx.x;
    const float *img = resid + L.out_off;
    if (nc == 2 * P && (reinterpret_cast<uintptr_t>(img) & 15) == 0 && (N % 4) == 0) {
        // every 16-byte piece in flight at once, straight into shared memory
        for (int i = tid; i < N * (2 * P / 4); i += NT) {
            const int y = i / (2 * P / 4), q = i % (2 * P / 4);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(uint32_t(__cvta_generic_to_shared(
                             strip + ((y + H) % N) * W + 4 * q))),
                         "l"(img + int64_t(y) * N + x0 + 4 * q)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    } else {
        for (int i = tid; i < N * 2 * P; i += NT) {
            const int y = i / (2 * P), c = i % (2 * P);
            strip[((y + H) % N) * W + c] = c < nc ? __ldcs(img + int64_t(y) * N + x0 + c) : 0.f;
        }
    }
    __syncthreads();
    degrid_cols_strip<N>(sm, ci.rows, x0, a.scratch + int64_t(lw) * a.r_alloc * N, tid);
}

// Grid: (bands of RB rows, layers in wave).  gamma goes to dvis at vis_off.
template <int N>
__global__ void __launch_bounds__(LargeCfg<N>::NT) k_degrid_rows(ImageArgs a, float2 *dvis, int l0) {
    constexpr int NT = LargeCfg<N>::NT, S = LargeCfg<N>::S, RB = LargeCfg<N>::RB;
    extern __shared__ float2 sm[];
    const int lw = blockIdx.y;
    const DevLayer L = a.layers[l0 + lw];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows;
    const int r0 = blockIdx.x * RB;
    const int tid = threadIdx.x;
    const uint32_t *code = a.codes + ci.code_off;
    float2 *g = dvis + L.vis_off;
    if (r0 >= R) return;
    const int nrows = min(RB, R - r0);
    const float2 *in = a.scratch + (int64_t(lw) * a.r_alloc + r0) * N;
    float2 *tw = sm + tw_offset<N>();
    stage_four_step<N>(tw, tid, NT);
    // the band's rows: every 8-byte copy in flight at once (the padded row
    // layout keeps only 8-byte alignment)
    for (int i = tid; i < nrows * N; i += NT)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(uint32_t(__cvta_generic_to_shared(
                         sm + (i / N) * S + RowLayout<N>::phys(i % N)))),
                     "l"(in + i)
                     : "memory");
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    rows_fft<N, -1, true>(sm, S, nrows, tid, NT, tw);
    const float *w = ci.weighting == 1 ? a.wgt + ci.wgt_off : nullptr;
    const float scale = 2.f * (((a.flags & kNormalize) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f) *
                        (a.lscale ? __ldg(a.lscale + L.layer) : 1.f);
    if (a.csr && ci.csr_off >= 0) {
        const CsrLayout cl(N, a.nb);
        const int32_t *ptr = reinterpret_cast<const int32_t *>(a.csr + ci.csr_off + cl.row_ptr);
        const uint2 *ents = reinterpret_cast<const uint2 *>(a.csr + ci.csr_off + cl.ents);
        if (r0 == 0)  // dropped baselines (last bucket) get a zero gradient
            for (int e = ptr[N / 2] + tid; e < ptr[N / 2 + 1]; e += NT) g[__ldg(ents + e).x] = make_float2(0.f, 0.f);
        const int e1 = ptr[r0 + nrows];
        for (int e = ptr[r0] + tid; e < e1; e += NT) {
            const uint2 en = __ldg(ents + e);
            const int r = int(code_row(en.y)), c = int(code_col(en.y));
            const float2 h = sm[(r - r0) * S + RowLayout<N>::phys(pos_after_rows<N>(c))];
            const float wv = scale * (w ? w[r * N + c] : 1.f);
            g[en.x] = make_float2(wv * h.x, code_conj(en.y) ? -wv * h.y : wv * h.y);
        }
        return;
    }
    for (int64_t b = tid; b < a.nb; b += NT) {
        const uint32_t cd = __ldg(code + b);
        if (cd == kCodeDropped) {
            if (r0 == 0) g[b] = make_float2(0.f, 0.f);
            continue;
        }
        const int r = int(code_row(cd));
        if (r < r0 || r >= r0 + nrows) continue;
        const int c = int(code_col(cd));
        const float2 h = sm[(r - r0) * S + RowLayout<N>::phys(pos_after_rows<N>(c))];
        const float wv = scale * (w ? w[r * N + c] : 1.f);
        g[b] = make_float2(wv * h.x, code_conj(cd) ? -wv * h.y : wv * h.y);
    }
}

template <int N>
Error launch_degrid_n(const ImageArgs &a, const float *resid, float2 *dvis, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    using C = DegridCfg<N>;
    const size_t per_layer = size_t(a.r_alloc) * N * sizeof(float2);
    if (!a.scratch || a.scratch_bytes < per_layer)
        return Error{-5, "degrid scratch too small for image size " + std::to_string(N)};
    const int wave = wave_size(a.n_layers, a.scratch_bytes, per_layer);
    const size_t smem_c = degrid_cols_smem<N>();
    const size_t smem_r = rows_smem<N>();
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_degrid_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_c)));
    // three CTAs per SM: ask for the largest shared-memory carveout
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_degrid_cols<N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_degrid_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_r)));
    const unsigned pchunks = unsigned((N + 2 * C::P - 1) / (2 * C::P));
    const unsigned bands = unsigned((a.r_alloc + C::RB - 1) / C::RB);
    // waves split over the auxiliary stream as in the forward path
    const bool two = a.aux && a.ev_fork && a.ev_join && wave >= 2;
    if (two) {
        BLINK_CUDA_TRY(cudaEventRecord(a.ev_fork, st));
        BLINK_CUDA_TRY(cudaStreamWaitEvent(a.aux, a.ev_fork, 0));
    }
    auto pass = [&](const ImageArgs &b, int l0, int cnt, cudaStream_t s) -> Error {
        k_degrid_cols<N><<<dim3(pchunks, unsigned(cnt)), C::NT, smem_c, s>>>(b, resid, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_degrid_rows<N><<<dim3(bands, unsigned(cnt)), LargeCfg<N>::NT, smem_r, s>>>(b, dvis, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
        return Error{0, ""};
    };
    const int half = wave / 2;
    ImageArgs hb = a;
    hb.scratch = a.scratch + size_t(half) * a.r_alloc * N;
    for (int l0 = 0; l0 < a.n_layers; l0 += wave) {
        const int cnt = std::min(wave, a.n_layers - l0);
        if (two && cnt >= 2) {
            const int h = std::min(half, cnt - 1);
            Error e = pass(a, l0, h, st);
            if (e.status) return e;
            e = pass(hb, l0 + h, cnt - h, a.aux);
            if (e.status) return e;
        } else {
            Error e = pass(a, l0, cnt, st);
            if (e.status) return e;
        }
    }
    if (two) {
        BLINK_CUDA_TRY(cudaEventRecord(a.ev_join, a.aux));
        BLINK_CUDA_TRY(cudaStreamWaitEvent(st, a.ev_join, 0));
    }
    return Error{0, ""};
}

// The adjoint's column transforms of every layer's image (resid) into the
// slots out[l][k][p] (r_alloc rows of N per layer, FFT-order columns): the
// first half of blink_degrid, kept for a later row pass.
template <int N>
Error launch_degrid_cols_n(const ImageArgs &a, const float *resid, float2 *out, cudaStream_t st) {
    using C = DegridCfg<N>;
    const size_t smem_c = degrid_cols_smem<N>();
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_degrid_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_c)));
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_degrid_cols<N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const unsigned pchunks = unsigned((N + 2 * C::P - 1) / (2 * C::P));
    for (int l0 = 0; l0 < a.n_layers; l0 += 65535) {
        const int cnt = std::min(65535, a.n_layers - l0);
        ImageArgs b = a;
        b.scratch = out + int64_t(l0) * a.r_alloc * N;
        k_degrid_cols<N><<<dim3(pchunks, unsigned(cnt)), C::NT, smem_c, st>>>(b, resid, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

// The adjoint's row pass from kept column transforms (slots as above).
template <int N>
Error launch_degrid_rows_n(const ImageArgs &a, const float2 *in, float2 *dvis, cudaStream_t st) {
    const size_t smem_r = rows_smem<N>();
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_degrid_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_r)));
    const unsigned bands = unsigned((a.r_alloc + LargeCfg<N>::RB - 1) / LargeCfg<N>::RB);
    for (int l0 = 0; l0 < a.n_layers; l0 += 65535) {
        const int cnt = std::min(65535, a.n_layers - l0);
        ImageArgs b = a;
        b.scratch = const_cast<float2 *>(in) + int64_t(l0) * a.r_alloc * N;
        k_degrid_rows<N><<<dim3(bands, unsigned(cnt)), LargeCfg<N>::NT, smem_r, st>>>(b, dvis, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

template <int N>
bool use_small(int r_alloc) {
    return N <= 256 && small_path_fits(N, r_alloc);
}

// The persistent launch of one size group (a.queue holds queue_bytes(n)).
template <int N>
Error launch_large_n(const ImageArgs &a, cudaStream_t st) {
    const size_t per_layer = size_t(a.r_alloc) * N * sizeof(float2);
    LargeSched q{};
    q.n = a.n_layers;
    // band height: at most RB rows, and about kBandEntries gridding entries
    // per row item, so a dense band does not hold up its layer's column items
    // (row items that read compact grids gather nothing: full bands)
    constexpr int kBandEntries = 4096;
    q.rb = a.row_entries > 0 && !a.cg ? std::max(1, std::min(RowsCfg<N>::RB, kBandEntries / a.row_entries))
                                      : RowsCfg<N>::RB;
    q.nR = (a.r_alloc + q.rb - 1) / q.rb;
    q.nC = (N / 2 + LargeCfg<N>::P - 1) / LargeCfg<N>::P;
    q.total = int64_t(q.n) * (q.nR + q.nC);
    q.wait_ns = a.wait_ns < 0 ? kWaitNs : static_cast<unsigned long long>(a.wait_ns);
    const size_t ring = a.wave_budget ? std::min(a.scratch_bytes, std::max(a.wave_budget, per_layer)) : a.scratch_bytes;
    q.slots = int(std::max<size_t>(1, std::min<size_t>(ring / per_layer, size_t(q.n))));
    const size_t smem = large_smem<N>(a.r_alloc);
    auto kern = (a.ref || a.sq_part || a.adj) ? k_large<N, true> : k_large<N, false>;
    BLINK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    // three CTAs per SM need the largest shared-memory carveout
    BLINK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int dev = 0, sms = 0, per_sm = 0;
    BLINK_CUDA_TRY(cudaGetDevice(&dev));
    BLINK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BLINK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
    if (per_sm < 1) return Error{-2, "persistent image kernel does not fit on an SM for size " + std::to_string(N)};
    const int64_t grid = std::min<int64_t>(q.total, int64_t(per_sm) * sms);
    // lag: up to eight grids of items between a layer's row and column items
    // (a dense band of rows takes several times as long as a column item).
    // A row item also waits for the column items of the layer `slots` back,
    // which sit slots - lag stages earlier: half the ring each way keeps both
    // gaps wide (and lag <= slots - 1).
    const int lag_want = int(8 * grid / int64_t(q.nR + q.nC)) + 1;
    q.lag = std::max(0, std::min({lag_want, q.slots / 2, q.n}));
    // look-ahead prefetch of row buckets: only when they do not all stay in L2
    q.ahead = a.csr_bytes > (size_t(32) << 20) && !a.cg
                  ? int(std::min<int64_t>(64, std::max<int64_t>(1, grid / int64_t(q.nR + q.nC))))
                  : 0;
    BLINK_CUDA_TRY(cudaMemsetAsync(a.queue, 0, image_queue_bytes(q.n), st));
    kern<<<unsigned(grid), 256, smem, st>>>(a, q, static_cast<float *>(a.out), a.ref);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

// The large-image path of a group (or of one wave of compact grids).
template <int N>
Error launch_large_body(const ImageArgs &a, cudaStream_t st) {
    using C = LargeCfg<N>;
    const size_t per_layer = size_t(a.r_alloc) * N * sizeof(float2);
    // the persistent queue by default; groups whose rows come from compact
    // grids (short row items, nothing to gather) run as waves unless path 3
    // is asked for: there the two kernels measured a few per cent faster
    const bool waves = a.force_path == 4 || (a.force_path == 0 && a.cg);
    if (!waves && a.queue && a.queue_bytes >= image_queue_bytes(a.n_layers)) return launch_large_n<N>(a, st);
    // wave path (no work queue, or chosen by the autotuner): pass 1 of a wave
    // of layers, then pass 2
    const int wave = wave_size(a.n_layers, a.scratch_bytes, per_layer, a.wave_budget);
    const size_t smem_rows = RowsCfg<N>::smem;
    const size_t smem_cols = cols_smem<N>(a.r_alloc);
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem_rows)));
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_rows<N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    auto cols = (a.ref || a.sq_part || a.adj) ? k_cols<N, true> : k_cols<N, false>;
    BLINK_CUDA_TRY(cudaFuncSetAttribute(cols, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_cols)));
    BLINK_CUDA_TRY(cudaFuncSetAttribute(cols, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const unsigned bands = unsigned((a.r_alloc + RowsCfg<N>::RB - 1) / RowsCfg<N>::RB);
    const unsigned pchunks = unsigned((N / 2 + C::P - 1) / C::P);
    for (int l0 = 0; l0 < a.n_layers; l0 += wave) {
        const int cnt = std::min(wave, a.n_layers - l0);
        k_rows<N><<<dim3(bands, unsigned(cnt)), RowsCfg<N>::NT, smem_rows, st>>>(a, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
        cols<<<dim3(pchunks, unsigned(cnt)), C::NT, smem_cols, st>>>(a, l0, static_cast<float *>(a.out), a.ref);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

template <int N>
Error launch_image_n(const ImageArgs &a, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    {
        Error e;
        if (launch_fused_n<N>(a, st, e)) {
            // the fused small-image kernels keep no column strips: the
            // adjoint's columns are transformed from the stored images
            if (!e.status && a.adj) e = launch_degrid_cols_n<N>(a, static_cast<const float *>(a.out), a.adj, st);
            return e;
        }
    }
    const size_t per_layer = size_t(a.r_alloc) * N * sizeof(float2);
    if (!a.scratch || a.scratch_bytes < per_layer)
        return Error{-5, "row-transform scratch too small for image size " + std::to_string(N)};
    if (!AdjFusable<N>::value && a.adj) {
        ImageArgs b = a;
        b.adj = nullptr;
        Error e = launch_image_n<N>(b, st);
        if (!e.status) e = launch_degrid_cols_n<N>(a, static_cast<const float *>(a.out), a.adj, st);
        return e;
    }
    if (!a.cg) return launch_large_body<N>(a, st);
    // compact gridding, one wave of the compact-grid buffer at a time, each
    // wave followed by its rows and columns
    for (int l0 = 0; l0 < a.n_layers; l0 += a.cg_cap) {
        ImageArgs b = a;
        b.layers = a.layers + l0;
        b.n_layers = std::min(a.cg_cap, a.n_layers - l0);
        b.cg_l0 = 0;
        if (a.adj) b.adj = a.adj + int64_t(l0) * a.r_alloc * N;
        Error e = launch_grid_compact(b, 0, b.n_layers, st);
        if (e.status) return e;
        e = launch_large_body<N>(b, st);
        if (e.status) return e;
    }
    return Error{0, ""};
}

template <int N>
size_t scratch_per_layer_n(int r_alloc) {
    return use_small<N>(r_alloc) ? 0 : size_t(r_alloc) * N * sizeof(float2);
}

}  // namespace

// Per-size entry points; each size is explicitly instantiated in exactly one
// blink_image_<sizes>.cu translation unit (they compile in parallel).
template <int N>
Error SizeOps<N>::image(const ImageArgs &a, cudaStream_t st) { return launch_image_n<N>(a, st); }

template <int N>
Error SizeOps<N>::rows_wave(const ImageArgs &a, int l0, int cnt, cudaStream_t st) {
    const size_t smem_rows = RowsCfg<N>::smem;
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_rows)));
    const unsigned bands = unsigned((a.r_alloc + RowsCfg<N>::RB - 1) / RowsCfg<N>::RB);
    k_rows<N><<<dim3(bands, unsigned(cnt)), RowsCfg<N>::NT, smem_rows, st>>>(a, l0);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

template <int N>
Error SizeOps<N>::degrid(const ImageArgs &a, const float *resid, float2 *dvis, cudaStream_t st) {
    return launch_degrid_n<N>(a, resid, dvis, st);
}

template <int N>
Error SizeOps<N>::degrid_rows(const ImageArgs &a, const float2 *in, float2 *dvis, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    return launch_degrid_rows_n<N>(a, in, dvis, st);
}

template <int N>
Error SizeOps<N>::degrid_cols(const ImageArgs &a, const float *resid, float2 *out, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    return launch_degrid_cols_n<N>(a, resid, out, st);
}

template <int N>
bool SizeOps<N>::small(int r_alloc) { return use_small<N>(r_alloc); }

template <int N>
size_t SizeOps<N>::scratch_per_layer(int r_alloc) { return scratch_per_layer_n<N>(r_alloc); }

template <int N>
int SizeOps<N>::sq_slots() { return (N / 2 + LargeCfg<N>::P - 1) / LargeCfg<N>::P; }

template <int N>
bool SizeOps<N>::adj_fusable() { return AdjFusable<N>::value; }

}  // namespace blink
