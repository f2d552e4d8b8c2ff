// blink_image.cu -- gridding (a3-a4) and the shifted inverse 2-D FFT (a5-a7).
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
// Paths.  Small images: one CTA grids a whole layer in shared memory
// (per-element shared atomics, no global atomics) and runs both passes there.
// Large images: k_rows grids a band of rows per CTA and writes transformed
// rows to a scratch buffer; k_cols runs pass 2 from it.
#include "blink_common.cuh"
#include "blink_fft.cuh"
#include "blink_kernels.cuh"

#include <algorithm>

namespace blink {

namespace {

constexpr int kNormalize = 1;

__device__ __forceinline__ float2 ld_stream(const float2 *p) { return __ldcs(p); }

// Weight the canonical cells and complete row 0.  G has row stride S.
// Cells outside the canonical half are zero on entry.
template <int N>
__device__ __forceinline__ void weight_and_complete(float2 *G, int S, int r_begin, int r_end,
                                                    const ChanInfo &ci, const float *wgt, int tid,
                                                    int nt) {
    constexpr int H = N / 2;
    const float *w = ci.weighting == 1 ? wgt + ci.wgt_off : nullptr;
    if (w) {
        const int first = max(r_begin, 1);
        for (int idx = tid; idx < (r_end - first) * N; idx += nt) {
            const int r = first + idx / N, c = idx % N;
            float2 &g = G[(r - r_begin) * S + c];
            const float wv = w[r * N + c];
            g.x *= wv;
            g.y *= wv;
        }
    }
    if (r_begin == 0) {
        for (int c = tid; c < H; c += nt) {
            const float wv = w ? w[c] : 1.f;
            float2 g = G[c];
            if (c == 0) {
                // origin: V and conj(V) of every baseline there
                G[0] = make_float2(2.f * g.x * wv, 0.f);
            } else {
                g.x *= wv;
                g.y *= wv;
                G[c] = g;
                G[N - c] = make_float2(g.x, -g.y);
            }
        }
    }
}

// Pass 1 on rows [0, nrows) of G (row stride S): N-point inverse DFT of each
// row in place.  Output frequency p ends at position N2 * (p % N1) + p / N1.
template <int N>
__device__ __forceinline__ void rows_fft(float2 *G, int S, int nrows, int tid, int nt) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    // step A: N1-point transforms along stride N2, then twiddle W_N^(n2 k1)
    for (int t = tid; t < nrows * N2; t += nt) {
        const int r = t % nrows, n2 = t / nrows;
        float2 *row = G + r * S + n2;
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = row[N2 * n1];
        dft<N1, +1>(x);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) x[k1] = cmulc(x[k1], c_roots<N, +1>.v[n2 * k1]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) row[N2 * k1] = x[k1];
    }
    __syncthreads();
    // step B: N2-point transforms on contiguous runs, result kept in place
    for (int t = tid; t < nrows * N1; t += nt) {
        const int r = t % nrows, k1 = t / nrows;
        float2 *run = G + r * S + N2 * k1;
        float2 y[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) y[n2] = run[n2];
        dft<N2, +1>(y);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) run[k2] = y[k2];
    }
    __syncthreads();
}

template <int N>
__device__ __forceinline__ int pos_after_rows(int p) {
    return Plan<N>::N2 * (p % Plan<N>::N1) + p / Plan<N>::N1;
}

// Pass 2, step A for column pairs (j0 + jj, j0 + jj + N/2), jj < P.  `hrow(k,
// p)` returns row k (< R) of the pass-1 output at frequency column p.  Writes
// the four-step intermediate of pair jj to Z + jj * S.
template <int N, int P, class HRow>
__device__ __forceinline__ void cols_step_a(float2 *Z, int S, int R, int j0, HRow hrow, int tid,
                                            int nt) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H = N / 2;
    for (int t = tid; t < P * N2; t += nt) {
        const int jj = t % P, n2 = t / P;
        const int ja = j0 + jj;
        if (ja >= H) continue;
        const int jb = ja + H;
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int k = N2 * n1 + n2;
            float2 z = make_float2(0.f, 0.f);
            if (k < H) {
                if (k < R) {
                    const float2 a = hrow(k, ja), b = hrow(k, jb);
                    z = make_float2(a.x - b.y, a.y + b.x);  // H_a + i H_b
                }
            } else if (k > H) {
                const int m = N - k;
                if (m < R) {
                    const float2 a = hrow(m, ja), b = hrow(m, jb);
                    z = make_float2(a.x + b.y, b.x - a.y);  // conj(H_a) + i conj(H_b)
                }
            }
            x[n1] = z;
        }
        dft<N1, +1>(x);
        float2 *zp = Z + jj * S + n2;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1)
            zp[N2 * k1] = k1 == 0 ? x[0] : cmulc(x[k1], c_roots<N, +1>.v[n2 * k1]);
    }
}

// Pass 2, step B: N2-point transforms, then the two real image columns with
// the fftshift folded into the addresses.
template <int N, int P>
__device__ __forceinline__ void cols_step_b(const float2 *Z, int S, int j0, float *img, float scale,
                                            int tid, int nt) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H = N / 2;
    for (int t = tid; t < P * N1; t += nt) {
        const int jj = t % P, k1 = t / P;
        const int ja = j0 + jj;
        if (ja >= H) continue;
        const float2 *zp = Z + jj * S + N2 * k1;
        float2 y[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) y[n2] = zp[n2];
        dft<N2, +1>(y);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int q = k1 + N1 * k2;               // FFT-order row
            const int row = q < H ? q + H : q - H;    // fftshift
            float *o = img + int64_t(row) * N;
            __stcs(o + ja + H, y[k2].x * scale);      // column ja   -> ja + N/2
            __stcs(o + ja, y[k2].y * scale);          // column ja+H -> ja
        }
    }
}

// Grid the canonical rows [r0, r0 + nrows) of one layer into G (stride S).
template <int NT>
__device__ __forceinline__ void grid_rows(float2 *G, int S, int r0, int nrows, const uint32_t *code,
                                          const float2 *vis, int64_t nb, int tid) {
    for (int64_t b = tid; b < nb; b += NT) {
        const uint32_t cd = __ldg(code + b);
        if (cd == kCodeDropped) continue;
        const int r = int(code_row(cd)) - r0;
        if (r < 0 || r >= nrows) continue;
        float2 v = ld_stream(vis + b);
        if (code_conj(cd)) v.y = -v.y;
        float2 *cell = G + r * S + code_col(cd);
        atomicAdd(&cell->x, v.x);
        atomicAdd(&cell->y, v.y);
    }
}

// ------------------------------------------------------------- small path
template <int N>
struct SmallCfg {
    static constexpr int NT = 384;
    static constexpr int P = std::min(32, NT / Plan<N>::N1);
};

template <int N>
__global__ void __launch_bounds__(SmallCfg<N>::NT) k_image_small(ImageArgs a) {
    constexpr int NT = SmallCfg<N>::NT, P = SmallCfg<N>::P, S = N + 1, H = N / 2;
    extern __shared__ float2 sm[];
    const DevLayer L = a.layers[blockIdx.x];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows;
    float2 *G = sm;
    float2 *Z = sm + size_t(a.r_alloc) * S;
    const int tid = threadIdx.x;
    for (int i = tid; i < R * S; i += NT) G[i] = make_float2(0.f, 0.f);
    __syncthreads();
    grid_rows<NT>(G, S, 0, R, a.codes + ci.code_off, a.vis + L.vis_off, a.nb, tid);
    __syncthreads();
    weight_and_complete<N>(G, S, 0, R, ci, a.wgt, tid, NT);
    __syncthreads();
    rows_fft<N>(G, S, R, tid, NT);
    const float scale = ((a.flags & kNormalize) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f;
    float *img = static_cast<float *>(a.out) + L.out_off;
    auto hrow = [&](int k, int p) { return G[k * S + pos_after_rows<N>(p)]; };
    for (int j0 = 0; j0 < H; j0 += P) {
        cols_step_a<N, P>(Z, S, R, j0, hrow, tid, NT);
        __syncthreads();
        cols_step_b<N, P>(Z, S, j0, img, scale, tid, NT);
        __syncthreads();
    }
    if (tid == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
}

template <int N>
size_t small_smem(int r_alloc) {
    return size_t(r_alloc + SmallCfg<N>::P) * (N + 1) * sizeof(float2);
}

// ------------------------------------------------------------- large path
template <int N>
struct LargeCfg {
    static constexpr int NT = 256;
    static constexpr int S = N + 1;
    static constexpr int RB = std::max(1, std::min(32, int(65536 / (S * sizeof(float2)))));
    static constexpr int P = std::max(1, std::min(32, NT / Plan<N>::N1));
};

// Pass 1 for a band of RB canonical rows of one layer, written in natural
// order to scratch[layer_in_wave][r][p].  Grid: (bands, layers in wave).
template <int N>
__global__ void __launch_bounds__(LargeCfg<N>::NT) k_rows(ImageArgs a, int l0) {
    constexpr int NT = LargeCfg<N>::NT, S = LargeCfg<N>::S, RB = LargeCfg<N>::RB;
    extern __shared__ float2 sm[];
    const int lw = blockIdx.y;
    const DevLayer L = a.layers[l0 + lw];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows;
    const int r0 = blockIdx.x * RB;
    if (r0 >= R) return;
    const int nrows = min(RB, R - r0);
    const int tid = threadIdx.x;
    for (int i = tid; i < nrows * S; i += NT) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    grid_rows<NT>(sm, S, r0, nrows, a.codes + ci.code_off, a.vis + L.vis_off, a.nb, tid);
    __syncthreads();
    weight_and_complete<N>(sm, S, r0, r0 + nrows, ci, a.wgt, tid, NT);
    __syncthreads();
    rows_fft<N>(sm, S, nrows, tid, NT);
    float2 *out = a.scratch + (int64_t(lw) * a.r_alloc + r0) * N;
    for (int i = tid; i < nrows * N; i += NT) {
        const int r = i / N, p = i % N;
        out[int64_t(r) * N + p] = sm[r * S + pos_after_rows<N>(p)];
    }
}

// Pass 2 for P column pairs of one layer.  Grid: (ceil(N/2 / P), layers in wave).
template <int N>
__global__ void __launch_bounds__(LargeCfg<N>::NT) k_cols(ImageArgs a, int l0) {
    constexpr int NT = LargeCfg<N>::NT, S = LargeCfg<N>::S, P = LargeCfg<N>::P;
    extern __shared__ float2 sm[];
    const int lw = blockIdx.y;
    const DevLayer L = a.layers[l0 + lw];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows;
    const int j0 = blockIdx.x * P;
    const float2 *Hs = a.scratch + int64_t(lw) * a.r_alloc * N;
    auto hrow = [&](int k, int p) { return Hs[int64_t(k) * N + p]; };
    cols_step_a<N, P>(sm, S, R, j0, hrow, threadIdx.x, NT);
    __syncthreads();
    const float scale = ((a.flags & kNormalize) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f;
    cols_step_b<N, P>(sm, S, j0, static_cast<float *>(a.out) + L.out_off, scale, threadIdx.x, NT);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
}

// ----------------------------------------------------- full grid (blink_grid)
// Output rows [y0, y0 + RB) of the Hermitian-complete grid, DC at (N/2, N/2).
// Slot s holds canonical row |y0 + s - N/2|.
constexpr int kGridRB = 8;
constexpr int kGridNT = 256;

__global__ void __launch_bounds__(kGridNT) k_grid_full(ImageArgs a, int n) {
    extern __shared__ float2 sm[];
    const int h = n / 2;
    const DevLayer L = a.layers[blockIdx.y];
    const ChanInfo ci = a.chans[L.chan];
    const int R = ci.rows;
    const int y0 = blockIdx.x * kGridRB;
    const int ny = min(kGridRB, n - y0);
    const int tid = threadIdx.x;
    for (int i = tid; i < ny * n; i += kGridNT) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const uint32_t *code = a.codes + ci.code_off;
    const float2 *vis = a.vis + L.vis_off;
    for (int64_t b = tid; b < a.nb; b += kGridNT) {
        const uint32_t cd = __ldg(code + b);
        if (cd == kCodeDropped) continue;
        const int r = int(code_row(cd));
        const int c = int(code_col(cd));
        const int ya = h + r - y0, yb = h - r - y0;
        const bool ina = ya >= 0 && ya < ny, inb = r > 0 && yb >= 0 && yb < ny;
        if (!ina && !inb) continue;
        float2 v = vis[b];
        if (code_conj(cd)) v.y = -v.y;
        if (ina) { atomicAdd(&sm[ya * n + c].x, v.x); atomicAdd(&sm[ya * n + c].y, v.y); }
        if (inb) { atomicAdd(&sm[yb * n + c].x, v.x); atomicAdd(&sm[yb * n + c].y, v.y); }
    }
    __syncthreads();
    const float *w = ci.weighting == 1 ? a.wgt + ci.wgt_off : nullptr;
    float2 *out = static_cast<float2 *>(a.out) + L.out_off;
    for (int i = tid; i < ny * n; i += kGridNT) {
        const int s = i / n, x = i % n;
        const int y = y0 + s;
        const int kv = y - h, ku = x - h;
        const int r = kv >= 0 ? kv : -kv;
        float2 val = make_float2(0.f, 0.f);
        if (r < R && y > 0 && x > 0) {
            const float2 *srow = sm + s * n;
            if (r == 0) {
                if (ku == 0) {
                    const float wv = w ? w[0] : 1.f;
                    val = make_float2(2.f * srow[0].x * wv, 0.f);
                } else {
                    const int c = ku > 0 ? ku : -ku;
                    const float wv = w ? w[c] : 1.f;
                    const float2 g = srow[c];
                    val = ku > 0 ? make_float2(g.x * wv, g.y * wv) : make_float2(g.x * wv, -g.y * wv);
                }
            } else {
                // k_v > 0: canonical (r, k_u); k_v < 0: conj of canonical (r, -k_u)
                const int cu = kv > 0 ? ku : -ku;
                const int c = cu < 0 ? cu + n : cu;
                const float wv = w ? w[r * n + c] : 1.f;
                const float2 g = srow[c];
                val = kv > 0 ? make_float2(g.x * wv, g.y * wv) : make_float2(g.x * wv, -g.y * wv);
            }
        }
        out[int64_t(y) * n + x] = val;
    }
    if (blockIdx.x == 0 && tid == 0 && a.wsum_out) a.wsum_out[L.layer] = ci.wsum;
}

constexpr size_t kSmallSmemLimit = 200 * 1024;

template <int N>
bool use_small(int r_alloc) {
    return N <= 256 && small_smem<N>(r_alloc) <= kSmallSmemLimit;
}

template <int N>
Error launch_image_n(const ImageArgs &a, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    if constexpr (N <= 256) {
      if (use_small<N>(a.r_alloc)) {
        const size_t smem = small_smem<N>(a.r_alloc);
        BLINK_CUDA_TRY(cudaFuncSetAttribute(k_image_small<N>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        for (int l0 = 0; l0 < a.n_layers; l0 += 1 << 30) {
            ImageArgs b = a;
            b.layers = a.layers + l0;
            const int cnt = std::min(a.n_layers - l0, 1 << 30);
            k_image_small<N><<<cnt, SmallCfg<N>::NT, smem, st>>>(b);
            BLINK_CUDA_TRY(cudaGetLastError());
        }
        return Error{0, ""};
      }
    }
    using C = LargeCfg<N>;
    const size_t per_layer = size_t(a.r_alloc) * N * sizeof(float2);
    if (!a.scratch || a.scratch_bytes < per_layer)
        return Error{-5, "row-transform scratch too small for image size " + std::to_string(N)};
    const int wave = int(std::min<size_t>(size_t(a.n_layers), std::min<size_t>(65535, a.scratch_bytes / per_layer)));
    const size_t smem_rows = size_t(C::RB) * C::S * sizeof(float2);
    const size_t smem_cols = size_t(C::P) * C::S * sizeof(float2);
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem_rows)));
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem_cols)));
    const unsigned bands = unsigned((a.r_alloc + C::RB - 1) / C::RB);
    const unsigned pchunks = unsigned((N / 2 + C::P - 1) / C::P);
    for (int l0 = 0; l0 < a.n_layers; l0 += wave) {
        const int cnt = std::min(wave, a.n_layers - l0);
        k_rows<N><<<dim3(bands, unsigned(cnt)), C::NT, smem_rows, st>>>(a, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_cols<N><<<dim3(pchunks, unsigned(cnt)), C::NT, smem_cols, st>>>(a, l0);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

template <int N>
size_t scratch_per_layer_n(int r_alloc) {
    return use_small<N>(r_alloc) ? 0 : size_t(r_alloc) * N * sizeof(float2);
}

}  // namespace

bool image_size_supported(int n_px) {
#define X(N_) if (n_px == N_) return true;
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return false;
}

int supported_sizes(int32_t *out, int cap) {
    int k = 0;
#define X(N_) { if (out && k < cap) out[k] = N_; ++k; }
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return k;
}

size_t image_scratch_per_layer(int n_px, int r_alloc) {
#define X(N_) if (n_px == N_) return scratch_per_layer_n<N_>(r_alloc);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return 0;
}

Error launch_image_group(int n_px, const ImageArgs &a, cudaStream_t st) {
#define X(N_) if (n_px == N_) return launch_image_n<N_>(a, st);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return Error{-2, "unsupported image size " + std::to_string(n_px)};
}

Error launch_grid_group(int n_px, const ImageArgs &a, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    const size_t smem = size_t(kGridRB) * n_px * sizeof(float2);
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_grid_full, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem)));
    const unsigned bands = unsigned((n_px + kGridRB - 1) / kGridRB);
    for (int l0 = 0; l0 < a.n_layers; l0 += 65535) {
        ImageArgs b = a;
        b.layers = a.layers + l0;
        b.n_layers = std::min(65535, a.n_layers - l0);
        k_grid_full<<<dim3(bands, unsigned(b.n_layers)), kGridNT, smem, st>>>(b, n_px);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

}  // namespace blink
