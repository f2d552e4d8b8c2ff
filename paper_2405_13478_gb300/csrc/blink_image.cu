// blink_image.cu -- size dispatch of the gridding / transform kernels and the
// full Hermitian grid of blink_grid.  The kernels themselves are templates in
// blink_image_impl.cuh, instantiated per image size in blink_image_<sizes>.cu.
#include "blink_common.cuh"
#include "blink_kernels.cuh"

#include <algorithm>
#include <string>

namespace blink {

namespace {

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

// ------------------------------------------- per-layer sums of squares
// One warp per layer: lane i adds slots i, i + 32, ... in order, then a fixed
// shuffle tree; the same bits on every run.
constexpr int kSqWarps = 8;

__global__ void __launch_bounds__(32 * kSqWarps) k_sq_totals(const double *part, int stride, int n_layers,
                                                             double *out) {
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * kSqWarps + (threadIdx.x >> 5);
    if (l >= n_layers) return;  // whole warps leave together
    const double *row = part + int64_t(l) * stride;
    double s = 0.0;
    for (int i = lane; i < stride; i += 32) s += row[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[l] = s;
}

// ------------------------------------------------------------ adjoint
// Gradient of a real image loss with respect to the visibilities:
// gamma_b = 2 w_b H[k_b], H = forward 2-D DFT (exp(-2 pi i k.(p - N/2)/N)) of
// the image gradient R, conjugated for baselines mirrored into the canonical
// half, zero for dropped baselines.  H is needed only on the canonical
// support rows.  Pass 1 (k_degrid_cols): the real columns of R, two at a time
// packed as one complex column, forward N-point transforms along v; rows
// k < R of both columns to scratch.  Pass 2 (k_degrid_rows): forward
// transforms of those rows along u, then every baseline of the band reads
// its cell.
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

bool image_small_path(int n_px, int r_alloc) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::small(r_alloc);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return false;
}

size_t image_rows_scratch_per_layer(int n_px, int r_alloc) { return size_t(r_alloc) * n_px * sizeof(float2); }

// a 64-bit item counter and the abort flag (four words), then two counters per layer
size_t image_queue_bytes(int n_layers) { return (4 + 2 * size_t(n_layers > 0 ? n_layers : 0)) * sizeof(int); }

size_t image_scratch_per_layer(int n_px, int r_alloc) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::scratch_per_layer(r_alloc);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return 0;
}

Error launch_image_group(int n_px, const ImageArgs &a, cudaStream_t st) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::image(a, st);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return Error{-2, "unsupported image size " + std::to_string(n_px)};
}

Error launch_rows_wave(int n_px, const ImageArgs &a, int l0, int cnt, cudaStream_t st) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::rows_wave(a, l0, cnt, st);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return Error{-2, "unsupported image size " + std::to_string(n_px)};
}

size_t degrid_scratch_per_layer(int n_px, int r_alloc) {
    return size_t(r_alloc) * n_px * sizeof(float2);
}

Error launch_degrid_group(int n_px, const ImageArgs &a, const float *resid, float2 *dvis, cudaStream_t st) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::degrid(a, resid, dvis, st);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return Error{-2, "unsupported image size " + std::to_string(n_px)};
}

bool adjoint_fusable(int n_px) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::adj_fusable();
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return false;
}

int sq_slots(int n_px) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::sq_slots();
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return 0;
}

Error launch_sq_totals(const double *part, int stride, int n_layers, double *out, cudaStream_t st) {
    if (n_layers <= 0) return Error{0, ""};
    const unsigned blocks = unsigned((n_layers + kSqWarps - 1) / kSqWarps);
    k_sq_totals<<<blocks, 32 * kSqWarps, 0, st>>>(part, stride, n_layers, out);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

Error launch_degrid_cols_group(int n_px, const ImageArgs &a, const float *resid, float2 *out, cudaStream_t st) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::degrid_cols(a, resid, out, st);
    BLINK_FOR_EACH_SIZE(X)
#undef X
    return Error{-2, "unsupported image size " + std::to_string(n_px)};
}

Error launch_degrid_rows_group(int n_px, const ImageArgs &a, const float2 *in, float2 *dvis, cudaStream_t st) {
#define X(N_) if (n_px == N_) return SizeOps<N_>::degrid_rows(a, in, dvis, st);
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
