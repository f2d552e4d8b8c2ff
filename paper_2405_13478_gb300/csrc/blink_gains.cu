// blink_gains.cu -- per-antenna complex gains: forward application and the
// chain rule of the image-loss gradient.
//
// Visibilities corrupted by antenna gains, V_ij = g_i conj(g_j) M_ij (the
// antenna-level calibration factors of Sec. 4.2 applied to model
// visibilities M).  With gamma = dL/dRe V + i dL/dIm V from blink_degrid,
//   gamma(g_i) = sum_{j>i} gamma(V_ij) g_j conj(M_ij)
//              + sum_{k<i} conj(gamma(V_ki)) g_k M_ki,
// summed over all layers.  Every sum runs in a fixed order, so the gradient
// is the same bits from run to run: per thread a compensated FP32 sum
// (Kahan 1965: the running error of each add is carried into the next), the
// partials then in FP64.  This part runs FP64 at about 1/75 of its FP32
// rate, so FP64 adds per baseline would bound the kernel.
#include "blink_common.cuh"
#include "blink_kernels.cuh"
#include "blink_pairs.cuh"

#include <algorithm>

namespace blink {

namespace {

// Grid: (ceil(B / 256), layers).
__global__ void k_apply_gains(const float2 *__restrict__ model, const float2 *__restrict__ gains,
                              const int64_t *__restrict__ vis_off, int n_ant, int64_t nb,
                              float2 *__restrict__ vis) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int i, j;
    baseline_pair(b, n_ant, i, j);
    const int64_t o = vis_off[blockIdx.y] + b;
    const float2 m = model[o], gi = gains[i], gj = gains[j];
    // g_i conj(g_j)
    const float2 p = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
    vis[o] = make_float2(p.x * m.x - p.y * m.y, p.x * m.y + p.y * m.x);
}

// Grid: (ceil(B / 256), rows).  Gain-product table of the fused epilogue.
__global__ void k_gain_products(const float2 *__restrict__ gains, int64_t stride, int n_ant, int64_t nb,
                                float2 *__restrict__ out) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int i, j;
    baseline_pair(b, n_ant, i, j);
    const float2 *g = gains + int64_t(blockIdx.y) * stride;
    const float2 gi = g[i], gj = g[j];
    out[int64_t(blockIdx.y) * nb + b] = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
}

// Compensated FP32 sum of a complex series (Kahan summation per component).
struct KSum {
    float2 s, c;  // running sum, running compensation (the negated lost low part)
    __device__ __forceinline__ void zero() {
        s = make_float2(0.f, 0.f);
        c = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void add(float x, float y) {
        const float ax = x - c.x, ay = y - c.y;
        const float tx = s.x + ax, ty = s.y + ay;
        c.x = (tx - s.x) - ax;
        c.y = (ty - s.y) - ay;
        s.x = tx;
        s.y = ty;
    }
    __device__ __forceinline__ double2 value() const {
        return make_double2(double(s.x) - double(c.x), double(s.y) - double(c.y));
    }
};

// Gain gradient, pass 1.  CTA (t, g) takes the antenna rows i of tile t
// (kGradTile rows) and the layers of group g; thread j walks the baselines
// (i, j), j > i, of every such row -- contiguous in the upper-triangle order,
// so every load is coalesced -- and adds
//   to row i's partial:     gamma(V_ij) g_j conj(M_ij)        (kept per thread,
//                                                              reduced at the end)
//   to column j's partial:  conj(gamma(V_ij)) g_i M_ij.
// Products in FP32, per-thread sums compensated FP32, the reduction of the
// row partials in FP64, all in a fixed order.  Partials (FP64):
// pcol[g][t][j] and prow[g][i].
constexpr int kGradTile = 8;
constexpr int kGradThreads = 256;
constexpr int kGradMaxJ = 4;  // antennas per thread: n_ant <= 1024

__global__ void __launch_bounds__(kGradThreads, 2) k_gain_grad_part(const float2 *__restrict__ dvis,
                                                                 const float2 *__restrict__ model,
                                                                 const float2 *__restrict__ gains,
                                                                 const int64_t *__restrict__ vis_off, int n_layers,
                                                                 int n_ant, int layers_per_group,
                                                                 double2 *__restrict__ pcol,
                                                                 double2 *__restrict__ prow) {
    const int t = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
    const int i0 = t * kGradTile;
    const int l0 = g * layers_per_group, l1 = min(n_layers, l0 + layers_per_group);
    KSum racc[kGradTile];
#pragma unroll
    for (int k = 0; k < kGradTile; ++k) racc[k].zero();
    // the tile's rows: g_i and the position of baseline (i, 0) in a layer
    float2 gik[kGradTile];
    int32_t rowoff[kGradTile];
#pragma unroll
    for (int k = 0; k < kGradTile; ++k) {
        const int i = min(i0 + k, n_ant - 1);
        gik[k] = gains[i];
        rowoff[k] = int32_t(pair_row_start(i, n_ant) - i - 1);  // baseline (i, j) at rowoff + j
    }
    double2 *pc = pcol + (int64_t(g) * gridDim.x + t) * n_ant;
#pragma unroll
    for (int q = 0; q < kGradMaxJ; ++q) {
        if (q * kGradThreads >= n_ant) break;  // CTA-uniform
        const int j = tid + q * kGradThreads;
        const float2 gj = j < n_ant ? gains[j] : make_float2(0.f, 0.f);
        KSum cacc;
        cacc.zero();
        for (int l = l0; l < l1; ++l) {
            const int64_t o = vis_off[l];
            // every row's loads of this layer first (sixteen in flight), then
            // the sums in the fixed order of the rows
            float2 gv[kGradTile], mv[kGradTile];
#pragma unroll
            for (int k = 0; k < kGradTile; ++k) {
                const int i = i0 + k;
                const bool live = i < n_ant - 1 && j > i && j < n_ant;
                gv[k] = live ? dvis[o + rowoff[k] + j] : make_float2(0.f, 0.f);
                mv[k] = live ? model[o + rowoff[k] + j] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < kGradTile; ++k) {
                const int i = i0 + k;
                if (i < n_ant - 1 && j > i && j < n_ant) {
                    const float2 v = gv[k], m = mv[k], gi = gik[k];
                    const float tr = gj.x * m.x + gj.y * m.y, ti = gj.y * m.x - gj.x * m.y;  // g_j conj(M)
                    racc[k].add(v.x * tr - v.y * ti, v.x * ti + v.y * tr);
                    const float ur = gi.x * m.x - gi.y * m.y, ui = gi.x * m.y + gi.y * m.x;  // g_i M
                    cacc.add(v.x * ur + v.y * ui, v.x * ui - v.y * ur);                      // conj(gamma) g_i M
                }
            }
        }
        if (j < n_ant) pc[j] = cacc.value();
    }
    // row partials: a fixed-order tree over the threads, one row at a time
    // (unrolled over the rows, so the accumulators stay in registers)
    __shared__ double2 red[kGradThreads];
#pragma unroll
    for (int k = 0; k < kGradTile; ++k) {
        const int i = i0 + k;
        if (i < n_ant) {  // CTA-uniform
            red[tid] = racc[k].value();
            __syncthreads();
            for (int s2 = kGradThreads / 2; s2 > 0; s2 >>= 1) {
                if (tid < s2) {
                    red[tid].x += red[tid + s2].x;
                    red[tid].y += red[tid + s2].y;
                }
                __syncthreads();
            }
            if (tid == 0) prow[int64_t(g) * n_ant + i] = red[0];
            __syncthreads();
        }
    }
}

// Gain gradient, pass 2: one warp per antenna.  Lane l takes the partials
// l, l + 32, ... of the antenna (row partials of every group, then the column
// partials of every (group, tile)), and a fixed shuffle tree adds the 32
// lane sums: the order never changes, so neither does the result.
__global__ void k_gain_grad_sum(const double2 *__restrict__ pcol, const double2 *__restrict__ prow, int groups,
                                int tiles, int n_ant, float2 *__restrict__ dgains) {
    const int a = blockIdx.x * (blockDim.x / 32) + int(threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (a >= n_ant) return;
    double re = 0.0, im = 0.0;
    const int terms = groups * (tiles + 1);
    for (int k = lane; k < terms; k += 32) {
        const int g = k / (tiles + 1), t = k % (tiles + 1);
        const double2 v = t == tiles ? prow[int64_t(g) * n_ant + a] : pcol[(int64_t(g) * tiles + t) * n_ant + a];
        re += v.x;
        im += v.y;
    }
    for (int d = 16; d > 0; d >>= 1) {
        re += __shfl_down_sync(0xFFFFFFFFu, re, d);
        im += __shfl_down_sync(0xFFFFFFFFu, im, d);
    }
    if (lane == 0) dgains[a] = make_float2(float(re), float(im));
}

}  // namespace

Error launch_gain_products(const float2 *gains, int64_t stride, int rows, int n_ant, int64_t nb, float2 *out,
                           cudaStream_t st) {
    if (rows <= 0 || nb <= 0) return Error{0, ""};
    for (int r0 = 0; r0 < rows; r0 += 65535) {
        const int cnt = std::min(65535, rows - r0);
        k_gain_products<<<dim3(unsigned((nb + 255) / 256), unsigned(cnt)), 256, 0, st>>>(
            gains + int64_t(r0) * stride, stride, n_ant, nb, out + int64_t(r0) * nb);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

Error launch_apply_gains(const float2 *model, const float2 *gains, const int64_t *vis_off, int n_layers, int n_ant,
                         int64_t nb, float2 *vis, cudaStream_t st) {
    for (int l0 = 0; l0 < n_layers; l0 += 65535) {
        const int cnt = std::min(65535, n_layers - l0);
        k_apply_gains<<<dim3(unsigned((nb + 255) / 256), unsigned(cnt)), 256, 0, st>>>(model, gains, vis_off + l0,
                                                                                         n_ant, nb, vis);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

// Layer groups of the gain gradient: about four CTAs per SM over all tiles.
int gain_grad_groups(int n_layers, int n_ant) {
    const int tiles = (n_ant + kGradTile - 1) / kGradTile;
    const int want = std::max(1, (4 * 152 + tiles - 1) / tiles);
    return std::max(1, std::min(n_layers, want));
}

size_t gain_grad_scratch_bytes(int n_layers, int n_ant) {
    const int tiles = (n_ant + kGradTile - 1) / kGradTile, groups = gain_grad_groups(n_layers, n_ant);
    return size_t(groups) * (size_t(tiles) + 1) * size_t(n_ant) * sizeof(double2);
}

Error launch_gain_grad(const float2 *dvis, const float2 *model, const float2 *gains, const int64_t *vis_off,
                       int n_layers, int n_ant, float2 *dgains, void *scratch, cudaStream_t st) {
    if (n_ant > kGradMaxJ * kGradThreads) return Error{-2, "gain gradient: more than 1024 antennas"};
    const int tiles = (n_ant + kGradTile - 1) / kGradTile, groups = gain_grad_groups(n_layers, n_ant);
    const int per = (n_layers + groups - 1) / groups;
    double2 *pcol = static_cast<double2 *>(scratch);
    double2 *prow = pcol + size_t(groups) * tiles * n_ant;
    k_gain_grad_part<<<dim3(unsigned(tiles), unsigned(groups)), kGradThreads, 0, st>>>(
        dvis, model, gains, vis_off, n_layers, n_ant, per, pcol, prow);
    BLINK_CUDA_TRY(cudaGetLastError());
    k_gain_grad_sum<<<(n_ant + 7) / 8, 256, 0, st>>>(pcol, prow, groups, tiles, n_ant, dgains);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

}  // namespace blink
