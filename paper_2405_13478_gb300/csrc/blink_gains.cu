// blink_gains.cu -- per-antenna complex gains: forward application and the
// chain rule of the image-loss gradient.
//
// Visibilities corrupted by antenna gains, V_ij = g_i conj(g_j) M_ij (the
// antenna-level calibration factors of Sec. 4.2 applied to model
// visibilities M).  With gamma = dL/dRe V + i dL/dIm V from blink_degrid,
//   gamma(g_i) = sum_{j>i} gamma(V_ij) g_j conj(M_ij)
//              + sum_{k<i} conj(gamma(V_ki)) g_k M_ki,
// summed over all layers.
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

// One CTA per antenna; FP64 accumulation, fixed-order block reduction.
__global__ void __launch_bounds__(256) k_gain_grad(const float2 *__restrict__ dvis, const float2 *__restrict__ model,
                                                   const float2 *__restrict__ gains,
                                                   const int64_t *__restrict__ vis_off, int n_layers, int n_ant,
                                                   float2 *__restrict__ dgains) {
    const int i = blockIdx.x;
    double re = 0.0, im = 0.0;
    const int64_t terms = int64_t(n_layers) * n_ant;
    for (int64_t t = threadIdx.x; t < terms; t += blockDim.x) {
        const int l = int(t / n_ant), j = int(t % n_ant);
        if (j == i) continue;
        const int64_t o = vis_off[l];
        const float2 gj = gains[j];
        if (j > i) {
            const int64_t b = o + baseline_index(i, j, n_ant);
            const float2 gv = dvis[b], m = model[b];
            const double tr = double(gj.x) * m.x + double(gj.y) * m.y;  // g_j conj(M)
            const double ti = double(gj.y) * m.x - double(gj.x) * m.y;
            re += gv.x * tr - gv.y * ti;
            im += gv.x * ti + gv.y * tr;
        } else {
            const int64_t b = o + baseline_index(j, i, n_ant);
            const float2 gv = dvis[b], m = model[b];
            const double ur = double(gj.x) * m.x - double(gj.y) * m.y;  // g_j M
            const double ui = double(gj.x) * m.y + double(gj.y) * m.x;
            re += gv.x * ur + gv.y * ui;  // conj(gamma) (g_j M)
            im += gv.x * ui - gv.y * ur;
        }
    }
    __shared__ double sr[256], si[256];
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) dgains[i] = make_float2(float(sr[0]), float(si[0]));
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

Error launch_gain_grad(const float2 *dvis, const float2 *model, const float2 *gains, const int64_t *vis_off,
                       int n_layers, int n_ant, float2 *dgains, cudaStream_t st) {
    k_gain_grad<<<n_ant, 256, 0, st>>>(dvis, model, gains, vis_off, n_layers, n_ant, dgains);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

}  // namespace blink
