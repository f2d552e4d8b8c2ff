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

#include <algorithm>

namespace blink {

namespace {

__device__ __forceinline__ int64_t pair_index(int i, int j, int n_ant) {  // i < j
    return int64_t(i) * n_ant - int64_t(i) * (i + 1) / 2 + (j - i - 1);
}

__device__ __forceinline__ void pair_of_b(int64_t b, int n_ant, int &i, int &j) {
    const double twon1 = 2.0 * n_ant - 1.0;
    int r = int((twon1 - sqrt(fmax(twon1 * twon1 - 8.0 * double(b), 0.0))) * 0.5);
    r = max(0, min(r, n_ant - 2));
    auto start = [n_ant](int64_t row) { return row * (2 * int64_t(n_ant) - row - 1) / 2; };
    while (r > 0 && start(r) > b) --r;
    while (r < n_ant - 2 && start(r + 1) <= b) ++r;
    i = r;
    j = int(b - start(r)) + r + 1;
}

// Grid: (ceil(B / 256), layers).
__global__ void k_apply_gains(const float2 *__restrict__ model, const float2 *__restrict__ gains,
                              const int64_t *__restrict__ vis_off, int n_ant, int64_t nb,
                              float2 *__restrict__ vis) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int i, j;
    pair_of_b(b, n_ant, i, j);
    const int64_t o = vis_off[blockIdx.y] + b;
    const float2 m = model[o], gi = gains[i], gj = gains[j];
    // g_i conj(g_j)
    const float2 p = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
    vis[o] = make_float2(p.x * m.x - p.y * m.y, p.x * m.y + p.y * m.x);
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
            const int64_t b = o + pair_index(i, j, n_ant);
            const float2 gv = dvis[b], m = model[b];
            const double tr = double(gj.x) * m.x + double(gj.y) * m.y;  // g_j conj(M)
            const double ti = double(gj.y) * m.x - double(gj.x) * m.y;
            re += gv.x * tr - gv.y * ti;
            im += gv.x * ti + gv.y * tr;
        } else {
            const int64_t b = o + pair_index(j, i, n_ant);
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
