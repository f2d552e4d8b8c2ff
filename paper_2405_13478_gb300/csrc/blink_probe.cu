// blink_probe.cu -- measured arithmetic peaks for roofline reports.
//
// The imaging kernels are bound by HBM bandwidth, by FP32 arithmetic (the
// transforms) or by the FP64 pipe (the cell assignment of the plan).  Their
// roofline fractions need the rate these pipes reach on the GPU at hand, so
// this file measures it: every thread runs eight independent fused
// multiply-add chains (enough to hide the pipe latency at full occupancy),
// and the rate is 2 flops per FMA over the CUDA-event time of one launch.
#include "blink.h"

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <class T>
__global__ void __launch_bounds__(512) k_fma_probe(T *sink, T a, T b, int iters) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // a, b keep every chain bounded, so this store never happens; the
    // compiler cannot know that and keeps the chains
    if (s == T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int run_probe(int iters, double *tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BLINK_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BLINK_ERR_CUDA;
    constexpr int threads = 512;
    const int blocks = sms * 4;  // 2048 threads per SM: full occupancy
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = BLINK_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return BLINK_ERR_CUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) status = BLINK_ERR_CUDA;
    const T a = T(0.999), b = T(1e-4);
    if (status == BLINK_OK) {
        k_fma_probe<T><<<blocks, threads, 0, st>>>(nullptr, a, b, iters / 8 + 1);  // warm-up
        cudaEventRecord(e0, st);
        k_fma_probe<T><<<blocks, threads, 0, st>>>(nullptr, a, b, iters);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || ms <= 0.f) {
            status = BLINK_ERR_CUDA;
        } else {
            const double fmas = double(blocks) * threads * double(iters) * kUnroll * kChains;
            *tflops = 2.0 * fmas / (double(ms) * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    return status;
}

}  // namespace

extern "C" BLINK_API int blink_probe_fma_peak(int device, int bits, double *tflops) {
    if (!tflops || (bits != 32 && bits != 64)) return BLINK_ERR_INVALID;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return BLINK_ERR_CUDA;
    if (device != prev && cudaSetDevice(device) != cudaSuccess) return BLINK_ERR_CUDA;
    // about 20-80 ms per launch on a GB300 in either precision
    const int st = bits == 32 ? run_probe<float>(4096, tflops) : run_probe<double>(64, tflops);
    if (device != prev) cudaSetDevice(prev);
    return st;
}
