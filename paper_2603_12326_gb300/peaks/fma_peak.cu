// Peak fused multiply-add throughput of the CUDA cores (FP64 DFMA, FP32 FFMA),
// measured with CUDA events.  This is a measurement utility for the roofline
// of the FP64 GPU path and of the FP32 pair-density kernel; it is not part of
// the screening path.
//
// Every thread runs NCHAIN independent multiply-add chains x <- x * b + c for
// `iters` steps (2 flops each); b and c come from arguments, so nothing folds,
// and each thread stores the sum of its chains.  The grid is blocks_per_sm CTAs
// of 256 threads per SM, enough independent work to cover the pipe latency.
#include <cuda_runtime.h>

namespace {

constexpr int NCHAIN = 8;
constexpr int THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(THREADS) k_fma(int iters, T b, T c, T* out) {
    T x[NCHAIN];
#pragma unroll
    for (int i = 0; i < NCHAIN; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int i = 0; i < NCHAIN; ++i) x[i] = fma(x[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < NCHAIN; ++i) s += x[i];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int device, int blocks_per_sm, int iters, int reps, double* out_tflops, double* out_ms) {
    if (blocks_per_sm < 1 || iters < 1 || reps < 1 || !out_tflops || !out_ms) return 1;
    if (cudaSetDevice(device) != cudaSuccess) return 2;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 2;
    const int grid = prop.multiProcessorCount * blocks_per_sm;
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * THREADS * sizeof(T)) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T b = (T)0.999999, c = (T)1e-7;
    k_fma<T><<<grid, THREADS>>>(iters / 8 + 1, b, c, out);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        k_fma<T><<<grid, THREADS>>>(iters, b, c, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return 3;
    const double flops = 2.0 * NCHAIN * 4.0 * (double)iters * grid * THREADS;
    *out_ms = best;
    *out_tflops = flops / (best * 1e-3) / 1e12;
    return 0;
}

}  // namespace

// Best of `reps` timed launches; returns 0 on success.  fp64 != 0: DFMA, else FFMA.
extern "C" int qcx_peak_fma(int device, int fp64, int blocks_per_sm, int iters, int reps, double* out_tflops,
                            double* out_ms) {
    return fp64 ? run<double>(device, blocks_per_sm, iters, reps, out_tflops, out_ms)
                : run<float>(device, blocks_per_sm, iters, reps, out_tflops, out_ms);
}
