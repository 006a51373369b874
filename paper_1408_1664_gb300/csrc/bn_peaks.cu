// bn_peaks.cu -- arithmetic-rate probes of the GPU, for the ALU rooflines of
// the benchmark (libbnpeaks.so, separate from the edge-posterior library).
//
// Each probe launches enough independent work to fill every SM (blocks of
// 256 threads, `blocks_per_sm` per SM), times it with CUDA events after one
// warm-up launch, and returns operations per second:
//   bn_peak_fp64_fma    FP64 fused multiply-adds, 2 flops each (8 independent
//                       chains per thread);
//   bn_peak_fp32_fma    FP32 fused multiply-adds, 2 flops each;
//   bn_peak_ex2_f32     MUFU base-2 exponentials (ex2.approx.ftz.f32), one
//                       operation each;
//   bn_peak_exp_f64     CUDA's double-precision exp(), one operation each
//                       (the cost of one FP64 log-domain term).
// The inputs keep every chain finite and data-dependent, and the results are
// written back, so nothing is folded away.  Returns 0 on success, -6 when a
// CUDA call fails.
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kThreads) k_ex2_chains(float* out, int iters)
{
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = -0.5f - 1e-4f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = -ex2_approx(x[k]);   // stays in [-1, -0.5]
    }
    float s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_exp64_chains(double* out, int iters)
{
    double x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = -0.5 - 1e-4 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = -exp(x[k]);           // stays in [-0.61, -0.54]
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Times `launch` (one warm-up call first); returns milliseconds or < 0.
template <typename L>
float timed(L launch)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    launch();
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess)
        cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

int grid_blocks(int blocks_per_sm)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return sms * (blocks_per_sm > 0 ? blocks_per_sm : 4);
}

template <typename T, typename K>
int run_probe(int blocks_per_sm, int iters, double ops_per_iter_thread, double* out, K kernel)
{
    const int grid = grid_blocks(blocks_per_sm);
    if (grid <= 0 || !out) return -6;
    T* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)grid * kThreads * sizeof(T)) != cudaSuccess) return -6;
    const float ms = timed([&] { kernel(buf, grid); });
    cudaFree(buf);
    if (!(ms > 0.f)) return -6;
    *out = (double)grid * kThreads * iters * ops_per_iter_thread / (ms * 1e-3);
    return 0;
}

}  // namespace

extern "C" int bn_peak_fp64_fma(int blocks_per_sm, double* flops_per_s)
{
    const int iters = 2048;
    return run_probe<double>(blocks_per_sm, iters, 16.0, flops_per_s, [&](double* b, int g) {
        k_fma_chains<double><<<g, kThreads>>>(b, iters, 0.999999, 1e-7);
    });
}

extern "C" int bn_peak_fp32_fma(int blocks_per_sm, double* flops_per_s)
{
    const int iters = 8192;
    return run_probe<float>(blocks_per_sm, iters, 16.0, flops_per_s, [&](float* b, int g) {
        k_fma_chains<float><<<g, kThreads>>>(b, iters, 0.999999f, 1e-7f);
    });
}

extern "C" int bn_peak_ex2_f32(int blocks_per_sm, double* ops_per_s)
{
    const int iters = 16384;
    return run_probe<float>(blocks_per_sm, iters, 8.0, ops_per_s, [&](float* b, int g) {
        k_ex2_chains<<<g, kThreads>>>(b, iters);
    });
}

extern "C" int bn_peak_exp_f64(int blocks_per_sm, double* ops_per_s)
{
    const int iters = 256;
    return run_probe<double>(blocks_per_sm, iters, 4.0, ops_per_s, [&](double* b, int g) {
        k_exp64_chains<<<g, kThreads>>>(b, iters);
    });
}
