// probe.cu -- measurement aids: the rates of FP32 shared-memory atomic adds and of
// 32-bit integer shared-memory adds to random bins, the ceilings that the privatised
// scatter-adds (method 2's row scatter; method 1's fixed-point scatter) run against.
// Not part of the method.
#include "kernels.cuh"

namespace tnsk {

namespace {
constexpr int kBins = 1024, kReps = 8, kIters = 64;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {  // a 32-bit integer finaliser
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
}  // namespace

__global__ void __launch_bounds__(512, 4) probe_shared_atomics_kernel(float* sink) {
    __shared__ float bins[kBins * kReps];
    for (int i = threadIdx.x; i < kBins * kReps; i += blockDim.x) bins[i] = 0.f;
    __syncthreads();
    uint32_t s = mix32(blockIdx.x * blockDim.x + threadIdx.x + 1);
    for (int it = 0; it < kIters; ++it)
#pragma unroll 4
        for (int r = 0; r < kReps; ++r) {
            s = mix32(s + r);
            atomicAdd(&bins[r * kBins + (s & (kBins - 1))], (s & 0x80000000u) ? -1.f : 1.f);
        }
    __syncthreads();
    float a = 0.f;
    for (int i = threadIdx.x; i < kBins * kReps; i += blockDim.x) a += bins[i];
    if (a == 1234567.f) sink[0] = a;  // keeps the adds live
}

// The same with 32-bit integer adds whose result is unused (the fixed-point scatter's
// update), values of either sign.
__global__ void __launch_bounds__(512, 4) probe_shared_int_adds_kernel(float* sink) {
    __shared__ int bins[kBins * kReps];
    for (int i = threadIdx.x; i < kBins * kReps; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    uint32_t s = mix32(blockIdx.x * blockDim.x + threadIdx.x + 1);
    for (int it = 0; it < kIters; ++it)
#pragma unroll 4
        for (int r = 0; r < kReps; ++r) {
            s = mix32(s + r);
            atomicAdd(&bins[r * kBins + (s & (kBins - 1))], (int)(s >> 20) - 2048);
        }
    __syncthreads();
    int a = 0;
    for (int i = threadIdx.x; i < kBins * kReps; i += blockDim.x) a += bins[i];
    if (a == 1234567) sink[0] = (float)a;  // keeps the adds live
}

cudaError_t run_probe_shared_int_adds(float* sink, cudaStream_t s, double* updates_per_s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 4 * sms;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    probe_shared_int_adds_kernel<<<blocks, 512, 0, s>>>(sink);  // warm-up
    float best = 0.f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(a, s);
        for (int k = 0; k < 8; ++k) probe_shared_int_adds_kernel<<<blocks, 512, 0, s>>>(sink);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (best == 0.f || ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double n = 8.0 * blocks * 512.0 * kIters * kReps;
    *updates_per_s = best > 0.f ? n / (best * 1e-3) : 0.0;
    return cudaGetLastError();
}

cudaError_t run_probe_shared_atomics(float* sink, cudaStream_t s, double* updates_per_s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 4 * sms;  // 2048 threads per SM: full occupancy
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    probe_shared_atomics_kernel<<<blocks, 512, 0, s>>>(sink);  // warm-up
    float best = 0.f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(a, s);
        for (int k = 0; k < 8; ++k) probe_shared_atomics_kernel<<<blocks, 512, 0, s>>>(sink);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (best == 0.f || ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double n = 8.0 * blocks * 512.0 * kIters * kReps;
    *updates_per_s = best > 0.f ? n / (best * 1e-3) : 0.0;
    return cudaGetLastError();
}

}  // namespace tnsk
