// Throughput microbenchmark of the pipes the pair kernels run on: FP32 FFMA,
// FP64 DFMA and the MUFU approximations (rsqrt.approx, ex2.approx).  A
// standalone program (not part of libbipb), built and run by
// `bench.py --mode peaks`; it prints one "name value" line per pipe, in
// lane-operations per second, after one warm-up launch.
//
// Every thread runs 8 (FFMA), 4 (DFMA) or 4 (MUFU) independent dependency
// chains, and the grid holds 8 CTAs of 256 threads per SM, so the issue
// slots, not latencies, bound each kernel.
#include <cstdio>
#include <cuda_runtime.h>

namespace {

constexpr int kIters = 4096;

__global__ void k_ffma(float* out, float a, float b) {
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, double a, double b) {
  double x[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < kIters / 32; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = fma(x[c], a, b);
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

__global__ void k_mufu(float* out) {
  float x[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) x[c] = threadIdx.x + 1.0f + c;
  for (int i = 0; i < kIters / 4; ++i) {
    asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[0]));
    asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[1]));
    asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[2]));
    asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[3]));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

}  // namespace

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) {
    std::printf("error no device\n");
    return 1;
  }
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  const double n = (double)blocks * threads;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)n * sizeof(double)) != cudaSuccess) {
    std::printf("error cudaMalloc\n");
    return 1;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](auto launch) {
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms / 1e3;
  };
  const double t_ffma = timed([&] { k_ffma<<<blocks, threads>>>((float*)buf, 0.999f, 0.001f); });
  const double t_dfma = timed([&] { k_dfma<<<blocks, threads>>>((double*)buf, 0.999, 0.001); });
  const double t_mufu = timed([&] { k_mufu<<<blocks, threads>>>((float*)buf); });
  std::printf("sms %d\n", p.multiProcessorCount);
  std::printf("ffma_per_s %.6e\n", n * kIters * 8 / t_ffma);
  std::printf("dfma_per_s %.6e\n", n * (kIters / 32) * 4 / t_dfma);
  std::printf("mufu_per_s %.6e\n", n * kIters / t_mufu);
  const cudaError_t err = cudaGetLastError();
  std::printf("status %s\n", err == cudaSuccess ? "ok" : cudaGetErrorString(err));
  cudaFree(buf);
  return err == cudaSuccess ? 0 : 1;
}
