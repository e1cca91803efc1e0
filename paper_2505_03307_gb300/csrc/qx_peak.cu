// Measured arithmetic rates of the GPU: the FP64 and FP32 fused multiply-add
// throughput that bounds the kernels whose bytes stay in cache (the merge
// wires' group sums).  Not part of the propagation; the bench reports the
// FP64-bound kernels against these numbers.
//
// Each thread runs kChains independent FMA chains (enough to cover the FMA
// pipeline's latency) for `iters` iterations; the chains' results are summed
// into one store so the compiler keeps every FMA.  Timed with CUDA events on
// a private stream after one untimed launch.
#include <cstdint>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int blocks_per_sm, int iters, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int blocks = sms * blocks_per_sm;
  T* out = nullptr;
  if (cudaMalloc(&out, size_t(blocks) * kThreads * sizeof(T)) != cudaSuccess) return 2;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = 3;
  } else {
    // a = 1 - 2^-20, b small: the values stay finite and normal
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1e-6);
    k_fma_chains<T><<<blocks, kThreads, 0, s>>>(out, iters, a, b);
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, kThreads, 0, s>>>(out, iters, a, b);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        ms <= 0.f) {
      rc = 4;
    } else {
      const double flops = 2.0 * kChains * double(iters) * double(blocks) * kThreads;
      *tflops = flops / (double(ms) * 1e-3) / 1e12;
      *ms_out = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  cudaGetLastError();
  return rc;
}

}  // namespace

// FP64 (bits = 64) or FP32 (bits = 32) FMA throughput of the current device
// in TFLOP/s (2 flops per FMA), from one timed launch of blocks_per_sm x SMs
// blocks of 256 threads, each thread running 8 independent chains of `iters`
// FMAs.  *ms receives the launch's duration.  Returns 0 on success.
extern "C" int qx_peak_fma(int bits, int blocks_per_sm, int iters, double* tflops, double* ms) {
  if (!tflops || !ms || iters <= 0 || blocks_per_sm <= 0) return 5;
  return bits == 64 ? measure<double>(blocks_per_sm, iters, tflops, ms)
                    : measure<float>(blocks_per_sm, iters, tflops, ms);
}
