// Arithmetic-pipe peak microbenchmark (tlqr_pipe_peak): independent FMA
// chains on every resident warp of the device, timed with CUDA events, give
// the FP32 and FP64 FMA throughput that the roofline of the ALU-bound kernels
// is measured against.  Not part of the solver's path.
#include <cuda_runtime.h>

#include "../../include/tlqr.h"

namespace {

constexpr int kChains = 8;     // independent accumulators per thread (hides the FMA latency)

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T b, T c) {
  T acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  if (s == (T)12345.678) out[blockIdx.x] = s;    // keeps the chains alive, practically never stores
}

template <typename T>
int run(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0, blocks_per_sm = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) return TLQR_ERR_CUDA;
  const int threads = 256;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_fma_chains<T>, threads, 0))
    return TLQR_ERR_CUDA;
  const int blocks = sms * blocks_per_sm;
  T* out = nullptr;
  if (cudaMallocAsync((void**)&out, blocks * sizeof(T), st)) { cudaGetLastError(); return TLQR_ERR_OOM; }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // about 10 ms (FP32) per timed launch on a B300; FP64 runs fewer iterations
  const int iters = sizeof(T) == 4 ? 1 << 16 : 1 << 12;
  k_fma_chains<T><<<blocks, threads, 0, st>>>(out, iters / 16, (T)0.999, (T)0.001);   // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(a, st);
    k_fma_chains<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms > 0 && ms < best) best = ms;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  if (e) return TLQR_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * threads * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return TLQR_OK;
}

}  // namespace

extern "C" int tlqr_pipe_peak(int32_t precision, double* tflops, void* stream) {
  if (!tflops) return TLQR_ERR_ARG;
  if (precision == TLQR_PREC_MIXED) return run<float>(tflops, (cudaStream_t)stream);
  if (precision == TLQR_PREC_FP64) return run<double>(tflops, (cudaStream_t)stream);
  return TLQR_ERR_ARG;
}
