// Measured FMA throughput of the FP64 and FP32 pipes: the compute ceilings
// of the step kernels' roofline (the FP64 form is bound by its FP64 pipe).
//
// Every thread runs kChains independent FMA chains (enough to cover the pipe
// latency), Iters FMAs each, on a grid of 8 blocks of 256 threads per SM; the
// chains are folded into one store so that none is dead code. Timed with CUDA
// events on a private stream after one warm-up launch, best of a few.
#include <cuda_runtime.h>

#include "rlbm.h"

namespace {

constexpr int kChains = 8;
// FMAs per chain: about a quarter of a second per launch on a GPU whose FP64
// rate is 1/64 of its FP32 rate
constexpr int kItersF64 = 64, kItersF32 = 4096;
constexpr int kThreadsPeak = 256;
constexpr int kBlocksPerSm = 8;

template <class T, int Iters>
__global__ void __launch_bounds__(kThreadsPeak) k_fma_chain(T a, T b, T* out) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 16
  for (int i = 0; i < Iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

template <class T, int Iters>
int time_chain(int sms, cudaStream_t st, T* sink, double* flops) {
  const int grid = sms * kBlocksPerSm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RLBM_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RLBM_E_CUDA;
  }
  // a = 1 - 2^-20, b = 2^-20: the chains stay near 1, no overflow or denormals
  const T a = (T)(1.0 - 9.5367431640625e-07), b = (T)9.5367431640625e-07;
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // the first launch is the warm-up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_fma_chain<T, Iters><<<grid, kThreadsPeak, 0, st>>>(a, b, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  const double fma_count = (double)grid * kThreadsPeak * kChains * (double)Iters;
  *flops = 2.0 * fma_count / (best * 1e-3);
  return RLBM_OK;
}

}  // namespace

extern "C" int rlbm_pipe_peaks(double* fp64_flops, double* fp32_flops, int* sm_count) {
  if (!fp64_flops || !fp32_flops) return RLBM_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RLBM_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RLBM_E_CUDA;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return RLBM_E_CUDA;
  // the sink is never written (see k_fma_chain); a null pointer would do, but
  // the kernels get a valid address anyway
  double* sink = nullptr;
  int r = cudaMallocAsync(&sink, (size_t)sms * kBlocksPerSm * sizeof(double), st) == cudaSuccess ? RLBM_OK
                                                                                                  : RLBM_E_CUDA;
  if (r == RLBM_OK) r = time_chain<double, kItersF64>(sms, st, sink, fp64_flops);
  if (r == RLBM_OK) r = time_chain<float, kItersF32>(sms, st, reinterpret_cast<float*>(sink), fp32_flops);
  if (sink) cudaFreeAsync(sink, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (r == RLBM_OK && sm_count) *sm_count = sms;
  return r;
}
