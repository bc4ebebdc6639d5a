// Arithmetic pipe rates of this GPU, measured with independent fused
// multiply-add chains (no memory traffic): the denominators of the rooflines of
// ALU-bound kernels (FP64 operator, FP32 sweeps).  No counterpart in the paper.
#include "nnmg_internal.h"

namespace {

constexpr int kChains = 8;      // independent chains per thread (covers the pipe latency)
constexpr int kUnroll = 4;

template <typename T>
__global__ void fma_chain_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = x[j] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == T(-1.2345)) out[threadIdx.x] = s;   // never true; keeps the chains alive
}

// Packed FP32 pairs: one instruction, two multiply-adds.
__global__ void fma2_chain_kernel(float* out, int iters, float a, float b) {
  float2 x[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = make_float2((threadIdx.x + j) * 1e-3f, (threadIdx.x - j) * 1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
  if (s == -1.2345f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" int nnmg_pipe_rate(int kind, int iters, void* stream, double* fma_per_s) {
  using namespace nnmg;
  if ((kind < 0 || kind > 2) || iters < 1 || !fma_per_s) {
    set_error("nnmg_pipe_rate: kind must be 0 (FP64), 1 (FP32) or 2 (packed FP32), iters >= 1");
    return NNMG_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  NNMG_CUDA(cudaGetDevice(&dev));
  NNMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;     // 2048 threads per SM
  void* out = nullptr;
  NNMG_CUDA(cudaMalloc(&out, threads * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first launch warms up
    e = cudaEventRecord(e0, s);
    if (kind == 0)
      fma_chain_kernel<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.9999999, 1e-7);
    else if (kind == 1)
      fma_chain_kernel<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.9999f, 1e-4f);
    else
      fma2_chain_kernel<<<blocks, threads, 0, s>>>((float*)out, iters, 0.9999f, 1e-4f);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  NNMG_CUDA(e);
  const double per_thread = (double)iters * kUnroll * kChains * (kind == 2 ? 2 : 1);
  *fma_per_s = per_thread * threads * blocks / (ms * 1e-3);
  return NNMG_OK;
}
