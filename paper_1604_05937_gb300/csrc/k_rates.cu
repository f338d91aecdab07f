// FP64 issue-rate measurement for the roofline of the FP64-bound kernels:
// GB300 runs DFMA and DADD/DMUL at different rates, so the ceiling of a
// kernel depends on its instruction mix.  Each probe kernel runs eight
// independent dependency chains per thread over a grid of 4 CTAs per SM.
#include "ext_internal.cuh"

namespace {

template <int KIND>
__global__ void __launch_bounds__(256) k_rate(double *out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (KIND == 0) x[i] = fma(x[i], a, b);
      else if (KIND == 1) x[i] = x[i] + b;
      else x[i] = x[i] * a;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 atomic adds executed by L2: every warp adds to 32 consecutive doubles of
// a 64 MiB buffer (resident in L2), a new region each iteration.
__global__ void __launch_bounds__(256) k_red_rate(double *buf, uint32_t mask, int iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (int it = 0; it < iters; ++it) atomicAdd(buf + ((tid + (uint32_t)it * stride) & mask), 1.0);
}

}  // namespace

extern "C" ext_status ext_fp64_rates(double *gops_host, void *stream) {
  if (!gops_host) return ext_fail(EXT_EINVAL, "ext_fp64_rates: output is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = 4 * sms, threads = 256, iters = 4096;
  double *out = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      if (kind == 0) k_rate<0><<<blocks, threads, 0, s>>>(out, iters, 1.0000001, 1e-9);
      else if (kind == 1) k_rate<1><<<blocks, threads, 0, s>>>(out, iters, 1.0000001, 1e-9);
      else k_rate<2><<<blocks, threads, 0, s>>>(out, iters, 1.0000001, 1e-9);
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;  // the first launch warms up
    }
    gops_host[kind] = (double)blocks * threads * iters * 8 / best / 1e6;
  }
  double *buf = nullptr;
  const uint32_t n = 1u << 23;  // 64 MiB of doubles
  if (e == cudaSuccess) e = cudaMalloc(&buf, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) {
    const int riters = 256;
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      k_red_rate<<<blocks, threads, 0, s>>>(buf, n - 1, riters);
      cudaEventRecord(e1, s);
      e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    gops_host[3] = (double)blocks * threads * riters / best / 1e6;
  }
  cudaFree(buf);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_fp64_rates: %s", cudaGetErrorString(e));
  return EXT_OK;
}
