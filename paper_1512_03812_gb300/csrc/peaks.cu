// peaks.cu -- micro-benchmarks of the device rates the kernels are measured
// against: FP64 and FP32 FMA throughput, L2 read bandwidth and shared-memory
// read bandwidth (sm_peak_*).  The HBM copy bandwidth comes from elsewhere.
#include <cuda_runtime.h>

#include "internal.h"
#include "schwinger.h"

namespace sm {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread
constexpr int kUnroll = 16;  // FMAs per chain per loop trip

template <typename R>
__global__ void __launch_bounds__(256) k_fma(R a, R b, int trips, R* sink) {
  R x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (R)(threadIdx.x + k);
  for (int i = 0; i < trips; ++i)
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  R s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == (R)-1.2345) *sink = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(512) k_l2_read(const uint4* __restrict__ p, long long n,
                                                 int passes, unsigned* sink) {
  unsigned acc = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int r = 0; r < passes; ++r)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
      const uint4 v = __ldcg(p + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x9e3779b9u) *sink = acc;
}

constexpr int kSmemF4 = 2048;  // 32 KB per block
__global__ void __launch_bounds__(1024) k_smem_read(int trips, float* sink) {
  __shared__ float4 buf[kSmemF4];
  for (int i = threadIdx.x; i < kSmemF4; i += blockDim.x)
    buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int j = threadIdx.x;
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 v = buf[(j + u * 256) & (kSmemF4 - 1)];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    j += 32;
  }
  if (acc.x + acc.y + acc.z + acc.w == -1.f) *sink = acc.x;
}

int nsm() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

// Times `launch` (after one untimed run) with events on the default stream;
// returns milliseconds or a negative value on error.
template <typename F>
float time_ms(F launch) {
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

}  // namespace
}  // namespace sm

using namespace sm;

int sm_peak_fma(int prec, double* tflops) {
  if (!tflops || (prec != SM_F64 && prec != SM_F32)) return fail(SM_ERR_ARG, "sm_peak_fma: bad argument");
  void* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return fail(SM_ERR_CUDA, "sm_peak_fma: alloc");
  const int blocks = nsm() * 8, threads = 256;
  const int trips = prec == SM_F64 ? 256 : 8192;
  float ms;
  if (prec == SM_F64)
    ms = time_ms([&] {
      k_fma<double><<<blocks, threads>>>(0.999999, 1e-7, trips, (double*)sink);
    });
  else
    ms = time_ms([&] {
      k_fma<float><<<blocks, threads>>>(0.9999f, 1e-4f, trips, (float*)sink);
    });
  cudaFree(sink);
  if (ms <= 0.f) return fail(SM_ERR_CUDA, "sm_peak_fma: %s", cudaGetErrorString(cudaGetLastError()));
  const double flops = 2.0 * blocks * threads * (double)trips * kUnroll * kChains;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SM_OK;
}

int sm_peak_l2_read(long long bytes, int passes, double* gbs) {
  if (!gbs || bytes < 16 || passes < 1) return fail(SM_ERR_ARG, "sm_peak_l2_read: bad argument");
  const long long n = bytes / 16;
  void *buf = nullptr, *sink = nullptr;
  if (cudaMalloc(&buf, n * 16) != cudaSuccess) return fail(SM_ERR_CUDA, "sm_peak_l2_read: alloc");
  if (cudaMalloc(&sink, 16) != cudaSuccess || cudaMemset(buf, 1, n * 16) != cudaSuccess) {
    cudaFree(buf);
    return fail(SM_ERR_CUDA, "sm_peak_l2_read: alloc");
  }
  const int blocks = nsm() * 4;
  const float ms = time_ms([&] {
    k_l2_read<<<blocks, 512>>>((const uint4*)buf, n, passes, (unsigned*)sink);
  });
  cudaFree(buf);
  cudaFree(sink);
  if (ms <= 0.f) return fail(SM_ERR_CUDA, "sm_peak_l2_read: %s", cudaGetErrorString(cudaGetLastError()));
  *gbs = 16.0 * n * passes / (ms * 1e-3) / 1e9;
  return SM_OK;
}

int sm_peak_smem_read(double* gbs) {
  if (!gbs) return fail(SM_ERR_ARG, "sm_peak_smem_read: bad argument");
  void* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return fail(SM_ERR_CUDA, "sm_peak_smem_read: alloc");
  const int blocks = nsm() * 2, threads = 1024, trips = 4096;
  const float ms = time_ms([&] { k_smem_read<<<blocks, threads>>>(trips, (float*)sink); });
  cudaFree(sink);
  if (ms <= 0.f) return fail(SM_ERR_CUDA, "sm_peak_smem_read: %s", cudaGetErrorString(cudaGetLastError()));
  *gbs = 16.0 * blocks * threads * (double)trips * 8 / (ms * 1e-3) / 1e9;
  return SM_OK;
}
