// Measurement utilities of the GB300 sparse-FCT library (no counterpart in
// the paper): the on-chip roofs that bound the solver when its working set
// stays in L2, measured on the device they run on.
//   - L2 read bandwidth: every block streams a buffer that fits in L2 with
//     16-byte loads that bypass L1 (ld.global.cg), many passes after a warm
//     pass; bytes read / time.
//   - L2 random-gather rate: 8-byte loads at pseudo-random positions of a
//     buffer that fits in L2 (the access pattern of the alias gathers); each
//     load moves one 32-byte sector, reported as loads/s and sector bytes/s.
//   - FP64 FMA rate: independent fma chains in registers, 2 flops per fma.
// None of them changes a GPU setting; each allocates and frees its own buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "fct_internal.h"

using namespace fct;

namespace {

fct_status peaks_cuda_fail(cudaError_t e, const char* what) {
  (void)cudaGetLastError();
  return fail(FCT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

__global__ void l2_stream_kernel(const float4* __restrict__ buf, int64_t n16, int passes, float* sink) {
  float acc = 0.0f;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = i + u * stride < n16 ? __ldcg(buf + i + u * stride) : make_float4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += (v[u].x + v[u].y) + (v[u].z + v[u].w);
    }
  }
  if (acc == 1.2345f) sink[blockIdx.x] = acc;  // keeps the loads; never true for a zero buffer
}

__global__ void l2_gather_kernel(const double* __restrict__ buf, int64_t n8, int loads, double* sink) {
  unsigned int s = 0x9E3779B9u * (blockIdx.x * blockDim.x + threadIdx.x + 1u);
  double acc = 0.0;
  for (int k = 0; k < loads; k += 8) {
    int64_t idx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s = s * 1664525u + 1013904223u;
      idx[u] = static_cast<int64_t>(s % static_cast<unsigned int>(n8));
    }
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(buf + idx[u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  if (acc == 1.2345) sink[blockIdx.x] = acc;
}

__global__ void fp64_fma_kernel(int iters, double seed, double* sink) {
  double a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = seed + 1e-3 * (threadIdx.x + u);
  const double m = 1.0 - 1e-9, c = 1e-9;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(a[u], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += a[u];
  if (s == 1.2345) sink[blockIdx.x] = s;
}

// Times one launch of `launch` between two events on the legacy stream.
template <typename L>
fct_status time_launch(L launch, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return peaks_cuda_fail(e, "peak measurement");
  return FCT_OK;
}

}  // namespace

extern "C" fct_status fct_measure_l2(int64_t bytes, int passes, double* read_gbs, double* gather_gloads,
                                     double* gather_sector_gbs) {
  if (!read_gbs || bytes < (int64_t{1} << 20) || bytes > (int64_t{96} << 20) || passes < 1 || passes > 100000)
    return fail(FCT_ERR_INVALID_ARG, "need bytes in [1 MiB, 96 MiB], passes in [1, 1e5], read_gbs != NULL");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return peaks_cuda_fail(e, "device query");
  bytes &= ~int64_t{15};
  void* buf = nullptr;
  float* sink = nullptr;
  e = cudaMalloc(&buf, static_cast<size_t>(bytes));
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double) * 4096);
  if (e == cudaSuccess) e = cudaMemset(buf, 0, static_cast<size_t>(bytes));
  if (e != cudaSuccess) {
    cudaFree(buf);
    cudaFree(sink);
    return peaks_cuda_fail(e, "L2 probe buffers");
  }
  const int blocks = 4 * nsm, threads = 512;
  const int64_t n16 = bytes / 16, n8 = bytes / 8;
  fct_status s = FCT_OK;
  float ms = 0.0f;
  // warm pass: the buffer becomes L2-resident
  s = time_launch([&] { l2_stream_kernel<<<blocks, threads>>>(static_cast<const float4*>(buf), n16, 1, sink); }, &ms);
  if (s == FCT_OK)
    s = time_launch([&] { l2_stream_kernel<<<blocks, threads>>>(static_cast<const float4*>(buf), n16, passes, sink); },
                    &ms);
  if (s == FCT_OK) *read_gbs = static_cast<double>(bytes) * passes / (1e-3 * ms) / 1e9;
  const int loads = 4096;
  if (s == FCT_OK && (gather_gloads || gather_sector_gbs)) {
    s = time_launch(
        [&] {
          l2_gather_kernel<<<blocks, threads>>>(static_cast<const double*>(buf), n8, loads,
                                                reinterpret_cast<double*>(sink));
        },
        &ms);
    const double nload = static_cast<double>(blocks) * threads * loads;
    if (s == FCT_OK && gather_gloads) *gather_gloads = nload / (1e-3 * ms) / 1e9;
    if (s == FCT_OK && gather_sector_gbs) *gather_sector_gbs = 32.0 * nload / (1e-3 * ms) / 1e9;
  }
  cudaFree(buf);
  cudaFree(sink);
  return s;
}

extern "C" fct_status fct_measure_fp64(int iters, double* tflops) {
  if (!tflops || iters < 1 || iters > (1 << 24)) return fail(FCT_ERR_INVALID_ARG, "need iters in [1, 2^24]");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return peaks_cuda_fail(e, "device query");
  double* sink = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * 8192);
  if (e != cudaSuccess) return peaks_cuda_fail(e, "FP64 probe buffer");
  const int blocks = 8 * nsm, threads = 256;
  float ms = 0.0f;
  fct_status s = time_launch([&] { fp64_fma_kernel<<<blocks, threads>>>(16, 0.5, sink); }, &ms);
  if (s == FCT_OK) s = time_launch([&] { fp64_fma_kernel<<<blocks, threads>>>(iters, 0.5, sink); }, &ms);
  if (s == FCT_OK) *tflops = 2.0 * 8.0 * static_cast<double>(iters) * blocks * threads / (1e-3 * ms) / 1e12;
  cudaFree(sink);
  return s;
}
