// probe.cu -- a measurement of the device, not a step of the method: the
// throughput of no-return shared-memory atomic adds, the unit the deposit's
// tile accumulation is bound by (its roofline peak).
#include <cstdint>

#include "../../include/mond_pm.h"
#include "internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeSlots = 8;  // words per thread: consecutive lanes hit consecutive words (no bank conflicts)

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_probe_atomics(int iters, T* sink) {
  __shared__ T s[kProbeThreads * kProbeSlots];
  for (int k = 0; k < kProbeSlots; k++) s[threadIdx.x + kProbeThreads * k] = 0;
  __syncthreads();
  const T v = (T)((threadIdx.x & 7) + 1);
#pragma unroll 8
  for (int i = 0; i < iters; i++) atomicAdd(&s[threadIdx.x + kProbeThreads * (i & (kProbeSlots - 1))], v);
  __syncthreads();
  T tot = 0;
  for (int k = 0; k < kProbeSlots; k++) tot += s[threadIdx.x + kProbeThreads * k];
  if (tot == (T)1) sink[blockIdx.x] = tot;  // never true for iters > 0; keeps the adds alive
}

template <typename T>
int run(cudaStream_t st, double* rate) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_probe_atomics<T>, kProbeThreads, 0) != cudaSuccess)
    return MOND_ECUDA;
  const int grid = sms * (per > 0 ? per : 1);
  const int iters = 8192;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return MOND_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return MOND_ECUDA;
  }
  float best = 0.f;
  for (int rep = 0; rep < 4; rep++) {  // the first run warms the clocks up; the best of the rest is kept
    cudaEventRecord(a, st);
    k_probe_atomics<T><<<grid, kProbeThreads, 0, st>>>(iters, nullptr);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cudaGetLastError() != cudaSuccess || best <= 0.f) return MOND_ECUDA;
  *rate = (double)grid * kProbeThreads * iters / (best * 1e-3);
  return MOND_OK;
}

}  // namespace

extern "C" int mond_pm_probe_smem_atomics(int bits, void* cuda_stream, double* adds_per_s) {
  if (!adds_per_s || (bits != 32 && bits != 64)) return MOND_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  return bits == 32 ? run<uint32_t>(st, adds_per_s) : run<unsigned long long>(st, adds_per_s);
}
