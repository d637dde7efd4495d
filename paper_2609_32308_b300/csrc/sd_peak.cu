// sd_peak.cu -- measured integer add/min throughput of the current GPU.
//
// The fill's min-plus work is bound by integer ALU issue (no tensor cores:
// min-plus is not a dense contraction).  The roofline denominator is the rate
// at which this GPU retires independent "x = min(x + s, t)" steps: one add and
// one min, in 32-bit or in 64-bit integers, with enough independent chains
// per thread and enough threads per SM that neither latency nor occupancy
// limits the rate.  The kernel's result is stored so nothing is optimised
// away; every chain has its own operands so no step folds into another.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sd.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_addmin(const T *__restrict__ seed, int iters,
                                                     T *__restrict__ out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  T x[kChains], s[kChains], t[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) {
    x[k] = seed[(tid + k) & 1023];
    s[k] = seed[(tid * 3 + 7 * k + 1) & 1023];
    t[k] = seed[(tid * 5 + 11 * k + 2) & 1023];
  }
#pragma unroll 1
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 16; u++)
#pragma unroll
      for (int k = 0; k < kChains; k++) {
        const T y = x[k] + s[k];
        x[k] = y < t[k] ? y : t[k];
      }
  }
  T acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) acc ^= x[k];
  out[tid] = acc;
}

template <class T>
int measure(int iters, double *ops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return SD_ECUDA;
  const int blocks = sms * 8;  // 2048 resident threads per SM
  const int nthreads = blocks * kThreads;
  T *seed = nullptr, *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SD_OK;
  if (cudaMalloc(&seed, sizeof(T) * 1024) != cudaSuccess ||
      cudaMalloc(&out, sizeof(T) * nthreads) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = SD_ECUDA;
  } else {
    T h[1024];
    for (int k = 0; k < 1024; k++) h[k] = (T)((k * 2654435761u) % 1000003u) - (T)500000;
    float best = 0.f;
    if (cudaMemcpy(seed, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) rc = SD_ECUDA;
    for (int rep = 0; rep < 4 && rc == SD_OK; rep++) {  // first run warms up
      cudaEventRecord(e0);
      k_addmin<T><<<blocks, kThreads>>>(seed, iters, out);
      cudaEventRecord(e1);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = SD_ECUDA;
      else if (rep > 0 && (best == 0.f || ms < best))
        best = ms;
    }
    if (rc == SD_OK) {
      // one add and one min per step
      const double ops = 2.0 * (double)nthreads * kChains * 16.0 * (double)iters;
      *ops_per_s = best > 0.f ? ops / (best * 1e-3) : 0.0;
    }
  }
  if (seed) cudaFree(seed);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" int sd_peak_addmin(int bits, int iters, double *ops_per_s) {
  if (!ops_per_s || iters <= 0 || !(bits == 32 || bits == 64)) return SD_EINVAL;
  *ops_per_s = 0.0;
  return bits == 32 ? measure<int32_t>(iters, ops_per_s) : measure<int64_t>(iters, ops_per_s);
}
