// Measured multiply-add throughput of the FP32 and FP64 pipes: the denominators of the
// collision kernel's ALU roofline (the kernel is bound by the FMA pipe of its precision, not by
// HBM or the tensor cores).  No counterpart in the paper; a measurement helper.
//
// Every thread runs kChains independent chains x <- x a + b (a dependent chain per register,
// so the compiler can neither fold nor reorder them), kUnroll steps per loop trip.  The grid
// fills every SM with kBlocksPerSm blocks of kThreads threads, enough warps to cover the FMA
// latency on every scheduler.  A short launch sizes the loop so that the timed launch takes
// about 50 ms; the rate is 2 flop per FMA over the CUDA-event time of that launch.
#include <cuda_runtime.h>

#include "dgfs_internal.h"

namespace dgfs {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(T* out, int trips, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T sum = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) sum += x[c];
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = sum;
}

template <typename T>
int measure(double* flop_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DGFS_ERR_CUDA;
  const int blocks = sms * kBlocksPerSm;
  T* out = nullptr;
  if (cudaMalloc(&out, size_t(blocks) * kThreads * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DGFS_OK;
  float ms = 0.f;
  // a and b keep |x| bounded (x -> b / (1 - a)), so no chain overflows or goes subnormal
  const T a = T(0.999999), b = T(1e-6);
  int trips = 64;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = DGFS_ERR_CUDA;
  } else {
    for (int pass = 0; pass < 3 && rc == DGFS_OK; ++pass) {
      cudaEventRecord(e0);
      fma_rate_kernel<T><<<blocks, kThreads>>>(out, trips, a, b);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = DGFS_ERR_CUDA;
        break;
      }
      if (pass < 2) {
        // size the next launch to ~50 ms (at most 2^24 trips)
        double next = double(trips) * 50.0 / (ms > 1e-3f ? ms : 1e-3f);
        trips = int(next < 1.0 ? 1.0 : (next > 16777216.0 ? 16777216.0 : next));
      }
    }
  }
  if (rc == DGFS_OK) {
    const double fma = double(blocks) * kThreads * double(trips) * kUnroll * kChains;
    *flop_per_s = 2.0 * fma / (double(ms) * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess && rc == DGFS_OK) rc = DGFS_ERR_CUDA;
  return rc;
}

}  // namespace
}  // namespace dgfs

extern "C" int dgfs_measure_fma_rate(int precision, double* flop_per_s) {
  if (!flop_per_s) return DGFS_ERR_INVALID_ARG;
  if (precision == DGFS_FP32) return dgfs::measure<float>(flop_per_s);
  if (precision == DGFS_FP64) return dgfs::measure<double>(flop_per_s);
  return DGFS_ERR_INVALID_ARG;
}
