// Homogeneous time stepping d_t f_i = sum_j kappa_ij Q_ij(f_i, f_j) with the second-order
// strong-stability-preserving Runge-Kutta scheme the paper uses in time (Sec. 5; the
// Krook-Wu evolution of Sec. 6.1 runs it with dt = 0.01):
//   f1 = f + dt R(f),   f <- f/2 + (f1 + dt R(f1)) / 2,
// R being the plan's species-summed collision operator.  The two combinations are the
// element-wise kernels below; the operator evaluations are the plan's collision kernel.
#include "dgfs_internal.h"

namespace dgfs {

namespace {

template <typename T>
__global__ void rk_stage1(const T* __restrict__ f, const T* __restrict__ r, T* __restrict__ f1, T dt, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    f1[i] = f[i] + dt * r[i];
}

template <typename T>
__global__ void rk_stage2(T* __restrict__ f, const T* __restrict__ f1, const T* __restrict__ r, T dt, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    f[i] = T(0.5) * f[i] + T(0.5) * (f1[i] + dt * r[i]);
}

unsigned blocks_for(size_t n) { return unsigned(n / 256 + 1 < 8192 ? n / 256 + 1 : 8192); }

}  // namespace

int launch_rk_stage(const Plan& p, int stage, void* f, void* f1, const void* r, double dt, size_t n, cudaStream_t st) {
  if (p.f32io()) {
    if (stage == 1)
      rk_stage1<float><<<blocks_for(n), 256, 0, st>>>(static_cast<const float*>(f), static_cast<const float*>(r),
                                                      static_cast<float*>(f1), float(dt), n);
    else
      rk_stage2<float><<<blocks_for(n), 256, 0, st>>>(static_cast<float*>(f), static_cast<const float*>(f1),
                                                      static_cast<const float*>(r), float(dt), n);
  } else {
    if (stage == 1)
      rk_stage1<double><<<blocks_for(n), 256, 0, st>>>(static_cast<const double*>(f), static_cast<const double*>(r),
                                                       static_cast<double*>(f1), dt, n);
    else
      rk_stage2<double><<<blocks_for(n), 256, 0, st>>>(static_cast<double*>(f), static_cast<const double*>(f1),
                                                       static_cast<const double*>(r), dt, n);
  }
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

}  // namespace dgfs
