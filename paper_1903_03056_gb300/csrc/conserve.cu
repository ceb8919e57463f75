// Conservation projection and species sum, applied after the collision kernel.
//
// conserve_kernel: one CTA per (node, block).  A block is a self pair Q_ii (5 constraint
// rows: 1, v_x, v_y, v_z, |v|^2) or a stacked cross pair [Q_ij; Q_ji] (6 rows: the two
// masses, m_i w_ij v + m_j w_ji v, m_i w_ij |v|^2 + m_j w_ji |v|^2), the discrete laws of
// Eq. consv.  The CTA sums C Q in FP64 over the grid, solves lambda = (C C^T)^-1 C Q with the
// plan's FP64 inverse and replaces Q by Q - C^T lambda, the nearest vector (in L2) that
// satisfies the laws exactly.
//
// species_sum_kernel: Q_i = sum_j kappa_ij Q_ij (Eq. NMBE right-hand side, kappa = 1/Kn).
#include "dgfs_internal.h"

namespace dgfs {

namespace {

constexpr int kConsThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kConsThreads) conserve_kernel(T* Q, int s, int N, double L,
                                                                const ConsBlock* blocks, int n_blocks) {
  const int b = blockIdx.x / n_blocks;
  const ConsBlock cb = blocks[blockIdx.x % n_blocks];
  const size_t N3 = size_t(N) * N * N;
  T* x1 = Q + ((size_t(b) * s + cb.i) * s + cb.j) * N3;
  T* x2 = Q + ((size_t(b) * s + cb.j) * s + cb.i) * N3;  // == x1 for a self pair
  const bool cross = cb.rows == 6;
  const double dv = 2.0 * L / N;

  // moments of the grid rows against Q (FP64)
  double acc[10] = {};  // per half: 1, vx, vy, vz, |v|^2
  for (size_t n = threadIdx.x; n < N3; n += kConsThreads) {
    const int ix = int(n / (size_t(N) * N)), iy = int((n / N) % N), iz = int(n % N);
    const double vx = -L + (ix + 0.5) * dv, vy = -L + (iy + 0.5) * dv, vz = -L + (iz + 0.5) * dv;
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double a = double(x1[n]);
    acc[0] += a;
    acc[1] += a * vx;
    acc[2] += a * vy;
    acc[3] += a * vz;
    acc[4] += a * v2;
    if (cross) {
      const double c = double(x2[n]);
      acc[5] += c;
      acc[6] += c * vx;
      acc[7] += c * vy;
      acc[8] += c * vz;
      acc[9] += c * v2;
    }
  }
  __shared__ double red[kConsThreads / 32][10];
  __shared__ double lam[6];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S[10];
    for (int k = 0; k < 10; ++k) {
      S[k] = 0.0;
      for (int w = 0; w < kConsThreads / 32; ++w) S[k] += red[w][k];
    }
    double cq[6];
    if (cross) {
      cq[0] = S[0];
      cq[1] = S[5];
      for (int d = 0; d < 3; ++d) cq[2 + d] = cb.a * S[1 + d] + cb.b * S[6 + d];
      cq[5] = cb.a * S[4] + cb.b * S[9];
    } else {
      for (int k = 0; k < 5; ++k) cq[k] = S[k];
    }
    for (int r = 0; r < cb.rows; ++r) {
      double v = 0.0;
      for (int c = 0; c < cb.rows; ++c) v += cb.minv[r * cb.rows + c] * cq[c];
      lam[r] = v;
    }
  }
  __syncthreads();
  // Q <- Q - C^T lambda
  for (size_t n = threadIdx.x; n < N3; n += kConsThreads) {
    const int ix = int(n / (size_t(N) * N)), iy = int((n / N) % N), iz = int(n % N);
    const double vx = -L + (ix + 0.5) * dv, vy = -L + (iy + 0.5) * dv, vz = -L + (iz + 0.5) * dv;
    const double v2 = vx * vx + vy * vy + vz * vz;
    if (cross) {
      const double mom = lam[2] * vx + lam[3] * vy + lam[4] * vz + lam[5] * v2;
      x1[n] = T(double(x1[n]) - lam[0] - cb.a * mom);
      x2[n] = T(double(x2[n]) - lam[1] - cb.b * mom);
    } else {
      x1[n] = T(double(x1[n]) - (lam[0] + lam[1] * vx + lam[2] * vy + lam[3] * vz + lam[4] * v2));
    }
  }
}

template <typename T>
__global__ void species_sum_kernel(const T* __restrict__ Qfull, T* __restrict__ Qsum, int batch, int s, size_t N3,
                                   const double* __restrict__ kappa) {
  for (int bi = blockIdx.y; bi < batch * s; bi += gridDim.y) {
    const int b = bi / s, i = bi % s;
    for (size_t n = blockIdx.x * size_t(blockDim.x) + threadIdx.x; n < N3; n += size_t(gridDim.x) * blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < s; ++j) acc += kappa[i * s + j] * double(Qfull[((size_t(b) * s + i) * s + j) * N3 + n]);
      Qsum[(size_t(b) * s + i) * N3 + n] = T(acc);
    }
  }
}

}  // namespace

int launch_conserve(const Plan& p, void* Q, int batch, cudaStream_t st) {
  const int nb = int(p.cons.size());
  if (nb == 0 || batch == 0) return DGFS_OK;
  const dim3 grid(unsigned(batch) * nb);
  if (p.f32io())
    conserve_kernel<float><<<grid, kConsThreads, 0, st>>>(static_cast<float*>(Q), p.s, p.N, p.L, p.d_cons, nb);
  else
    conserve_kernel<double><<<grid, kConsThreads, 0, st>>>(static_cast<double*>(Q), p.s, p.N, p.L, p.d_cons, nb);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int launch_species_sum(const Plan& p, const void* Qfull, void* Qsum, int batch, cudaStream_t st) {
  if (batch == 0) return DGFS_OK;
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const unsigned gx = unsigned((N3 + 255) / 256 < 64 ? (N3 + 255) / 256 : 64);
  const unsigned gy = unsigned(batch) * p.s < 65535u ? unsigned(batch) * p.s : 65535u;
  const dim3 grid(gx, gy);
  if (p.f32io())
    species_sum_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(Qfull), static_cast<float*>(Qsum),
                                                    batch, p.s, N3, p.d_kappa);
  else
    species_sum_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(Qfull), static_cast<double*>(Qsum),
                                                     batch, p.s, N3, p.d_kappa);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

}  // namespace dgfs
