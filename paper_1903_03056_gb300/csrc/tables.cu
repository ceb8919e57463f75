// On-device construction of the FP64 VHS weight tables of a plan (the plan's own stream):
//   Fw[o][q][k] = w_q 4 pi b_o rho_q^(4 - 2 omega_o) / N^3 * sinc(pi rho_q c_j |k| / L)
//   Gm[o][k]    = sum_q 16 pi^2 b_o w_q rho_q^(4 - 2 omega_o) sinc(pi rho_q |k| / L)
// (the VHS gain weight F of Eq. GG with the radial weight and the 1/N^3 of the forward
// transform folded in, and the loss weight on the same radial rule).  The per-(pair, rho)
// prefactors and sinc scales come from the host; the N^3-sized loops run here.
#include "dgfs_internal.h"

namespace dgfs {

namespace {

__device__ __forceinline__ double sinc(double x) { return fabs(x) < 1e-300 ? 1.0 : sin(x) / x; }

__device__ __forceinline__ double kabs_at(size_t n, int N) {
  const int a = int(n / (size_t(N) * N)), b = int((n / N) % N), c = int(n % N);
  const double kx = a < N / 2 ? a : a - N, ky = b < N / 2 ? b : b - N, kz = c < N / 2 ? c : c - N;
  return sqrt(kx * kx + ky * ky + kz * kz);
}

__global__ void gain_table_kernel(double* __restrict__ Fw, size_t count, int N, const double* __restrict__ coef) {
  const size_t N3 = size_t(N) * N * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < count; idx += size_t(gridDim.x) * blockDim.x) {
    const size_t oq = idx / N3;
    Fw[idx] = coef[2 * oq] * sinc(coef[2 * oq + 1] * kabs_at(idx % N3, N));
  }
}

__global__ void loss_table_kernel(double* __restrict__ Gm, size_t count, int N, int NR, const double* __restrict__ gcoef,
                                  const double* __restrict__ gscale) {
  const size_t N3 = size_t(N) * N * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < count; idx += size_t(gridDim.x) * blockDim.x) {
    const size_t o = idx / N3;
    const double ka = kabs_at(idx % N3, N);
    double g = 0.0;
    for (int q = 0; q < NR; ++q) g += gcoef[o * NR + q] * sinc(gscale[q] * ka);
    Gm[idx] = g;
  }
}

}  // namespace

int launch_vhs_tables(Plan& p, const double* d_fcoef, const double* d_gcoef, const double* d_gscale) {
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t nF = size_t(p.s) * p.s * p.N_rho * N3, nG = size_t(p.s) * p.s * N3;
  auto blocks = [](size_t n) { return unsigned(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096); };
  gain_table_kernel<<<blocks(nF), 256, 0, p.home>>>(p.d_Fw, nF, p.N, d_fcoef);
  loss_table_kernel<<<blocks(nG), 256, 0, p.home>>>(p.d_Gm, nG, p.N, p.N_rho, d_gcoef, d_gscale);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

}  // namespace dgfs
