// On-device construction of the FP64 weight tables of a plan (the plan's own stream):
//   VHS  Fw[o][q][k]    = w_q 4 pi b_o rho_q^(4 - 2 omega_o) / N^3 * sinc(pi rho_q c_j |k| / L)
//   VSS  Fv[o][q][r][k] = w_q 2 pi b_o rho_q^(4 - 2 omega_o) / N^3
//                         * sum_t w_t exp(-i a t cos th) J0(a sqrt(1 - t^2) sin th),
//        a = pi rho_q c_j |k| / L, cos th = k_hat . sigma_m, m = reps[r], (t, w_t) the
//        Gauss-Jacobi rule of the weight (1 + t)^(alpha_o - 1)  (the sphere integral of
//        Eq. GG with the azimuth integrated to J0); one slot r per antipodal pair of
//        directions, since F(k, -sigma) = conj F(k, sigma)
//   loss Gm[o][k]       = sum_q (8 pi^2 2^alpha / alpha) b_o w_q rho_q^(4 - 2 omega_o) sinc(pi rho_q |k| / L)
// (the radial weight and the 1/N^3 of the forward transform folded into F).  The per-(pair,
// rho) prefactors and scales and the quadrature nodes come from the host; the N^3-sized
// loops run here.
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
    for (int q = 0; q < NR; ++q) g += gcoef[o * NR + q] * sinc(gscale[o * NR + q] * ka);
    Gm[idx] = g;
  }
}

__global__ void vss_table_kernel(double2* __restrict__ Fv, int P, int NR, int N, const double* __restrict__ coef,
                                 const double* __restrict__ gj, int n_t, const double* __restrict__ sigma,
                                 const int* __restrict__ reps, int n_reps) {
  const size_t N3 = size_t(N) * N * N;
  const size_t count = size_t(P) * NR * n_reps * N3;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < count; idx += size_t(gridDim.x) * blockDim.x) {
    const size_t n = idx % N3;
    const int r = int((idx / N3) % n_reps);
    const size_t oq = idx / (N3 * n_reps);  // o * NR + q
    const int o = int(oq / NR);
    const int m = reps[r];
    const int a_ = int(n / (size_t(N) * N)), b_ = int((n / N) % N), c_ = int(n % N);
    const double kx = a_ < N / 2 ? a_ : a_ - N, ky = b_ < N / 2 ? b_ : b_ - N, kz = c_ < N / 2 ? c_ : c_ - N;
    const double kn = sqrt(kx * kx + ky * ky + kz * kz);
    const double a = coef[2 * oq + 1] * kn;
    double mu = 0.0;
    if (kn > 0.0) mu = (kx * sigma[3 * m] + ky * sigma[3 * m + 1] + kz * sigma[3 * m + 2]) / kn;
    const double smu = sqrt(fmax(0.0, 1.0 - mu * mu));
    const double* t = gj + size_t(o) * 3 * n_t;  // nodes, weights, sqrt(1 - t^2)
    double re = 0.0, im = 0.0;
    for (int k = 0; k < n_t; ++k) {
      double sv, cv;
      sincos(a * t[k] * mu, &sv, &cv);
      const double j = t[n_t + k] * j0(a * t[2 * n_t + k] * smu);
      re += cv * j;
      im -= sv * j;
    }
    const double pref = coef[2 * oq];
    Fv[(oq * n_reps + r) * N3 + n] = make_double2(pref * re, pref * im);
  }
}

// The VSS gain weight depends on (k, rho, sigma) only through two numbers (Sec. 4, F after
// Eq. GG): F = pref(rho) Phi_alpha(p, q) with p = s k.sigma, q = s |k x sigma|, s = pi rho c_j / L,
// and Phi_alpha(p, q) = int_{-1}^{1} (1+t)^(alpha-1) exp(-i t p) J0(sqrt(1-t^2) q) dt.
// phi_grid_kernel tabulates Phi on a uniform grid p = p0 + i h, q = q0 + j h (q0 = -2h: J0 is
// even, so the rows below q = 0 mirror the ones above); vss_from_phi_kernel fills the gain table
// by 4 x 4-point Lagrange interpolation on that grid, in FP64.
__global__ void phi_grid_kernel(double2* __restrict__ phi, int np, int nq, double p0, double q0, double h,
                                const double* __restrict__ gj, int n_t) {
  const size_t count = size_t(np) * nq;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < count; idx += size_t(gridDim.x) * blockDim.x) {
    const double p = p0 + double(idx % np) * h, q = q0 + double(idx / np) * h;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < n_t; ++k) {
      double sv, cv;
      sincos(gj[k] * p, &sv, &cv);
      const double j = gj[n_t + k] * j0(gj[2 * n_t + k] * q);
      re += cv * j;
      im -= sv * j;
    }
    phi[idx] = make_double2(re, im);
  }
}

// cubic Lagrange weights of the stencil points -1, 0, 1, 2 at the fraction f in [0, 1)
__device__ __forceinline__ void lagrange4(double f, double (&w)[4]) {
  w[0] = -f * (f - 1.0) * (f - 2.0) / 6.0;
  w[1] = (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0;
  w[2] = -(f + 1.0) * f * (f - 2.0) / 2.0;
  w[3] = (f + 1.0) * f * (f - 1.0) / 6.0;
}

__global__ void vss_from_phi_kernel(double2* __restrict__ Fv, int P, int NR, int N, const double* __restrict__ coef,
                                    const double2* __restrict__ phi, const int* __restrict__ grid_of_pair, int np,
                                    int nq, double p0, double q0, double h, const double* __restrict__ sigma,
                                    const int* __restrict__ reps, int n_reps) {
  const size_t N3 = size_t(N) * N * N;
  const size_t count = size_t(P) * NR * n_reps * N3;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < count; idx += size_t(gridDim.x) * blockDim.x) {
    const size_t n = idx % N3;
    const int r = int((idx / N3) % n_reps);
    const size_t oq = idx / (N3 * n_reps);  // o * NR + q
    const int o = int(oq / NR);
    const int m = reps[r];
    const int a_ = int(n / (size_t(N) * N)), b_ = int((n / N) % N), c_ = int(n % N);
    const double kx = a_ < N / 2 ? a_ : a_ - N, ky = b_ < N / 2 ? b_ : b_ - N, kz = c_ < N / 2 ? c_ : c_ - N;
    const double s = coef[2 * oq + 1];
    const double kd = kx * sigma[3 * m] + ky * sigma[3 * m + 1] + kz * sigma[3 * m + 2];
    const double pv = s * kd;
    const double qv = s * sqrt(fmax(0.0, kx * kx + ky * ky + kz * kz - kd * kd));
    const double u = (pv - p0) / h, v = (qv - q0) / h;
    int iu = int(floor(u)), iv = int(floor(v));
    iu = iu < 1 ? 1 : (iu > np - 3 ? np - 3 : iu);
    iv = iv < 1 ? 1 : (iv > nq - 3 ? nq - 3 : iv);
    double wu[4], wv[4];
    lagrange4(u - iu, wu);
    lagrange4(v - iv, wv);
    const double2* g = phi + size_t(grid_of_pair[o]) * np * nq;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double rr = 0.0, ii = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double2 z = g[size_t(iv - 1 + b) * np + (iu - 1 + a)];
        rr += wu[a] * z.x;
        ii += wu[a] * z.y;
      }
      re += wv[b] * rr;
      im += wv[b] * ii;
    }
    const double pref = coef[2 * oq];
    Fv[(oq * n_reps + r) * N3 + n] = make_double2(pref * re, pref * im);
  }
}

__global__ void gain_to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    dst[i] = float(src[i]);
}

__global__ void vss_to_f32_kernel(const double2* __restrict__ src, float2* __restrict__ dst, int s, int NR,
                                  int n_slot, size_t N3, int self_sum) {
  const size_t n = size_t(s) * s * NR * n_slot * N3;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const int o = int(i / (N3 * n_slot * NR));
    double2 v = src[i];
    // F(sigma) + F(-sigma) = F + conj F
    if (self_sum && o / s == o % s) v = make_double2(v.x + v.x, 0.0);
    dst[i] = make_float2(float(v.x), float(v.y));
  }
}

}  // namespace

int launch_to_f32(const Plan& p, const double* src, float* dst, size_t n) {
  gain_to_f32_kernel<<<unsigned(n / 256 + 1 < 8192 ? n / 256 + 1 : 8192), 256, 0, p.home>>>(src, dst, n);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int launch_gain_tables_f32(Plan& p, int self_sum) {
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t P = size_t(p.s) * p.s;
  if (!p.vss) {
    const size_t n = P * p.N_rho * N3;
    gain_to_f32_kernel<<<unsigned(n / 256 + 1 < 8192 ? n / 256 + 1 : 8192), 256, 0, p.home>>>(p.d_Fw, p.d_Fwf, n);
  } else {
    const size_t n = P * p.N_rho * p.n_fslot * N3;
    vss_to_f32_kernel<<<unsigned(n / 256 + 1 < 65536 ? n / 256 + 1 : 65536), 256, 0, p.home>>>(
        p.d_Fv, p.d_Fvf, p.s, p.N_rho, p.n_fslot, N3, self_sum);
  }
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int launch_loss_table(Plan& p, const double* d_gcoef, const double* d_gscale, int n_loss) {
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t nG = size_t(p.s) * p.s * N3;
  const unsigned blocks = unsigned(nG / 256 + 1 < 4096 ? nG / 256 + 1 : 4096);
  loss_table_kernel<<<blocks, 256, 0, p.home>>>(p.d_Gm, nG, p.N, n_loss, d_gcoef, d_gscale);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int launch_vss_tables(Plan& p, const double* d_fcoef, const double* d_gj, int n_t, const double* d_sigma,
                      const int* d_reps, int n_reps) {
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t n = size_t(p.s) * p.s * p.N_rho * n_reps * N3;
  const unsigned blocks = unsigned(n / 256 + 1 < 65536 ? n / 256 + 1 : 65536);
  vss_table_kernel<<<blocks, 256, 0, p.home>>>(p.d_Fv, p.s * p.s, p.N_rho, p.N, d_fcoef, d_gj, n_t, d_sigma,
                                               d_reps, n_reps);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int launch_vss_tables_grid(Plan& p, const double* d_fcoef, double2* d_phi, const double* d_gj, int n_alpha, int n_t,
                           const VssGrid& gr, const int* d_grid_of_pair, const double* d_sigma, const int* d_reps,
                           int n_reps) {
  const size_t cells = size_t(gr.np) * gr.nq;
  for (int a = 0; a < n_alpha; ++a) {
    const unsigned blocks = unsigned(cells / 256 + 1 < 65536 ? cells / 256 + 1 : 65536);
    phi_grid_kernel<<<blocks, 256, 0, p.home>>>(d_phi + a * cells, gr.np, gr.nq, gr.p0, gr.q0, gr.h,
                                                d_gj + size_t(a) * 3 * n_t, n_t);
  }
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t n = size_t(p.s) * p.s * p.N_rho * n_reps * N3;
  const unsigned blocks = unsigned(n / 256 + 1 < 65536 ? n / 256 + 1 : 65536);
  vss_from_phi_kernel<<<blocks, 256, 0, p.home>>>(p.d_Fv, p.s * p.s, p.N_rho, p.N, d_fcoef, d_phi, d_grid_of_pair,
                                                  gr.np, gr.nq, gr.p0, gr.q0, gr.h, d_sigma, d_reps, n_reps);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int launch_vhs_tables(Plan& p, const double* d_fcoef, const double* d_gcoef, const double* d_gscale, int n_loss) {
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t nF = size_t(p.s) * p.s * p.N_rho * N3, nG = size_t(p.s) * p.s * N3;
  auto blocks = [](size_t n) { return unsigned(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096); };
  gain_table_kernel<<<blocks(nF), 256, 0, p.home>>>(p.d_Fw, nF, p.N, d_fcoef);
  loss_table_kernel<<<blocks(nG), 256, 0, p.home>>>(p.d_Gm, nG, p.N, n_loss, d_gcoef, d_gscale);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

}  // namespace dgfs
