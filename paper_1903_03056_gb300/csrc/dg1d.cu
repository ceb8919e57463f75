// One-dimensional nodal DG transport and the RKDG step of the full equation (Sec. 5), with
// the Maxwell wall boundary condition of Sec. 2.  Entry points declared in include/dgfs.h.
//
// Scheme, per element of width h with K GLL nodes xi_m and weights w_m and the Lagrange
// basis on them (Sec. 5):
//   mass matrix (GLL rule)     M_ml = (h/2) w_m delta_ml
//   stiffness (exact)          S_ml = int phi_l d/dx phi_m dx = w_l D_lm,  D_lm = phi_m'(xi_l)
//   transport                  d_t F_m = (2 / (h w_m)) [ v_x sum_l S_ml F_l
//                                                       - delta_{m,K} F*_right + delta_{m,1} F*_left ]
//   upwind face flux           F* = v_x f(interior trace) when v . n >= 0, else v_x f(exterior)
//   collision (GLL rule, H diagonal)  d_t F_m += sum_j kappa_ij Q_ij(F_m^i, F_m^j)
// Wall exterior state for velocities entering the domain ((v - u_w) . n < 0):
//   (1 - acc) f_int(v_x -> -v_x) + acc n_w exp(-m_i |v - u_w|^2 / T_w),
//   n_w = - sum_{(v-u_w).n >= 0} (v-u_w).n f_int / sum_{(v-u_w).n < 0} (v-u_w).n exp(...),
// the mass-conservation condition of Sec. 2 with the integrals as velocity-grid sums.
//
// Kernels: one FP64 reduction of the outgoing wall fluxes per stage, and one transport
// kernel in which a thread owns one (element, species, velocity) and computes all K nodes.
// It reads the K nodal values and the one upwind neighbour or wall trace it needs, and
// writes K values, so it streams the state once and is bound by HBM bandwidth.  The RK stage
// combinations are fused into the transport kernel.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dgfs_internal.h"

namespace {

constexpr int kMaxK = 8;
constexpr int kMaxS = 8;

struct DGKParams {
  int Ne, K, s, N, bc;
  double S[kMaxK * kMaxK];    // S_ml, row m
  double coef[kMaxK];         // 2 / (h w_m)
  double acc[2];
  double den[2 * kMaxS];      // wall flux denominators [side][species]
  double vx0, dv;             // v_x of velocity index a: vx0 + (a + 1/2) dv
  double dt;
  int inflow[2];              // side is an in-flow boundary
  double cin[2 * kMaxS];      // in-flow coefficient n_in (m / (pi T))^(3/2) [side][species]
  // the same coefficients rounded once to FP32 for the FP32 kernel (GB300's FP64 rate is a
  // small fraction of its FP32 rate, so the FP32 kernel does no FP64 arithmetic per element)
  float Sf[kMaxK * kMaxK];
  float coeff[kMaxK];
  float vx0f, dvf;
  const void* F;              // stage input (the state whose transport is taken)
  const void* F0;             // stage 2: the state at the start of the step
  const void* C;              // collision term [Ne*K][s][N^3], or null
  void* out;
  const void* W;              // wall Maxwellian shapes [2][s][N^3]
  const double* num;          // outgoing wall fluxes [2][s]
};

// 16 bytes of consecutive velocities per thread: 4 floats or 2 doubles.  N^2 is a multiple of
// 4 for the even grids the library supports, so a thread's velocities share their v_x index
// (and their reflected block); every access is a 16-byte vector access.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vload(const T* p, T (&x)[Vec16<T>::n]) {
  const typename Vec16<T>::type v = *reinterpret_cast<const typename Vec16<T>::type*>(p);
  memcpy(x, &v, sizeof(v));
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, const T (&x)[Vec16<T>::n]) {
  typename Vec16<T>::type v;
  memcpy(&v, x, sizeof(v));
  *reinterpret_cast<typename Vec16<T>::type*>(p) = v;
}

// MODE 0: out = transport rhs; 1: out = F + dt (rhs + C); 2: out = F0/2 + (F + dt (rhs + C))/2
template <typename T, int MODE, int K>
__global__ void __launch_bounds__(256) dg_transport_kernel(const DGKParams p) {
  constexpr int V = Vec16<T>::n;
  const size_t N3 = size_t(p.N) * p.N * p.N;
  const size_t v = (blockIdx.x * size_t(blockDim.x) + threadIdx.x) * V;  // first velocity
  if (v >= N3) return;
  const int e = int(blockIdx.y) / p.s;
  const int i = int(blockIdx.y) % p.s;
  const T* F = static_cast<const T*>(p.F);
  const int s_ = p.s;
  auto at = [=](int ee, int m) { return ((size_t(ee) * K + m) * s_ + i) * N3 + v; };
  const int a = int(v / (size_t(p.N) * p.N));
  // the same velocities with v_x -> -v_x (the grid is symmetric: index a -> N - 1 - a)
  const size_t v_refl = size_t(static_cast<long long>(v) + static_cast<long long>(p.N - 1 - 2 * a) * p.N * p.N);
  constexpr bool F32 = sizeof(T) == 4;
  const T vx = F32 ? T(p.vx0f + (float(a) + 0.5f) * p.dvf) : T(p.vx0 + (a + 0.5) * p.dv);

  T Fl[K][V];
#pragma unroll
  for (int m = 0; m < K; ++m) vload<T>(F + at(e, m), Fl[m]);

  // upwind values at the two faces (v_x is the same for the thread's velocities)
  T up_l[V], up_r[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    up_l[j] = Fl[0][j];
    up_r[j] = Fl[K - 1][j];
  }
  if (vx > T(0)) {
    if (e > 0) {
      vload<T>(F + at(e - 1, K - 1), up_l);
    } else if (p.bc == DGFS_BC_PERIODIC) {
      vload<T>(F + at(p.Ne - 1, K - 1), up_l);
    } else {
      const T c_w = T(p.inflow[0] ? p.cin[i] : p.acc[0] * (-p.num[i] / p.den[i]));
      const T c_s = T(p.inflow[0] ? 0.0 : 1.0 - p.acc[0]);
      T fr[V], wv[V];
      vload<T>(F + (size_t(0) * s_ + i) * N3 + v_refl, fr);
      vload<T>(static_cast<const T*>(p.W) + size_t(i) * N3 + v, wv);
#pragma unroll
      for (int j = 0; j < V; ++j) up_l[j] = c_s * fr[j] + c_w * wv[j];
    }
  }
  if (vx < T(0)) {
    if (e < p.Ne - 1) {
      vload<T>(F + at(e + 1, 0), up_r);
    } else if (p.bc == DGFS_BC_PERIODIC) {
      vload<T>(F + at(0, 0), up_r);
    } else {
      const T c_w = T(p.inflow[1] ? p.cin[kMaxS + i] : p.acc[1] * (-p.num[s_ + i] / p.den[kMaxS + i]));
      const T c_s = T(p.inflow[1] ? 0.0 : 1.0 - p.acc[1]);
      T fr[V], wv[V];
      vload<T>(F + ((size_t(p.Ne) * K - 1) * s_ + i) * N3 + v_refl, fr);
      vload<T>(static_cast<const T*>(p.W) + (size_t(s_) + i) * N3 + v, wv);
#pragma unroll
      for (int j = 0; j < V; ++j) up_r[j] = c_s * fr[j] + c_w * wv[j];
    }
  }

  T* out = static_cast<T*>(p.out);
  const T* C = static_cast<const T*>(p.C);
  const T* F0 = static_cast<const T*>(p.F0);
  const T dt = T(p.dt);  // one conversion per thread
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const size_t o = at(e, m);
    const T cm = F32 ? T(p.coeff[m]) : T(p.coef[m]);
    T r[V], c[V], f0[V];
    if constexpr (MODE != 0) vload<T>(C + o, c);
    if constexpr (MODE == 2) vload<T>(F0 + o, f0);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      T vol = T(0);
#pragma unroll
      for (int l = 0; l < K; ++l) vol += (F32 ? T(p.Sf[m * kMaxK + l]) : T(p.S[m * kMaxK + l])) * Fl[l][j];
      T rr = vx * vol;
      if (m == K - 1) rr -= vx * up_r[j];
      if (m == 0) rr += vx * up_l[j];
      rr *= cm;
      if constexpr (MODE == 0) r[j] = rr;
      else if constexpr (MODE == 1) r[j] = Fl[m][j] + dt * (rr + c[j]);
      else r[j] = T(0.5) * f0[j] + T(0.5) * (Fl[m][j] + dt * (rr + c[j]));
    }
    vstore<T>(out + o, r);
  }
}

// outgoing normal mass flux sum_{(v-u_w).n >= 0} (v-u_w).n f_trace in FP64, one block per
// (side, species); the trace is the first node of the first element (side 0) or the last
// node of the last element (side 1)
template <typename T>
__global__ void __launch_bounds__(256) dg_wall_flux_kernel(const T* __restrict__ F, int Ne, int K, int s, int N,
                                                           double vx0, double dv, double* __restrict__ num) {
  const int side = blockIdx.x / s, i = blockIdx.x % s;
  const size_t N3 = size_t(N) * N * N;
  const size_t node = side == 0 ? 0 : size_t(Ne) * K - 1;
  const T* f = F + (node * s + i) * N3;
  const double n_out = side == 0 ? -1.0 : 1.0;
  double acc = 0.0;
  for (size_t v = threadIdx.x; v < N3; v += blockDim.x) {
    const int a = int(v / (size_t(N) * N));
    const double cn = (vx0 + (a + 0.5) * dv) * n_out;
    if (cn >= 0.0) acc += cn * double(f[v]);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) num[side * s + i] = red[0];
}

// GLL nodes (endpoints and the roots of P'_{K-1}, by Newton's method from the
// Chebyshev-Gauss-Lobatto points) and weights 2 / (K (K-1) P_{K-1}(xi)^2)
void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (x * p1 - p0) / (x * x - 1.0);
}

void gll(int K, std::vector<double>& xi, std::vector<double>& w) {
  const int n = K - 1;
  xi.assign(K, 0.0);
  w.assign(K, 0.0);
  xi[0] = -1.0;
  xi[n] = 1.0;
  for (int k = 1; k < n; ++k) {
    double x = -std::cos(M_PI * k / n);
    for (int it = 0; it < 100; ++it) {
      // Newton on q(x) = P'_n(x): q' = (2x P'_n - n(n+1) P_n) / (1 - x^2)
      double P, dP;
      legendre(n, x, P, dP);
      const double d2P = (2.0 * x * dP - n * (n + 1.0) * P) / (1.0 - x * x);
      const double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    xi[k] = x;
  }
  for (int k = 0; k < K; ++k) {
    double P, dP;
    if (k == 0 || k == n) {
      P = (k == 0 && (n % 2 == 1)) ? -1.0 : 1.0;
    } else {
      legendre(n, xi[k], P, dP);
    }
    w[k] = 2.0 / (K * (K - 1.0) * P * P);
  }
}

// D_lm = phi_m'(xi_l) of the Lagrange basis on the GLL nodes
void diff_matrix(const std::vector<double>& xi, std::vector<double>& D) {
  const int K = int(xi.size());
  D.assign(size_t(K) * K, 0.0);
  for (int l = 0; l < K; ++l)
    for (int m = 0; m < K; ++m) {
      double d = 0.0;
      for (int k = 0; k < K; ++k) {
        if (k == m) continue;
        double term = 1.0 / (xi[m] - xi[k]);
        for (int n = 0; n < K; ++n)
          if (n != m && n != k) term *= (xi[l] - xi[n]) / (xi[m] - xi[n]);
        d += term;
      }
      D[size_t(l) * K + m] = d;
    }
}

}  // namespace

struct dgfs_dg_plan_s {
  dgfs_plan coll = nullptr;  // not owned
  int Ne = 0, K = 0, bc = 0, B = 0;
  double x0 = 0, x1 = 0, h = 0;
  std::vector<double> xi, w;
  DGKParams kp{};
  void* d_W = nullptr;       // wall Maxwellian shapes [2][s][N^3]
  double* d_num = nullptr;   // [2][s]
  void* d_F1 = nullptr;      // RK stage state
  void* d_C = nullptr;       // collision term
};

namespace {

template <typename T, int K>
void launch_k(int mode, dim3 grid, const DGKParams& kp, cudaStream_t st) {
  if (mode == 0) dg_transport_kernel<T, 0, K><<<grid, 256, 0, st>>>(kp);
  else if (mode == 1) dg_transport_kernel<T, 1, K><<<grid, 256, 0, st>>>(kp);
  else dg_transport_kernel<T, 2, K><<<grid, 256, 0, st>>>(kp);
}

template <typename T>
int launch_transport(dgfs_dg_plan_s& d, int mode, const void* F, const void* F0, const void* C, void* out,
                     double dt, cudaStream_t st) {
  const dgfs::Plan& p = d.coll->plan;
  DGKParams kp = d.kp;
  kp.dt = dt;
  kp.F = F;
  kp.F0 = F0;
  kp.C = C;
  kp.out = out;
  const size_t N3 = size_t(p.N) * p.N * p.N;
  if (d.bc == DGFS_BC_WALLS) {
    dg_wall_flux_kernel<T><<<2 * p.s, 256, 0, st>>>(static_cast<const T*>(F), d.Ne, d.K, p.s, p.N, kp.vx0, kp.dv,
                                                   d.d_num);
  }
  const size_t threads = N3 / (16 / sizeof(T));  // one 16-byte vector of velocities each
  const dim3 grid(unsigned((threads + 255) / 256), unsigned(d.Ne * p.s));
  switch (d.K) {
    case 2: launch_k<T, 2>(mode, grid, kp, st); break;
    case 3: launch_k<T, 3>(mode, grid, kp, st); break;
    case 4: launch_k<T, 4>(mode, grid, kp, st); break;
    case 5: launch_k<T, 5>(mode, grid, kp, st); break;
    case 6: launch_k<T, 6>(mode, grid, kp, st); break;
    case 7: launch_k<T, 7>(mode, grid, kp, st); break;
    default: launch_k<T, 8>(mode, grid, kp, st); break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

int transport(dgfs_dg_plan_s& d, int mode, const void* F, const void* F0, const void* C, void* out, double dt,
              cudaStream_t st) {
  return d.coll->plan.f32io() ? launch_transport<float>(d, mode, F, F0, C, out, dt, st)
                                             : launch_transport<double>(d, mode, F, F0, C, out, dt, st);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct DevGuard {
  int prev = -1;
  bool ok = true;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void release(dgfs_dg_plan_s* d) {
  if (d->d_W) cudaFree(d->d_W);
  if (d->d_num) cudaFree(d->d_num);
  if (d->d_F1) cudaFree(d->d_F1);
  if (d->d_C) cudaFree(d->d_C);
  delete d;
}

}  // namespace

extern "C" {

int dgfs_dg_create(const dgfs_dg_desc* desc, dgfs_plan collision, dgfs_dg_plan* out) {
  if (!desc || !collision || !out) return DGFS_ERR_INVALID_ARG;
  *out = nullptr;
  const dgfs::Plan& p = collision->plan;
  const int Ne = desc->Ne, K = desc->K;
  if (Ne < 1 || K < 2 || K > kMaxK || p.s > kMaxS || !(desc->x1 > desc->x0) || !std::isfinite(desc->x0) ||
      !std::isfinite(desc->x1))
    return DGFS_ERR_INVALID_ARG;
  if (desc->bc != DGFS_BC_PERIODIC && desc->bc != DGFS_BC_WALLS) return DGFS_ERR_INVALID_ARG;
  if (desc->bc == DGFS_BC_WALLS) {
    for (int side = 0; side < 2; ++side) {
      const int kind = desc->side[side];
      if (kind != DGFS_SIDE_WALL && kind != DGFS_SIDE_INFLOW) return DGFS_ERR_INVALID_ARG;
      if (!(desc->Tw[side] > 0.0) || !std::isfinite(desc->Tw[side]) || !std::isfinite(desc->uw[3 * side]) ||
          !std::isfinite(desc->uw[3 * side + 1]) || !std::isfinite(desc->uw[3 * side + 2]))
        return DGFS_ERR_INVALID_ARG;
      if (kind == DGFS_SIDE_WALL &&
          (!(desc->acc[side] >= 0.0) || !(desc->acc[side] <= 1.0) || desc->uw[3 * side] != 0.0))
        return DGFS_ERR_INVALID_ARG;
      if (kind == DGFS_SIDE_INFLOW) {
        if (!desc->n_in) return DGFS_ERR_INVALID_ARG;
        for (int i = 0; i < p.s; ++i)
          if (!(desc->n_in[side * p.s + i] >= 0.0) || !std::isfinite(desc->n_in[side * p.s + i]))
            return DGFS_ERR_INVALID_ARG;
      }
    }
  }
  if (long(Ne) * K > 1 << 30) return DGFS_ERR_INVALID_ARG;
  dgfs_dg_plan_s* d = new (std::nothrow) dgfs_dg_plan_s();
  if (!d) return DGFS_ERR_OOM;
  d->coll = collision;
  d->Ne = Ne;
  d->K = K;
  d->bc = desc->bc;
  d->B = Ne * K;
  d->x0 = desc->x0;
  d->x1 = desc->x1;
  d->h = (desc->x1 - desc->x0) / Ne;
  gll(K, d->xi, d->w);
  std::vector<double> D;
  diff_matrix(d->xi, D);
  DGKParams& kp = d->kp;
  kp.Ne = Ne;
  kp.K = K;
  kp.s = p.s;
  kp.N = p.N;
  kp.bc = desc->bc;
  for (int m = 0; m < K; ++m) {
    kp.coef[m] = 2.0 / (d->h * d->w[m]);
    kp.coeff[m] = float(kp.coef[m]);
    for (int l = 0; l < K; ++l) {
      kp.S[m * kMaxK + l] = d->w[l] * D[size_t(l) * K + m];
      kp.Sf[m * kMaxK + l] = float(kp.S[m * kMaxK + l]);
    }
  }
  kp.dv = 2.0 * p.L / p.N;
  kp.vx0 = -p.L;
  kp.dvf = float(kp.dv);
  kp.vx0f = float(kp.vx0);
  const int N = p.N;
  const size_t N3 = size_t(N) * N * N;
  DevGuard g(p.device);
  if (!g.ok) { release(d); return DGFS_ERR_CUDA; }
  // side Maxwellian shapes exp(-m_i |v - u|^2 / T); for walls also the denominators of n_w
  // in FP64, for in-flow sides the constant factor n_in (m_i / (pi T))^(3/2)
  std::vector<double> Wd(2 * size_t(p.s) * N3, 0.0);
  if (desc->bc == DGFS_BC_WALLS) {
    for (int side = 0; side < 2; ++side) {
      const bool inflow = desc->side[side] == DGFS_SIDE_INFLOW;
      kp.inflow[side] = inflow ? 1 : 0;
      kp.acc[side] = inflow ? 0.0 : desc->acc[side];
      const double n_out = side == 0 ? -1.0 : 1.0;
      const double* u = &desc->uw[3 * side];
      for (int i = 0; i < p.s; ++i) {
        double den = 0.0;
        for (size_t v = 0; v < N3; ++v) {
          const int a = int(v / (size_t(N) * N)), b = int((v / N) % N), c = int(v % N);
          const double vx = kp.vx0 + (a + 0.5) * kp.dv, vy = kp.vx0 + (b + 0.5) * kp.dv,
                       vz = kp.vx0 + (c + 0.5) * kp.dv;
          const double d2 = (vx - u[0]) * (vx - u[0]) + (vy - u[1]) * (vy - u[1]) + (vz - u[2]) * (vz - u[2]);
          const double wv = std::exp(-p.mass[i] * d2 / desc->Tw[side]);
          Wd[(size_t(side) * p.s + i) * N3 + v] = wv;
          const double cn = vx * n_out;
          if (cn < 0.0) den += cn * wv;
        }
        kp.den[side * kMaxS + i] = inflow ? 1.0 : den;
        kp.cin[side * kMaxS + i] =
            inflow ? desc->n_in[side * p.s + i] * std::pow(p.mass[i] / (M_PI * desc->Tw[side]), 1.5) : 0.0;
      }
    }
  }
  const size_t esz = p.f32io() ? sizeof(float) : sizeof(double);
  const size_t state = size_t(d->B) * p.s * N3 * esz;
  if (cudaMalloc(&d->d_W, Wd.size() * esz) != cudaSuccess || cudaMalloc((void**)&d->d_num, 2 * kMaxS * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d->d_F1, state) != cudaSuccess || cudaMalloc(&d->d_C, state) != cudaSuccess) {
    cudaGetLastError();
    release(d);
    return DGFS_ERR_OOM;
  }
  cudaError_t ce;
  if (p.f32io()) {
    std::vector<float> Wf(Wd.begin(), Wd.end());
    ce = cudaMemcpy(d->d_W, Wf.data(), Wf.size() * sizeof(float), cudaMemcpyHostToDevice);
  } else {
    ce = cudaMemcpy(d->d_W, Wd.data(), Wd.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (ce != cudaSuccess || cudaMemset(d->d_num, 0, 2 * kMaxS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    release(d);
    return DGFS_ERR_CUDA;
  }
  kp.W = d->d_W;
  kp.num = d->d_num;
  *out = d;
  return DGFS_OK;
}

int dgfs_dg_destroy(dgfs_dg_plan plan) {
  if (!plan) return DGFS_OK;
  DevGuard g(plan->coll->plan.device);
  cudaDeviceSynchronize();
  release(plan);
  return DGFS_OK;
}

int dgfs_dg_nodes(dgfs_dg_plan plan, double* x_out) {
  if (!plan || !x_out) return DGFS_ERR_INVALID_ARG;
  for (int e = 0; e < plan->Ne; ++e)
    for (int m = 0; m < plan->K; ++m)
      x_out[size_t(e) * plan->K + m] = plan->x0 + plan->h * e + (plan->xi[m] + 1.0) * plan->h / 2.0;
  return DGFS_OK;
}

int dgfs_dg_transport(dgfs_dg_plan plan, const void* f_dev, void* rhs_dev, void* stream) {
  if (!plan || !f_dev || !rhs_dev || !aligned16(f_dev) || !aligned16(rhs_dev) || f_dev == rhs_dev)
    return DGFS_ERR_INVALID_ARG;
  dgfs::NvtxRange range("dgfs_dg_transport");
  DevGuard g(plan->coll->plan.device);
  if (!g.ok) return DGFS_ERR_CUDA;
  return transport(*plan, 0, f_dev, nullptr, nullptr, rhs_dev, 0.0, static_cast<cudaStream_t>(stream));
}

int dgfs_dg_step(dgfs_dg_plan plan, void* f_dev, double dt, void* stream) {
  if (!plan || !f_dev || !aligned16(f_dev) || !std::isfinite(dt)) return DGFS_ERR_INVALID_ARG;
  const dgfs::Plan& p = plan->coll->plan;
  if (!(p.flags & DGFS_SUM_SPECIES)) return DGFS_ERR_INVALID_ARG;
  if (plan->B > p.max_batch) return DGFS_ERR_BUDGET;
  dgfs::NvtxRange range("dgfs_dg_step");
  DevGuard g(p.device);
  if (!g.ok) return DGFS_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  // stage 1: F1 = F + dt (T(F) + C(F))
  if ((rc = dgfs_eval_collision(plan->coll, f_dev, plan->d_C, plan->B, stream)) != DGFS_OK) return rc;
  if ((rc = transport(*plan, 1, f_dev, nullptr, plan->d_C, plan->d_F1, dt, st)) != DGFS_OK) return rc;
  // stage 2: F <- F/2 + (F1 + dt (T(F1) + C(F1)))/2
  if ((rc = dgfs_eval_collision(plan->coll, plan->d_F1, plan->d_C, plan->B, stream)) != DGFS_OK) return rc;
  return transport(*plan, 2, plan->d_F1, f_dev, plan->d_C, f_dev, dt, st);
}

}  // extern "C"
