// dgfs_eval_collision_noalloc: the collision evaluation for callers that cannot allocate
// device memory.
//
// Callers such as a solver plugin whose host application owns every device allocation
// through its own pool, code running where cudaMalloc is forbidden after start-up, or a
// process with a fixed device-memory budget cannot create a plan (dgfs_create_plan allocates
// tables and a workspace).  This entry point needs no plan and allocates nothing: the
// quadrature and kernel constants are built on the host into the kernel's parameter block,
// the gain/loss weights and the phase factors are evaluated inside the kernel, and the
// workspace is a file-scope static __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
//
// Limits (larger requests return an error before any work): FP32, N in {8, 12, 16}, s <= 3,
// M <= 12, N_rho <= 16, alpha = 1 (VHS).  The workspace holds kSlots = 64 work slots of
// 7 N^3 complex floats at N = 16: 64 * 7 * 16^3 * 8 bytes = 14.7 MB.  Batches of any size are
// processed by at most 64 CTAs looping over the (node, pair) items.
#include <cmath>
#include <mutex>

#include <cuda.h>

#include "collision_kernel.cuh"

namespace dgfs {
namespace {

constexpr int kMaxN = 16;
constexpr int kMaxS = 3;
constexpr int kMaxPairs = kMaxS * kMaxS;
constexpr int kMaxM = 12;
constexpr int kMaxRho = 16;
constexpr int kMaxEnt = kMaxPairs * kMaxM;
constexpr int kSlots = 64;
constexpr size_t kSlotComplex = size_t(7) * kMaxN * kMaxN * kMaxN;
constexpr int kMaxDevices = 64;
constexpr double kPi = 3.141592653589793238462643383279502884;

// the workspace: shared by every call on a device; each call writes every element it reads
static __device__ __align__(256) float2 g_noalloc_scratch[size_t(kSlots) * kSlotComplex];

struct NoAllocParams {
  const float* f;
  float* Q;
  float2* scratch;
  int batch, s, n_tasks, n_rho;
  double L;
  TaskDesc tasks[kMaxPairs];
  GroupDesc groups[kMaxEnt];
  float ent_w[kMaxEnt];
  double ent_sigma[kMaxEnt][3];
  double rho[kMaxRho];
  double c[kMaxPairs][2];          // per task: (c_i, c_j)
  float fpref[kMaxPairs][kMaxRho];  // per ordered pair: w_q 4 pi b rho_q^(4-2 omega) / N^3
  float fscale[kMaxPairs][kMaxRho]; // rho_q c_j / L
  float gpref[kMaxPairs][kMaxRho];  // 16 pi^2 b w_q rho_q^(4-2 omega)
  float gscale[kMaxRho];            // rho_q / L
};

__device__ __forceinline__ int centred(int n, int N) { return n < N / 2 ? n : n - N; }

// sin(pi y) / (pi y)
__device__ __forceinline__ float sinc_pi(float y) {
  return fabsf(y) < 1e-20f ? 1.0f : sinpif(y) / (float(kPi) * y);
}

template <int N>
__device__ __forceinline__ float kabs(int n0, int pp) {
  const float kx = float(centred(n0, N)), ky = float(centred(pp / N, N)), kz = float(centred(pp % N, N));
  return sqrtf(kx * kx + ky * ky + kz * kz);
}

// one work item per CTA at a time (no cluster); plane groups of N threads, one plane each
template <int N>
__global__ void __launch_bounds__(N * N, 1) collision_noalloc_kernel(const __grid_constant__ NoAllocParams p) {
  using T = float;
  using CT = float2;
  constexpr int N2 = N * N, N3 = N * N * N, GP = N, NT = N * N, PITCH = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int grp = tid / N;
  const int t = tid % N;
  CT* tb = reinterpret_cast<CT*>(smem_raw) + size_t(grp) * 2 * N * PITCH;
  CT* ab = tb + N * PITCH;
  CT* phs = reinterpret_cast<CT*>(smem_raw) + size_t(GP) * 2 * N * PITCH;  // [e][role][axis][N]

  CT* scr = p.scratch + size_t(blockIdx.x) * 7 * N3;
  CT* const FI = scr;
  CT* const FJ = scr + N3;
  CT* const HA = scr + 2 * N3;
  CT* const HB = scr + 3 * N3;
  CT* const PV = scr + 4 * N3;
  CT* const QA = scr + 5 * N3;
  CT* const QB = scr + 6 * N3;
  const T inv_n3 = T(1) / T(N3);

  const int n_items = p.batch * p.n_tasks;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int b = item / p.n_tasks;
    const int task = item % p.n_tasks;
    const TaskDesc tk = p.tasks[task];
    const T* fb = p.f + size_t(b) * p.s * N3;
    const int nspec = tk.j == tk.i ? 1 : 2;

    // Fourier coefficients of f_i (and f_j): planes, then pencils
    {
      const int x = grp;
      for (int sp = 0; sp < nspec; ++sp) {
        const T* src = fb + size_t(sp == 0 ? tk.i : tk.j) * N3 + size_t(x) * N2;
        CT v[N];
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = make_float2(__ldg(src + t * N + c), 0.0f);
        fft_line<T, N, -1>(v);
        rows_to_cols<T, N, GP>(v, tb, t);
        fft_line<T, N, -1>(v);
        CT* dst = (sp == 0 ? FI : FJ) + size_t(x) * N2;
#pragma unroll
        for (int r = 0; r < N; ++r) st2<T>(dst + r * N + t, v[r]);
      }
    }
    __syncthreads();
    for (int u = tid; u < nspec * N2; u += NT) {
      CT* vol = u < N2 ? FI : FJ;
      const int pp = u % N2;
      CT v[N];
#pragma unroll
      for (int n = 0; n < N; ++n) v[n] = ld2<T>(vol + n * N2 + pp);
      fft_line<T, N, -1>(v);
#pragma unroll
      for (int n = 0; n < N; ++n) st2<T>(vol + n * N2 + pp, scale<T>(v[n], inv_n3));
    }
    __syncthreads();
    const CT* FJs = nspec == 2 ? FJ : FI;

    for (int q = 0; q < p.n_rho; ++q) {
      // phase factors exp(i pi shift_d k / L) of this task and radial node
      for (int u = tid; u < tk.n_ent * 6 * N; u += NT) {
        const int n = u % N;
        const int axis = (u / N) % 3;
        const int role = (u / (3 * N)) % 2;
        const int e = u / (6 * N);
        const double sh = (role == 0 ? p.rho[q] * p.c[task][1] : -p.rho[q] * p.c[task][0]) *
                          p.ent_sigma[tk.ent_off + e][axis];
        const double x = sh * centred(n, N) / p.L;
        const float r = float(x - 2.0 * rint(0.5 * x));
        float sv, cv;
        sincospif(r, &sv, &cv);
        phs[u] = make_float2(cv, sv);
      }
      __syncthreads();
      for (int gi = 0; gi < tk.n_grp; ++gi) {
        const GroupDesc gd = p.groups[tk.grp_off + gi];
        for (int u = tid; u < 2 * N2; u += NT) {
          const int role = u / N2;
          const int pp = u % N2;
          const CT* src = role == 0 ? FI : FJs;
          const CT* ph = phs + ((gd.first * 2 + role) * 3 + 0) * N;
          CT v[N];
#pragma unroll
          for (int n = 0; n < N; ++n) v[n] = cmul<T>(ld2<T>(src + n * N2 + pp), ph[n]);
          fft_line<T, N, +1>(v);
          CT* dst = role == 0 ? HA : HB;
#pragma unroll
          for (int n = 0; n < N; ++n) st2<T>(dst + n * N2 + pp, v[n]);
        }
        __syncthreads();
        const bool last = gi == tk.n_grp - 1;
        const int x = grp;
        CT P[N];
#pragma unroll
        for (int c = 0; c < N; ++c) P[c] = gi == 0 ? make_float2(0.0f, 0.0f) : ld2<T>(PV + x * N2 + c * N + t);
        for (int e = gd.first; e < gd.first + gd.count; ++e) {
          const T w = p.ent_w[tk.ent_off + e];
          CT v[N];
          for (int role = 0; role < 2; ++role) {
            const CT* vol = (role == 0 ? HA : HB) + size_t(x) * N2;
            const CT* phy = phs + ((e * 2 + role) * 3 + 1) * N;
            const CT* phz = phs + ((e * 2 + role) * 3 + 2) * N;
#pragma unroll
            for (int r = 0; r < N; ++r) v[r] = cmul<T>(ld2<T>(vol + r * N + t), phy[r]);
            fft_line<T, N, +1>(v);
            cols_to_rows<T, N, GP>(v, tb, t);
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] = cmul<T>(v[c], phz[c]);
            fft_line<T, N, +1>(v);
            if (role == 0) {
#pragma unroll
              for (int c = 0; c < N; ++c) ab[t * PITCH + c] = v[c];
            }
          }
#pragma unroll
          for (int c = 0; c < N; ++c) {
            const CT prod = cmul<T>(ab[t * PITCH + c], v[c]);
            P[c] = make_float2(P[c].x + w * prod.x, P[c].y + w * prod.y);
          }
        }
        if (last) {
          fft_line<T, N, -1>(P);
          rows_to_cols<T, N, GP>(P, tb, t);
          fft_line<T, N, -1>(P);
#pragma unroll
          for (int r = 0; r < N; ++r) st2<T>(PV + x * N2 + r * N + t, P[r]);
        } else {
#pragma unroll
          for (int c = 0; c < N; ++c) st2<T>(PV + x * N2 + c * N + t, P[c]);
        }
        __syncthreads();
      }
      for (int pp = tid; pp < N2; pp += NT) {
        CT v[N];
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = ld2<T>(PV + n * N2 + pp);
        fft_line<T, N, -1>(v);
        for (int o = 0; o < 2; ++o) {
          const int pair = o == 0 ? tk.out0 : tk.out1;
          if (pair < 0) break;
          const float pref = p.fpref[pair][q], sc = p.fscale[pair][q];
          CT* acc = o == 0 ? QA : QB;
#pragma unroll
          for (int n = 0; n < N; ++n) {
            CT val = scale<T>(v[n], pref * sinc_pi(sc * kabs<N>(n, pp)));
            if (q > 0) val = add<T>(val, ld2<T>(acc + n * N2 + pp));
            st2<T>(acc + n * N2 + pp, val);
          }
        }
      }
      __syncthreads();
    }

    // Q_ij = Re IFFT(Q_hat^+) - f_i Re IFFT(G^- f_hat_j)
    for (int o = 0; o < 2; ++o) {
      const int pair = o == 0 ? tk.out0 : tk.out1;
      if (pair < 0) break;
      const int io = o == 0 ? tk.i : tk.j;
      const int jo = o == 0 ? tk.j : tk.i;
      const CT* acc = o == 0 ? QA : QB;
      const CT* Fj = jo == tk.i ? FI : FJs;
      for (int pp = tid; pp < N2; pp += NT) {
        CT v[N];
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = ld2<T>(acc + n * N2 + pp);
        fft_line<T, N, +1>(v);
#pragma unroll
        for (int n = 0; n < N; ++n) st2<T>(HA + n * N2 + pp, v[n]);
#pragma unroll
        for (int n = 0; n < N; ++n) {
          const float ka = kabs<N>(n, pp);
          float g = 0.0f;
          for (int q = 0; q < p.n_rho; ++q) g += p.gpref[pair][q] * sinc_pi(p.gscale[q] * ka);
          v[n] = scale<T>(ld2<T>(Fj + n * N2 + pp), g);
        }
        fft_line<T, N, +1>(v);
#pragma unroll
        for (int n = 0; n < N; ++n) st2<T>(HB + n * N2 + pp, v[n]);
      }
      __syncthreads();
      T* Qout = p.Q + ((size_t(b) * p.s + io) * p.s + jo) * N3;
      const T* fi = fb + size_t(io) * N3;
      const int x = grp;
      CT v[N];
      T gain[N];
#pragma unroll
      for (int r = 0; r < N; ++r) v[r] = ld2<T>(HA + x * N2 + r * N + t);
      fft_line<T, N, +1>(v);
      cols_to_rows<T, N, GP>(v, tb, t);
      fft_line<T, N, +1>(v);
#pragma unroll
      for (int c = 0; c < N; ++c) gain[c] = v[c].x;
#pragma unroll
      for (int r = 0; r < N; ++r) v[r] = ld2<T>(HB + x * N2 + r * N + t);
      fft_line<T, N, +1>(v);
      cols_to_rows<T, N, GP>(v, tb, t);
      fft_line<T, N, +1>(v);
      T* rb = reinterpret_cast<T*>(tb);
#pragma unroll
      for (int c = 0; c < N; ++c) rb[t * PITCH + c] = gain[c] - __ldg(fi + x * N2 + t * N + c) * v[c].x;
      __syncthreads();
#pragma unroll
      for (int r = 0; r < N; ++r) Qout[x * N2 + r * N + t] = rb[r * PITCH + t];
      __syncthreads();
    }
  }
}

template <int N>
constexpr size_t smem_bytes() {
  return size_t(N) * 2 * N * (N + 1) * sizeof(float2) + size_t(kMaxM) * 6 * N * sizeof(float2);
}

// ---- once-per-context set-up ----------------------------------------------------------------
// The workspace's device address and the kernels' shared-memory limits belong to the CUDA
// context that loaded this module.  A cudaDeviceReset, or a new primary context, reloads the
// module, so the set-up is keyed on the current context's unique id (read through the
// driver's cuCtxGetCurrent / cuCtxGetId, looked up by the runtime without linking the driver
// library) and redone when that id changes.
struct DeviceState {
  unsigned long long ctx_id = 0;
  bool ready = false;
  float2* scratch = nullptr;
};
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// unique id of the context current on this thread (the device's primary context when the
// runtime made none current yet); 0 on failure
unsigned long long current_context_id(int dev) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return 0;
    }
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return 0;
  if (ctx == nullptr) {
    // no context current yet: make the device's primary context current (cudaSetDevice
    // initialises it) and read again
    if (cudaSetDevice(dev) != cudaSuccess || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) {
      cudaGetLastError();
      return 0;
    }
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int setup_device(int dev, float2** scratch) {
  if (dev < 0 || dev >= kMaxDevices) return DGFS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long ctx = current_context_id(dev);
  if (ctx == 0) return DGFS_ERR_CUDA;
  if (!g_state[dev].ready || g_state[dev].ctx_id != ctx) {
    g_state[dev].ready = false;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return DGFS_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(collision_noalloc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes<8>())) != cudaSuccess ||
        cudaFuncSetAttribute(collision_noalloc_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes<12>())) != cudaSuccess ||
        cudaFuncSetAttribute(collision_noalloc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes<16>())) != cudaSuccess) {
      cudaGetLastError();
      return DGFS_ERR_CUDA;
    }
    g_state[dev].scratch = static_cast<float2*>(ptr);
    g_state[dev].ctx_id = ctx;
    g_state[dev].ready = true;
  }
  *scratch = g_state[dev].scratch;
  return DGFS_OK;
}

// ---- host-side constants, without heap allocation -------------------------------------------
int builtin_design_fixed(int M, double (*sg)[3]) {
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  int m = 0;
  auto push = [&](double a, double b, double c) {
    const double n = std::sqrt(a * a + b * b + c * c);
    sg[m][0] = a / n;
    sg[m][1] = b / n;
    sg[m][2] = c / n;
    ++m;
  };
  if (M == 6) {
    for (int d = 0; d < 3; ++d)
      for (double s : {1.0, -1.0}) push(d == 0 ? s : 0.0, d == 1 ? s : 0.0, d == 2 ? s : 0.0);
    return DGFS_OK;
  }
  if (M == 12) {
    for (double a : {1.0, -1.0})
      for (double b : {g, -g}) {
        push(0.0, a, b);
        push(a, b, 0.0);
        push(b, 0.0, a);
      }
    return DGFS_OK;
  }
  return DGFS_ERR_INVALID_ARG;
}

int build_params(const dgfs_plan_desc* d, NoAllocParams& p) {
  if (d->precision != DGFS_FP32 || d->flags != 0u) return DGFS_ERR_UNSUPPORTED;
  if (d->N != 8 && d->N != 12 && d->N != 16) return DGFS_ERR_UNSUPPORTED_N;
  if (!(d->L > 0.0) || !std::isfinite(d->L) || d->s < 1 || !d->mass || !d->omega || !d->alpha || d->N_rho < 1 ||
      d->M < 1 || std::isnan(d->R) || std::isinf(d->R))
    return DGFS_ERR_INVALID_ARG;
  if (d->s > kMaxS || d->M > kMaxM || d->N_rho > kMaxRho) return DGFS_ERR_UNSUPPORTED;
  const int s = d->s, N = d->N, M = d->M, NR = d->N_rho;
  for (int i = 0; i < s; ++i)
    if (!(d->mass[i] > 0.0) || !std::isfinite(d->mass[i])) return DGFS_ERR_INVALID_ARG;
  for (int k = 0; k < s * s; ++k) {
    if (!(d->omega[k] >= 0.5 && d->omega[k] <= 1.0)) return DGFS_ERR_INVALID_ARG;
    if (d->alpha[k] != 1.0) return DGFS_ERR_UNSUPPORTED;
    if (d->b_override && !std::isfinite(d->b_override[k])) return DGFS_ERR_INVALID_ARG;
  }
  double sg[kMaxM][3], ws[kMaxM];
  if (d->sigma) {
    for (int m = 0; m < M; ++m) {
      for (int a = 0; a < 3; ++a) sg[m][a] = d->sigma[3 * m + a];
      const double n = std::sqrt(sg[m][0] * sg[m][0] + sg[m][1] * sg[m][1] + sg[m][2] * sg[m][2]);
      if (!(std::fabs(n - 1.0) < 1e-9)) return DGFS_ERR_INVALID_ARG;  // also rejects NaN
    }
  } else if (builtin_design_fixed(M, sg) != DGFS_OK) {
    return DGFS_ERR_INVALID_ARG;
  }
  for (int m = 0; m < M; ++m) {
    ws[m] = d->w_sigma ? d->w_sigma[m] : 4.0 * kPi / M;
    if (!std::isfinite(ws[m])) return DGFS_ERR_INVALID_ARG;
  }
  // radial truncation (Eq. domain, all pairs) and Gauss-Legendre rule
  double R = d->R;
  if (!(R > 0.0)) {
    double S = 1e300;
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) {
        const double cj = d->mass[j] / (d->mass[i] + d->mass[j]);
        const double den = std::fmax(4.0 * cj, 2.0) + std::sqrt(1.0 + d->mass[j] / d->mass[i]) + 1.0;
        S = std::fmin(S, 2.0 * d->L / den);
      }
    R = 2.0 * S;
  }
  double wr[kMaxRho];
  gauss_legendre_rule(NR, p.rho, wr);
  for (int q = 0; q < NR; ++q) {
    p.rho[q] = 0.5 * R * (p.rho[q] + 1.0);
    wr[q] *= 0.5 * R;
  }
  // kernel prefactors (Eq. NVSS unless overridden) and the weight constants per pair
  const double n3 = double(N) * N * N;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      const int o = i * s + j;
      const double mi = d->mass[i], mj = d->mass[j], om = d->omega[o];
      const double b = d->b_override ? d->b_override[o]
                                     : 1.0 / (std::sqrt(1.0 + mi / mj) * std::pow(mi * mj / (mi + mj), om - 0.5) *
                                              4.0 * std::tgamma(2.5 - om) * kPi);
      const double cj = mj / (mi + mj);
      for (int q = 0; q < NR; ++q) {
        const double rp = std::pow(p.rho[q], 4.0 - 2.0 * om);
        p.fpref[o][q] = float(wr[q] * 4.0 * kPi * b * rp / n3);
        p.fscale[o][q] = float(p.rho[q] * cj / d->L);
        p.gpref[o][q] = float(16.0 * kPi * kPi * b * wr[q] * rp);
      }
    }
  for (int q = 0; q < NR; ++q) p.gscale[q] = float(p.rho[q] / d->L);
  // tasks: unordered pairs with reuse when the rule is antipodal, else every ordered pair
  bool antipodal = true;
  for (int m = 0; m < M && antipodal; ++m) {
    bool found = false;
    for (int k = 0; k < M; ++k)
      if (std::fabs(sg[m][0] + sg[k][0]) < 1e-12 && std::fabs(sg[m][1] + sg[k][1]) < 1e-12 &&
          std::fabs(sg[m][2] + sg[k][2]) < 1e-12 && std::fabs(ws[m] - ws[k]) <= 1e-14 * std::fabs(ws[m]))
        found = true;
    antipodal = found;
  }
  int nt = 0, ne = 0, ng = 0;
  for (int i = 0; i < s; ++i)
    for (int j = antipodal ? i : 0; j < s; ++j) {
      int idx[kMaxM];
      double wt[kMaxM];
      int n = 0;
      for (int m = 0; m < M; ++m) {
        if (antipodal && i == j) {
          bool pos = true;
          for (int a = 0; a < 3; ++a) {
            if (sg[m][a] > 1e-12) { pos = true; break; }
            if (sg[m][a] < -1e-12) { pos = false; break; }
          }
          if (!pos) continue;
          idx[n] = m;
          wt[n++] = 2.0 * ws[m];
        } else {
          idx[n] = m;
          wt[n++] = ws[m];
        }
      }
      for (int a = 1; a < n; ++a)  // stable insertion sort by sigma_x
        for (int k = a; k > 0 && sg[idx[k]][0] < sg[idx[k - 1]][0] - 1e-12; --k) {
          const int ti = idx[k]; idx[k] = idx[k - 1]; idx[k - 1] = ti;
          const double tw = wt[k]; wt[k] = wt[k - 1]; wt[k - 1] = tw;
        }
      TaskDesc& tk = p.tasks[nt];
      tk.i = i;
      tk.j = j;
      tk.out0 = i * s + j;
      tk.out1 = (antipodal && i != j) ? j * s + i : -1;
      tk.ent_off = ne;
      tk.n_ent = n;
      tk.grp_off = ng;
      int first = 0;
      for (int e = 1; e <= n; ++e)
        if (e == n || std::fabs(sg[idx[e]][0] - sg[idx[first]][0]) > 1e-12) {
          p.groups[ng].first = first;
          p.groups[ng].count = e - first;
          ++ng;
          first = e;
        }
      tk.n_grp = ng - tk.grp_off;
      for (int e = 0; e < n; ++e) {
        p.ent_w[ne + e] = float(wt[e]);
        for (int a = 0; a < 3; ++a) p.ent_sigma[ne + e][a] = sg[idx[e]][a];
      }
      p.c[nt][0] = d->mass[i] / (d->mass[i] + d->mass[j]);
      p.c[nt][1] = d->mass[j] / (d->mass[i] + d->mass[j]);
      ne += n;
      ++nt;
    }
  p.s = s;
  p.n_tasks = nt;
  p.n_rho = NR;
  p.L = d->L;
  return DGFS_OK;
}

template <int N>
int launch_noalloc(const NoAllocParams& p, cudaStream_t st) {
  const int items = p.batch * p.n_tasks;
  const int grid = items < kSlots ? items : kSlots;
  collision_noalloc_kernel<N><<<grid, N * N, smem_bytes<N>(), st>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

}  // namespace
}  // namespace dgfs

extern "C" int dgfs_eval_collision_noalloc(const dgfs_plan_desc* desc, const void* f_dev, void* Q_dev, int batch,
                                           void* stream) {
  using namespace dgfs;
  if (!desc || batch < 0) return DGFS_ERR_INVALID_ARG;
  NoAllocParams p;
  const int rc = build_params(desc, p);
  if (rc != DGFS_OK) return rc;
  if (batch == 0) return DGFS_OK;
  if (!f_dev || !Q_dev || (reinterpret_cast<uintptr_t>(f_dev) & 15u) || (reinterpret_cast<uintptr_t>(Q_dev) & 15u))
    return DGFS_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DGFS_ERR_CUDA;
  float2* scratch = nullptr;
  const int src = setup_device(dev, &scratch);
  if (src != DGFS_OK) return src;
  p.f = static_cast<const float*>(f_dev);
  p.Q = static_cast<float*>(Q_dev);
  p.scratch = scratch;
  p.batch = batch;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (desc->N) {
    case 8: return launch_noalloc<8>(p, st);
    case 12: return launch_noalloc<12>(p, st);
    default: return launch_noalloc<16>(p, st);
  }
}
