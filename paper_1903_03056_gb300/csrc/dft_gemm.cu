// DGFS_BF16X3 collision path and the batched 3D DFT on the tensor cores.
//
// gemm_collision_kernel<N> evaluates the same steps as the FFT kernel (Sec. 4, the fast gain
// sum after Eq. GG and the loss convolution): per work item (node, task),
//   f_hat = N^-3 DFT3(f) of the task's species;
//   per radial node rho: for every entry (rho, sigma): a = IDFT3 of f_hat_i with the phase
//   e^{+i pi rho c_j k.sigma / L}, b = IDFT3 of f_hat_j with e^{-i pi rho c_i k.sigma / L},
//   P += w_sigma a b; then Q_hat^+ += w_rho F(k, rho) N^-3 DFT3(P) for (i,j) and, with the
//   antipodal reuse, (j,i);
//   Q_ij = Re IDFT3(Q_hat^+) - f_i Re IDFT3(G^- f_hat_j).
// Every 3D transform is three tensor-core passes (dft_gemm.cuh); the per-axis phase of a shifted
// transform is folded into that axis's matrix, precomputed per (task, rho, entry, role, axis).
// One CTA holds one work item at a time; its volumes between transforms (f_hat, a, the gain
// accumulators, the loss) live in a per-CTA workspace that stays in L2, the product sum P in
// tensor memory next to the pass output.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "dft_gemm.cuh"
#include "dgfs_internal.h"

namespace dgfs {

struct GemmParams {
  const float* f;            // [batch][s][N^3]
  float* Q;                  // [batch][s][s][N^3]
  int batch, s, n_tasks, n_rho, max_ent;
  const TaskDesc* tasks;
  const double* ent_w;
  const uint16_t* mats;      // matrix images: [task][rho][max_ent][role][axis], forward, inverse
  const float* Fw;           // [s*s][n_rho][N^3]: w_rho F / N^3
  const float* Gm;           // [s*s][N^3]: G^-
  float2* scratch;           // [CTAs][6][N^3] complex
  unsigned* work_counter;
  unsigned* status;
};

namespace {

// a CTA's volumes between transforms, in its workspace slot: f_hat_i, f_hat_j, the shifted
// f_i of the current entry, the two gain accumulators, the loss convolution
struct Vol {
  float2 *FI, *FJ, *AV, *QA, *QB;
  float* LS;
};

// One 3D transform: pass 1 from `src` (writes the A rows), passes 2 and 3 by transposes
// through shared memory, `epi` reads the result (thread t = row t of the last pass).
// XYZ: passes along x, y, z (orders kPX, kPY, kPZ); the result's rows are kPZ lines (x, y)
// with z along the columns.  ZYX: passes along z, y, x (kPZ, kPY2, kPX2); the result's rows
// are kPX2 lines (y, z) with x along the columns.  Each pass's matrix is copied in (bulk copy)
// while the previous pass runs.
template <int N, bool ZYX, class Src, class Epi>
__device__ __forceinline__ bool dft3(GemmCta<N>& cta, int t, const uint16_t* m0, const uint16_t* m1,
                                     const uint16_t* m2, Src&& src, Epi&& epi) {
  __syncthreads();  // workspace written by other threads' epilogues is read below
  cta.prefetch_matrix(m0, t);
  src(t);
  if (!cta.mma_pass(t, m1)) return false;
  if constexpr (ZYX) convert_pass<N, kPZ, kPY2>(cta, t); else convert_pass<N, kPX, kPY>(cta, t);
  if (!cta.mma_pass(t, m2)) return false;
  if constexpr (ZYX) convert_pass<N, kPY2, kPX2>(cta, t); else convert_pass<N, kPY, kPZ>(cta, t);
  if (!cta.mma_pass(t, nullptr)) return false;
  epi(t);
  return true;
}

// natural index x N^2 + y N of the line (y, z) of row t of the x pass (add x N^2 for a point)
template <int N>
__device__ __forceinline__ int px_base(int t) {
  int c[3];
  line_of<N, kPX>(t, c);
  return c[1] * N + c[2];
}
// natural index (x N + y) N of the line (x, y) of row t of the z pass (add z for a point)
template <int N>
__device__ __forceinline__ int pz_base(int t) {
  int c[3];
  line_of<N, kPZ>(t, c);
  return (c[0] * N + c[1]) * N;
}

// pass-1 source of an XYZ transform: the x line of row t of a volume in natural layout
// [x][y][z]; real (im = 0) or complex, optionally times a real table
template <int N>
__device__ __forceinline__ void src_real(const GemmCta<N>& cta, int t, const float* vol) {
  using G = GemmGeo<N>;
  if ((t & ~31) >= G::N2) return;
  const int o = px_base<N>(t);
  float v[G::K];
#pragma unroll
  for (int x = 0; x < N; ++x) {
    v[2 * x] = __ldg(vol + x * G::N2 + o);
    v[2 * x + 1] = 0.f;
  }
  cta.put_row(t, v);
}
template <int N>
__device__ __forceinline__ void src_cplx(const GemmCta<N>& cta, int t, const float2* vol, const float* g) {
  using G = GemmGeo<N>;
  if ((t & ~31) >= G::N2) return;
  const int o = px_base<N>(t);
  float v[G::K];
#pragma unroll
  for (int x = 0; x < N; ++x) {
    float2 c = vol[x * G::N2 + o];
    if (g) {
      const float s = __ldg(g + x * G::N2 + o);
      c.x *= s;
      c.y *= s;
    }
    v[2 * x] = c.x;
    v[2 * x + 1] = c.y;
  }
  cta.put_row(t, v);
}
// pass-1 source of a ZYX transform: row t of the product sum in tensor memory (kPZ order, the
// z pass's own order)
template <int N>
__device__ __forceinline__ void src_tmem(const GemmCta<N>& cta, int t) {
  using G = GemmGeo<N>;
  if ((t & ~31) >= G::N2) return;
  float v[G::K];
  const uint32_t ta = cta.lane_addr(t, 1);
#pragma unroll
  for (int ch = 0; ch < G::NN / 16; ++ch) {
    float c[16];
    tc::tmem_ld16(ta + uint32_t(16 * ch), c);
    tc::tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[16 * ch + i] = c[i];
  }
  cta.put_row(t, v);
}

// XYZ result, row t: hand each (natural index, re, im) of its z line to fn
template <int N, class Fn>
__device__ __forceinline__ void for_result(const GemmCta<N>& cta, int t, Fn&& fn) {
  using G = GemmGeo<N>;
  if ((t & ~31) >= G::N2) return;
  const uint32_t ta = cta.lane_addr(t, 0);
  const int o = pz_base<N>(t);
#pragma unroll 1
  for (int ch = 0; ch < G::NN / 16; ++ch) {
    float d[16];
    tc::tmem_ld16(ta + uint32_t(16 * ch), d);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) fn(o + 8 * ch + j, d[2 * j], d[2 * j + 1]);
  }
}

template <int N>
__device__ __forceinline__ void init_cta(GemmCta<N>& cta, unsigned char* smem, uint64_t* bar, uint64_t* bbar, int* abort_flag,
                                         unsigned* status, int t) {
  using G = GemmGeo<N>;
  cta.A = reinterpret_cast<uint16_t*>(smem);
  cta.B = cta.A + G::A_ELEMS;
  cta.bar = bar;
  cta.bbar = bbar;
  cta.abort_flag = abort_flag;
  cta.status = status;
  cta.phase = 0;
  cta.bphase = 0;
  cta.bsel = 0;
  if (t == 0) {
    *abort_flag = 0;
    tc::mbar_init(bar, 1);
    tc::mbar_init(&bbar[0], 1);
    tc::mbar_init(&bbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

template <int N>
__global__ void __launch_bounds__(GemmGeo<N>::THREADS, GemmGeo<N>::MINB) gemm_collision_kernel(const GemmParams p) {
  using G = GemmGeo<N>;
  constexpr int N2 = G::N2, N3 = G::N3;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t s_bar, s_bbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort, s_item;
  const int t = threadIdx.x;

  GemmCta<N> cta;
  init_cta<N>(cta, smem_raw, &s_bar, s_bbar, &s_abort, p.status, t);
  // padding rows of the A operand hold zeros (their outputs are never read)
  for (int i = t; i < G::A_ELEMS / 8; i += G::THREADS) reinterpret_cast<uint4*>(cta.A)[i] = make_uint4(0, 0, 0, 0);
  if (t < 32) {
    tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  cta.tmem = s_tmem;

  const int n_items = p.batch * p.n_tasks;
  const size_t img = size_t(G::B_ELEMS);
  const uint16_t* fwd = p.mats + size_t(p.n_tasks) * p.n_rho * p.max_ent * 6 * img;
  const uint16_t* inv = fwd + img;
  Vol V;
  float2* scr = p.scratch + size_t(blockIdx.x) * 6 * N3;
  V.FI = scr;
  V.FJ = scr + N3;
  V.AV = scr + 2 * N3;
  V.QA = scr + 3 * N3;
  V.QB = scr + 4 * N3;
  V.LS = reinterpret_cast<float*>(scr + 5 * N3);

  for (;;) {
    if (t == 0) s_item = int(atomicAdd(p.work_counter, 1u));
    __syncthreads();
    const int item = s_item;
    if (item >= n_items || s_abort) break;
    const int b = item / p.n_tasks;
    const int task = item % p.n_tasks;
    const TaskDesc tk = p.tasks[task];
    const float* fb = p.f + size_t(b) * p.s * N3;
    const int nspec = tk.i == tk.j ? 1 : 2;
    bool ok = true;

    // f_hat = N^-3 DFT3(f) of species i (and j)
    const float inv_n3 = 1.f / float(N3);
    for (int sp = 0; sp < nspec && ok; ++sp) {
      const float* fs = fb + size_t(sp == 0 ? tk.i : tk.j) * N3;
      float2* dst = sp == 0 ? V.FI : V.FJ;
      ok = dft3<N, false>(cta, t, fwd, fwd, fwd, [&](int tt) { src_real<N>(cta, tt, fs); },
                          [&](int tt) {
                            for_result<N>(cta, tt, [&](int idx, float re, float im) {
                              dst[idx] = make_float2(re * inv_n3, im * inv_n3);
                            });
                          });
    }
    const float2* FJs = nspec == 2 ? V.FJ : V.FI;

    // gain: radial nodes, entries
    for (int q = 0; q < p.n_rho && ok; ++q) {
      for (int e = 0; e < tk.n_ent && ok; ++e) {
        const float w = float(p.ent_w[tk.ent_off + e]);
        const uint16_t* ma = p.mats + ((size_t(task) * p.n_rho + q) * p.max_ent + e) * 6 * img;
        const uint16_t* mb = ma + 3 * img;
        // a: shifted f_i, kept in the workspace (line t of the result is written and read by thread t)
        ok = dft3<N, false>(cta, t, ma, ma + img, ma + 2 * img, [&](int tt) { src_cplx<N>(cta, tt, V.FI, nullptr); },
                            [&](int tt) {
                              for_result<N>(cta, tt, [&](int idx, float re, float im) { V.AV[idx] = make_float2(re, im); });
                            });
        if (!ok) break;
        // b: shifted f_j; P (+)= w a b in tensor memory
        const bool first = e == 0;
        ok = dft3<N, false>(cta, t, mb, mb + img, mb + 2 * img, [&](int tt) { src_cplx<N>(cta, tt, FJs, nullptr); },
                            [&](int tt) {
                              if ((tt & ~31) >= N2) return;
                              const uint32_t tD = cta.lane_addr(tt, 0), tP = cta.lane_addr(tt, 1);
                              const float2* a = V.AV + pz_base<N>(tt);
#pragma unroll 1
                              for (int ch = 0; ch < G::NN / 16; ++ch) {
                                float d[16], pv[16];
                                tc::tmem_ld16(tD + uint32_t(16 * ch), d);
                                if (!first) tc::tmem_ld16(tP + uint32_t(16 * ch), pv);
                                tc::tmem_wait_ld();
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                  const float2 av = a[8 * ch + j];
                                  const float pr = av.x * d[2 * j] - av.y * d[2 * j + 1];
                                  const float pi = av.x * d[2 * j + 1] + av.y * d[2 * j];
                                  pv[2 * j] = first ? w * pr : pv[2 * j] + w * pr;
                                  pv[2 * j + 1] = first ? w * pi : pv[2 * j + 1] + w * pi;
                                }
                                tc::tmem_st16(tP + uint32_t(16 * ch), pv);
                              }
                              tc::tmem_wait_st();
                            });
      }
      if (!ok) break;
      // Q_hat^+ (+)= w_rho F N^-3 DFT3(P) for (i,j) and the reused (j,i)
      ok = dft3<N, true>(cta, t, fwd, fwd, fwd, [&](int tt) { src_tmem<N>(cta, tt); },
                         [&](int tt) {
                           if ((tt & ~31) >= N2) return;
                           const uint32_t tD = cta.lane_addr(tt, 0);
                           int c[3];
                           line_of<N, kPX2>(tt, c);
                           const int o = c[1] * N + c[2];
#pragma unroll 1
                           for (int ch = 0; ch < G::NN / 16; ++ch) {
                             float d[16];
                             tc::tmem_ld16(tD + uint32_t(16 * ch), d);
                             tc::tmem_wait_ld();
#pragma unroll
                             for (int j = 0; j < 8; ++j) {
                               const int idx = (8 * ch + j) * N2 + o;  // (x, y, z) of the x line (y, z)
#pragma unroll
                               for (int o = 0; o < 2; ++o) {
                                 const int pair = o == 0 ? tk.out0 : tk.out1;
                                 if (pair < 0) break;
                                 const float fw = __ldg(p.Fw + (size_t(pair) * p.n_rho + q) * N3 + idx);
                                 float2* acc = o == 0 ? V.QA : V.QB;
                                 float2 val = make_float2(d[2 * j] * fw, d[2 * j + 1] * fw);
                                 if (q > 0) {
                                   const float2 old = acc[idx];
                                   val.x += old.x;
                                   val.y += old.y;
                                 }
                                 acc[idx] = val;
                               }
                             }
                           }
                         });
    }

    // finish: Q_ij = Re IDFT3(Q_hat^+) - f_i Re IDFT3(G^- f_hat_j), for (i,j) and (j,i)
    for (int o = 0; o < 2 && ok; ++o) {
      const int pair = o == 0 ? tk.out0 : tk.out1;
      if (pair < 0) break;
      const int io = o == 0 ? tk.i : tk.j;
      const int jo = o == 0 ? tk.j : tk.i;
      const float2* acc = o == 0 ? V.QA : V.QB;
      const float2* Fj = jo == tk.i ? V.FI : FJs;
      ok = dft3<N, false>(cta, t, inv, inv, inv, [&](int tt) { src_cplx<N>(cta, tt, Fj, p.Gm + size_t(pair) * N3); },
                          [&](int tt) { for_result<N>(cta, tt, [&](int idx, float re, float) { V.LS[idx] = re; }); });
      if (!ok) break;
      float* Qo = p.Q + ((size_t(b) * p.s + io) * p.s + jo) * N3;
      const float* fi = fb + size_t(io) * N3;
      ok = dft3<N, false>(cta, t, inv, inv, inv, [&](int tt) { src_cplx<N>(cta, tt, acc, nullptr); },
                          [&](int tt) {
                            for_result<N>(cta, tt, [&](int idx, float re, float) {
                              Qo[idx] = re - __ldg(fi + idx) * V.LS[idx];
                            });
                          });
    }
    if (!ok) break;
  }
  // release the tensor memory once no MMA of this CTA is in flight (each pass waited for its
  // MMAs, or gave up waiting: then the barrier is left behind with the CTA)
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(cta.tmem, G::TMEM_COLS);
}

// batched 3D DFT of complex volumes (XYZ passes, natural layout in and out)
template <int N>
__global__ void __launch_bounds__(GemmGeo<N>::THREADS, GemmGeo<N>::MINB)
    dft3_batch_kernel(const float2* x, float2* y, int count, const uint16_t* mat, unsigned* status) {
  using G = GemmGeo<N>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t s_bar, s_bbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int t = threadIdx.x;
  GemmCta<N> cta;
  init_cta<N>(cta, smem_raw, &s_bar, s_bbar, &s_abort, status, t);
  for (int i = t; i < G::A_ELEMS / 8; i += G::THREADS) reinterpret_cast<uint4*>(cta.A)[i] = make_uint4(0, 0, 0, 0);
  if (t < 32) {
    tc::tmem_alloc(&s_tmem, G::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  cta.tmem = s_tmem;
  for (int v = blockIdx.x; v < count; v += gridDim.x) {
    const float2* src = x + size_t(v) * G::N3;
    float2* dst = y + size_t(v) * G::N3;
    const bool ok = dft3<N, false>(cta, t, mat, mat, mat, [&](int tt) { src_cplx<N>(cta, tt, src, nullptr); },
                                   [&](int tt) {
                                     for_result<N>(cta, tt, [&](int idx, float re, float im) {
                                       dst[idx] = make_float2(re, im);
                                     });
                                   });
    if (!ok) break;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(cta.tmem, G::TMEM_COLS);
}

// One CTA waits, with the tensor-core kernels' bounded wait, on an mbarrier that nothing
// completes; the wait must give up after `limit_cycles` and report it in *status.
__global__ void bounded_wait_check_kernel(long long limit_cycles, unsigned* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = tc::mbar_wait_bounded(&bar, 0, limit_cycles);
  if (!ok && threadIdx.x == 0) atomicOr(status, 1u);
}

// ---- host: matrix images ---------------------------------------------------------------

constexpr double kPiD = 3.141592653589793238462643383279502884;

// round to the nearest BF16, ties to even (finite inputs)
uint16_t bf16_rn(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return uint16_t(u >> 16);
}
double bf16_value(uint16_t h) {
  const uint32_t u = uint32_t(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return double(f);
}

// Image of the line transform W (W[n_out * N + k_in], complex) as the B operand: the real form
// rows (2 n + ro) x columns (2 k + ri), each value split into three BF16 terms.
void matrix_image(int N, const std::complex<double>* W, uint16_t* img) {
  const int K = 2 * N, part = 2 * N * K;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      const double wr = W[n * N + k].real(), wi = W[n * N + k].imag();
      const double val[2][2] = {{wr, -wi}, {wi, wr}};  // [ro][ri]
      for (int ro = 0; ro < 2; ++ro)
        for (int ri = 0; ri < 2; ++ri) {
          double rem = val[ro][ri];
          const int at = op_index(2 * n + ro, 2 * k + ri, K);
          for (int s = 0; s < 3; ++s) {
            const uint16_t h = bf16_rn(float(rem));
            img[s * part + at] = h;
            rem -= bf16_value(h);
          }
        }
    }
}

// e^{dir 2 pi i n k / N} with the angle reduced exactly
std::complex<double> twiddle_host(long nk, int N, int dir) {
  const long m = ((nk % N) + N) % N;
  const double a = 2.0 * kPiD * double(m) / double(N);
  return std::complex<double>(std::cos(a), dir * std::sin(a));
}

int centred(int n, int N) { return n < N / 2 ? n : n - N; }

template <int N>
int configure_gemm_impl(Plan& p) {
  using G = GemmGeo<N>;
  auto kern = gemm_collision_kernel<N>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(G::SMEM)) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::THREADS, G::SMEM) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  // the CTAs of one SM share its 512 tensor-memory columns
  if (per_sm > 512 / G::TMEM_COLS) per_sm = 512 / G::TMEM_COLS;
  p.shape.cluster = 1;
  p.shape.groups = G::TILES;
  p.shape.threads = G::THREADS;
  p.shape.smem = G::SMEM;
  p.shape.phase_smem = 0;
  p.shape.clusters = sms * per_sm;
  p.scratch_bytes = size_t(p.shape.clusters) * 6 * G::N3 * sizeof(float2);
  return DGFS_OK;
}

template <int N>
int launch_gemm_impl(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws) {
  using G = GemmGeo<N>;
  GemmParams kp;
  kp.f = static_cast<const float*>(f);
  kp.Q = static_cast<float*>(Q);
  kp.batch = batch;
  kp.s = p.s;
  kp.n_tasks = int(p.tasks.size());
  kp.n_rho = p.N_rho;
  kp.max_ent = p.max_ent;
  kp.tasks = p.d_tasks;
  kp.ent_w = p.d_ent_w;
  kp.mats = p.d_mats;
  kp.Fw = p.d_Fwf;
  kp.Gm = p.d_Gmf;
  kp.scratch = static_cast<float2*>(p.scratch_of(ws));
  kp.work_counter = p.counter_of(ws);
  kp.status = p.counter_of(ws) + 1;
  const int items = batch * kp.n_tasks;
  int limit = int(p.shape.clusters * p.shape.share);
  if (limit < 1) limit = 1;
  const int grid = items < limit ? items : limit;
  if (cudaMemsetAsync(kp.work_counter, 0, sizeof(unsigned), st) != cudaSuccess) return DGFS_ERR_CUDA;
  gemm_collision_kernel<N><<<grid, G::THREADS, G::SMEM, st>>>(kp);
  return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
}

template <int N>
int dft3_impl(int dir, const void* x, void* y, int count, cudaStream_t st) {
  using G = GemmGeo<N>;
  std::vector<std::complex<double>> W(size_t(N) * N);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) W[size_t(n) * N + k] = twiddle_host(long(n) * k, N, dir);
  std::vector<uint16_t> img(G::B_ELEMS);
  matrix_image(N, W.data(), img.data());
  void* d = nullptr;
  const size_t bytes = img.size() * sizeof(uint16_t) + 256;
  if (cudaMallocAsync(&d, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_OOM;
  }
  unsigned* status = reinterpret_cast<unsigned*>(static_cast<char*>(d) + img.size() * sizeof(uint16_t));
  int rc = DGFS_OK;
  int sms = 0, dev = 0;
  if (cudaMemcpyAsync(d, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaFuncSetAttribute(dft3_batch_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(G::SMEM)) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    rc = DGFS_ERR_CUDA;
  } else {
    const int grid = count < sms ? count : sms;
    dft3_batch_kernel<N><<<grid, G::THREADS, G::SMEM, st>>>(static_cast<const float2*>(x), static_cast<float2*>(y),
                                                               count, static_cast<const uint16_t*>(d), status);
    if (cudaPeekAtLastError() != cudaSuccess) rc = DGFS_ERR_CUDA;
  }
  unsigned host_status = 0;
  if (rc == DGFS_OK &&
      (cudaMemcpyAsync(&host_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = DGFS_ERR_CUDA;
  cudaFreeAsync(d, st);
  if (rc != DGFS_OK) cudaGetLastError();
  if (rc == DGFS_OK && host_status != 0) rc = DGFS_ERR_DEVICE_TIMEOUT;
  return rc;
}

}  // namespace

bool gemm_supported_n(int N) { return N == 8 || N == 16 || N == 24; }

size_t gemm_image_elems(int N) {
  switch (N) {
    case 8: return GemmGeo<8>::B_ELEMS;
    case 16: return GemmGeo<16>::B_ELEMS;
    default: return GemmGeo<24>::B_ELEMS;
  }
}

// Matrix images of a DGFS_BF16X3 plan: every shifted transform's per-axis matrix
// W[n][k] = e^{+2 pi i n k / N} ph(k), ph the plan's phase factor of (task, rho, entry, role,
// axis), then the plain forward (e^{-2 pi i n k / N}) and inverse matrices.
void build_gemm_images(const Plan& p, const std::vector<std::complex<double>>& phase, std::vector<uint16_t>& out) {
  const int N = p.N;
  const size_t img = gemm_image_elems(N);
  const int NT = int(p.tasks.size());
  const size_t n_ph = size_t(NT) * p.N_rho * p.max_ent * 6;
  out.assign((n_ph + 2) * img, 0);
  std::vector<std::complex<double>> W(size_t(N) * N);
  for (size_t m = 0; m < n_ph; ++m) {
    const std::complex<double>* ph = &phase[m * N];
    if (ph[0] == std::complex<double>(0.0, 0.0)) continue;  // an entry slot the task does not use
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < N; ++k) W[size_t(n) * N + k] = twiddle_host(long(n) * k, N, +1) * ph[k];
    matrix_image(N, W.data(), &out[m * img]);
  }
  for (int dir = -1; dir <= 1; dir += 2) {
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < N; ++k) W[size_t(n) * N + k] = twiddle_host(long(n) * k, N, dir);
    matrix_image(N, W.data(), &out[(n_ph + (dir < 0 ? 0 : 1)) * img]);
  }
}

int configure_bf16x3(Plan& p) {
  switch (p.N) {
    case 8: return configure_gemm_impl<8>(p);
    case 16: return configure_gemm_impl<16>(p);
    case 24: return configure_gemm_impl<24>(p);
    default: return DGFS_ERR_UNSUPPORTED_N;
  }
}

int launch_bf16x3(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws) {
  switch (p.N) {
    case 8: return launch_gemm_impl<8>(p, f, Q, batch, st, ws);
    case 16: return launch_gemm_impl<16>(p, f, Q, batch, st, ws);
    case 24: return launch_gemm_impl<24>(p, f, Q, batch, st, ws);
    default: return DGFS_ERR_UNSUPPORTED_N;
  }
}

}  // namespace dgfs

extern "C" int dgfs_check_bounded_wait(double seconds) {
  if (!(seconds > 0.0) || seconds > 10.0) return DGFS_ERR_INVALID_ARG;
  int dev = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  unsigned* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_OOM;
  }
  unsigned host = 0;
  int rc = DGFS_OK;
  const long long cycles = (long long)(seconds * double(khz) * 1e3);
  if (cudaMemset(d, 0, sizeof(unsigned)) != cudaSuccess) rc = DGFS_ERR_CUDA;
  if (rc == DGFS_OK) {
    dgfs::bounded_wait_check_kernel<<<1, 32>>>(cycles, d);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&host, d, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = DGFS_ERR_CUDA;
  }
  cudaFree(d);
  if (rc != DGFS_OK) return rc;
  return host != 0 ? DGFS_ERR_DEVICE_TIMEOUT : DGFS_OK;
}

extern "C" int dgfs_dft3_bf16x3(int N, int dir, const void* x_dev, void* y_dev, int count, void* stream) {
  if (count < 0 || (dir != 1 && dir != -1)) return DGFS_ERR_INVALID_ARG;
  if (!dgfs::gemm_supported_n(N)) return DGFS_ERR_UNSUPPORTED_N;
  if (count == 0) return DGFS_OK;
  if (!x_dev || !y_dev || (reinterpret_cast<uintptr_t>(x_dev) & 15u) || (reinterpret_cast<uintptr_t>(y_dev) & 15u))
    return DGFS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (N) {
    case 8: return dgfs::dft3_impl<8>(dir, x_dev, y_dev, count, st);
    case 16: return dgfs::dft3_impl<16>(dir, x_dev, y_dev, count, st);
    default: return dgfs::dft3_impl<24>(dir, x_dev, y_dev, count, st);
  }
}
