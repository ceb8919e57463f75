// Persistent collision kernel: one thread-block cluster per work item (node b, task).
//
// For a task (i, j) the cluster evaluates, for every radial node rho_q (Sec. 4):
//
//   step A  pencil pass along x: for the entries of one sigma_x group, the spectra
//           f_hat_i e^{+i pi rho c_j k_x sigma_x / L} and f_hat_j e^{-i pi rho c_i k_x sigma_x / L}
//           are inverse-transformed along x (the x phase is shared by the group);
//   step B  plane pass over (y, z): per entry, the y and z phases are applied, the inverse
//           transforms along y and z finish a_e and b_e on the plane, and
//           P += w_e a_e b_e accumulates in registers (entries with the previous entry's
//           sigma_y reuse its y pass where a third plane buffer fits); after the last group
//           P is transformed forward along z and y;
//   step C  pencil pass along x: forward transform of P, then Q_hat^+_(ij) += w_rho F^(ij) P_hat
//           (and Q_hat^+_(ji) += w_rho F^(ji) P_hat for a cross pair).
//
// then finishes Q_ij = Re IFFT(Q_hat^+_ij) - f_i Re IFFT(G^(ij)- f_hat_j) (the loss
// convolution of Sec. 4) and writes it.  The 3D transforms are split into a pencil pass
// (x, strided by N^2) and a plane pass (y, z, contiguous), each line transformed in the
// registers of one thread; the planes of a volume are spread over the cluster's CTAs and the
// pencils likewise, with cluster barriers between passes.  The volumes live in a per-cluster
// workspace accessed through L2 only; when the workspaces of all resident clusters exceed L2
// (N >= 24) part of them streams through HBM, and each plane is prefetched into L2 one read
// ahead of its use.
#pragma once

#include <cuda_runtime.h>

#include "dgfs_internal.h"
#include "fft_line.cuh"
#include "tcgen05.cuh"

namespace dgfs {

// compile-time launch shape per (precision, N): cluster size, plane groups per CTA, CTAs per SM
template <typename T, int N> struct Shape;
#define DGFS_SHAPE3(TT, NN, CC, GG, MB)                              \
  template <> struct Shape<TT, NN> {                                 \
    static constexpr int cluster = CC;                               \
    static constexpr int groups = GG;                                \
    static constexpr int min_blocks = MB;                            \
  };
#define DGFS_SHAPE(TT, NN, CC, GG) DGFS_SHAPE3(TT, NN, CC, GG, 1)
#include "tuned_shapes.h"
#undef DGFS_SHAPE
#undef DGFS_SHAPE3

template <typename T, int N>
struct Geo {
  static constexpr int N2 = N * N;
  static constexpr int N3 = N * N * N;
  static constexpr int PITCH = N + 1;  // padded smem row (complex elements)
  // P accumulates in registers when a second line of N complex values still fits (FP32 up to
  // N = 48: ~50 bytes of spills there, and one plane buffer per group less; measured 8-10 %
  // faster than P in shared memory at N = 48)
  static constexpr bool PREG = (sizeof(T) == 4 && N <= 48) || N <= 16;
  static constexpr int CL = Shape<T, N>::cluster;
  static constexpr int GP = Shape<T, N>::groups;
  static constexpr int MINB = Shape<T, N>::min_blocks;  // CTAs per SM the registers are sized for
  static constexpr int THREADS = GP * N;
  static constexpr int PLANES = N / CL;       // planes per CTA
  static constexpr int PENCILS = N2 / CL;     // pencils per CTA
  static_assert(PLANES % GP == 0, "planes must split evenly over plane groups");
  static_assert(N2 % CL == 0, "pencils must split evenly over the cluster");
  static constexpr size_t BUF = size_t(N) * PITCH * sizeof(C<T>);  // one padded plane
  // CTAs an SM holds at once: the register budget's count, or two when a CTA of at most 128
  // threads (at up to 256 registers each) and two plane buffers per group leave room
  static constexpr int RES =
      MINB > 1 ? MINB : (THREADS <= 128 && 2 * (GP * 2 * BUF + 1024) <= 228 * 1024 ? 2 : 1);
  // y-pass sharing: entries of a group with equal sigma_y reuse the y pass of both shifted
  // volumes, kept in a transpose buffer per role; needs P in registers and a third buffer per
  // group that still leaves RES CTAs per SM with 8 KB for the z phases.  Measured on the
  // 8192-node N = 16 batch: FP32 -4 %, FP64 -11 %; at N = 24 and 32 the third buffer takes
  // the room of the phase block and of L1 and the kernel ran 5-8 % slower, so it stays off.
  static constexpr bool YSH = N <= 16 && PREG && RES * (GP * 3 * BUF + 1024 + 8 * 1024) <= 228 * 1024;
  // Tensor-memory accumulators: the sigma sum P of each of a group's planes and the role-0 line
  // a_e live in TMEM columns (2N FP32 columns per line) instead of registers and shared memory,
  // which leaves the registers to the line transform and keeps P on chip across the sigma_x
  // groups of a radial node.  FP32, groups of one whole warp and at most 128 threads (each
  // thread owns one TMEM lane), and the allocations of the CTAs an SM holds within its 512
  // columns.
  static constexpr int PPG = PLANES / GP;  // planes per group
  static constexpr int TM_COLS = 2 * N * (PPG + 1);
  static constexpr int TM_ALLOC =
      TM_COLS <= 32 ? 32 : TM_COLS <= 64 ? 64 : TM_COLS <= 128 ? 128 : TM_COLS <= 256 ? 256 : 512;
  static constexpr bool TM = sizeof(T) == 4 && N % 32 == 0 && THREADS <= 128 && !YSH &&
                             TM_COLS <= 512 && RES * TM_ALLOC <= 512;
  // smem planes per plane group: transpose (role 0), a, then P (!PREG) or the role-1 transpose;
  // with TMEM accumulators the transpose buffer only
  static constexpr int NBUF = TM ? 1 : (PREG && !YSH) ? 2 : 3;
  static constexpr size_t SMEM = size_t(GP) * NBUF * BUF;
  // L2 prefetch of the workspace reads (measured: a gain from N = 24 on, where the clusters'
  // workspaces together exceed L2; a loss at N = 16); bulk prefetches need whole 16-byte rows
  static constexpr bool PF = N >= 24 && (PENCILS * sizeof(C<T>)) % 16 == 0;
  // staged plane pass (step B): the two plane buffers of a group take turns receiving the next
  // shifted plane by a bulk copy, issued one (entry, role) ahead of its use, so the plane's
  // L2/HBM latency overlaps the transforms of the previous role instead of stalling the loads
  // (P in registers, no y-pass sharing or TMEM accumulators, N >= 24; a plane is a whole
  // number of 16-byte rows)
  static constexpr bool STAGE = !TM && PREG && !YSH && N >= 24 && (N2 * sizeof(C<T>)) % 16 == 0 && (BUF % 16) == 0;
  // Buffers of the shifted-volume pair: three for clusters of several CTAs, whose VHS phases
  // split the cluster barrier (a CTA arrives when its step A is written and waits at the end
  // of the phase, so a CTA may still read pair k-1 while another writes pair k+1), two otherwise.
  // Measured at N = 32: 2-CTA clusters 2.6 % faster with the split; the TMEM shape (8-CTA
  // clusters) as fast without it, and the third buffer raised its DRAM traffic from 28 to 45 GB
  // per 288-node launch (L2 hit rate 86 % -> 74 %), so TMEM shapes keep two.
  static constexpr int NBV = CL > 1 && !TM ? 3 : 2;
  // workspace volumes per cluster: f_hat_i, f_hat_j, the NBV pairs of shifted volumes, two P
  // volumes (the second used by the VSS pipeline), two gain accumulators
  static constexpr int SLOT = 2 + 2 * NBV + 4;
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// the two halves of the cluster barrier (CL > 1)
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int CL>
__device__ __forceinline__ void cluster_sync() {
  if constexpr (CL == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}

// read an int in the shared memory of the cluster's rank-0 CTA (distributed shared memory)
__device__ __forceinline__ int ld_rank0(const int* local) {
  const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(local));
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(remote) : "r"(addr));
  int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(remote) : "memory");
  return v;
}

// workspace loads/stores go to L2 only: the data is written by other SMs of the cluster
template <typename T> __device__ __forceinline__ C<T> ld2(const C<T>* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void st2(C<T>* p, C<T> v) { __stcg(p, v); }

// Hint that [p, p + bytes) (16-byte aligned, a multiple of 16 bytes) is read soon: one bulk
// prefetch into L2, so the loads that follow meet L2 rather than DRAM latency.  The workspace
// of all clusters exceeds L2, so a volume written in one phase is partly evicted before it is
// read in the next.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Order this thread's generic-proxy accesses to global memory before later async-proxy (bulk
// copy) accesses: the workspace planes are written with ordinary stores and read back by bulk
// copies after a barrier.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}


// Barrier of one plane group.  A group of N threads that divides a warp lives inside one warp
// and synchronises only that warp.  Otherwise SG = lcm(N, 32) / N consecutive groups form a
// warp-aligned super-group that synchronises on its own named barrier (ids 1, 2, ...), so
// super-groups run independently; when the groups of a CTA do not split into super-groups
// the CTA barrier is used (every group then runs the same control flow).
constexpr int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }

template <int N, int GP>
struct GroupSync {
  static constexpr int LCM = N / gcd_int(N, 32) * 32;
  static constexpr int SG = LCM / N;  // plane groups per super-group
  static constexpr bool WARP = N <= 32 && 32 % N == 0;
  static constexpr bool NAMED = !WARP && GP % SG == 0 && GP / SG <= 15;
};

template <int N, int GP>
__device__ __forceinline__ void group_sync() {
  using S = GroupSync<N, GP>;
  if constexpr (S::WARP) {
    __syncwarp();
  } else if constexpr (S::NAMED) {
    const int sg = int(threadIdx.x) / S::LCM;
    asm volatile("bar.sync %0, %1;" ::"r"(1 + sg), "n"(S::LCM) : "memory");
  } else {
    __syncthreads();
  }
}

// transpose a plane held as column t (x[r] = V[r][t]) into row t (x[c] = V[t][c]) and back
template <typename T, int N, int GP>
__device__ __forceinline__ void cols_to_rows(C<T> (&x)[N], C<T>* tb, int t) {
  constexpr int P = N + 1;
#pragma unroll
  for (int r = 0; r < N; ++r) tb[r * P + t] = x[r];
  group_sync<N, GP>();
#pragma unroll
  for (int c = 0; c < N; ++c) x[c] = tb[t * P + c];
  group_sync<N, GP>();
}
template <typename T, int N, int GP>
__device__ __forceinline__ void rows_to_cols(C<T> (&x)[N], C<T>* tb, int t) {
  constexpr int P = N + 1;
#pragma unroll
  for (int c = 0; c < N; ++c) tb[t * P + c] = x[c];
  group_sync<N, GP>();
#pragma unroll
  for (int r = 0; r < N; ++r) x[r] = tb[r * P + t];
  group_sync<N, GP>();
}

// A line of N complex FP32 values in 2N consecutive TMEM columns of the thread's lane (16
// columns per access; every thread of the warp takes part).  The load waits for its data inside
// the same asm statement, so no use of the registers can move ahead of the wait.
__device__ __forceinline__ void tm_ld16w(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
template <int N>
__device__ __forceinline__ void tm_store_line(uint32_t ta, const C<float> (&v)[N]) {
#pragma unroll
  for (int ch = 0; ch < N / 8; ++ch) {
    float f[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      f[2 * j] = v[8 * ch + j].x;
      f[2 * j + 1] = v[8 * ch + j].y;
    }
    tc::tmem_st16(ta + uint32_t(16 * ch), f);
  }
}
template <int N>
__device__ __forceinline__ void tm_load_line(uint32_t ta, C<float> (&v)[N]) {
#pragma unroll
  for (int ch = 0; ch < N / 8; ++ch) {
    float f[16];
    tm_ld16w(ta + uint32_t(16 * ch), f);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[8 * ch + j] = mk<float>(f[2 * j], f[2 * j + 1]);
  }
}

// v[r] *= ph[r] for a phase array of N complex values.  Every phase array starts on a multiple
// of N complex values (N even), so FP32 phases can be read two at a time with 16-byte loads
// (broadcast reads: the arrays are the same for every thread of a group).  Measured: 1.3 % and
// 0.8 % faster at N = 24 and 16; at N = 32 and 48 the line transform's register allocation
// came out 2-3 % slower, so there the phases are read one at a time.
template <typename T, int N>
__device__ __forceinline__ void mul_phases(C<T> (&v)[N], const C<T>* ph) {
  if constexpr (sizeof(T) == 4 && N % 2 == 0 && N <= 24) {
#pragma unroll
    for (int r = 0; r < N; r += 2) {
      const float4 q = *reinterpret_cast<const float4*>(ph + r);
      v[r] = cmul<T>(v[r], mk<T>(q.x, q.y));
      v[r + 1] = cmul<T>(v[r + 1], mk<T>(q.z, q.w));
    }
  } else {
#pragma unroll
    for (int r = 0; r < N; ++r) v[r] = cmul<T>(v[r], ph[r]);
  }
}

// Two-pass transform of a plane: the first line pass, the transpose (columns to rows when
// COLS_FIRST, rows to columns otherwise), an optional per-element phase, the second line pass.
// For N >= 32 the passes run as a two-trip loop over one copy of the unrolled line transform,
// which keeps the kernel's instruction footprint small (measured: +3% at N = 32 and 48); the
// smaller transforms are faster unrolled.
template <typename T, int N, int GP, int DIR, bool COLS_FIRST>
__device__ __forceinline__ void plane_pass2(C<T> (&v)[N], C<T>* tb, int t, const C<T>* ph2) {
  auto between = [&]() {
    if constexpr (COLS_FIRST) cols_to_rows<T, N, GP>(v, tb, t); else rows_to_cols<T, N, GP>(v, tb, t);
    if (ph2 != nullptr) mul_phases<T, N>(v, ph2);
  };
  if constexpr (N >= 32) {
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) between();
      fft_line<T, N, DIR>(v);
    }
  } else {
    fft_line<T, N, DIR>(v);
    between();
    fft_line<T, N, DIR>(v);
  }
}

template <typename T, int N>
__device__ __forceinline__ const C<T>* phase_ptr(const KernelParams& p, int task, int q, int e,
                                                  int role, int axis) {
  const C<T>* ph = reinterpret_cast<const C<T>*>(p.phase);
  return ph + ((((size_t(task) * p.n_rho + q) * p.max_ent + e) * 2 + role) * 3 + axis) * N;
}

template <typename T, int N>
__global__ void __launch_bounds__(Geo<T, N>::THREADS, Geo<T, N>::MINB) collision_kernel(const KernelParams p) {
  using G = Geo<T, N>;
  using CT = C<T>;
  constexpr int N2 = G::N2, N3 = G::N3, CL = G::CL, GP = G::GP, NT = G::THREADS;
  constexpr int PITCH = G::PITCH;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int grp = tid / N;  // plane group
  const int t = tid % N;    // line within the plane group
  CT* tb = reinterpret_cast<CT*>(smem_raw) + size_t(grp) * G::NBUF * N * PITCH;
  CT* ab = tb + N * PITCH;
  CT* pb = ab + N * PITCH;  // used only when !PREG
  CT* const tbB = pb;       // used only when YSH: transpose buffer of role 1
  // phase block of the current (task, rho): [entry][role][axis][N], when staged in smem
  CT* const phs = reinterpret_cast<CT*>(smem_raw) + size_t(GP) * G::NBUF * N * PITCH;
  // phase block in shared memory: 1 = all axes, 2 = the z phases only (YSH shapes, where the
  // x and y phases are read once per group or per unshared entry)
  const bool ph_smem = p.phase_smem != 0;
  const bool ph_zonly = G::YSH && p.phase_smem == 2;

  const int rank = CL == 1 ? 0 : int(cluster_rank());
  const int cid = blockIdx.x / CL;
  CT* scr = reinterpret_cast<CT*>(p.scratch) + size_t(cid) * G::SLOT * N3;
  CT* const FI = scr;
  CT* const FJ = scr + N3;
  CT* const HA0 = scr + 2 * N3;               // shifted volumes of role 0: HA0 + b N^3
  CT* const HB0 = scr + (2 + G::NBV) * N3;    // and of role 1
  CT* const PV = scr + (2 + 2 * G::NBV) * N3;
  CT* const PV1 = PV + N3;
  CT* const QA = PV + 2 * N3;
  CT* const QB = PV + 3 * N3;
  const bool vss = p.vss != 0;
  const int plane0 = rank * G::PLANES;
  const int pencil0 = rank * G::PENCILS;
  const T inv_n3 = T(1) / T(N3);

  // Work items (node, task) are taken from a counter: thread 0 of the rank-0 CTA takes the
  // next item and the cluster reads it from that CTA's shared memory after a cluster barrier,
  // so clusters that start late (other kernels holding SMs) find no work left instead of
  // owning a share of it.  The value for the next item is taken after the first barrier of
  // the current one, when every CTA has read the current value.
  __shared__ int s_next_item;
  const int n_items = p.batch * p.n_tasks;

  // Staged plane pass: one mbarrier per plane buffer of each group (tb = buffer 0, ab =
  // buffer 1), armed by the group's first thread for one bulk copy of N^2 complex values.
  // Every thread of the group keeps the same bookkeeping: fill_par bit b is the parity of
  // buffer b's next completion, fill_out bit b a copy in flight.  A wait gives up after about
  // a second: the status word beside the work counter records it, and the group stops issuing
  // and waiting (its results are then invalid, which the status reports).
  __shared__ __align__(8) uint64_t s_fill[2 * GP];
  unsigned fill_par = 0, fill_out = 0;
  bool stalled = false;
  if constexpr (G::STAGE) {
    if (tid == 0) {
      for (int b = 0; b < 2 * GP; ++b) tc::mbar_init(&s_fill[b], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  // start a bulk copy of the plane at src into buffer bi (called by every thread of the group
  // after the buffer's last readers have passed a group barrier behind a proxy fence)
  auto fill = [&](int bi, const CT* src) {
    if (stalled) return;
    if (t == 0) {
      uint64_t* bar = &s_fill[2 * grp + bi];
      tc::mbar_expect_tx(bar, unsigned(N2 * sizeof(CT)));
      tc::bulk_g2s(bi ? ab : tb, src, unsigned(N2 * sizeof(CT)), bar);
    }
    fill_out |= 1u << bi;
  };
  auto wait_fill = [&](int bi) {
    if (stalled) return;
    if (tc::mbar_wait_bounded(&s_fill[2 * grp + bi], (fill_par >> bi) & 1u, 2000000000LL)) {
      fill_par ^= 1u << bi;
      fill_out &= ~(1u << bi);
    } else {
      stalled = true;
      atomicOr(p.work_counter + 1, 2u);
    }
  };

  // TMEM accumulators: warp 0 allocates the CTA's columns; thread t of warp w reaches lane
  // 32 (w % 4) + t
  __shared__ uint32_t s_tmem;
  uint32_t tm_row = 0;
  if constexpr (G::TM) {
    if (tid < 32) {
      tc::tmem_alloc(&s_tmem, G::TM_ALLOC);
      tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tm_row = s_tmem + (uint32_t(32 * ((tid / 32) & 3)) << 16);
  }

  if (rank == 0 && tid == 0) s_next_item = int(atomicAdd(p.work_counter, 1u));
  cluster_sync<CL>();
  for (int item = CL == 1 ? s_next_item : ld_rank0(&s_next_item); item < n_items;
       item = CL == 1 ? s_next_item : ld_rank0(&s_next_item)) {
    const int b = item / p.n_tasks;
    const int task = item % p.n_tasks;
    const TaskDesc tk = p.tasks[task];
    const T* fb = reinterpret_cast<const T*>(p.f) + size_t(b) * p.s * N3;
    const int nspec = tk.j == tk.i ? 1 : 2;

    // ---- step 0: Fourier coefficients f_hat = N^-3 FFT(f) of species i (and j) ----------
    for (int xl = grp; xl < G::PLANES; xl += GP) {
      const int x = plane0 + xl;
      for (int sp = 0; sp < nspec; ++sp) {
        const T* src = fb + size_t(sp == 0 ? tk.i : tk.j) * N3 + size_t(x) * N2;
        CT v[N];
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = mk<T>(__ldg(src + t * N + c), T(0));
        plane_pass2<T, N, GP, -1, false>(v, tb, t, nullptr);
        CT* dst = (sp == 0 ? FI : FJ) + size_t(x) * N2;
#pragma unroll
        for (int r = 0; r < N; ++r) st2<T>(dst + r * N + t, v[r]);
      }
    }
    cluster_sync<CL>();
    if (rank == 0 && tid == 0) s_next_item = int(atomicAdd(p.work_counter, 1u));
    for (int u = tid; u < nspec * G::PENCILS; u += NT) {
      const int sp = u / G::PENCILS;
      const int pp = pencil0 + u % G::PENCILS;
      CT* vol = sp == 0 ? FI : FJ;
      CT v[N];
#pragma unroll
      for (int n = 0; n < N; ++n) v[n] = ld2<T>(vol + n * N2 + pp);
      fft_line<T, N, -1>(v);
#pragma unroll
      for (int n = 0; n < N; ++n) st2<T>(vol + n * N2 + pp, scale<T>(v[n], inv_n3));
    }
    cluster_sync<CL>();
    const CT* FJs = nspec == 2 ? FJ : FI;

    // ---- gain: radial nodes, sigma_x groups, entries ----------------------------------------
    // Phase k runs step A of group k (into buffer k&1) and step B of group k-1 (from buffer
    // (k-1)&1); one cluster barrier per phase, n_grp + 1 phases per radial node.  With VSS
    // every group is one entry whose product is transformed forward on its own: step B of
    // entry k-1 writes P volume (k-1)&1 and step C of entry k-2 weights P volume (k-2)&1 by
    // F(k, rho, sigma) in the same phase (n_grp + 2 phases).
    for (int q = 0; q < p.n_rho; ++q) {
      const CT* const phq = phase_ptr<T, N>(p, task, q, 0, 0, 0);
      if (ph_zonly) {
        for (int u = tid; u < tk.n_ent * 2 * N; u += NT) phs[u] = __ldg(phq + ((u / N) * 3 + 2) * N + u % N);
        __syncthreads();
      } else if (ph_smem) {
        for (int u = tid; u < tk.n_ent * 6 * N; u += NT) phs[u] = __ldg(phq + u);
        __syncthreads();
      }
      const CT* const phb = ph_smem && !ph_zonly ? phs : phq;  // x and y phases
      const int n_phase = tk.n_grp + (vss ? 2 : 1);
      // Split cluster barrier (VHS, CL > 1): the CTA arrives once its step A of the phase is
      // written and waits at the end of the phase, so its step B covers the other CTAs' lag.
      // Pair k is written in phase k and read in phase k + 1, so with three buffers the pair
      // written in phase k + 1 is one that no CTA reads after arriving in phase k.  The VSS
      // pipeline's step B writes P volumes other CTAs read in the next phase: one full barrier.
      const bool split = G::NBV == 3 && !vss;
      const int nbv = split ? 3 : 2;
      for (int k = 0; k < n_phase; ++k) {
        if constexpr (G::STAGE) {
          // step B of this phase starts on planes written before the last cluster barrier:
          // copy the first entry's two planes now, so that they land during step A
          if (k > 0 && k <= tk.n_grp) {
            fence_proxy_async_global();
            tc::fence_async_smem();
            group_sync<N, GP>();
            const size_t x0 = size_t(plane0 + grp) * N2;
            fill(0, HA0 + size_t((k - 1) % nbv) * N3 + x0);
            fill(1, HB0 + size_t((k - 1) % nbv) * N3 + x0);
          }
        }
        if (k < tk.n_grp) {
          const GroupDesc gd = p.groups[tk.grp_off + k];
          CT* const dA = HA0 + size_t(k % nbv) * N3;
          CT* const dB = HB0 + size_t(k % nbv) * N3;
          // step A: x-pencils with the group's shared x phase.  The CTA's pencils of f_hat_i
          // and f_hat_j are N rows of PENCILS contiguous elements each; prefetch them first.
          if constexpr (G::PF) {
            for (int u = tid; u < 2 * N; u += NT)
              prefetch_l2((u < N ? FI : FJs) + size_t(u % N) * N2 + pencil0, G::PENCILS * sizeof(CT));
          }
          for (int u = tid; u < 2 * G::PENCILS; u += NT) {
            const int role = u / G::PENCILS;
            const int pp = pencil0 + u % G::PENCILS;
            const CT* src = role == 0 ? FI : FJs;
            const CT* ph = phb + ((gd.first * 2 + role) * 3 + 0) * N;
            CT v[N];
#pragma unroll
            for (int n = 0; n < N; ++n) v[n] = ld2<T>(src + n * N2 + pp);
            mul_phases<T, N>(v, ph);
            fft_line<T, N, +1>(v);
            CT* dst = role == 0 ? dA : dB;
#pragma unroll
            for (int n = 0; n < N; ++n) st2<T>(dst + n * N2 + pp, v[n]);
          }
          // the next phase reads these planes with bulk copies
          if constexpr (G::STAGE) fence_proxy_async_global();
        }
        if constexpr (CL > 1) {
          if (split && k < tk.n_grp) cluster_arrive();
        }
        if (G::STAGE && k > 0 && k <= tk.n_grp) {
          const int gi = k - 1;
          const GroupDesc gd = p.groups[tk.grp_off + gi];
          const CT* const sA = HA0 + size_t(gi % nbv) * N3;
          const CT* const sB = HB0 + size_t(gi % nbv) * N3;
          const bool last = vss || gi == tk.n_grp - 1;
          const bool fresh = vss || gi == 0;
          CT* const PVw = (vss && (gi & 1)) ? PV1 : PV;
          const int e_end = gd.first + gd.count;
          // staged step B.  Role 0 of an entry reads buffer `cur` and leaves a_e in it; role 1
          // reads the other buffer.  After role 1's transpose its buffer takes the next
          // entry's role-0 plane; after the product, `cur` takes the next entry's role-1 plane.
          // Every entry of the group reads the same two planes (the x pass is shared).
          int cur = 0;
          for (int xl = grp; xl < G::PLANES; xl += GP) {
            const int x = plane0 + xl;
            CT P[N];
#pragma unroll
            for (int c = 0; c < N; ++c) P[c] = fresh ? mk<T>(0, 0) : ld2<T>(PV + x * N2 + c * N + t);
            for (int e = gd.first; e < e_end; ++e) {
              const T w = T(p.ent_w[tk.ent_off + e]);
              CT v[N];
#pragma unroll 1
              for (int role = 0; role < 2; ++role) {
                const int bi = role == 0 ? cur : 1 - cur;
                CT* const B = bi ? ab : tb;
                const CT* phy = phb + ((e * 2 + role) * 3 + 1) * N;
                const CT* phz = phb + ((e * 2 + role) * 3 + 2) * N;
                wait_fill(bi);
                // column t of the plane as copied (unpadded rows), with the y phase
#pragma unroll
                for (int r = 0; r < N; ++r) v[r] = B[r * N + t];
                mul_phases<T, N>(v, phy);
                group_sync<N, GP>();  // every column read: the buffer is re-laid out in place
#pragma unroll 1
                for (int pass = 0; pass < 2; ++pass) {
                  if (pass == 1) {
#pragma unroll
                    for (int r = 0; r < N; ++r) B[r * PITCH + t] = v[r];
                    group_sync<N, GP>();
#pragma unroll
                    for (int c = 0; c < N; ++c) v[c] = B[t * PITCH + c];
                    mul_phases<T, N>(v, phz);
                    if (role == 1) {
                      // the buffer is free: the next entry's role-0 plane
                      const CT* nxt = e + 1 < e_end ? sA + size_t(x) * N2
                                    : xl + GP < G::PLANES ? sA + size_t(x + GP) * N2 : nullptr;
                      tc::fence_async_smem();
                      group_sync<N, GP>();
                      if (nxt != nullptr) fill(bi, nxt);
                    }
                  }
                  fft_line<T, N, +1>(v);
                }
                if (role == 0) {
#pragma unroll
                  for (int c = 0; c < N; ++c) B[t * PITCH + c] = v[c];
                }
              }
              const CT* A0 = cur ? ab : tb;
#pragma unroll
              for (int c = 0; c < N; ++c) {
                const CT ab_ = cmul<T>(A0[t * PITCH + c], v[c]);
                P[c] = mk<T>(P[c].x + w * ab_.x, P[c].y + w * ab_.y);
              }
              if (e + 1 < e_end) {
                tc::fence_async_smem();
                group_sync<N, GP>();
                fill(cur, sB + size_t(x) * N2);
              }
              cur = 1 - cur;
            }
            // the last entry's role-0 buffer (1 - cur) is free once every row has been read
            CT* const Pb = cur ? tb : ab;
            if (last) {
              plane_pass2<T, N, GP, -1, false>(P, Pb, t, nullptr);
#pragma unroll
              for (int r = 0; r < N; ++r) st2<T>(PVw + x * N2 + r * N + t, P[r]);
            } else {
#pragma unroll
              for (int c = 0; c < N; ++c) st2<T>(PV + x * N2 + c * N + t, P[c]);
            }
            if (xl + GP < G::PLANES) {
              tc::fence_async_smem();
              group_sync<N, GP>();
              fill(1 - cur, sB + size_t(x + GP) * N2);
            }
          }
        } else if (k > 0 && k <= tk.n_grp) {
          const int gi = k - 1;
          const GroupDesc gd = p.groups[tk.grp_off + gi];
          const CT* const sA = HA0 + size_t(gi % nbv) * N3;
          const CT* const sB = HB0 + size_t(gi % nbv) * N3;
          // step B: (y, z) planes
          const bool last = vss || gi == tk.n_grp - 1;
          const bool fresh = vss || gi == 0;
          CT* const PVw = (vss && (gi & 1)) ? PV1 : PV;
          // each plane is prefetched one (plane, entry, role) read ahead of its use
          constexpr bool PF = G::PF;
          if (PF && t == 0) prefetch_l2(sA + size_t(plane0 + grp) * N2, N2 * sizeof(CT));
          for (int xl = grp; xl < G::PLANES; xl += GP) {
            const int x = plane0 + xl;
            // TMEM columns of this plane's P and of a_e (TMEM accumulators)
            const uint32_t tp = tm_row + uint32_t(((xl - grp) / GP) * 2 * N);
            const uint32_t ta = tm_row + uint32_t(G::PPG * 2 * N);
            CT P[G::PREG && !G::TM ? N : 1];
            if constexpr (G::TM) {
              // P stays in TMEM from the first group of the radial node to the last
            } else if constexpr (G::PREG) {
#pragma unroll
              for (int c = 0; c < N; ++c) P[c] = fresh ? mk<T>(0, 0) : ld2<T>(PV + x * N2 + c * N + t);
            } else {
#pragma unroll
              for (int c = 0; c < N; ++c) pb[t * PITCH + c] = fresh ? mk<T>(0, 0) : ld2<T>(PV + x * N2 + c * N + t);
            }
            for (int e = gd.first; e < gd.first + gd.count; ++e) {
              const T w = T(p.ent_w[tk.ent_off + e]);
              // with YSH, an entry whose sigma_y equals the previous entry's in the group reads
              // the y pass of both volumes back from the role's transpose buffer
              const bool reuse = G::YSH && e > gd.first && p.ent_ysh[tk.ent_off + e] != 0;
              CT v[N];
              for (int role = 0; role < 2; ++role) {
                const CT* vol = (role == 0 ? sA : sB) + size_t(x) * N2;
                const CT* phy = phb + ((e * 2 + role) * 3 + 1) * N;
                const CT* phz = ph_zonly ? phs + (e * 2 + role) * N : phb + ((e * 2 + role) * 3 + 2) * N;
                if (PF && t == 0 && !reuse) {
                  // next plane read: the other role, the next entry that does not reuse, or
                  // the group's next plane
                  const CT* nxt = nullptr;
                  if (role == 0) {
                    nxt = sB + size_t(x) * N2;
                  } else {
                    int en = e + 1;
                    if constexpr (G::YSH) {
                      while (en < gd.first + gd.count && p.ent_ysh[tk.ent_off + en] != 0) ++en;
                    }
                    if (en < gd.first + gd.count) nxt = sA + size_t(x) * N2;
                    else if (xl + GP < G::PLANES) nxt = sA + size_t(x + GP) * N2;
                  }
                  if (nxt != nullptr) prefetch_l2(nxt, N2 * sizeof(CT));
                }
                if constexpr (G::YSH) {
                  CT* const yb = role == 0 ? tb : tbB;
                  constexpr int P_ = PITCH;
                  if (!reuse) {
#pragma unroll
                    for (int r = 0; r < N; ++r) v[r] = ld2<T>(vol + r * N + t);
                    mul_phases<T, N>(v, phy);
                  }
                  // pass 0: y transform of the column (skipped on reuse); pass 1: z transform
                  // of row t read back from the role's buffer, with the entry's z phase
#pragma unroll 1
                  for (int pass = reuse ? 1 : 0; pass < 2; ++pass) {
                    if (pass == 1) {
                      if (!reuse) {
                        group_sync<N, GP>();  // the previous rows of yb have been read
#pragma unroll
                        for (int r = 0; r < N; ++r) yb[r * P_ + t] = v[r];
                        group_sync<N, GP>();
                      }
#pragma unroll
                      for (int c = 0; c < N; ++c) v[c] = yb[t * P_ + c];
                      mul_phases<T, N>(v, phz);
                    }
                    fft_line<T, N, +1>(v);
                  }
                } else {
#pragma unroll
                  for (int r = 0; r < N; ++r) v[r] = ld2<T>(vol + r * N + t);
                  mul_phases<T, N>(v, phy);
                  plane_pass2<T, N, GP, +1, true>(v, tb, t, phz);
                }
                if (role == 0) {
                  if constexpr (G::TM) {
                    __syncwarp();
                    tm_store_line<N>(ta, v);
                  } else {
#pragma unroll
                    for (int c = 0; c < N; ++c) ab[t * PITCH + c] = v[c];
                  }
                }
              }
              if constexpr (G::TM) {
                // P += w a_e b_e in chunks of 8 values (the first entry of the radial node's first
                // group writes P)
                const bool p_first = fresh && e == gd.first;
                __syncwarp();
                tc::tmem_wait_st();
#pragma unroll
                for (int ch = 0; ch < N / 8; ++ch) {
                  float a16[16], p16[16];
                  tm_ld16w(ta + uint32_t(16 * ch), a16);
                  if (!p_first) tm_ld16w(tp + uint32_t(16 * ch), p16);
#pragma unroll
                  for (int j = 0; j < 8; ++j) {
                    const CT ab_ = cmul<T>(mk<T>(a16[2 * j], a16[2 * j + 1]), v[8 * ch + j]);
                    // one rounding per update, as P + w ab in registers (P = 0 at the start)
                    p16[2 * j] = fmaf(w, ab_.x, p_first ? 0.f : p16[2 * j]);
                    p16[2 * j + 1] = fmaf(w, ab_.y, p_first ? 0.f : p16[2 * j + 1]);
                  }
                  tc::tmem_st16(tp + uint32_t(16 * ch), p16);
                }
              } else if constexpr (G::PREG) {
#pragma unroll
                for (int c = 0; c < N; ++c) {
                  const CT a = ab[t * PITCH + c];
                  const CT ab_ = cmul<T>(a, v[c]);
                  P[c] = mk<T>(P[c].x + w * ab_.x, P[c].y + w * ab_.y);
                }
              } else {
#pragma unroll
                for (int c = 0; c < N; ++c) {
                  const CT a = ab[t * PITCH + c];
                  const CT ab_ = cmul<T>(a, v[c]);
                  const CT o = pb[t * PITCH + c];
                  pb[t * PITCH + c] = mk<T>(o.x + w * ab_.x, o.y + w * ab_.y);
                }
              }
            }
            if (last) {
              CT v[N];
              if constexpr (G::TM) {
                __syncwarp();
                tc::tmem_wait_st();
                tm_load_line<N>(tp, v);
              } else {
#pragma unroll
                for (int c = 0; c < N; ++c) {
                  if constexpr (G::PREG) v[c] = P[c]; else v[c] = pb[t * PITCH + c];
                }
              }
              plane_pass2<T, N, GP, -1, false>(v, tb, t, nullptr);
#pragma unroll
              for (int r = 0; r < N; ++r) st2<T>(PVw + x * N2 + r * N + t, v[r]);
            } else if constexpr (!G::TM) {
#pragma unroll
              for (int c = 0; c < N; ++c) {
                CT val;
                if constexpr (G::PREG) val = P[c]; else val = pb[t * PITCH + c];
                st2<T>(PV + x * N2 + c * N + t, val);
              }
            }
          }
        }
        if (vss && k >= 2) {
          // step C (VSS) of entry k-2: forward x transform, Q_hat^+ += F(k, rho, sigma) P_hat;
          // for a halved self pair F(sigma) + F(-sigma), for the reused (j,i) pair F^(ji)(-sigma)
          const int e = k - 2;
          const CT* const PVr = (e & 1) ? PV1 : PV;
          const int c0 = p.ent_m[2 * (tk.ent_off + e)], c1 = p.ent_m[2 * (tk.ent_off + e) + 1];
          const bool self_sum = tk.i == tk.j && c1 >= 0;
          const bool first = q == 0 && e == 0;
          for (int u = tid; u < G::PENCILS; u += NT) {
            const int pp = pencil0 + u;
            CT v[N];
#pragma unroll
            for (int n = 0; n < N; ++n) v[n] = ld2<T>(PVr + n * N2 + pp);
            fft_line<T, N, -1>(v);
            for (int o = 0; o < 2; ++o) {
              const int pair = o == 0 ? tk.out0 : tk.out1;
              if (pair < 0) break;
              // slot code of this output's direction: 2 slot + 1 when the slot holds the
              // antipode's weight (read conjugated)
              const int code = o == 0 ? c0 : c1;
              const size_t fo = ((size_t(pair) * p.n_rho + q) * p.n_fslot + (code >> 1)) * N3;
              const T sgn = (code & 1) ? T(-1) : T(1);
              CT* acc = o == 0 ? QA : QB;
              if constexpr (sizeof(T) == 4) {
                // FP32 table; a self pair's slot already holds F(sigma) + F(-sigma)
                const float2* F0 = static_cast<const float2*>(p.Fv) + fo;
#pragma unroll
                for (int n = 0; n < N; ++n) {
                  const float2 fw = __ldg(F0 + n * N2 + pp);
                  CT val = cmul<T>(v[n], mk<T>(fw.x, sgn * fw.y));
                  if (!first) val = add<T>(val, ld2<T>(acc + n * N2 + pp));
                  st2<T>(acc + n * N2 + pp, val);
                }
              } else {
                const double2* F0 = static_cast<const double2*>(p.Fv) + fo;
#pragma unroll
                for (int n = 0; n < N; ++n) {
                  double2 fw = __ldg(F0 + n * N2 + pp);
                  // a halved self pair takes F(sigma) + F(-sigma) = F + conj F
                  fw = self_sum ? make_double2(fw.x + fw.x, 0.0) : make_double2(fw.x, sgn * fw.y);
                  CT val = cmul<T>(v[n], mk<T>(T(fw.x), T(fw.y)));
                  if (!first) val = add<T>(val, ld2<T>(acc + n * N2 + pp));
                  st2<T>(acc + n * N2 + pp, val);
                }
              }
            }
          }
        }
        if constexpr (CL > 1) {
          if (split && k < tk.n_grp) cluster_wait(); else cluster_sync<CL>();
        } else {
          cluster_sync<CL>();
        }
      }
      if (vss) continue;
      // step C: forward transform of P along x, weight, accumulate
      for (int u = tid; u < G::PENCILS; u += NT) {
        const int pp = pencil0 + u;
        CT v[N];
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = ld2<T>(PV + n * N2 + pp);
        fft_line<T, N, -1>(v);
        for (int o = 0; o < 2; ++o) {
          const int pair = o == 0 ? tk.out0 : tk.out1;
          if (pair < 0) break;
          // the table is in the plan's real type (FP32 plans: rounded once at plan creation)
          const T* Fw = static_cast<const T*>(p.Fw) + (size_t(pair) * p.n_rho + q) * N3;
          CT* acc = o == 0 ? QA : QB;
#pragma unroll
          for (int n = 0; n < N; ++n) {
            const T fw = __ldg(Fw + n * N2 + pp);
            CT val = scale<T>(v[n], fw);
            if (q > 0) val = add<T>(val, ld2<T>(acc + n * N2 + pp));
            st2<T>(acc + n * N2 + pp, val);
          }
        }
      }
    }
    __syncthreads();

    // ---- finish: Q_ij = Re IFFT(Q_hat^+) - f_i Re IFFT(G^- f_hat_j) --------------------------
    for (int o = 0; o < 2; ++o) {
      const int pair = o == 0 ? tk.out0 : tk.out1;
      if (pair < 0) break;
      const int io = o == 0 ? tk.i : tk.j;
      const int jo = o == 0 ? tk.j : tk.i;
      const CT* acc = o == 0 ? QA : QB;
      const CT* Fj = jo == tk.i ? FI : FJs;
      const T* Gm = static_cast<const T*>(p.Gm) + size_t(pair) * N3;
      for (int u = tid; u < G::PENCILS; u += NT) {
        const int pp = pencil0 + u;
        CT v[N];
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = ld2<T>(acc + n * N2 + pp);
        fft_line<T, N, +1>(v);
#pragma unroll
        for (int n = 0; n < N; ++n) st2<T>(HA0 + n * N2 + pp, v[n]);
#pragma unroll
        for (int n = 0; n < N; ++n) v[n] = scale<T>(ld2<T>(Fj + n * N2 + pp), __ldg(Gm + n * N2 + pp));
        fft_line<T, N, +1>(v);
#pragma unroll
        for (int n = 0; n < N; ++n) st2<T>(HB0 + n * N2 + pp, v[n]);
      }
      cluster_sync<CL>();
      T* Qout = reinterpret_cast<T*>(p.Q) + ((size_t(b) * p.s + io) * p.s + jo) * N3;
      const T* fi = fb + size_t(io) * N3;
      for (int xl = grp; xl < G::PLANES; xl += GP) {
        const int x = plane0 + xl;
        CT v[N];
        T gain[N];
#pragma unroll
        for (int r = 0; r < N; ++r) v[r] = ld2<T>(HA0 + x * N2 + r * N + t);
        plane_pass2<T, N, GP, +1, true>(v, tb, t, nullptr);
#pragma unroll
        for (int c = 0; c < N; ++c) gain[c] = v[c].x;
#pragma unroll
        for (int r = 0; r < N; ++r) v[r] = ld2<T>(HB0 + x * N2 + r * N + t);
        plane_pass2<T, N, GP, +1, true>(v, tb, t, nullptr);
        // row t of this plane; stage through shared memory for a coalesced store
        T* rb = reinterpret_cast<T*>(tb);
#pragma unroll
        for (int c = 0; c < N; ++c) rb[t * PITCH + c] = gain[c] - __ldg(fi + x * N2 + t * N + c) * v[c].x;
        group_sync<N, GP>();
#pragma unroll
        for (int r = 0; r < N; ++r) Qout[x * N2 + r * N + t] = rb[r * PITCH + t];
        group_sync<N, GP>();
      }
      cluster_sync<CL>();
    }
  }
  // a group that gave up waiting lets its copies in flight land (bounded) before it leaves
  if constexpr (G::STAGE) {
    if (stalled && t == 0) {
      for (int b = 0; b < 2; ++b)
        if ((fill_out >> b) & 1u) tc::mbar_wait_bounded(&s_fill[2 * grp + b], (fill_par >> b) & 1u, 2000000000LL);
    }
  }
  if constexpr (G::TM) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(s_tmem, G::TM_ALLOC);
  }
  // no CTA leaves while another may still read its shared memory (the last item index)
  if constexpr (CL > 1) cluster_sync<CL>();
}

// ------------------------------------------------------------------------------------------
template <typename T, int N>
int configure_impl(Plan& pl) {
  using G = Geo<T, N>;
  auto kern = collision_kernel<T, N>;
  // stage the phase block of the current (task, rho) in shared memory when it fits
  // (with YSH: only while the SM still holds G::RES CTAs with it)
  const size_t ph_bytes = size_t(pl.max_ent) * 6 * N * sizeof(C<T>);
  // (with YSH: only while the SM still holds G::RES CTAs with it, else the z phases only)
  const size_t z_bytes = size_t(pl.max_ent) * 2 * N * sizeof(C<T>);
  int ph_mode = 0;
  if (G::YSH) {
    if (G::RES * (G::SMEM + ph_bytes + 1024) <= size_t(228) * 1024) ph_mode = 1;
    else if (G::RES * (G::SMEM + z_bytes + 1024) <= size_t(228) * 1024) ph_mode = 2;
  } else if (G::MINB * (G::SMEM + ph_bytes) <= size_t(200) * 1024) {
    ph_mode = 1;
  }
  const size_t smem = G::SMEM + (ph_mode == 1 ? ph_bytes : ph_mode == 2 ? z_bytes : 0);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return DGFS_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(G::CL);
  cfg.blockDim = dim3(G::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters <= 0) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  if constexpr (G::TM) {
    // The CTAs an SM can hold by the built kernel's registers, shared memory and threads must
    // stay within the TMEM columns: a CTA that could not allocate would wait inside its
    // cluster.  (The launch bounds size the registers for RES CTAs, whose allocations fit; a
    // build with fewer registers could let more in.)
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return DGFS_ERR_CUDA;
    const int warps = (G::THREADS + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_warp > 0 ? 65536 / (regs_warp * warps) : 32;
    const int by_smem = int(size_t(228) * 1024 / (smem + fa.sharedSizeBytes + 1024));
    int most = 2048 / G::THREADS;
    if (by_regs < most) most = by_regs;
    if (by_smem < most) most = by_smem;
    if (most < 1 || most * G::TM_ALLOC > 512) return DGFS_ERR_CUDA;
    // The occupancy calculator grants a kernel that allocates tensor memory one CTA per SM; the
    // device co-schedules `most`.  Clusters beyond what it places wait, and the work counter
    // leaves them the items still open when they start.
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return DGFS_ERR_CUDA;
    const int cap = most * sms / G::CL;
    if (cap > clusters) clusters = cap;
  }
  pl.shape.cluster = G::CL;
  pl.shape.groups = G::GP;
  pl.shape.threads = G::THREADS;
  pl.shape.smem = smem;
  pl.shape.phase_smem = ph_mode;
  pl.shape.clusters = clusters;
  pl.scratch_bytes = size_t(clusters) * G::SLOT * G::N3 * sizeof(C<T>);
  return DGFS_OK;
}

template <typename T, int N>
int launch_impl(const Plan& pl, const void* f, void* Q, int batch, cudaStream_t st, int ws) {
  using G = Geo<T, N>;
  KernelParams kp;
  kp.f = f;
  kp.Q = Q;
  kp.batch = batch;
  kp.s = pl.s;
  kp.n_tasks = int(pl.tasks.size());
  kp.n_rho = pl.N_rho;
  kp.max_ent = pl.max_ent;
  kp.tasks = pl.d_tasks;
  kp.groups = pl.d_groups;
  kp.ent_w = pl.d_ent_w;
  kp.phase = pl.d_phase;
  kp.Fw = pl.d_Fwf ? static_cast<const void*>(pl.d_Fwf) : static_cast<const void*>(pl.d_Fw);
  kp.Gm = pl.d_Gmf ? static_cast<const void*>(pl.d_Gmf) : static_cast<const void*>(pl.d_Gm);
  kp.scratch = pl.scratch_of(ws);
  kp.phase_smem = pl.shape.phase_smem;
  kp.work_counter = pl.counter_of(ws);
  kp.vss = pl.vss ? 1 : 0;
  kp.n_fslot = pl.n_fslot;
  kp.Fv = pl.d_Fvf ? static_cast<const void*>(pl.d_Fvf) : static_cast<const void*>(pl.d_Fv);
  kp.ent_m = pl.d_ent_m;
  kp.ent_ysh = pl.d_ent_ysh;
  const int items = batch * kp.n_tasks;
  int limit = int(pl.shape.clusters * pl.shape.share);
  if (limit < 1) limit = 1;
  const int clusters = items < limit ? items : limit;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(clusters * G::CL);
  cfg.blockDim = dim3(G::THREADS);
  cfg.dynamicSmemBytes = pl.shape.smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaMemsetAsync(kp.work_counter, 0, sizeof(unsigned), st) != cudaSuccess) return DGFS_ERR_CUDA;
  if (cudaLaunchKernelEx(&cfg, collision_kernel<T, N>, kp) != cudaSuccess) return DGFS_ERR_CUDA;
  return DGFS_OK;
}

#define DGFS_DISPATCH(T, N_, CALL) \
  switch (N_) {                    \
    case 4: return CALL(T, 4);     \
    case 6: return CALL(T, 6);     \
    case 8: return CALL(T, 8);     \
    case 12: return CALL(T, 12);   \
    case 16: return CALL(T, 16);   \
    case 24: return CALL(T, 24);   \
    case 32: return CALL(T, 32);   \
    case 48: return CALL(T, 48);   \
    default: return DGFS_ERR_UNSUPPORTED_N; \
  }

}  // namespace dgfs
