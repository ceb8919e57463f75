// Internal plan and kernel-parameter structures shared by the host plan builder, the
// kernel launchers and the C ABI.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "dgfs.h"

namespace dgfs {

// One unit of gain work: the product sum P_rho(v) = sum_e w_e a_e(v) b_e(v) over the entries
// e of the task, where a_e is f_i shifted by +rho c_j sigma_e and b_e is f_j shifted by
// -rho c_i sigma_e (Sec. 4, the gain formula after Eq. GG).  out0 = i*s+j always receives
// F^(ij) P_hat; out1 = j*s+i (or -1) receives F^(ji) P_hat, which is exact when the sphere
// rule is antipodal with equal weights on antipodes, since then P^(ji) = P^(ij).
struct TaskDesc {
  int i, j;
  int out0, out1;
  int ent_off, n_ent;  // entries (sigma, weight) of this task
  int grp_off, n_grp;  // groups of entries sharing sigma_x
};

struct GroupDesc {
  int first, count;  // entry range within the task, all with the same sigma_x
};

struct KernelParams {
  const void* f;          // [batch][s][N^3] real
  void* Q;                // [batch][s][s][N^3] real
  int batch, s, n_tasks, n_rho, max_ent;
  const TaskDesc* tasks;
  const GroupDesc* groups;
  const double* ent_w;    // [entries] sigma weight (x2 for halved self pairs)
  const void* phase;      // complex: [task][rho][max_ent][role 2][axis 3][N]
  const void* Fw;         // [s*s][n_rho][N^3]: w_rho F^(ij)(k, rho) / N^3, in the plan's real
                          // type (FP32 plans: each FP64 value rounded once)
  const void* Gm;         // [s*s][N^3]: G^(ij)-(k), in the plan's real type
  void* scratch;          // complex: [clusters][SLOT][N^3]
  int phase_smem;         // 1: the task's phase block of the current rho is staged in smem;
                          // 2: only its z phases are
  unsigned* work_counter; // next work item (reset to 0 before every launch)
  // VSS (alpha != 1): sigma-dependent complex gain weights, one forward transform per entry
  int vss;
  int n_fslot;            // table slots per (pair, rho): M, or M / 2 with an antipodal design
  const void* Fv;         // [s*s][n_rho][n_fslot][N^3]: w_rho F^(ij)(k, rho, sigma) / N^3,
                          // complex in the plan's real type; with an antipodal design a slot
                          // holds the direction of lower index, its antipode reads it
                          // conjugated, and in FP32 plans a self pair's slots hold
                          // F(sigma) + F(-sigma) = 2 Re F(sigma) (summed in FP64)
  const int* ent_m;       // [entries][2]: slot code (2 slot + conjugation bit) of the entry's
                          // direction and of its antipode (-1: none); a self pair's entry with
                          // an antipode takes F(sigma) + F(-sigma)
  const int* ent_ysh;     // [entries]: 1 when the entry has the previous entry's sigma_x and
                          // sigma_y (same group), so both its shifted volumes share that
                          // entry's x and y passes
};

// Conservation projection of one self pair (rows = 5) or one stacked cross pair (rows = 6):
// constraint rows built from the grid, (C C^T)^-1 precomputed in FP64 on the host.
struct ConsBlock {
  int i, j, rows;
  double a, b;        // m_i w_ij and m_j w_ji (cross pairs), w = 1 / b_ij
  double minv[36];    // (C C^T)^-1, row-major rows x rows
};

struct LaunchShape {
  int cluster = 1;        // CTAs cooperating on one work item
  int groups = 1;         // plane groups per CTA
  int threads = 0;        // groups * N
  size_t smem = 0;        // dynamic shared memory per CTA
  int phase_smem = 0;     // phases staged in shared memory
  int clusters = 0;       // resident clusters (persistent grid)
  double share = 1.0;     // fraction of the resident clusters one launch may use
};

struct Plan {
  int device = 0;
  cudaStream_t home = nullptr;     // the plan's own stream: table builds, stream-ordered alloc/free
  cudaEvent_t last_eval = nullptr; // recorded after every evaluation
  cudaStream_t last_stream = nullptr;  // the stream of that evaluation
  bool has_eval = false;
  int N = 0;
  double L = 0;
  int s = 0;
  int M = 0;
  int N_rho = 0;
  double R = 0;
  int precision = DGFS_FP64;
  // f and Q in float: the FP32 path and the split-BF16 tensor-core path
  bool f32io() const { return precision != DGFS_FP64; }
  unsigned flags = 0;
  int max_batch = 0;
  std::vector<double> mass, omega, alpha, b, sigma, w_sigma, rho, w_rho;
  std::vector<double> pair_R;            // [s*s] radial truncation of every ordered pair
  std::vector<double> rho_p, w_rho_p;    // [s*s][N_rho] radial rule of every ordered pair

  std::vector<TaskDesc> tasks;
  std::vector<GroupDesc> groups;
  std::vector<double> ent_w;
  std::vector<int> ent_sigma;   // design index of each entry
  std::vector<int> ent_m;       // [entries][2] VSS table slot codes of the entry and its antipode
  std::vector<int> fslot;       // [M] VSS table slot code of each direction: 2 slot + conj bit
  int n_fslot = 0;              // slots per (pair, rho) of the VSS table
  int n_t = 64;                 // points of the VSS gain weight's Gauss-Jacobi rule in t
  double vss_a_max = 0;         // largest argument pi rho c_j |k| / L of that table
  bool vss_grid = false;        // the table was built from the grid of Phi_alpha(p, q)
  bool antipodal = false;       // every direction has an antipode of equal weight
  std::vector<int> ent_ysh;     // [entries] shares the previous entry's y pass
  int max_ent = 0;
  bool vss = false;             // some alpha_ij != 1

  std::vector<double> kappa;       // species-sum weights [s*s]
  std::vector<ConsBlock> cons;     // conservation blocks (DGFS_CONSERVE)

  // device tables
  ConsBlock* d_cons = nullptr;
  double* d_kappa = nullptr;
  void* d_Qfull = nullptr;         // full operators staged for DGFS_SUM_SPECIES
  double* d_Fw = nullptr;
  double2* d_Fv = nullptr;         // VSS gain weights (complex)
  float* d_Fwf = nullptr;          // FP32 plans: the gain and loss tables the kernel reads
  float2* d_Fvf = nullptr;
  float* d_Gmf = nullptr;
  int* d_ent_m = nullptr;
  int* d_ent_ysh = nullptr;
  double* d_Gm = nullptr;
  double* d_ent_w = nullptr;
  void* d_phase = nullptr;
  TaskDesc* d_tasks = nullptr;
  GroupDesc* d_groups = nullptr;
  size_t table_bytes = 0;

  // workspace
  LaunchShape shape;
  void* d_scratch = nullptr;       // kGuardBytes into d_scratch_raw
  void* d_scratch_raw = nullptr;   // guard | workspace | guard
  static constexpr size_t kGuardBytes = 4096;
  static constexpr unsigned char kGuardByte = 0xA5;
  unsigned* d_counter = nullptr;   // work-item counter of the persistent kernel; the next word is
                                   // the device status (set when a bounded device wait gave up)
  uint16_t* d_mats = nullptr;      // DGFS_BF16X3: line-transform matrix images (split BF16)
  // second workspace and work counter (allocated by the first host-buffer call): consecutive
  // chunks of a host-buffer evaluation alternate between the two, on two streams, so that one
  // chunk's kernel starts while the previous one finishes its last work items
  void* d_scratch2_raw = nullptr;
  void* d_scratch2 = nullptr;
  unsigned* d_counter2 = nullptr;
  cudaStream_t eval2 = nullptr;
  void* scratch_of(int ws) const { return ws == 0 ? d_scratch : d_scratch2; }
  unsigned* counter_of(int ws) const { return ws == 0 ? d_counter : d_counter2; }
  size_t scratch_bytes = 0;
  void* d_rk = nullptr;             // SSP-RK2 workspace: f1 and the right-hand side
  void* d_stage_f = nullptr;
  void* d_stage_Q = nullptr;
  int stage_batch = 0;
  int last_launches = 0;
  // host-buffer pipeline: copy streams and per-chunk events
  cudaStream_t h2d = nullptr, d2h = nullptr;
  static constexpr int kMaxChunks = 8;
  cudaEvent_t ev_h2d[kMaxChunks] = {}, ev_done[kMaxChunks] = {}, ev_start = nullptr;
};

size_t real_size(const Plan& p);

// NVTX range over a scope of host code (plan construction, evaluation stages): shown by
// profilers on the CPU timeline and usable as a kernel filter (ncu --nvtx); a no-op without
// an attached tool
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// host plan construction (plan.cpp)
// Gauss-Legendre rule of n points on [-1, 1] into the caller's arrays (no allocation)
void gauss_legendre_rule(int n, double* x, double* w);
int build_plan(const dgfs_plan_desc* d, Plan& p);
int upload_plan(Plan& p);
void free_plan(Plan& p);

// kernel configuration and launch, per precision (collision_f32.cu / collision_f64.cu)
int configure_f32(Plan& p);
int configure_f64(Plan& p);
int launch_f32(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws = 0);
int launch_f64(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws = 0);

// on-device FP64 weight tables on the plan's stream (tables.cu)
int launch_vhs_tables(Plan& p, const double* d_fcoef, const double* d_gcoef, const double* d_gscale, int n_loss);
int launch_loss_table(Plan& p, const double* d_gcoef, const double* d_gscale, int n_loss);
// FP32 copies of the gain tables (d_Fwf from d_Fw, or d_Fvf from d_Fv; self_sum: the self
// pairs' slots take F(sigma) + conj F(sigma), the sum their halved entries read)
int launch_gain_tables_f32(Plan& p, int self_sum);
// FP32 copy of an FP64 table (each value rounded once)
int launch_to_f32(const Plan& p, const double* src, float* dst, size_t n);
int launch_vss_tables(Plan& p, const double* d_fcoef, const double* d_gj, int n_t, const double* d_sigma,
                      const int* d_reps, int n_reps);
// the grid of Phi_alpha(p, q) behind the fast build of a VSS table (FP32 plans)
struct VssGrid {
  int np = 0, nq = 0;
  double p0 = 0, q0 = 0, h = 0;
};
// Phi grids of the distinct alpha (rules d_gj [n_alpha][3][n_t]) into d_phi [n_alpha][nq][np],
// then the gain table by interpolation (pair o reads grid d_grid_of_pair[o])
int launch_vss_tables_grid(Plan& p, const double* d_fcoef, double2* d_phi, const double* d_gj, int n_alpha, int n_t,
                           const VssGrid& gr, const int* d_grid_of_pair, const double* d_sigma, const int* d_reps,
                           int n_reps);

// split-BF16 tensor-core path (dft_gemm.cu): N it supports, matrix images from the plan's
// phase factors [task][rho][max_ent][role][axis][N], kernel configuration and launch
bool gemm_supported_n(int N);
void build_gemm_images(const Plan& p, const std::vector<std::complex<double>>& phase, std::vector<uint16_t>& out);
int configure_bf16x3(Plan& p);
int launch_bf16x3(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws = 0);

// SSP-RK2 stage combinations (stepper.cu): stage 1 f1 = f + dt r; stage 2 f = (f + f1 + dt r)/2
int launch_rk_stage(const Plan& p, int stage, void* f, void* f1, const void* r, double dt, size_t n, cudaStream_t st);

// conservation projection (in place on Q[batch][s][s][N^3]) and species sum (conserve.cu)
int launch_conserve(const Plan& p, void* Q, int batch, cudaStream_t st);
int launch_species_sum(const Plan& p, const void* Qfull, void* Qsum, int batch, cudaStream_t st);

}  // namespace dgfs

// the opaque plan handle of the C ABI
struct dgfs_plan_s {
  dgfs::Plan plan;
};
