// extern "C" entry points of libdgfs.so (declared in include/dgfs.h).
#include <cmath>
#include <cstdint>
#include <new>

#include "dgfs_internal.h"

namespace {

// make the plan's device current for the duration of a call
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool aligned16(const void* p) { return (reinterpret_cast<std::uintptr_t>(p) & 15u) == 0; }

// collision kernel on workspace `ws`, then (flags) the conservation projection and the species
// sum (the full operators staged at node `stage_node` of the plan's staging array); returns a
// status and adds the kernels it enqueued to *launches.  No ordering against other streams.
int launch_core(dgfs::Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws, int stage_node,
                int* launches) {
  const bool sum = (p.flags & DGFS_SUM_SPECIES) != 0u;
  if (sum && (stage_node + batch > p.max_batch || !p.d_Qfull)) return DGFS_ERR_BUDGET;
  const size_t n3 = size_t(p.N) * p.N * p.N;
  void* Qfull = sum ? static_cast<char*>(p.d_Qfull) + size_t(stage_node) * p.s * p.s * n3 * dgfs::real_size(p) : Q;
  int rc = p.precision == DGFS_FP32     ? dgfs::launch_f32(p, f, Qfull, batch, st, ws)
           : p.precision == DGFS_BF16X3 ? dgfs::launch_bf16x3(p, f, Qfull, batch, st, ws)
                                        : dgfs::launch_f64(p, f, Qfull, batch, st, ws);
  if (rc != DGFS_OK) return rc;
  *launches += 1;
  if (p.flags & DGFS_CONSERVE) {
    dgfs::NvtxRange r2("dgfs conservation projection");
    if ((rc = dgfs::launch_conserve(p, Qfull, batch, st)) != DGFS_OK) return rc;
    *launches += 1;
  }
  if (sum) {
    dgfs::NvtxRange r2("dgfs species sum");
    if ((rc = dgfs::launch_species_sum(p, Qfull, Q, batch, st)) != DGFS_OK) return rc;
    *launches += 1;
  }
  return DGFS_OK;
}

// one evaluation on the caller's stream, ordered after the plan's previous evaluation;
// p.last_launches = the kernels it enqueued
int launch(dgfs::Plan& p, const void* f, void* Q, int batch, cudaStream_t st) {
  dgfs::NvtxRange range("dgfs collision");
  p.last_launches = 0;
  // the plan's workspace and work counter serve one kernel at a time: an evaluation enqueued
  // on another stream than the previous one waits for it.  Launches recorded into a CUDA graph
  // (stream capture) are ordered by the graph and leave this bookkeeping alone.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (!capturing && p.has_eval && st != p.last_stream && cudaStreamWaitEvent(st, p.last_eval, 0) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  int launches = 0;
  const int rc = launch_core(p, f, Q, batch, st, 0, 0, &launches);
  p.last_launches = launches;
  if (rc != DGFS_OK) return rc;
  if (capturing) return cudaPeekAtLastError() == cudaSuccess ? DGFS_OK : (cudaGetLastError(), DGFS_ERR_CUDA);
  if (cudaEventRecord(p.last_eval, st) != cudaSuccess || cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  p.has_eval = true;
  p.last_stream = st;
  return DGFS_OK;
}

size_t output_pairs(const dgfs::Plan& p) { return (p.flags & DGFS_SUM_SPECIES) ? size_t(p.s) : size_t(p.s) * p.s; }

}  // namespace

extern "C" {

int dgfs_create_plan(const dgfs_plan_desc* desc, dgfs_plan* out) {
  if (!desc || !out) return DGFS_ERR_INVALID_ARG;
  dgfs::NvtxRange range("dgfs_create_plan");
  *out = nullptr;
  dgfs_plan_s* h = new (std::nothrow) dgfs_plan_s;
  if (!h) return DGFS_ERR_OOM;
  dgfs::Plan& p = h->plan;
  int rc = dgfs::build_plan(desc, p);
  if (rc == DGFS_OK && cudaGetDevice(&p.device) != cudaSuccess) rc = DGFS_ERR_CUDA;
  if (rc == DGFS_OK)
    rc = p.precision == DGFS_FP32     ? dgfs::configure_f32(p)
         : p.precision == DGFS_BF16X3 ? dgfs::configure_bf16x3(p)
                                      : dgfs::configure_f64(p);
  if (rc == DGFS_OK) rc = dgfs::upload_plan(p);
  if (rc != DGFS_OK) {
    dgfs::free_plan(p);
    cudaGetLastError();
    delete h;
    return rc;
  }
  *out = h;
  return DGFS_OK;
}

int dgfs_destroy_plan(dgfs_plan plan) {
  if (!plan) return DGFS_ERR_INVALID_ARG;
  {
    DeviceGuard g(plan->plan.device);
    // wait for the plan's last evaluation only; other streams keep running
    if (plan->plan.has_eval) cudaEventSynchronize(plan->plan.last_eval);
    dgfs::free_plan(plan->plan);
  }
  delete plan;
  return DGFS_OK;
}

int dgfs_eval_collision(dgfs_plan plan, const void* f_dev, void* Q_dev, int batch, void* stream) {
  if (!plan || batch < 0) return DGFS_ERR_INVALID_ARG;
  if (batch == 0) return DGFS_OK;
  if (!f_dev || !Q_dev || !aligned16(f_dev) || !aligned16(Q_dev)) return DGFS_ERR_INVALID_ARG;
  DeviceGuard g(plan->plan.device);
  if (!g.ok) return DGFS_ERR_CUDA;
  return launch(plan->plan, f_dev, Q_dev, batch, static_cast<cudaStream_t>(stream));
}

int dgfs_eval_collision_host(dgfs_plan plan, const void* f_host, void* Q_host, int batch, void* stream) {
  if (!plan || batch < 0) return DGFS_ERR_INVALID_ARG;
  if (batch == 0) return DGFS_OK;
  if (!f_host || !Q_host) return DGFS_ERR_INVALID_ARG;
  dgfs::Plan& p = plan->plan;
  if (batch > p.max_batch) return DGFS_ERR_BUDGET;
  dgfs::NvtxRange range("dgfs_eval_collision_host");
  DeviceGuard g(p.device);
  if (!g.ok) return DGFS_ERR_CUDA;
  const size_t n3 = size_t(p.N) * p.N * p.N;
  const size_t f_node = size_t(p.s) * n3 * dgfs::real_size(p);
  const size_t q_node = output_pairs(p) * n3 * dgfs::real_size(p);
  if (!p.d_stage_f) {
    if (cudaMallocAsync(&p.d_stage_f, size_t(p.max_batch) * f_node, p.home) != cudaSuccess ||
        cudaMallocAsync(&p.d_stage_Q, size_t(p.max_batch) * q_node, p.home) != cudaSuccess ||
        cudaStreamSynchronize(p.home) != cudaSuccess) {
      cudaGetLastError();
      if (p.d_stage_f) cudaFreeAsync(p.d_stage_f, p.home);
      if (p.d_stage_Q) cudaFreeAsync(p.d_stage_Q, p.home);
      cudaStreamSynchronize(p.home);
      p.d_stage_f = nullptr;
      p.d_stage_Q = nullptr;
      return DGFS_ERR_OOM;
    }
    p.stage_batch = p.max_batch;
  }
  if (!p.d_scratch2_raw) {
    // the second workspace (with its guard blocks) and work counter of the pipelined chunks
    if (cudaMallocAsync(&p.d_scratch2_raw, p.scratch_bytes + 2 * dgfs::Plan::kGuardBytes, p.home) != cudaSuccess ||
        cudaMallocAsync((void**)&p.d_counter2, 256, p.home) != cudaSuccess) {
      cudaGetLastError();
      if (p.d_scratch2_raw) cudaFreeAsync(p.d_scratch2_raw, p.home);
      if (p.d_counter2) cudaFreeAsync(p.d_counter2, p.home);
      cudaStreamSynchronize(p.home);
      p.d_scratch2_raw = nullptr;
      p.d_counter2 = nullptr;
      return DGFS_ERR_OOM;
    }
    p.d_scratch2 = static_cast<char*>(p.d_scratch2_raw) + dgfs::Plan::kGuardBytes;
    if (cudaMemsetAsync(p.d_scratch2_raw, dgfs::Plan::kGuardByte, dgfs::Plan::kGuardBytes, p.home) != cudaSuccess ||
        cudaMemsetAsync(static_cast<char*>(p.d_scratch2) + p.scratch_bytes, dgfs::Plan::kGuardByte,
                        dgfs::Plan::kGuardBytes, p.home) != cudaSuccess ||
        cudaMemsetAsync(p.d_counter2, 0, 256, p.home) != cudaSuccess || cudaStreamSynchronize(p.home) != cudaSuccess) {
      cudaGetLastError();
      return DGFS_ERR_CUDA;
    }
  }
  if (!p.h2d) {
    bool ok = cudaStreamCreateWithFlags(&p.h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.d2h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.eval2, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.ev_start, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < dgfs::Plan::kMaxChunks; ++k)
      ok = cudaEventCreateWithFlags(&p.ev_h2d[k], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&p.ev_done[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return DGFS_ERR_CUDA;
    }
  }
  // chunks of >= 256 nodes: the input copy of chunk k+1 and the output copy of chunk k-1
  // overlap the evaluation of chunk k (copies on the plan's two copy streams).  Chunks
  // alternate between two evaluation streams (the caller's and the plan's second one) and two
  // workspaces, so chunk k+1's kernel starts while chunk k's finishes its last work items;
  // chunk k+2 reuses chunk k's stream and workspace and so runs after it.  Measured on the
  // 4096-node N = 32 batch in 8 chunks: 312.9 ms per batch with two workspaces against
  // 337.6 ms with one (the device-resident launch: 309.1 ms).
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStream_t evs[2] = {st, p.eval2};
  int nchunks = batch / 256;
  nchunks = nchunks < 1 ? 1 : (nchunks > dgfs::Plan::kMaxChunks ? dgfs::Plan::kMaxChunks : nchunks);
  const int chunk = (batch + nchunks - 1) / nchunks;
  // every stream starts after the work already on the caller's stream and after the plan's
  // previous evaluation (wherever it ran)
  if (p.has_eval && cudaStreamWaitEvent(st, p.last_eval, 0) != cudaSuccess) return DGFS_ERR_CUDA;
  if (cudaEventRecord(p.ev_start, st) != cudaSuccess || cudaStreamWaitEvent(p.h2d, p.ev_start, 0) != cudaSuccess ||
      cudaStreamWaitEvent(p.eval2, p.ev_start, 0) != cudaSuccess)
    return DGFS_ERR_CUDA;
  int launches = 0;
  for (int k = 0; k < nchunks; ++k) {
    const int b0 = k * chunk;
    const int nb = batch - b0 < chunk ? batch - b0 : chunk;
    if (nb <= 0) break;
    cudaStream_t es = evs[k & 1];
    char* sf = static_cast<char*>(p.d_stage_f) + size_t(b0) * f_node;
    char* sq = static_cast<char*>(p.d_stage_Q) + size_t(b0) * q_node;
    if (cudaMemcpyAsync(sf, static_cast<const char*>(f_host) + size_t(b0) * f_node, size_t(nb) * f_node,
                        cudaMemcpyHostToDevice, p.h2d) != cudaSuccess ||
        cudaEventRecord(p.ev_h2d[k], p.h2d) != cudaSuccess || cudaStreamWaitEvent(es, p.ev_h2d[k], 0) != cudaSuccess)
      return DGFS_ERR_CUDA;
    {
      dgfs::NvtxRange range("dgfs collision");
      const int rc = launch_core(p, sf, sq, nb, es, k & 1, b0, &launches);
      if (rc != DGFS_OK) return rc;
    }
    if (cudaEventRecord(p.ev_done[k], es) != cudaSuccess || cudaStreamWaitEvent(p.d2h, p.ev_done[k], 0) != cudaSuccess ||
        cudaMemcpyAsync(static_cast<char*>(Q_host) + size_t(b0) * q_node, sq, size_t(nb) * q_node,
                        cudaMemcpyDeviceToHost, p.d2h) != cudaSuccess)
      return DGFS_ERR_CUDA;
  }
  // the caller's stream ends after both evaluation streams; that is the plan's last evaluation
  if (cudaEventRecord(p.ev_start, p.eval2) != cudaSuccess || cudaStreamWaitEvent(st, p.ev_start, 0) != cudaSuccess ||
      cudaEventRecord(p.last_eval, st) != cudaSuccess)
    return DGFS_ERR_CUDA;
  p.has_eval = true;
  p.last_stream = st;
  p.last_launches = launches;
  if (cudaStreamSynchronize(p.d2h) != cudaSuccess) return DGFS_ERR_CUDA;
  return DGFS_OK;
}

int dgfs_ssp_rk2_step(dgfs_plan plan, void* f_dev, double dt, int batch, void* stream) {
  if (!plan || batch < 0 || !std::isfinite(dt)) return DGFS_ERR_INVALID_ARG;
  dgfs::Plan& p = plan->plan;
  if (!(p.flags & DGFS_SUM_SPECIES)) return DGFS_ERR_INVALID_ARG;
  if (batch == 0) return DGFS_OK;
  if (!f_dev || !aligned16(f_dev)) return DGFS_ERR_INVALID_ARG;
  if (batch > p.max_batch) return DGFS_ERR_BUDGET;
  dgfs::NvtxRange range("dgfs_ssp_rk2_step");
  DeviceGuard g(p.device);
  if (!g.ok) return DGFS_ERR_CUDA;
  const size_t n = size_t(p.max_batch) * p.s * p.N * p.N * p.N;
  const size_t bytes = n * dgfs::real_size(p);
  if (!p.d_rk) {
    if (cudaMallocAsync(&p.d_rk, 2 * bytes, p.home) != cudaSuccess || cudaStreamSynchronize(p.home) != cudaSuccess) {
      cudaGetLastError();
      p.d_rk = nullptr;
      return DGFS_ERR_OOM;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* f1 = p.d_rk;
  void* r = static_cast<char*>(p.d_rk) + bytes;
  const size_t cnt = size_t(batch) * p.s * p.N * p.N * p.N;
  int rc, launches = 0;
  if ((rc = launch(p, f_dev, r, batch, st)) != DGFS_OK) return rc;
  launches += p.last_launches;
  if ((rc = dgfs::launch_rk_stage(p, 1, f_dev, f1, r, dt, cnt, st)) != DGFS_OK) return rc;
  if ((rc = launch(p, f1, r, batch, st)) != DGFS_OK) return rc;
  launches += p.last_launches;
  if ((rc = dgfs::launch_rk_stage(p, 2, f_dev, f1, r, dt, cnt, st)) != DGFS_OK) return rc;
  p.last_launches = launches + 2;
  return DGFS_OK;
}

int dgfs_plan_set_sm_share(dgfs_plan plan, double share) {
  if (!plan || !(share > 0.0) || share > 1.0) return DGFS_ERR_INVALID_ARG;
  plan->plan.shape.share = share;
  return DGFS_OK;
}

int dgfs_plan_bytes(dgfs_plan plan, int batch, size_t* tables, size_t* workspace) {
  if (!plan || batch < 0) return DGFS_ERR_INVALID_ARG;
  const dgfs::Plan& p = plan->plan;
  const size_t n3 = size_t(p.N) * p.N * p.N;
  if (tables) *tables = p.table_bytes;
  if (workspace)
    *workspace = p.scratch_bytes + 2 * dgfs::Plan::kGuardBytes + (p.d_Qfull ? size_t(p.max_batch) * p.s * p.s * n3 * dgfs::real_size(p) : 0) +
                 (batch > 0 ? size_t(batch) * (p.s + output_pairs(p)) * n3 * dgfs::real_size(p) +
                                  p.scratch_bytes + 2 * dgfs::Plan::kGuardBytes + 256
                            : 0);
  return DGFS_OK;
}

int dgfs_plan_radius(dgfs_plan plan, double* R) {
  if (!plan || !R) return DGFS_ERR_INVALID_ARG;
  *R = plan->plan.R;
  return DGFS_OK;
}

int dgfs_plan_check(dgfs_plan plan, int* intact) {
  if (!plan || !intact) return DGFS_ERR_INVALID_ARG;
  dgfs::Plan& p = plan->plan;
  if (!p.d_scratch_raw) return DGFS_ERR_INVALID_ARG;
  dgfs::NvtxRange range("dgfs_plan_check");
  DeviceGuard g(p.device);
  if (!g.ok) return DGFS_ERR_CUDA;
  constexpr size_t G = dgfs::Plan::kGuardBytes;
  static thread_local unsigned char host[2 * G];
  // after the plan's last evaluation, on the plan's own stream; both workspaces (the second
  // exists once a host-buffer call has run)
  if (p.has_eval && cudaStreamWaitEvent(p.home, p.last_eval, 0) != cudaSuccess) {
    cudaGetLastError();
    return DGFS_ERR_CUDA;
  }
  int ok = 1;
  unsigned status = 0;
  for (int ws = 0; ws < 2; ++ws) {
    void* raw = ws == 0 ? p.d_scratch_raw : p.d_scratch2_raw;
    if (!raw) continue;
    const char* body = static_cast<const char*>(p.scratch_of(ws));
    unsigned st = 0;
    if (cudaMemcpyAsync(host, raw, G, cudaMemcpyDeviceToHost, p.home) != cudaSuccess ||
        cudaMemcpyAsync(host + G, body + p.scratch_bytes, G, cudaMemcpyDeviceToHost, p.home) != cudaSuccess ||
        cudaMemcpyAsync(&st, p.counter_of(ws) + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, p.home) != cudaSuccess ||
        cudaStreamSynchronize(p.home) != cudaSuccess) {
      cudaGetLastError();
      return DGFS_ERR_CUDA;
    }
    for (size_t k = 0; k < 2 * G; ++k) ok &= host[k] == dgfs::Plan::kGuardByte ? 1 : 0;
    // the device status word beside the work counter: a bounded device-side wait gave up
    status |= st;
  }
  *intact = ok;
  return status != 0 ? DGFS_ERR_DEVICE_TIMEOUT : DGFS_OK;
}

int dgfs_plan_launches(dgfs_plan plan, int* launches) {
  if (!plan || !launches) return DGFS_ERR_INVALID_ARG;
  *launches = plan->plan.last_launches;
  return DGFS_OK;
}

const char* dgfs_strerror(int code) {
  switch (code) {
    case DGFS_OK: return "ok";
    case DGFS_ERR_INVALID_ARG: return "invalid argument";
    case DGFS_ERR_UNSUPPORTED_N: return "unsupported grid size N";
    case DGFS_ERR_OOM: return "out of memory";
    case DGFS_ERR_BUDGET: return "batch exceeds the plan's max_batch";
    case DGFS_ERR_CUDA: return "CUDA runtime error";
    case DGFS_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case DGFS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

}  // extern "C"
