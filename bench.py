"""Benchmark: collision evaluations per second on the 4096-node N=32^3 two-species VHS batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step evaluates all s^2 collision operators Q_ij at every node of the batch (the whole
hot path: forward transforms, gain over every radial node and design direction, loss,
assembly) in one call of the C ABI.  `value` is the FP32 (mixed-precision) path with inputs
resident in HBM; `fp64` is the plain FP64 path on the same batch; `e2e` times the host-buffer
entry point with both copies inside the timed region.  Inputs (1.07 GB in, 2.15 GB out) are
larger than L2.  Under torchrun every rank evaluates its own 4096-node batch (weak scaling,
no collective on the data path).
"""

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "collision evals/s at N=32^3 mixed-precision vs FP64 plain; p50/p99 stream latency"
WORKLOAD_KEY = "dg_batch_n32"
FP32_LANES_PER_SM = 128


def workload():
    from paper_1903_03056_gb300 import synth
    return synth.WORKLOADS[WORKLOAD_KEY]


def transforms_per_node(w):
    """Algorithmic 3D transforms per node (antipodal design): s forward (f), P*N_rho*M inverse
    (a(sigma) of (i,j) is b(-sigma) of (j,i)), the forward transforms of the products, 2P
    inverse (gain and loss).  VHS sums the products over sigma first: s(s+1)/2 forward per
    radial node; VSS transforms each (rho, sigma) product, M per cross pair and M/2 per self
    pair (p(sigma) = p(-sigma))."""
    s, P = w.s, w.s * w.s
    if w.alpha == 1.0:
        fwd = (s * (s + 1) // 2) * w.N_rho
    else:
        fwd = (s * (s - 1) // 2 * w.M + s * (w.M // 2)) * w.N_rho
    return s + P * w.N_rho * w.M + fwd + 2 * P


def flops_per_transform(N):
    n3 = N ** 3
    return 5.0 * n3 * np.log2(n3)


# the sources that define the collision kernel's code and launch shape
COLLISION_KERNEL_SOURCES = ("collision_kernel.cuh", "fft_line.cuh", "tcgen05.cuh", "collision_f32.cu", "collision_f64.cu",
                            "dgfs_internal.h", "tuned_shapes.h", "tuned_radix.h")


def kernel_sources_sha1():
    """SHA-1 over the collision kernel's sources, to tie a stored ncu traffic figure to the
    kernel it measured."""
    import hashlib
    d = os.path.join(ROOT, "paper_1903_03056_gb300", "csrc")
    h = hashlib.sha1()
    for name in COLLISION_KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()


def hbm_peak_gbs():
    """HBM copy bandwidth from the measured-peaks file beside this script (a STREAM-style copy
    measured on this GPU model), else an earlier copy measurement on a GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the kernel
    sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_sha1") != kernel_sources_sha1():
        return None
    return rec.get("bytes_per_launch")


def measured_alu_peaks(torch, dgfs, local):
    """FP32 and FP64 multiply-add rates of this GPU, measured by the library's dependent-FMA
    loop on every SM (dgfs_measure_fma_rate), with the SM clock sampled meanwhile.  Falls back
    to the FP32 lane count x 2 flop x the maximum clock of this device's SM count when the
    measurement fails."""
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    with ClockSampler(local) as clk:
        c32, r32 = dgfs.dgfs_measure_fma_rate("fp32")
        c64, r64 = dgfs.dgfs_measure_fma_rate("fp64")
    clocks = clk.summary()
    out = {"sms": sms, "clocks": clocks}
    if c32 == 0 and c64 == 0 and r32 > 0 and r64 > 0:
        out.update({"fp32_tflops": r32 / 1e12, "fp64_tflops": r64 / 1e12, "source": "measured"})
    else:
        mhz = clocks.get("sm_max_mhz") or 2070.0
        out.update({"fp32_tflops": sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, "fp64_tflops": None,
                    "source": "derived (measurement failed: %d, %d)" % (c32, c64)})
    return out


def config_dict(w):
    return {"workload": w.name, "batch": w.batch, "N": w.N, "species": w.s,
            "masses": list(w.masses), "omega": w.omega, "alpha": w.alpha, "L": w.L, "M": w.M,
            "N_rho": w.N_rho, "inputs": "seeded bi-Maxwellians, 5% multiplicative noise",
            "l2": "inputs larger than L2 (1.07 GB f + 2.15 GB Q per step)"}


# ---- clocks ---------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ---- CPU oracle (baseline and reference arm) ----------------------------------------------------

def _oracle_node(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    key, node = args
    from oracle import fast_spectral as fs
    from paper_1903_03056_gb300 import synth
    w = synth.WORKLOADS[key]
    prob = fs.make_problem(w.N, w.L, list(w.masses), omega=w.omega, alpha=w.alpha, M=w.M,
                           N_rho=w.N_rho)
    f = synth.node_distribution(w, node)
    t0 = time.perf_counter()
    fs.collision(f, prob)
    return time.perf_counter() - t0


class OraclePool:
    """A spawn pool of single-threaded oracle workers (spawn: a pool forked after CUDA was
    initialised can hang).  Each call times one sample of nodes, one node per task."""

    def __init__(self, workers, key=None):
        self.workers = workers
        self.key = key or WORKLOAD_KEY
        self.env_backup = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ["OMP_NUM_THREADS"] = "1"
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        self.pool = mp.get_context("spawn").Pool(workers)
        self.pool.map(_oracle_node, [(self.key, 0)] * workers)  # import warm-up

    def sample(self, nodes):
        t0 = time.perf_counter()
        self.pool.map(_oracle_node, [(self.key, n) for n in nodes])
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()
        for k, v in self.env_backup.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def run_oracle_sample(nodes, workers):
    """Time the FP64 oracle on `nodes` nodes with a spawn pool of `workers` processes."""
    pool = OraclePool(workers)
    try:
        return pool.sample(nodes)
    finally:
        pool.close()


def cpu_baseline(w, cores):
    nodes = list(range(cores))
    wall = run_oracle_sample(nodes, cores)
    return {"value": len(nodes) / wall, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": "%d nodes of the %d-node batch, one per process (FP64 numpy oracle, dense "
                      "DFT matrices, literal (rho, sigma, pair) loop), %.1f s wall" % (len(nodes), w.batch, wall)}


def reference_arm(args, key=None):
    """The oracle timed on the host cores: W untimed and K timed steps, each a sample of one
    node per core taken from the bench workload's batch (consecutive node ranges).  Under
    torchrun only rank 0 runs it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from paper_1903_03056_gb300 import synth
    w = synth.WORKLOADS[key] if key else workload()
    cores = os.cpu_count() or 1
    pool = OraclePool(cores, key)
    try:
        step = 0
        for _ in range(args.warmup):
            pool.sample([(step * cores + c) % w.batch for c in range(cores)])
            step += 1
        times = []
        for _ in range(args.steps):
            times.append(pool.sample([(step * cores + c) % w.batch for c in range(cores)]))
            step += 1
    finally:
        pool.close()
    per_step = sum(times) / len(times)
    value = cores / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(w),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": "%d nodes per step (one per host core) of the %d-node batch, "
                                       "FP64 numpy oracle" % (cores, w.batch)},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


# ---- GPU arm ---------------------------------------------------------------------------------

def rank_nodes(rank, batch):
    """Node indices of one rank: every rank evaluates its own batch (weak scaling)."""
    return range(rank * batch, (rank + 1) * batch)


def aggregate_ranks(ms_local, batch, world, dist=None, device="cpu"):
    """Max of the ranks' per-step times and the whole-job rate world * batch / max time.
    The only collective of the path: an all_reduce(MAX) of one number."""
    ms = float(ms_local)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * batch / (ms * 1e-3)


def time_steps(torch, fn, steps, warmup, stream, dist=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end) / steps
    if dist is not None:
        ms, _ = aggregate_ranks(ms, 1, dist.get_world_size(), dist, device="cuda")
        dist.barrier()
    return ms


def serving_leg(args):
    """The mixed request stream: N in {16, 24, 32, 48}, s in {2, 3}, masses U[1, 4], VHS
    omega U[0.5, 1], batches of 1..4096 nodes, FP32, 120 GB HBM budget, 8 slots, requests
    served in chunks of ~50 ms of device work, shortest remaining work first.  The device
    time per node of every (N, s) is measured first; the Poisson arrivals are then scaled so
    that the stream's device work keeps the GPU 75 % busy over the stream.  A closed-loop run
    of the first requests reports the engine's capacity on the mix."""
    from paper_1903_03056_gb300 import serve
    budget = 120 << 30
    ex = serve.GpuExecutor(slots=8, sm_share=args.serve_sm_share)
    warm_s = ex.warmup()
    chunk = args.serve_chunk_s if args.serve_chunk_s > 0 else None
    eng = serve.ServingEngine(ex, budget_bytes=budget, slots=8, chunk_s=chunk, policy=args.serve_policy)
    calib = serve.mixed_stream(args.serve_calib, math.inf, seed=5000)
    st0 = eng.run(calib)
    stream = serve.mixed_stream(args.serve_requests, 1.0, seed=5001)
    keys = sorted({(r.N, r.s) for r in stream})
    spn32 = ex.service_seconds_per_node(keys, precision="fp32")
    work = sum(r.batch * spn32[(r.N, r.s)] for r in stream)
    span = max(r.arrival for r in stream)
    scale = (work / 0.75) / span
    for r in stream:
        r.arrival *= scale
    rate = len(stream) / (span * scale)
    st = eng.run(stream)
    out = st.as_dict()
    out["fp64_comparison"] = fp64_serving_replay(ex, stream, st, chunk, args.serve_policy, spn32, budget)
    out.update({"arrival_rate_per_s": rate, "target_utilisation": 0.75, "stream_device_work_s": work,
                "closed_loop_requests": st0.n, "closed_loop_evals_per_s": st0.evals_per_s,
                "closed_loop_req_per_s": st0.n / st0.makespan, "sm_share": args.serve_sm_share,
                "warmup_s": warm_s, "policy": args.serve_policy, "chunk_s": chunk,
                "mix": "N in {16,24,32,48}, s in {2,3}, masses U[1,4], omega U[0.5,1], batch "
                       "round(exp U[0, ln 4096]), M=12, N_rho=N/2, FP32, 8 slots, 120 GB budget"})
    return out


def fp64_serving_replay(ex, stream, measured, chunk, policy, spn32, budget):
    """The plain FP64 path on the same request stream.  Serving the mix in FP64 for real takes
    tens of minutes (one 4096-node N=48 three-species request alone is ~6 min of device time),
    so the stream's arrival trace is replayed through the same chunk scheduler in virtual time
    (serve.replay_chunked) with device service times measured per (N, s) for both precisions.
    The FP32 replay is checked against the FP32 stream measured above; the FP64 replay is given
    at the same arrivals (the FP64 path is then overloaded) and with the arrivals slowed to 75 %
    of the FP64 path's own capacity."""
    from paper_1903_03056_gb300 import serve
    keys = sorted({(r.N, r.s) for r in stream})
    spn64 = ex.service_seconds_per_node(keys, precision="fp64")
    chunk_s = chunk if chunk else 0.05
    b32 = lambda r: serve.request_bytes(r, 4)  # noqa: E731
    b64 = lambda r: serve.request_bytes(r, 8)  # noqa: E731
    r32 = serve.replay_chunked(stream, lambda r: spn32[(r.N, r.s)], chunk_s, policy, bytes_of=b32, budget=budget)
    r64 = serve.replay_chunked(stream, lambda r: spn64[(r.N, r.s)], chunk_s, policy, bytes_of=b64, budget=budget)
    work32 = sum(r.batch * spn32[(r.N, r.s)] for r in stream)
    work64 = sum(r.batch * spn64[(r.N, r.s)] for r in stream)
    span = max(r.arrival for r in stream) - min(r.arrival for r in stream)
    # arrivals stretched so that the FP64 path is 75 % busy over the stream
    scale = (work64 / 0.75) / span if span > 0 else 1.0
    r64s = serve.replay_chunked(stream, lambda r: spn64[(r.N, r.s)], chunk_s, policy, rate_scale=scale,
                                bytes_of=b64, budget=budget)

    def brief(s):
        return {"requests": s.n, "p50_ms": s.p50 * 1e3, "p99_ms": s.p99 * 1e3, "mean_ms": s.mean_latency * 1e3,
                "makespan_s": s.makespan, "evals_per_s": s.evals_per_s}

    return {"method": "trace replay of the measured stream's arrivals through the same SRPT chunk scheduler and "
                      "HBM-budget admission, device modelled as processor sharing, service times per (N, s) "
                      "measured on this GPU (plan building not modelled)",
            "service_ms_per_node_fp32": {"%d,%d" % k: v * 1e3 for k, v in spn32.items()},
            "service_ms_per_node_fp64": {"%d,%d" % k: v * 1e3 for k, v in spn64.items()},
            "fp32_replay": brief(r32), "fp32_measured": {"p50_ms": measured.p50 * 1e3, "p99_ms": measured.p99 * 1e3},
            "fp64_same_arrivals": brief(r64), "fp64_utilisation_at_same_arrivals": work64 / span if span > 0 else None,
            "fp64_at_75pct_of_its_capacity": dict(brief(r64s), arrival_rate_per_s=len(stream) / (span * scale)),
            "fp64_over_fp32_device_work": work64 / work32}


def bf16x3_tensor_flops_per_node(w):
    """BF16 tensor-core work of one node on the DGFS_BF16X3 path: every 3D transform is 3 passes
    over ceil(N^2 / 128) tiles of 128 lines, 6 split-term products of 2 x 128 x 2N x 2N flop.
    Transforms per node (antipodal rule): a self-pair task does its f_hat, 2 (M/2) N_rho shifted
    transforms, N_rho forward transforms of P and 2 final ones; a cross-pair task 2 f_hat,
    2 M N_rho shifted, N_rho forward and 4 final."""
    s, M, NR, N = w.s, w.M, w.N_rho, w.N
    self_t = 1 + 2 * (M // 2) * NR + NR + 2
    cross_t = 2 + 2 * M * NR + NR + 4
    transforms = s * self_t + s * (s - 1) // 2 * cross_t
    tiles = (N * N + 127) // 128
    return transforms, transforms * 3 * tiles * 6 * 2 * 128 * (2 * N) * (2 * N)


def tensor_leg(torch, stream, steps=3):
    """The split-BF16 tensor-core path against the FP32 FFT kernel on the 16384-node N = 24
    hard-sphere batch (the workload that path is defined on), same inputs, CUDA events."""
    from paper_1903_03056_gb300 import dgfs, synth
    w = synth.WORKLOADS["hs_n24"]
    f = synth.batch_distribution(w)
    with torch.cuda.stream(stream):
        fd = torch.from_numpy(f.astype(np.float32)).cuda()
        Q = torch.empty((w.batch, w.s, w.s, w.N, w.N, w.N), dtype=torch.float32, device="cuda")
    stream.synchronize()
    out = {"config": {"workload": w.name, "batch": w.batch, "N": w.N, "species": w.s, "masses": list(w.masses),
                      "omega": w.omega, "M": w.M, "N_rho": w.N_rho}}
    for prec in ("fp32", "bf16x3"):
        plan = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho, precision=prec)
        ms = time_steps(torch, lambda: plan.eval_ptr(fd.data_ptr(), Q.data_ptr(), w.batch, stream), steps, 1, stream)
        out[prec] = {"ms_per_step": ms, "evals_per_s": w.batch / (ms * 1e-3)}
        plan.close()
    transforms, flops = bf16x3_tensor_flops_per_node(w)
    achieved = flops * w.batch / (out["bf16x3"]["ms_per_step"] * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, how = float(json.load(fh)["bf16_tflops_sustained"]), "measured, sustained"
    except (OSError, ValueError, KeyError):
        peak, how = 1700.0, "fallback, sustained"
    out["bf16x3"]["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                 "frac": achieved / peak, "peak_source": how, "transforms_per_node": transforms,
                                 "tensor_flops_per_node": flops, "kernel": "gemm_collision_kernel<24>"}
    out["bf16x3_over_fp32"] = out["bf16x3"]["evals_per_s"] / out["fp32"]["evals_per_s"]
    del fd, Q
    return out


def dg_leg(torch, w, stream, Ne=1024, K=4):
    """The 1D DG path on Ne elements of K GLL nodes (Ne K = 4096 nodes of the batch's grid and
    species) between Maxwell walls: one transport pass (HBM-bound kernel, algorithmic bytes = the
    state read once and the right-hand side written once) and one full SSP-RK2 step (two
    transport passes and two collision evaluations of all nodes), FP32."""
    from paper_1903_03056_gb300 import dgfs, synth
    B = Ne * K
    f = synth.batch_distribution(w, nodes=range(min(B, w.batch)))
    f = np.concatenate([f] * (B // len(f) + 1))[:B]
    with torch.cuda.stream(stream):
        fd = torch.from_numpy(f.astype(np.float32)).cuda()
        rhs = torch.empty_like(fd)
    stream.synchronize()
    coll = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho,
                     precision="fp32", flags=dgfs.DGFS_SUM_SPECIES, max_batch=B)
    dgp = dgfs.DGPlan(coll, Ne, K, 0.0, 1.0, bc="walls", Tw=(0.9, 1.2),
                      uw=((0.0, 0.2, 0.0), (0.0, -0.2, 0.0)), acc=(1.0, 1.0))
    ms_t = time_steps(torch, lambda: dgp.transport(fd, rhs, stream), 10, 3, stream)
    ms_s = time_steps(torch, lambda: dgp.step(fd, 1e-3, stream), 1, 0, stream)
    peak, how = hbm_peak_gbs()
    nbytes = 2 * fd.numel() * fd.element_size()
    gbs = nbytes / (ms_t * 1e-3) / 1e9
    out = {"config": {"elements": Ne, "gll_nodes": K, "nodes": B, "N": w.N, "species": w.s,
                      "bc": "Maxwell walls (diffuse)", "dtype": "f32"},
           "transport_ms": ms_t, "step_ms": ms_s,
           "transport_roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak, "peak_source": how,
                                  "bytes_per_launch": nbytes, "kernel": "dg_transport_kernel<float,0,4>"}}
    dgp.close()
    coll.close()
    del fd, rhs
    return out


def gpu_arm(args):
    import torch
    from paper_1903_03056_gb300 import build, dgfs, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    dgfs.load()
    w = workload()
    B = w.batch
    cores = os.cpu_count() or 1

    # CPU baseline first (spawned pool before heavy GPU work; rank 0, N=1 only)
    cpu = cpu_baseline(w, cores) if (world == 1 and not args.no_cpu_baseline) else None
    peaks = measured_alu_peaks(torch, dgfs, local)

    f64 = synth.batch_distribution(w, nodes=rank_nodes(rank, B))  # [B, s, N, N, N]
    stream = torch.cuda.Stream()
    flops_node = transforms_per_node(w) * flops_per_transform(w.N)

    with torch.cuda.stream(stream):
        f32 = torch.from_numpy(f64.astype(np.float32)).cuda()
        Q32 = torch.empty((B, w.s, w.s, w.N, w.N, w.N), dtype=torch.float32, device="cuda")
    stream.synchronize()
    plan32 = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho,
                       precision="fp32", max_batch=B)

    def step32():
        plan32.eval_ptr(f32.data_ptr(), Q32.data_ptr(), B, stream)

    with ClockSampler(local) as clk:
        ms32 = time_steps(torch, step32, args.steps, args.warmup, stream, dist)
    launches = plan32.launches() * args.steps
    value = world * B / (ms32 * 1e-3)

    # e2e: host buffers (pinned), copies inside the timed region
    f_host = torch.from_numpy(f64.astype(np.float32)).pin_memory()
    Q_host = torch.empty((B, w.s, w.s, w.N, w.N, w.N), dtype=torch.float32).pin_memory()

    def step_e2e():
        plan32.eval_host(f_host, Q_host, stream)

    # the same warm-up and step counts as the device-resident measurement
    ms_e2e = time_steps(torch, step_e2e, args.steps, max(3, args.warmup), stream, dist)
    e2e = {"value": world * B / (ms_e2e * 1e-3), "unit": "evals/s",
           "h2d_bytes_per_step": int(f_host.numel() * 4), "d2h_bytes_per_step": int(Q_host.numel() * 4)}
    del f_host, Q_host

    # FP64 plain path on the same batch
    fp64 = None
    if not args.no_fp64:
        del Q32
        with torch.cuda.stream(stream):
            fd = torch.from_numpy(f64).cuda()
            Qd = torch.empty((B, w.s, w.s, w.N, w.N, w.N), dtype=torch.float64, device="cuda")
        stream.synchronize()
        plan64 = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M,
                           N_rho=w.N_rho, precision="fp64")

        def step64():
            plan64.eval_ptr(fd.data_ptr(), Qd.data_ptr(), B, stream)

        ms64 = time_steps(torch, step64, args.fp64_steps, 1, stream, dist)
        fp64 = {"value": world * B / (ms64 * 1e-3), "unit": "evals/s", "ms_per_step": ms64,
                "steps": args.fp64_steps, "dtype": "f64",
                "mixed_over_fp64": value / (world * B / (ms64 * 1e-3))}
        plan64.close()
        del fd, Qd

    dg = None
    if not args.no_dg and world == 1:
        dg = dg_leg(torch, w, stream)

    tensor = None
    if not args.no_tensor and world == 1:
        tensor = tensor_leg(torch, stream)

    serving = None
    if not args.no_serving and world == 1:
        del f32
        torch.cuda.empty_cache()
        serving = serving_leg(args)

    if rank == 0:
        achieved = flops_node * B / (ms32 * 1e-3) / 1e12
        peak = peaks["fp32_tflops"]
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic("collision_kernel<float,32>"),
                "kernel": "collision_kernel<float,32>",
                "peak_note": "FP32 FMA rate %s: dependent-FMA loop on all %d SMs (dgfs_measure_fma_rate) "
                             "at a median SM clock of %s MHz" % (peaks["source"], peaks["sms"],
                                                                  peaks["clocks"].get("sm_mhz")),
                "fp64_peak_tflops": peaks["fp64_tflops"],
                "flops_per_node": flops_node}
        if fp64 is not None and peaks["fp64_tflops"]:
            fp64["achieved_tflops"] = flops_node * B / (fp64["ms_per_step"] * 1e-3) / 1e12
            fp64["frac_of_fp64_peak"] = fp64["achieved_tflops"] / peaks["fp64_tflops"]
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_dict(w), "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "fp64": fp64, "dg": dg, "tensor_path": tensor, "serving": serving,
                "parity": {"fp32_bar": "1e-5 of the node's max |Q| over its s^2 operators (per-node scale) "
                                       "against the FP64 oracle", "fp64_bar": "1e-11 of max |Q| per pair"}}
        print(json.dumps(line), flush=True)
    plan32.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-dg", action="store_true")
    ap.add_argument("--no-tensor", action="store_true", help="skip the split-BF16 tensor-core leg")
    ap.add_argument("--serve-calib", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-sm-share", type=float, default=1.0)
    ap.add_argument("--serve-chunk-s", type=float, default=0.05,
                    help="device seconds per chunk of a request (0: whole requests)")
    ap.add_argument("--serve-policy", default="srpt", choices=["srpt", "fifo"])
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
