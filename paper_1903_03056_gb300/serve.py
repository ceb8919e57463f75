"""Serving: a continuous-batching request loop over the collision library.

A request asks for the s^2 collision operators of a batch of DG nodes on a velocity grid of
its own (N, L, masses, omega, M, N_rho).  Node states live on the device (in a DG solver the
operator feeds the next Runge-Kutta stage there), so a request arrives with its input f in
device memory and completes when its Q is in device memory.

Loop (one host thread, ``ServingEngine.run``):

* arrival -- the request enters the pending queue and its plan is built on a worker thread
  (tables are computed on the device on the plan's own stream; plans with identical
  parameters are shared through a cache);
* admission -- in arrival order, a pending request whose plan is ready is admitted when a
  slot (a CUDA stream) is free and the HBM budget covers its plan, its input copy and its
  output; requests that arrive while others run are admitted as soon as slots and memory
  free up, so their kernels overlap on the device;
* completion -- an event per request; on completion the slot and the memory are released.

The budget covers admitted requests (plan tables, workspace, input and output); plans built
ahead for waiting requests are bounded by the prefetch depth.

Chunked mode (``chunk_s`` set): an admitted request does not hold a slot.  A free slot takes
the next chunk of some admitted request -- consecutive nodes worth about ``chunk_s`` seconds
of device work by a cost model -- chosen by ``policy``: "srpt" takes the request with the
least remaining work (small requests overtake large ones between chunks), "fifo" the
earliest.  Chunks of one request may run on several slots at once; results do not depend on
how a batch is split, since every node is evaluated independently.

Latency = completion - arrival.  The executor is pluggable: ``GpuExecutor`` drives the CUDA
library, ``FakeExecutor`` (tests) models durations on the CPU.
"""

import collections
import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

L_FOR_N = {8: 4.0, 12: 5.0, 16: 6.0, 24: 6.0, 32: 7.0, 48: 8.0}


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    N: int
    L: float
    masses: tuple
    omega: float
    M: int
    N_rho: int
    batch: int
    pool_offset: int = 0    # first node of the input pool tiled into this request
    admitted: float = None
    done: float = None
    bytes: int = 0
    slot: int = -1
    next_node: int = 0      # chunked mode: first node not yet submitted
    nodes_done: int = 0     # chunked mode: nodes whose chunks completed

    @property
    def s(self):
        return len(self.masses)

    @property
    def plan_key(self):
        return (self.N, self.L, self.masses, self.omega, self.M, self.N_rho)

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


def mixed_stream(n_requests, rate, seed=5000, sizes=(16, 24, 32, 48), max_batch=4096):
    """Seeded request mix: N uniform over `sizes`, s in {2, 3}, masses U[1, 4], one VHS
    omega U[0.5, 1] for all pairs, M = 12, N_rho = N/2, batch = round(exp U[0, ln max_batch]),
    Poisson arrivals at `rate` requests/s (rate = inf: all at t = 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(n_requests):
        if math.isfinite(rate):
            t += rng.exponential(1.0 / rate)
        N = int(rng.choice(sizes))
        s = int(rng.integers(2, 4))
        masses = tuple(float(m) for m in np.round(rng.uniform(1.0, 4.0, size=s), 6))
        omega = float(np.round(rng.uniform(0.5, 1.0), 6))
        batch = int(max(1, min(max_batch, round(math.exp(rng.uniform(0.0, math.log(max_batch)))))))
        out.append(Request(k, t if math.isfinite(rate) else 0.0, N, L_FOR_N[N], masses, omega, 12,
                           N // 2, batch, pool_offset=int(rng.integers(0, 1 << 20))))
    return out


# seconds per node of one evaluation on the whole device, by the transform count
# s^2 N_rho M N^3 log2 N^3 (calibrated on the 4096-node N=32, s=2, N_rho=16, M=12 batch:
# 79 us per node)
COST_PER_TRANSFORM_POINT = 79e-6 / (4 * 16 * 12 * 32 ** 3 * 15)


def cost_per_node(r):
    n3 = r.N ** 3
    return COST_PER_TRANSFORM_POINT * r.s * r.s * r.N_rho * r.M * n3 * math.log2(n3)


def request_bytes(r, elem=4, plan_bytes=0):
    """Device bytes a request holds while admitted: its input f [batch][s][N^3] and output Q
    [batch][s][s][N^3] in the precision's element size, plus its plan."""
    return plan_bytes + r.batch * (r.s + r.s * r.s) * r.N ** 3 * elem


def percentile(values, p):
    v = sorted(values)
    if not v:
        return None
    k = (len(v) - 1) * p / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


@dataclass
class Stats:
    n: int
    nodes: int
    makespan: float
    p50: float
    p99: float
    mean_latency: float
    peak_bytes: int
    peak_inflight: int
    budget: int
    extra: dict = field(default_factory=dict)

    @property
    def evals_per_s(self):
        return self.nodes / self.makespan if self.makespan > 0 else 0.0

    def as_dict(self):
        d = {"requests": self.n, "nodes": self.nodes, "makespan_s": self.makespan,
             "evals_per_s": self.evals_per_s, "p50_ms": self.p50 * 1e3, "p99_ms": self.p99 * 1e3,
             "mean_ms": self.mean_latency * 1e3, "peak_bytes": self.peak_bytes,
             "peak_inflight": self.peak_inflight, "budget_bytes": self.budget}
        d.update(self.extra)
        return d


class ServingEngine:
    def __init__(self, executor, budget_bytes, slots=8, prefetch=8, chunk_s=None, policy="srpt"):
        if policy not in ("srpt", "fifo"):
            raise ValueError(policy)
        self.ex = executor
        self.budget = int(budget_bytes)
        self.slots = slots
        self.prefetch = prefetch
        self.chunk_s = chunk_s
        self.policy = policy

    def run(self, requests, poll_s=50e-6):
        """Serve `requests` (arrival times relative to the start); returns Stats."""
        if self.chunk_s is not None:
            return self._run_chunked(requests, poll_s)
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        arrivals = collections.deque(reqs)
        pending = collections.deque()       # arrived, waiting for admission (FIFO)
        plans = {}                          # rid -> future of the plan
        inflight = {}                       # slot -> request
        free_slots = list(range(self.slots))
        in_use = 0
        peak_bytes, peak_inflight = 0, 0
        builder = ThreadPoolExecutor(max_workers=2)
        t0 = time.perf_counter()
        try:
            while arrivals or pending or inflight:
                now = time.perf_counter() - t0
                while arrivals and arrivals[0].arrival <= now:
                    pending.append(arrivals.popleft())
                # build plans for the first few waiting requests, in arrival order
                for r in list(pending)[: self.prefetch]:
                    if r.rid not in plans:
                        plans[r.rid] = builder.submit(self.ex.prepare, r)
                # admission in arrival order: the head must fit before later requests go
                while pending and free_slots:
                    r = pending[0]
                    fut = plans.get(r.rid)
                    if fut is None or not fut.done():
                        break
                    need = fut.result()
                    if need > self.budget:
                        raise RuntimeError("request %d needs %d bytes, budget %d" % (r.rid, need, self.budget))
                    if in_use + need > self.budget:
                        break
                    pending.popleft()
                    slot = free_slots.pop()
                    r.slot, r.bytes = slot, need
                    r.admitted = time.perf_counter() - t0
                    in_use += need
                    self.ex.submit(r, slot)
                    inflight[slot] = r
                    peak_bytes = max(peak_bytes, in_use)
                    peak_inflight = max(peak_inflight, len(inflight))
                # completions
                for slot, r in list(inflight.items()):
                    if self.ex.done(r):
                        r.done = time.perf_counter() - t0
                        self.ex.release(r)
                        plans.pop(r.rid, None)
                        in_use -= r.bytes
                        del inflight[slot]
                        free_slots.append(slot)
                if not inflight and not pending and arrivals:
                    wait = arrivals[0].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                else:
                    time.sleep(poll_s)
        finally:
            builder.shutdown(wait=True)
        lat = [r.latency for r in reqs]
        first = min(r.arrival for r in reqs)
        makespan = max(r.done for r in reqs) - first
        return Stats(n=len(reqs), nodes=sum(r.batch for r in reqs), makespan=makespan,
                     p50=percentile(lat, 50), p99=percentile(lat, 99),
                     mean_latency=sum(lat) / len(lat), peak_bytes=peak_bytes,
                     peak_inflight=peak_inflight, budget=self.budget)

    def _run_chunked(self, requests, poll_s):
        """Chunked loop (see the module docstring); returns Stats."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        arrivals = collections.deque(reqs)
        pending = collections.deque()       # arrived, waiting for admission (FIFO)
        plans = {}                          # rid -> future of the plan
        active = []                         # admitted, nodes left to submit or running
        running = {}                        # slot -> (request, lo, hi)
        free_slots = list(range(self.slots))
        in_use = 0
        peak_bytes, peak_inflight = 0, 0
        builder = ThreadPoolExecutor(max_workers=2)
        t0 = time.perf_counter()

        def pick():
            # one chunk per plan at a time: a plan's evaluations share its workspace and the library
            # serialises them, so a second chunk of the same plan would only hold a slot
            busy = {r.plan_key for (r, _, _) in running.values()}
            cand = [r for r in active if r.next_node < r.batch and r.plan_key not in busy]
            if not cand:
                return None
            if self.policy == "fifo":
                return min(cand, key=lambda r: (r.arrival, r.rid))
            return min(cand, key=lambda r: ((r.batch - r.next_node) * cost_per_node(r), r.arrival, r.rid))

        try:
            while arrivals or pending or active:
                now = time.perf_counter() - t0
                while arrivals and arrivals[0].arrival <= now:
                    pending.append(arrivals.popleft())
                for r in list(pending)[: self.prefetch]:
                    if r.rid not in plans:
                        plans[r.rid] = builder.submit(self.ex.prepare, r)
                # admission in arrival order under the memory budget (no slot needed)
                while pending:
                    r = pending[0]
                    fut = plans.get(r.rid)
                    if fut is None or not fut.done():
                        break
                    need = fut.result()
                    if need > self.budget:
                        raise RuntimeError("request %d needs %d bytes, budget %d" % (r.rid, need, self.budget))
                    if in_use + need > self.budget:
                        break
                    pending.popleft()
                    r.bytes = need
                    r.admitted = time.perf_counter() - t0
                    r.next_node, r.nodes_done = 0, 0
                    in_use += need
                    self.ex.begin(r)
                    active.append(r)
                    peak_bytes = max(peak_bytes, in_use)
                # fill free slots with chunks
                while free_slots:
                    r = pick()
                    if r is None:
                        break
                    n = max(1, int(self.chunk_s / cost_per_node(r)))
                    lo, hi = r.next_node, min(r.batch, r.next_node + n)
                    r.next_node = hi
                    slot = free_slots.pop()
                    self.ex.submit_chunk(r, slot, lo, hi)
                    running[slot] = (r, lo, hi)
                    peak_inflight = max(peak_inflight, len(running))
                # chunk completions
                for slot, (r, lo, hi) in list(running.items()):
                    if self.ex.chunk_done(slot):
                        del running[slot]
                        free_slots.append(slot)
                        r.nodes_done += hi - lo
                        if r.nodes_done == r.batch:
                            r.done = time.perf_counter() - t0
                            self.ex.finish(r)
                            plans.pop(r.rid, None)
                            in_use -= r.bytes
                            active.remove(r)
                if not running and not pending and not active and arrivals:
                    wait = arrivals[0].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                else:
                    time.sleep(poll_s)
        finally:
            builder.shutdown(wait=True)
        lat = [r.latency for r in reqs]
        first = min(r.arrival for r in reqs)
        makespan = max(r.done for r in reqs) - first
        return Stats(n=len(reqs), nodes=sum(r.batch for r in reqs), makespan=makespan,
                     p50=percentile(lat, 50), p99=percentile(lat, 99),
                     mean_latency=sum(lat) / len(lat), peak_bytes=peak_bytes,
                     peak_inflight=peak_inflight, budget=self.budget,
                     extra={"policy": self.policy, "chunk_s": self.chunk_s})


def replay_chunked(requests, seconds_per_node, chunk_s, policy="srpt", slots=8, rate_scale=1.0,
                   bytes_of=None, budget=None):
    """The chunked scheduler of ServingEngine._run_chunked replayed in virtual time: the same
    arrivals (times multiplied by rate_scale), the same chunk sizes (cost model), the same
    admission in arrival order under the memory budget (when bytes_of and budget are given)
    and the same choice of the next chunk (srpt or fifo, one chunk per plan at a time), with
    the device modelled as one server that works through the chunks in flight side by side
    (processor sharing: k chunks in flight each advance at 1/k of the device).
    seconds_per_node(r) is the measured device time per node of the request's (N, s) when it
    has the whole device.  Plan building is not modelled.  Returns Stats (latency =
    completion - arrival)."""
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    arr = [(r.arrival * rate_scale, r) for r in reqs]
    left = {r.rid: r.batch for r in reqs}     # nodes not yet handed out
    todo = {r.rid: r.batch for r in reqs}     # nodes not yet completed
    done_at = {}
    waiting = collections.deque()             # arrived, not yet admitted (arrival order)
    active = []                               # admitted requests with nodes to hand out
    running = []                              # [remaining device seconds, request, nodes]
    t, i = 0.0, 0
    peak = 0
    in_use, peak_bytes = 0, 0

    def pick():
        busy = {r.plan_key for (_, r, _) in running}
        cand = [r for r in active if left[r.rid] > 0 and r.plan_key not in busy]
        if not cand:
            return None
        if policy == "fifo":
            return min(cand, key=lambda r: (r.arrival, r.rid))
        return min(cand, key=lambda r: (left[r.rid] * cost_per_node(r), r.arrival, r.rid))

    while i < len(arr) or running or waiting or any(left[r.rid] > 0 for r in active):
        while i < len(arr) and arr[i][0] <= t + 1e-15:
            waiting.append(arr[i][1])
            i += 1
        while waiting:
            need = bytes_of(waiting[0]) if bytes_of else 0
            if budget is not None and in_use + need > budget and (active or running):
                break
            r = waiting.popleft()
            in_use += need
            peak_bytes = max(peak_bytes, in_use)
            active.append(r)
        while len(running) < slots:
            r = pick()
            if r is None:
                break
            n = min(left[r.rid], max(1, int(chunk_s / cost_per_node(r))))
            left[r.rid] -= n
            running.append([n * seconds_per_node(r), r, n])
        peak = max(peak, len(running))
        if not running:
            if i < len(arr):
                t = arr[i][0]
                continue
            break
        k = len(running)
        # next event: a chunk finishes (at rate 1/k) or a request arrives
        dt_finish = min(c[0] for c in running) * k
        dt_arrive = arr[i][0] - t if i < len(arr) else float("inf")
        dt = min(dt_finish, dt_arrive)
        for c in running:
            c[0] -= dt / k
        t += dt
        for c in [c for c in running if c[0] <= 1e-12]:
            running.remove(c)
            r = c[1]
            todo[r.rid] -= c[2]
            if todo[r.rid] == 0:
                done_at[r.rid] = t
                active.remove(r)
                in_use -= bytes_of(r) if bytes_of else 0
    lat = [done_at[r.rid] - r.arrival * rate_scale for r in reqs]
    first = min(r.arrival for r in reqs) * rate_scale
    return Stats(n=len(reqs), nodes=sum(r.batch for r in reqs), makespan=max(done_at.values()) - first,
                 p50=percentile(lat, 50), p99=percentile(lat, 99), mean_latency=sum(lat) / len(lat),
                 peak_bytes=peak_bytes, peak_inflight=peak, budget=budget or 0,
                 extra={"policy": policy, "chunk_s": chunk_s, "rate_scale": rate_scale})


class FakeExecutor:
    """CPU model of the device for scheduler tests: a request occupies its slot for
    `seconds_per_node * batch` and needs a fixed number of bytes per node."""

    def __init__(self, seconds_per_node=1e-5, bytes_per_node=1 << 20, plan_bytes=1 << 24):
        self.spn, self.bpn, self.pb = seconds_per_node, bytes_per_node, plan_bytes
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.log = []

    def prepare(self, r):
        return self.pb + self.bpn * r.batch

    def submit(self, r, slot):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.log.append(("submit", r.rid, slot))
        r._t_end = time.perf_counter() + self.spn * r.batch

    def done(self, r):
        return time.perf_counter() >= r._t_end

    def release(self, r):
        with self.lock:
            self.active -= 1
            self.log.append(("release", r.rid, r.slot))

    # chunked mode: a chunk of n nodes occupies its slot for seconds_per_node * n
    def begin(self, r):
        self.log.append(("begin", r.rid))

    def submit_chunk(self, r, slot, lo, hi):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.log.append(("chunk", r.rid, slot, lo, hi))
        if not hasattr(self, "_slot_end"):
            self._slot_end = {}
        self._slot_end[slot] = time.perf_counter() + self.spn * (hi - lo)

    def chunk_done(self, slot):
        if time.perf_counter() >= self._slot_end[slot]:
            with self.lock:
                self.active -= 1
            self._slot_end[slot] = float("inf")
            return True
        return False

    def finish(self, r):
        self.log.append(("finish", r.rid))


class GpuExecutor:
    """Drives libdgfs: plans from a cache (shared by requests with equal parameters), one
    CUDA stream per slot, device-resident inputs tiled from a seeded node pool.  Every kernel
    is limited to `sm_share` of the SMs so that concurrent slots share the device."""

    def __init__(self, slots=8, precision="fp32", pool_nodes=32, keep_outputs=False, device=0,
                 sm_share=0.5):
        import torch

        from . import dgfs, synth
        self.torch, self.dgfs, self.synth = torch, dgfs, synth
        self.dev = torch.device("cuda", device)
        self.dt = torch.float32 if precision == "fp32" else torch.float64
        self.precision = precision
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.pool_nodes = pool_nodes
        self.pools = {}
        self.plans = {}
        self.plan_users = collections.Counter()
        self.lock = threading.Lock()
        self.keep_outputs = keep_outputs
        self.sm_share = sm_share
        self.outputs = {}
        self.state = {}
        self.slot_events = {}

    def _pool(self, N, s):
        """Seeded input nodes per (N, s), on the device (bi-Maxwellians with 5% noise)."""
        key = (N, s)
        if key not in self.pools:
            w = self.synth.Workload("serving pool", self.pool_nodes, N, L_FOR_N[N],
                                    tuple([1.0] * s), 0.75, 1.0, 12, N // 2, "bimaxwellian", 0.05,
                                    9000 + 100 * N + s)
            f = self.synth.batch_distribution(w)
            self.pools[key] = self.torch.from_numpy(f).to(device=self.dev, dtype=self.dt)
        return self.pools[key]

    def prepare(self, r):
        torch = self.torch
        with torch.cuda.device(self.dev):
            with self.lock:
                plan = self.plans.get(r.plan_key)
                if plan is None:
                    plan = self.dgfs.Plan(r.N, r.L, list(r.masses), r.omega, M=r.M, N_rho=r.N_rho,
                                          precision=self.precision)
                    # a kernel takes at most this share of the SMs, so requests in other
                    # slots run beside it instead of queueing behind it
                    plan.set_sm_share(self.sm_share)
                    self.plans[r.plan_key] = plan
                self.plan_users[r.plan_key] += 1
            self._pool(r.N, r.s)
        tables, work = plan.bytes(0)
        esz = 4 if self.precision == "fp32" else 8
        n3 = r.N ** 3
        return tables + work + r.batch * (r.s + r.s * r.s) * n3 * esz

    def submit(self, r, slot):
        torch = self.torch
        st = self.streams[slot]
        plan = self.plans[r.plan_key]
        pool = self._pool(r.N, r.s)
        with torch.cuda.stream(st):
            idx = (torch.arange(r.batch, device=self.dev) + r.pool_offset) % self.pool_nodes
            f = pool.index_select(0, idx)
            Q = torch.empty((r.batch, r.s, r.s, r.N, r.N, r.N), dtype=self.dt, device=self.dev)
            plan.eval_ptr(f.data_ptr(), Q.data_ptr(), r.batch, st)
            ev = torch.cuda.Event()
            ev.record(st)
        self.state[r.rid] = (f, Q, ev)

    def done(self, r):
        return self.state[r.rid][2].query()

    def release(self, r):
        f, Q, ev = self.state.pop(r.rid)
        if self.keep_outputs:
            self.outputs[r.rid] = Q
        with self.lock:
            self.plan_users[r.plan_key] -= 1
            if self.plan_users[r.plan_key] == 0:
                self.plans.pop(r.plan_key).close()
                del self.plan_users[r.plan_key]

    # chunked mode: inputs and outputs of the whole request at admission, one launch per chunk
    def begin(self, r):
        torch = self.torch
        pool = self._pool(r.N, r.s)
        with torch.cuda.device(self.dev):
            idx = (torch.arange(r.batch, device=self.dev) + r.pool_offset) % self.pool_nodes
            f = pool.index_select(0, idx)
            Q = torch.empty((r.batch, r.s, r.s, r.N, r.N, r.N), dtype=self.dt, device=self.dev)
            ready = torch.cuda.Event()
            ready.record(torch.cuda.current_stream(self.dev))
        self.state[r.rid] = (f, Q, ready)

    def submit_chunk(self, r, slot, lo, hi):
        torch = self.torch
        st = self.streams[slot]
        f, Q, ready = self.state[r.rid]
        plan = self.plans[r.plan_key]
        with torch.cuda.stream(st):
            st.wait_event(ready)
            plan.eval_ptr(f[lo].data_ptr(), Q[lo].data_ptr(), hi - lo, st)
            ev = torch.cuda.Event()
            ev.record(st)
        self.slot_events[slot] = ev

    def chunk_done(self, slot):
        return self.slot_events[slot].query()

    def finish(self, r):
        self.release(r)

    def warmup(self, grids=(16, 24, 32, 48), species=(2, 3)):
        """One small evaluation per (N, s) through the same calls as `submit`, so the first
        requests of a run do not pay the one-time start-up of the library and of torch's
        device operators.  Returns the seconds it took."""
        torch = self.torch
        t0 = time.perf_counter()
        for N in grids:
            for s in species:
                r = Request(rid=-1, arrival=0.0, N=N, L=L_FOR_N[N], masses=tuple([1.0] * s),
                            omega=0.75, M=12, N_rho=N // 2, batch=2)
                self.prepare(r)
                self.submit(r, 0)
                self.streams[0].synchronize()
                self.release(r)
        torch.cuda.synchronize(self.dev)
        return time.perf_counter() - t0

    # nodes per timed evaluation: enough work items to fill the device at every N
    SERVICE_NODES = {8: 1024, 12: 1024, 16: 512, 24: 256, 32: 128, 48: 48}

    def service_seconds_per_node(self, keys, precision=None):
        """Device seconds per node with the whole device, per (N, s) in keys, measured with
        CUDA events on one evaluation of SERVICE_NODES[N] nodes (after one warm-up evaluation)
        with a plan of the serving mix's parameters (masses 1 .. 2.5, omega 0.75, M = 12,
        N_rho = N/2) in `precision` (default: the executor's)."""
        torch = self.torch
        prec = precision or self.precision
        dt = torch.float32 if prec != "fp64" else torch.float64
        out = {}
        for N, s in keys:
            nodes = self.SERVICE_NODES[N]
            masses = list(np.linspace(1.0, 2.5, s))
            plan = self.dgfs.Plan(N, L_FOR_N[N], masses, 0.75, M=12, N_rho=N // 2, precision=prec)
            pool = self._pool(N, s).to(dt)
            idx = torch.arange(nodes, device=self.dev) % self.pool_nodes
            f = pool.index_select(0, idx).contiguous()
            Q = torch.empty((nodes, s, s, N, N, N), dtype=dt, device=self.dev)
            st = torch.cuda.current_stream(self.dev)
            plan.eval_ptr(f.data_ptr(), Q.data_ptr(), nodes, st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            plan.eval_ptr(f.data_ptr(), Q.data_ptr(), nodes, st)
            e1.record(st)
            torch.cuda.synchronize(self.dev)
            out[(N, s)] = e0.elapsed_time(e1) * 1e-3 / nodes
            plan.close()
            del f, Q
        return out

    def run_alone(self, r):
        """Evaluate one request by itself (fresh plan, default stream); returns Q."""
        torch = self.torch
        plan = self.dgfs.Plan(r.N, r.L, list(r.masses), r.omega, M=r.M, N_rho=r.N_rho,
                              precision=self.precision)
        pool = self._pool(r.N, r.s)
        idx = (torch.arange(r.batch, device=self.dev) + r.pool_offset) % self.pool_nodes
        Q = plan.eval(pool.index_select(0, idx).contiguous())
        torch.cuda.synchronize()
        plan.close()
        return Q
