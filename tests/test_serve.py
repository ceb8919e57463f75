"""Serving loop: admission by slots and HBM budget, arrival order, latency statistics (CPU,
fake executor), and on the GPU: every request's result equals its result alone."""

import math

import pytest

from paper_1903_03056_gb300 import serve


def _small_stream(n, rate, seed=1):
    return serve.mixed_stream(n, rate, seed=seed, sizes=(8, 12, 16), max_batch=64)


def test_stream_is_seeded_and_shaped():
    a, b = _small_stream(20, 100.0), _small_stream(20, 100.0)
    assert [(r.N, r.masses, r.batch, r.arrival) for r in a] == [(r.N, r.masses, r.batch, r.arrival) for r in b]
    assert all(r.N in (8, 12, 16) and r.s in (2, 3) and 1 <= r.batch <= 64 for r in a)
    assert all(1.0 <= m <= 4.0 for r in a for m in r.masses)
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))


def test_percentile():
    assert serve.percentile([1, 2, 3, 4], 50) == 2.5
    assert serve.percentile(list(range(101)), 99) == 99


def test_admission_respects_budget_and_slots():
    fake = serve.FakeExecutor(seconds_per_node=2e-5, bytes_per_node=1 << 20, plan_bytes=1 << 24)
    budget = (1 << 24) * 3 + (1 << 20) * 150
    eng = serve.ServingEngine(fake, budget_bytes=budget, slots=4)
    reqs = _small_stream(40, math.inf)
    st = eng.run(reqs)
    assert st.n == 40 and all(r.done is not None for r in reqs)
    assert st.peak_bytes <= budget and st.peak_inflight <= 4 and fake.max_active <= 4
    assert st.peak_inflight > 1
    assert st.p50 <= st.p99


def test_admission_in_arrival_order():
    fake = serve.FakeExecutor(seconds_per_node=1e-5)
    eng = serve.ServingEngine(fake, budget_bytes=1 << 40, slots=3)
    reqs = _small_stream(30, 2000.0, seed=3)
    eng.run(reqs)
    order = [rid for kind, rid, _ in fake.log if kind == "submit"]
    assert order == sorted(order)


def test_request_larger_than_budget_is_an_error():
    fake = serve.FakeExecutor(bytes_per_node=1 << 30)
    eng = serve.ServingEngine(fake, budget_bytes=1 << 30, slots=2)
    with pytest.raises(RuntimeError):
        eng.run(_small_stream(3, math.inf))


@pytest.mark.gpu
@pytest.mark.parametrize("chunk_s", [None, 2e-4])
def test_each_result_equals_its_result_alone(chunk_s):
    """Whole-request and chunked (SRPT) service: every request's output in the mix is bitwise
    equal to its output evaluated alone."""
    import torch
    from paper_1903_03056_gb300 import build
    build.build()
    ex = serve.GpuExecutor(slots=4, keep_outputs=True)
    reqs = _small_stream(16, 400.0, seed=11)
    st = serve.ServingEngine(ex, budget_bytes=8 << 30, slots=4, chunk_s=chunk_s).run(reqs)
    print("serving mix:", st.as_dict())
    assert st.peak_inflight > 1
    for r in reqs:
        alone = ex.run_alone(r)
        assert torch.equal(ex.outputs[r.rid], alone), r.rid


def test_chunked_srpt_lets_small_requests_overtake_a_large_one():
    """Chunked mode: a large request admitted first is split into chunks, and a small request
    that arrives later finishes long before it (FIFO whole-request service would finish it
    after the large one); every node of every request is submitted exactly once."""
    # wall-clock timing: the large request takes 200 ms, so a few ms of thread-scheduling jitter
    # on a loaded host stays well inside the margin
    fake = serve.FakeExecutor(seconds_per_node=5e-5)
    big = serve.Request(0, 0.0, 16, 6.0, (1.0, 2.0), 0.7, 12, 8, 4000)
    small = serve.Request(1, 0.02, 16, 6.0, (1.0, 3.0), 0.7, 12, 8, 20)
    eng = serve.ServingEngine(fake, budget_bytes=1 << 40, slots=1, chunk_s=0.005, policy="srpt")
    st = eng.run([big, small])
    assert small.done < big.done
    assert small.latency < 0.25 * big.latency
    covered = {}
    for ev in fake.log:
        if ev[0] == "chunk":
            _, rid, slot, lo, hi = ev
            covered.setdefault(rid, []).append((lo, hi))
    for r in (big, small):
        spans = sorted(covered[r.rid])
        assert spans[0][0] == 0 and spans[-1][1] == r.batch
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    assert st.n == 2


def test_chunked_fifo_serves_in_arrival_order():
    fake = serve.FakeExecutor(seconds_per_node=2e-5)
    big = serve.Request(0, 0.0, 16, 6.0, (1.0, 2.0), 0.7, 12, 8, 2000)
    small = serve.Request(1, 0.01, 16, 6.0, (1.0, 3.0), 0.7, 12, 8, 20)
    eng = serve.ServingEngine(fake, budget_bytes=1 << 40, slots=1, chunk_s=0.005, policy="fifo")
    eng.run([big, small])
    assert big.done < small.done


def test_chunked_mode_runs_one_chunk_per_plan_at_a_time():
    fake = serve.FakeExecutor(seconds_per_node=1e-5)
    reqs = [serve.Request(k, 0.0, 16, 6.0, (1.0, 2.0), 0.7, 12, 8, 300) for k in range(3)]
    eng = serve.ServingEngine(fake, budget_bytes=1 << 40, slots=4, chunk_s=0.0005, policy="srpt")
    eng.run(reqs)
    assert fake.max_active == 1   # all three share one plan key


# ---- replay of a stream in virtual time (the FP64 comparison of the serving report) --------

def _req(rid, arrival, N, batch, s=2):
    return serve.Request(rid, arrival, N, serve.L_FOR_N[N], tuple([1.0] * s), 0.75, 12, N // 2, batch)


def test_replay_single_request_takes_its_service_time():
    r = _req(0, 0.5, 16, 300)
    st = serve.replay_chunked([r], lambda q: 1e-4, chunk_s=0.05)
    assert abs(st.p50 - 300 * 1e-4) < 1e-9 and abs(st.makespan - 300 * 1e-4) < 1e-9


def test_replay_conserves_work_and_lets_small_requests_overtake():
    """All requests at t = 0 on an idle device: the makespan is the total work (the device never
    idles), and under SRPT the one-node request finishes long before the large one."""
    reqs = [_req(0, 0.0, 32, 4000), _req(1, 0.0, 32, 1), _req(2, 0.0, 16, 50)]
    spn = {32: 1e-4, 16: 1e-5}
    st = serve.replay_chunked(reqs, lambda q: spn[q.N], chunk_s=0.05)
    work = 4000 * 1e-4 + 1e-4 + 50 * 1e-5
    assert abs(st.makespan - work) < 1e-9
    st_f = serve.replay_chunked(reqs, lambda q: spn[q.N], chunk_s=0.05, policy="fifo")
    assert abs(st_f.makespan - work) < 1e-9
    # the small requests' latencies: SRPT far below FIFO
    assert st.p50 < 0.05 * st_f.p50


def test_replay_latency_grows_with_the_service_time_and_the_arrival_scale():
    reqs = serve.mixed_stream(40, 20.0, seed=77)
    fast = serve.replay_chunked(reqs, lambda q: 1e-5, chunk_s=0.05)
    slow = serve.replay_chunked(reqs, lambda q: 3e-4, chunk_s=0.05)
    assert slow.p50 > fast.p50 and slow.p99 > fast.p99
    # stretching the arrivals by the slowdown relieves the queue
    relaxed = serve.replay_chunked(reqs, lambda q: 3e-4, chunk_s=0.05, rate_scale=30.0)
    assert relaxed.p99 < slow.p99
    assert relaxed.n == slow.n == 40 and relaxed.nodes == sum(r.batch for r in reqs)


def test_replay_admits_in_arrival_order_under_the_budget():
    """Two requests that do not fit the budget together: the second is admitted only when the
    first completes, so its latency includes the first's service time."""
    a = _req(0, 0.0, 32, 100)
    b = serve.Request(1, 0.0, 32, serve.L_FOR_N[32], (1.0, 1.5), 0.75, 12, 16, 100)  # another plan
    spn = lambda q: 1e-3  # noqa: E731
    one = serve.request_bytes(a)
    st = serve.replay_chunked([a, b], spn, chunk_s=0.05, bytes_of=serve.request_bytes, budget=int(1.5 * one))
    assert abs(st.makespan - 0.2) < 1e-9 and st.peak_bytes == one
    both = serve.replay_chunked([a, b], spn, chunk_s=0.05, bytes_of=serve.request_bytes, budget=3 * one)
    assert both.peak_bytes == 2 * one
    # serialised by the budget: latencies 0.1 s and 0.2 s (median 0.15 s); sharing the device,
    # both finish at 0.2 s
    assert abs(st.p50 - 0.15) < 1e-9
    assert abs(both.p50 - 0.2) < 1e-9
