"""Host logic of the streaming service (admission, micro-batching, completion order), on CPU.

A fake backend completes each batch a fixed simulated time after its launch and echoes the
syndromes as corrections, so every output row can be traced back to its request.
"""
import numpy as np
import pytest

from paper_2508_15743_gb300 import service as S

STATS = np.dtype([("status", "u1"), ("lsd_invoked", "u1"), ("n_converged", "u1"), ("chosen_member", "u1"),
                  ("iters", "<u2"), ("largest_cluster", "<u2"), ("n_clusters", "<u4")])


class Clock:
    def __init__(self, step):
        self.t, self.step = 0.0, step

    def __call__(self):
        return self.t

    def idle(self):
        self.t += self.step


class FakeBackend:
    def __init__(self, clock, pipelines, latency, max_batch):
        self.clock, self.pipelines, self.latency, self.max_batch = clock, pipelines, latency, max_batch
        self.due = [None] * pipelines
        self.out = [None] * pipelines
        self.launches = []

    def launch(self, pipe, problems, syndromes):
        assert self.due[pipe] is None, "launch on a busy pipeline"
        assert len(problems) <= self.max_batch
        self.due[pipe] = self.clock() + self.latency
        self.out[pipe] = (np.asarray(syndromes).copy(), np.asarray(problems).reshape(-1, 1).astype(np.uint32))
        self.launches.append((self.clock(), len(problems)))

    def done(self, pipe):
        return self.due[pipe] is not None and self.clock() >= self.due[pipe]

    def results(self, pipe):
        syn, prob = self.out[pipe]
        self.due[pipe] = None
        return syn, prob, np.zeros(len(syn), STATS)


def run_fake(rate, count, capacity, max_batch, latency, pipelines=2, wait=1e-4, step=1e-5, seed=0):
    clk = Clock(step)
    be = FakeBackend(clk, pipelines, latency, max_batch)
    svc = S.StreamingService(be, capacity=capacity, max_batch=max_batch, max_wait_s=wait)
    arr = S.poisson_arrivals(rate, count, seed)
    rng = np.random.default_rng(seed)
    prob = rng.integers(0, 3, count).astype(np.int32)
    syn = rng.integers(0, 2**31, (count, 2)).astype(np.uint32)
    rep, corr, logi, st = svc.run(arr, prob, syn, clock=clk, idle=clk.idle)
    return rep, corr, logi, syn, prob, be, arr


def test_poisson_arrivals_are_seeded_with_the_right_rate():
    a = S.poisson_arrivals(1000.0, 20000, 3)
    assert np.array_equal(a, S.poisson_arrivals(1000.0, 20000, 3))
    gaps = np.diff(a)
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() - 1e-3) < 3 * 1e-3 / np.sqrt(len(gaps))   # exponential: sd = mean
    # exponential gaps: P(gap > mean) = 1/e
    assert abs((gaps > 1e-3).mean() - np.exp(-1)) < 0.02


def test_every_request_completes_in_order_with_its_own_output():
    rep, corr, logi, syn, prob, be, arr = run_fake(rate=5e4, count=3000, capacity=512, max_batch=256,
                                                   latency=2e-3)
    assert rep.requests == 3000
    assert np.array_equal(corr, syn)               # row i holds request i's output
    assert np.array_equal(logi[:, 0], prob)
    assert rep.max_inflight <= 512
    assert all(n <= 256 for _, n in be.launches)
    assert sum(n for _, n in be.launches) == 3000
    assert rep.latency_ms["p50"] <= rep.latency_ms["p99"] <= rep.latency_ms["p999"] <= rep.latency_ms["max"]
    assert rep.latency_ms["p50"] >= 2.0 - 1e-9     # nothing completes before the backend latency


def test_capacity_bounds_the_batches_below_max_batch():
    rep, corr, logi, syn, prob, be, arr = run_fake(rate=1e6, count=2000, capacity=100, max_batch=1000,
                                                   latency=1e-3)
    assert all(n <= 100 for _, n in be.launches)
    assert rep.max_inflight <= 100
    assert np.array_equal(corr, syn)


def test_batches_wait_for_max_wait_or_a_full_batch():
    # slow arrivals: each batch leaves when its oldest request has waited max_wait
    rep, corr, logi, syn, prob, be, arr = run_fake(rate=1e3, count=200, capacity=10_000, max_batch=10_000,
                                                   latency=1e-4, wait=5e-3, step=1e-5)
    starts = [t for t, _ in be.launches]
    assert len(starts) < 200                       # requests were grouped
    assert rep.latency_ms["max"] <= 5.0 + 0.1 + 0.2   # wait + latency + polling steps (ms)


def test_overload_makes_latency_grow():
    # arrivals faster than the backend can serve: the queue and the latency grow over the run
    rep, corr, logi, syn, prob, be, arr = run_fake(rate=2e6, count=20000, capacity=500, max_batch=250,
                                                   latency=1e-3)
    lat = rep.latency_ms
    assert lat["p99"] > 5 * lat["p50"] or lat["max"] > 5.0
    assert rep.throughput < 0.6e6                  # at most capacity / latency = 5e5 per second


def test_rejects_bad_arguments():
    clk = Clock(1e-5)
    with pytest.raises(ValueError):
        S.StreamingService(FakeBackend(clk, 1, 1e-3, 4), capacity=0, max_batch=4)
    svc = S.StreamingService(FakeBackend(clk, 1, 1e-3, 4), capacity=4, max_batch=4)
    with pytest.raises(ValueError):
        svc.run(np.array([1.0, 0.5]), np.zeros(2, np.int32), np.zeros((2, 1), np.uint32), clock=clk, idle=clk.idle)


def test_device_bytes_per_shot_counts_io_and_workspace():
    assert S.device_bytes_per_shot(1, 1, 1, 10) == 4 * 3 + 12 + 4 + 4 + 40


def test_make_requests_is_seeded_and_mixes_problems():
    from paper_2508_15743_gb300 import dem as D
    dems = [D.build_workload("cc666_d5_codecap"), D.phenomenological_dem(3, 2, 0.05, 0.05)]
    a = S.make_requests(dems, 2000, 5e4, seed=3)
    b = S.make_requests(dems, 2000, 5e4, seed=3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    arrivals, problems, syn, obs = a
    assert np.all(np.diff(arrivals) >= 0)
    assert set(np.unique(problems)) == {0, 1}
    assert syn.shape == (2000, max(D.words(d.m) for d in dems))
    # each row's syndrome uses only its own problem's words and bits
    for i, dm in enumerate(dems):
        rows = problems == i
        assert not syn[rows][:, D.words(dm.m):].any()
        rem = dm.m % 32
        if rem:
            assert not (syn[rows][:, D.words(dm.m) - 1] >> rem).any()


def test_bench_binomial_interval():
    import bench
    r = bench.ler_ci(100, 10_000)
    assert r["ler"] == 0.01 and r["failures"] == 100 and r["shots"] == 10_000
    half = 2 * np.sqrt(0.01 * 0.99 / 10_000)
    assert np.isclose(r["two_sigma"][0], 0.01 - half) and np.isclose(r["two_sigma"][1], 0.01 + half)
    z = bench.ler_ci(0, 1000)           # no failures: the interval still has width
    assert z["two_sigma"][0] == 0.0 and z["two_sigma"][1] > 0.0
