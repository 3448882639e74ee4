"""Streaming decoding service: syndrome requests arrive over time and are decoded in micro-batches.

The paper motivates VibeLSD by real-time decoding (Sec. I): syndromes arrive continuously and each
must be decoded with low latency. This module is the serving loop around the library:

  * resident problems: one vibe handle per detector error model (Tanner graph, schedules and
    wavefronts built once and kept on the device), grouped in mixed batches (vibe_batch_*) so that
    one launch pair decodes requests of different codes;
  * admission by a device-memory budget: a request enters the GPU only while the shots in flight
    fit in what the budget leaves after the resident tables and the fixed workspaces; the others
    wait in arrival order;
  * micro-batching: a batch is launched when `max_batch` requests are waiting, when the oldest has
    waited `max_wait_s`, or when no more arrivals are due; `pipelines` batches can be in flight on
    their own CUDA streams (each pipeline owns a vibe_batch and its workspace, so they never share
    scratch memory);
  * per-request latency = completion time (the host sees the batch's event complete) minus the
    request's arrival time; reported as p50 / p99 / p99.9 beside the sustained throughput.

Arrivals are a seeded Poisson process (exponential inter-arrival times). The loop itself is host
code; every decoding step runs in the CUDA library through the C ABI.
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass, field

import numpy as np


def poisson_arrivals(rate_hz: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of `count` requests of a Poisson process of rate `rate_hz`."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


@dataclass
class ServiceReport:
    requests: int
    duration_s: float
    throughput: float                 # requests completed per second of wall time
    latency_ms: dict                  # p50 / p99 / p999 / max
    batches: int
    mean_batch: float
    max_inflight: int
    capacity: int
    failures: int = -1                # logical failures against the given observables (-1: not given)
    extra: dict = field(default_factory=dict)

    def to_json(self) -> str:
        return json.dumps(self.__dict__)


class StreamingService:
    """Admission, micro-batching and completion tracking over a backend that decodes batches.

    backend: an object with
        pipelines: int
        launch(pipe, problem_ids, syndromes) -> None    (asynchronous; one batch per pipeline)
        done(pipe) -> bool                              (the pipeline's batch has completed)
        results(pipe) -> (corrections, logical, stats)  (host arrays of the completed batch)
    capacity: the largest number of shots in flight that the memory budget admits.
    """

    def __init__(self, backend, capacity: int, max_batch: int, max_wait_s: float = 0.0005):
        if capacity < 1 or max_batch < 1:
            raise ValueError("capacity and max_batch must be positive")
        self.backend = backend
        self.capacity = int(capacity)
        self.max_batch = int(max_batch)
        self.max_wait_s = float(max_wait_s)

    def run(self, arrivals, problems, syndromes, observables=None, clock=time.perf_counter, idle=lambda: None):
        """Serve requests i = 0..N-1 (arrival time arrivals[i], problem problems[i], syndrome row i).

        Returns (ServiceReport, corrections [N, nw], logical [N, kw], stats [N]) with the outputs of
        every request in arrival order.
        """
        arrivals = np.asarray(arrivals, dtype=np.float64)
        N = len(arrivals)
        if N == 0:
            raise ValueError("no requests")
        if np.any(np.diff(arrivals) < 0):
            raise ValueError("arrival times must be non-decreasing")
        done_t = np.full(N, np.nan)
        corr = logi = stats = None
        inflight = {}                     # pipe -> (first request, count)
        free = list(range(self.backend.pipelines))
        head = 0                          # first request not yet launched
        completed = 0
        batches = 0
        max_inflight = 0
        t0 = clock()
        while completed < N:
            now = clock() - t0
            # completions
            for pipe in list(inflight):
                if self.backend.done(pipe):
                    first, cnt = inflight.pop(pipe)
                    c, l, s = self.backend.results(pipe)
                    if corr is None:
                        corr = np.zeros((N, c.shape[1]), c.dtype)
                        logi = np.zeros((N, l.shape[1]), l.dtype)
                        stats = np.zeros(N, s.dtype)
                    corr[first:first + cnt] = c[:cnt]
                    logi[first:first + cnt] = l[:cnt]
                    stats[first:first + cnt] = s[:cnt]
                    done_t[first:first + cnt] = clock() - t0
                    completed += cnt
                    free.append(pipe)
            # arrivals up to now: requests head .. arrived - 1 are waiting
            arrived = int(np.searchsorted(arrivals, now, side="right"))
            waiting = arrived - head
            in_flight = sum(c for _, c in inflight.values())
            room = self.capacity - in_flight
            if free and waiting > 0 and room > 0:
                due = (waiting >= self.max_batch or now - arrivals[head] >= self.max_wait_s or arrived == N)
                if due:
                    cnt = min(waiting, self.max_batch, room)
                    pipe = free.pop(0)
                    self.backend.launch(pipe, problems[head:head + cnt], syndromes[head:head + cnt])
                    inflight[pipe] = (head, cnt)
                    head += cnt
                    batches += 1
                    max_inflight = max(max_inflight, in_flight + cnt)
                    continue
            idle()
        lat = (done_t - arrivals) * 1e3
        span = float(np.nanmax(done_t) - arrivals[0])
        rep = ServiceReport(
            requests=N, duration_s=span, throughput=N / span if span > 0 else float("inf"),
            latency_ms=dict(p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                            p999=float(np.percentile(lat, 99.9)), max=float(lat.max())),
            batches=batches, mean_batch=N / max(batches, 1), max_inflight=max_inflight, capacity=self.capacity)
        if observables is not None:
            kwn = observables.shape[1]
            rep.failures = int((logi[:, :kwn] != observables).any(axis=1).sum())
        return rep, corr, logi, stats


# ---------------------------------------------------------------------------------------------
# GPU backend: mixed batches through the C ABI, one CUDA stream and pinned buffers per pipeline
# ---------------------------------------------------------------------------------------------

class GpuBackend:
    """Decodes micro-batches with vibe_batch_decode; outputs come back through pinned host memory."""

    def __init__(self, decoders, max_batch: int, pipelines: int = 2):
        import torch

        from . import vibe as V
        self.torch, self.V = torch, V
        self.pipelines = int(pipelines)
        self.max_batch = int(max_batch)
        self.mw = max(d.mw for d in decoders)
        self.nw = max(d.nw for d in decoders)
        self.kw = max(d.kw for d in decoders)
        self.handles = [V.vibe_batch_create([d.handle for d in decoders]) for _ in range(self.pipelines)]
        self.streams = [torch.cuda.Stream() for _ in range(self.pipelines)]
        self.events = [torch.cuda.Event() for _ in range(self.pipelines)]
        B = self.max_batch
        i32, u8 = torch.int32, torch.uint8

        def pinned(shape, dt):
            return torch.zeros(shape, dtype=dt, pin_memory=True)

        def dev(shape, dt):
            return torch.zeros(shape, dtype=dt, device="cuda")

        self.h = [dict(syn=pinned((B, self.mw), i32), pid=pinned((B,), i32), corr=pinned((B, self.nw), i32),
                       log=pinned((B, self.kw), i32), st=pinned((B, 12), u8)) for _ in range(self.pipelines)]
        self.d = [dict(syn=dev((B, self.mw), i32), pid=dev((B,), i32), corr=dev((B, self.nw), i32),
                       log=dev((B, self.kw), i32), st=dev((B, 12), u8)) for _ in range(self.pipelines)]
        self.n = [0] * self.pipelines

    def launch(self, pipe, problems, syndromes):
        torch, V = self.torch, self.V
        n = len(problems)
        h, d, s = self.h[pipe], self.d[pipe], self.streams[pipe]
        h["syn"].numpy()[:n] = np.asarray(syndromes).view(np.int32)
        h["pid"].numpy()[:n] = problems
        with torch.cuda.stream(s):
            d["syn"][:n].copy_(h["syn"][:n], non_blocking=True)
            d["pid"][:n].copy_(h["pid"][:n], non_blocking=True)
            d["corr"][:n].zero_()
            d["log"][:n].zero_()
            V.vibe_batch_decode(self.handles[pipe], d["pid"], d["syn"], self.mw, n, d["corr"], self.nw, d["log"],
                                self.kw, d["st"], None, None, stream=s)
            h["corr"][:n].copy_(d["corr"][:n], non_blocking=True)
            h["log"][:n].copy_(d["log"][:n], non_blocking=True)
            h["st"][:n].copy_(d["st"][:n], non_blocking=True)
            self.events[pipe].record(s)
        self.n[pipe] = n

    def done(self, pipe):
        return self.events[pipe].query()

    def results(self, pipe):
        n, h = self.n[pipe], self.h[pipe]
        return (h["corr"].numpy()[:n].view(np.uint32).copy(), h["log"].numpy()[:n].view(np.uint32).copy(),
                self.V.stats_to_numpy(h["st"][:n]).copy())

    def close(self):
        for b in self.handles:
            self.V.vibe_batch_destroy(b)
        self.handles = []


def device_bytes_per_shot(mw: int, nw: int, kw: int, n_max: int) -> int:
    """Device memory one in-flight shot holds: the service's syndrome, problem id and output rows and
    the library's per-shot workspace (LSD queue entry and soft vector)."""
    return 4 * (mw + nw + kw) + 12 + 4 + 4 + 4 * n_max


# Problems the command line knows: name -> (DEM builder, K, T, M, natural order)
def _problem_specs():
    from . import circuit as C
    from . import dem as D
    return {
        "codecap_d5": (lambda: D.build_workload("cc666_d5_codecap"), 1, 20, 1, True),
        "pheno_d9": (lambda: D.build_workload("cc666_d9_pheno"), 16, 30, 5, False),
        "circuit_d9": (lambda: C.circuit_dem(9, 9, 0.001, noise="si1000", basis="X"), 32, 50, 5, False),
        "circuit_d13": (lambda: C.circuit_dem(13, 13, 0.001, noise="si1000", basis="X"), 32, 50, 7, False),
    }


def build_service(names, budget_bytes: int, fp16: bool, max_batch: int, pipelines: int = 2,
                  max_wait_s: float = 0.0005, seed: int = 0, pair_mode: bool = False):
    """Creates the resident problems, sizes the micro-batches to the device-memory budget, warms the
    pipelines up and returns (service, backend, decoders, dems). pair_mode decodes each shot's members
    at the same time on different warps (vibe_params.pair_mode): same outputs, lower latency per
    request when the GPU is not saturated."""
    import torch

    from . import dem as D
    from . import vibe as V
    specs = _problem_specs()
    free0, _ = torch.cuda.mem_get_info()
    dems, decs = [], []
    for i, name in enumerate(names):
        build, K, T, M, natural = specs[name]
        dm = build()
        dems.append(dm)
        decs.append(V.Decoder(dm, K, D.schedules(dm.n, K, seed + i, natural=natural), T=T, M=M, msg_fp16=fp16,
                              pair_mode=pair_mode))
    mw = max(d.mw for d in decs)
    nw = max(d.nw for d in decs)
    kw = max(d.kw for d in decs)
    per_shot = device_bytes_per_shot(mw, nw, kw, max(d.n for d in decs))
    # fixed part: resident tables and the pipelines' shot-independent workspaces (measured)
    probe = GpuBackend(decs, 1, pipelines)
    for p in range(pipelines):
        probe.launch(p, np.zeros(1, np.int32), np.zeros((1, mw), np.uint32))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    probe.close()
    fixed = max(free0 - free1, 0)
    fit = (budget_bytes - fixed) // (pipelines * per_shot)
    if fit < 1:
        raise MemoryError(f"budget {budget_bytes} B leaves no room for a shot (fixed part {fixed} B)")
    mb = int(min(max_batch, fit))
    backend = GpuBackend(decs, mb, pipelines)
    for p in range(pipelines):   # grow every workspace to the batch size before serving
        backend.launch(p, np.zeros(mb, np.int32), np.zeros((mb, mw), np.uint32))
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    svc = StreamingService(backend, capacity=pipelines * mb, max_batch=mb, max_wait_s=max_wait_s)
    svc.budget = dict(budget_bytes=int(budget_bytes), fixed_bytes=int(fixed), per_shot_bytes=int(per_shot),
                      max_batch=mb, pipelines=pipelines, used_bytes=int(max(free0 - free2, 0)),
                      pair_mode=bool(pair_mode))
    return svc, backend, decs, dems


def make_requests(dems, count: int, rate_hz: float, seed: int):
    """Seeded request stream: Poisson arrival times, uniformly mixed problems, sampled syndromes."""
    from . import dem as D
    rng = np.random.default_rng(seed)
    arrivals = poisson_arrivals(rate_hz, count, seed + 1)
    problems = rng.integers(0, len(dems), count).astype(np.int32)
    mw = max(D.words(dm.m) for dm in dems)
    kw = max(D.words(dm.k) for dm in dems)
    syn = np.zeros((count, mw), np.uint32)
    obs = np.zeros((count, kw), np.uint32)
    for i, dm in enumerate(dems):
        rows = np.nonzero(problems == i)[0]
        if len(rows):
            s, o = D.sample(dm, len(rows), seed + 100 + i)
            syn[rows, :s.shape[1]] = s
            obs[rows, :o.shape[1]] = o
    return arrivals, problems, syn, obs


def main():
    import argparse
    ap = argparse.ArgumentParser(description="Streaming VibeLSD decoding with Poisson arrivals")
    ap.add_argument("--mix", default="codecap_d5,pheno_d9", help="comma-separated problems: "
                    + ",".join(sorted(_problem_specs())))
    ap.add_argument("--rate", type=float, default=200_000.0, help="arrivals per second")
    ap.add_argument("--requests", type=int, default=200_000)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--fp16", action="store_true")
    ap.add_argument("--max-batch", type=int, default=65_536)
    ap.add_argument("--max-wait-us", type=float, default=500.0)
    ap.add_argument("--pipelines", type=int, default=2)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--pair-mode", action="store_true", help="one warp per (shot, member) pair")
    args = ap.parse_args()
    names = args.mix.split(",")
    svc, backend, decs, dems = build_service(names, int(args.budget_gb * 2**30), args.fp16, args.max_batch,
                                             args.pipelines, args.max_wait_us * 1e-6, args.seed, args.pair_mode)
    arrivals, problems, syn, obs = make_requests(dems, args.requests, args.rate, args.seed)
    rep, corr, logi, stats = svc.run(arrivals, problems, syn, observables=obs)
    rep.extra = dict(mix=names, rate=args.rate, fp16=args.fp16, budget=svc.budget,
                     ler=rep.failures / rep.requests, lsd_fraction=float(stats["lsd_invoked"].mean()))
    print(rep.to_json())
    backend.close()
    for d in decs:
        d.close()


if __name__ == "__main__":
    main()
