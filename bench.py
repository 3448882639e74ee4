"""Benchmark: decoded shots/s of the VibeLSD hot path on GB300, FP32 and FP16 messages.

One step = one vibe_decode call over the whole batch: BP ensemble on every shot, ensemble ranking,
LSD on the shots no member resolved, logical flips and per-shot records. The batch is the d=9
colour-code phenomenological workload (9 noisy + 1 perfect round, p = q = 0.01; m = 300 detectors,
n = 819 mechanisms; K = 16 seeded schedules, T = 30, M = 5, LSD-0), 10^6 shots sampled on the host
with a seeded generator and resident in HBM before timing. Between timed steps a 256 MB buffer is
written to flush L2; each step is timed with CUDA events on the decoding stream.

`--impl reference` times the CPU oracle (plain C, all host cores) on a bounded sample of the same
workload instead. Under torchrun each rank decodes its own 10^6 shots (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2508_15743_gb300 import dem as D  # noqa: E402

WORKLOAD = "cc666_d9_pheno"
METRIC = "decoded shots/s and p50/p99 latency at fixed logical error rate, FP16 vs FP32"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def make_inputs(shots, seed):
    dm = D.build_workload(WORKLOAD)
    w = D.WORKLOADS[WORKLOAD]
    syn, obs = D.sample(dm, shots, seed)
    perms = D.schedules(dm.n, w["K"], w["seed"])
    return dm, w, syn, obs, perms


def cpu_baseline(dm, w, syn, perms, target_s=12.0, max_shots=200_000):
    """The oracle as it stands, all host cores, on a bounded prefix of the same shots."""
    import oracle
    cores = os.cpu_count() or 1
    cal = min(len(syn), 2000)
    t0 = time.perf_counter()
    oracle.decode(dm, perms, syn[:cal], w["T"], w["alpha"], w["M"], nthreads=cores, want_soft=False)
    rate = cal / max(time.perf_counter() - t0, 1e-6)
    S = int(min(len(syn), max_shots, max(cal, rate * target_s)))
    t0 = time.perf_counter()
    ref = oracle.decode(dm, perms, syn[:S], w["T"], w["alpha"], w["M"], nthreads=cores, want_soft=False)
    dt = time.perf_counter() - t0
    return {"value": S / dt, "unit": "shots/s", "cores": cores, "kind": "oracle",
            "sample": f"first {S} shots of the {len(syn)}-shot workload (seed {w['seed']}), FP32 oracle, "
                      f"{cores} threads, {dt:.1f} s"}, ref, S


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w_shots = 60_000
    dm, w, syn, obs, perms = make_inputs(w_shots, D.WORKLOADS[WORKLOAD]["seed"])
    import oracle
    cores = os.cpu_count() or 1
    per_step = 2000
    t0 = time.perf_counter()
    oracle.decode(dm, perms, syn[:per_step], w["T"], w["alpha"], w["M"], nthreads=cores, want_soft=False)
    rate0 = per_step / (time.perf_counter() - t0)
    per_step = int(max(500, min(20_000, rate0 * 6.0)))
    for s in range(args.warmup):
        oracle.decode(dm, perms, syn[:min(per_step, 500)], w["T"], w["alpha"], w["M"], nthreads=cores, want_soft=False)
    times = []
    fails = 0
    for s in range(args.steps):
        lo = (s * per_step) % max(1, w_shots - per_step)
        t0 = time.perf_counter()
        ref = oracle.decode(dm, perms, syn[lo:lo + per_step], w["T"], w["alpha"], w["M"], nthreads=cores,
                            want_soft=False)
        times.append(time.perf_counter() - t0)
        fails += int((ref["logical"] != obs[lo:lo + per_step]).any(axis=1).sum())
    value = per_step * args.steps / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{WORKLOAD}: d=9 colour code, 9+1 phenomenological rounds, p=q=0.01, "
                                   f"K=16, T=30, M=5, LSD-0; {per_step} shots per step (bounded sample of 10^6)",
                       "shots_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "shots/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} shots per step from a 60000-shot prefix (seed {w['seed']})"},
            "e2e": {"value": value, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "ler": fails / (per_step * args.steps)}
    print(json.dumps(line))
    return 0


def ler_ci(fails, shots):
    p = fails / shots if shots else 0.0
    sd = (p * (1 - p) / shots) ** 0.5 if shots else 0.0
    return {"ler": p, "two_sigma": [max(0.0, p - 2 * sd), p + 2 * sd], "failures": int(fails), "shots": int(shots)}


def run_vibe(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2508_15743_gb300 import vibe as V

    w = D.WORKLOADS[WORKLOAD]
    shots = args.shots or w["shots"]
    dm, w, syn, obs, perms = make_inputs(shots, w["seed"] + 1000 * rank)
    B = len(syn)
    syn_d = torch.from_numpy(syn.view(np.int32)).to(dev)
    obs_d = torch.from_numpy(obs.view(np.int32)).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    results = {}
    for label, fp16 in [("f32", False), ("f16", True)]:
        dec = V.Decoder(dm, w["K"], perms, T=w["T"], alpha=w["alpha"], M=w["M"], msg_fp16=fp16)
        out = None
        cnt = torch.zeros(8, dtype=torch.int64, device=dev)
        for _ in range(args.warmup):
            out = dec.decode(syn_d, observables=obs_d, counters=cnt, out=out)
        torch.cuda.synchronize()
        cnt.zero_()
        dec.profile(True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for s in range(args.steps):
            flush.fill_(s)
            starts[s].record(stream)
            out = dec.decode(syn_d, observables=obs_d, counters=cnt, out=out)
            ends[s].record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        prof = dec.profile_read()
        dec.profile(False)
        c = cnt.cpu().numpy()
        total_ms = max_over_ranks(sum(step_ms))
        results[label] = dict(step_ms=step_ms, total_ms=total_ms, prof=prof, counters=c, clocks=clk, wall=wall,
                              corr=out["corrections"].clone(), logical=out["logical"].clone())
        # end to end through the host-buffer entry point (H2D + decode + D2H every step)
        if label == "f32":
            hsyn = torch.from_numpy(syn.view(np.int32)).pin_memory()
            hobs = torch.from_numpy(obs.view(np.int32)).pin_memory()
            hcorr = torch.empty((B, dm.n // 32 + (dm.n % 32 > 0)), dtype=torch.int32).pin_memory()
            hlog = torch.empty((B, 1), dtype=torch.int32).pin_memory()
            hst = torch.empty((B, 12), dtype=torch.uint8).pin_memory()
            hcnt = np.zeros(8, np.uint64)
            V.vibe_decode_host(dec.handle, hsyn, B, hcorr, hlog, hst, hobs, hcnt, stream)
            e2e_times = []
            for s in range(max(1, min(args.steps, 3))):
                flush.fill_(s)
                torch.cuda.synchronize()
                barrier()
                t0 = time.perf_counter()
                V.vibe_decode_host(dec.handle, hsyn, B, hcorr, hlog, hst, hobs, hcnt, stream)
                e2e_times.append(time.perf_counter() - t0)
            e2e_s = max_over_ranks(statistics.mean(e2e_times))
            results["e2e"] = dict(value=B * world / e2e_s,
                                  h2d=int(hsyn.numel() * 4 + hobs.numel() * 4),
                                  d2h=int(hcorr.numel() * 4 + hlog.numel() * 4 + hst.numel() + 8 * 8))
        dec.close()

    r32, r16 = results["f32"], results["f16"]
    f32_fail = int(r32["counters"][1]) // args.steps
    f16_fail = int(r16["counters"][1]) // args.steps
    differ = int((r32["corr"] != r16["corr"]).any(dim=1).sum().item())
    value = B * world * args.steps / (r32["total_ms"] / 1000.0)
    v16 = B * world * args.steps / (r16["total_ms"] / 1000.0)
    peaks, peak_src = measured_peaks()
    E = dm.H.nnz
    pair_iters = int(r32["counters"][3]) // args.steps
    io_bytes_per_shot = 4 * (dm.m + 31) // 32 + 4 * ((dm.n + 31) // 32) + 4 + 12
    bp_bytes = pair_iters * 2 * E * 4 + B * io_bytes_per_shot
    bp_ms = r32["prof"]["bp_ms"] / max(1, r32["prof"]["bp_launches"])
    achieved = bp_bytes / (bp_ms / 1000.0) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    lat = sorted(r32["step_ms"])
    lat16 = sorted(r16["step_ms"])

    def pct(a, q):
        return a[min(len(a) - 1, int(round(q * (len(a) - 1))))]

    line = {
        "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(r32["step_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: d=9 6.6.6 colour code, 9 noisy + 1 perfect phenomenological rounds, "
                               f"p=q=0.01, m={dm.m}, n={dm.n}, E={E}; K=16 seeded serial schedules, T=30, M=5, "
                               f"alpha=0.625, LSD-0; {B} shots per GPU per step",
                   "shots_per_gpu": B, "l2": "flushed between steps (256 MB write)"},
        "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "per": "batch of %d shots" % B},
        "fp16": {"value": v16, "ms_per_step": statistics.mean(r16["step_ms"]),
                 "latency_ms": {"p50": pct(lat16, 0.5), "p99": pct(lat16, 0.99)},
                 "ler": ler_ci(f16_fail, B), "corrections_differ_vs_f32": differ / B},
        "ler": ler_ci(f32_fail, B),
        "lsd_fraction": int(r32["counters"][2]) / (B * args.steps),
        "pair_iters_per_shot": pair_iters / B,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_bp (persistent BP ensemble)",
                     "peak_source": peak_src,
                     "bytes_per_launch": bp_bytes, "launch_ms": bp_ms,
                     "lsd_kernel_ms": r32["prof"]["lsd_ms"] / max(1, r32["prof"]["lsd_launches"])},
        "e2e": {"value": results["e2e"]["value"], "unit": "shots/s", "h2d_bytes_per_step": results["e2e"]["h2d"],
                "d2h_bytes_per_step": results["e2e"]["d2h"]},
        "gpu_launches": int(r32["prof"]["bp_launches"] + r32["prof"]["lsd_launches"]),
        "clocks": r32["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, ref, S = cpu_baseline(dm, w, syn, perms)
        gpu_corr = r32["corr"][:S].cpu().numpy().view(np.uint32)
        line["cpu_baseline"] = cb
        line["parity_sample"] = {"shots": S, "corrections_equal": bool(np.array_equal(gpu_corr, ref["corrections"]))}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vibe", choices=["vibe", "reference"])
    ap.add_argument("--shots", type=int, default=0, help="override shots per GPU (default: the workload's 10^6)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_vibe(args)


if __name__ == "__main__":
    sys.exit(main())
