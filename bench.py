"""Benchmark: LapH baryon+meson block contraction, algorithmic complex TFLOP/s.

Workload (default): L=32 (32768 sites), T=64 timeslices, N=64 orthonormal
complex64 vectors per timeslice, 19 momenta |n|^2 <= 2; B (i<j<k) and M.
A step is one pass of the whole contraction over the T timeslices.

Algorithmic flops per step = T * 8 * 3V * (C(N,3) + N^2) * P (8 real flops per
complex multiply-add, 3V = sites x colours, only i<j<k counted).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--mode f16x3|bf16x3|fp32|f16|bf16]
       python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)
Under torchrun each rank runs the full workload on its own GPU with its own
seeds (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_26313_gb300 import synth  # noqa: E402

WORKLOADS = {
    # name: (L, T, N, n2max)
    "metric": (32, 64, 64, 2),
    "medium": (24, 48, 32, 1),
    "small": (8, 1, 16, None),
    # a case small enough for full ncu captures (inputs still larger than L2 once staged)
    "profile": (24, 2, 64, 2),
}
METRIC = "baryon+meson block complex TFLOP/s at L=32,N=64,Np=19; tensor-pipe %; rel err vs FP64"

# DRAM bytes (read + write) of tc_kernel per byte of B-operand stage images it consumes, from the ncu captures
# summarised in profiles/, by (tile rows, tile columns): tc_kernel_L24_T2_N64_P19_full.md (1.941 GB for 2 x 12 x 1728
# stage images of 39,936 B, tc_kernel<0,3,104,0>) and tc_kernel_rowdoubled208_L24_T2_N64_P19_full.md (1.071 GB for
# 2 x 6 x 1728 images of 39,936 B, tc_kernel<0,3,208,1>).  The contraction's DRAM traffic is dominated by those images,
# so a launch's traffic is the ratio times its image bytes; a plan of another tile shape reports no traffic.  To be
# retaken whenever the kernel changes.
TC_DRAM_PER_IMAGE_BYTE = {(128, 104): 1.941e9 / (2 * 12 * 1728 * 39936),
                          (64, 208): 1.071e9 / (2 * 6 * 1728 * 39936)}
TC_PROFILE = {(128, 104): "profiles/tc_kernel_L24_T2_N64_P19_full.md",
              (64, 208): "profiles/tc_kernel_rowdoubled208_L24_T2_N64_P19_full.md"}


def momenta_for(name):
    L, T, N, n2 = WORKLOADS[name]
    if n2 is None:
        return np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    return synth.momentum_shell(n2)


def flops_per_timeslice(L, N, P):
    V = L ** 3
    return 8.0 * 3 * V * (math.comb(N, 3) + N * N) * P


def rel_frob(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def schedule_of(plan, tuned: bool) -> dict:
    """The tensor-core schedule a plan runs (and, when autotuned, every candidate it timed)."""
    d = plan.describe()
    sch = plan.schedule()
    out = {"layout": 1 if d["tile_rows"] == 64 else 0, "tile_cols": d["tile_cols"], "tile_rows": d["tile_rows"],
           "chunk_sites": d["chunk_sites"], "chunk_sites_b": plan.drain_sites()[1], "sum_sites": plan.sum_sites()[0],
           "timeslices_per_chunk": sch["timeslices_per_chunk"], "tile_order": sch["tile_order"], "autotuned": tuned}
    if tuned:
        out["candidates"] = [[r["layout"], r["tile_cols"], r["tile_order"], r["timeslices_per_chunk"], r["sum_sites"],
                              r["chunk_sites"], r["chunk_sites_b"], round(r["ms"], 3), r["probe_err"]]
                             for r in plan.tuning()]
        out["candidate_fields"] = ["layout", "tile_cols", "tile_order", "timeslices_per_chunk", "sum_sites",
                                   "chunk_sites", "chunk_sites_b", "ms", "probe_err"]
    return out


def pinned_copy_rates(nbytes: int = 1 << 30):
    """This box's pinned host <-> device copy rates (GB/s) on one buffer of nbytes, timed with CUDA events; they
    vary a lot between boxes and bound the end-to-end figure."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(s):
        d.copy_(h, non_blocking=True)
        h.copy_(d, non_blocking=True)
        ev[0].record()
        d.copy_(h, non_blocking=True)
        ev[1].record()
        h.copy_(d, non_blocking=True)
        ev[2].record()
    torch.cuda.synchronize()
    out = {"h2d_gbs": nbytes / ev[0].elapsed_time(ev[1]) / 1e6, "d2h_gbs": nbytes / ev[1].elapsed_time(ev[2]) / 1e6}
    del h, d
    return out


def max_over_ranks(ms: float, device) -> float:
    """The largest of a per-rank duration over all ranks of the process group (the duration
    itself for one rank): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(flops_per_rank: float, ms: float, world: int) -> float:
    """Whole-job TFLOP/s: every rank processes its own batch of the same size."""
    return world * flops_per_rank / (ms / 1e3) / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def oracle_sample(phi_t, L, mom, n_trip_sample=None, seed=0):
    """Oracle B (all or a seeded sample of triples) and M for one timeslice; returns
    (B or (idx, Bsample), M, seconds, algorithmic flops, threads)."""
    from oracle import oracle as O
    N = phi_t.shape[0]
    V = L ** 3
    P = mom.shape[0]
    t0 = time.perf_counter()
    if n_trip_sample is None:
        B = O.baryon_blocks(phi_t, L, mom)
        nt = math.comb(N, 3)
    else:
        rng = np.random.default_rng(seed)
        trip = sorted({tuple(sorted(rng.choice(N, 3, replace=False))) for _ in range(n_trip_sample)})
        Bs = O.baryon_triples(phi_t, L, mom, trip)
        B = (np.array([math.comb(k, 3) + math.comb(j, 2) + i for (i, j, k) in trip]), Bs)
        nt = len(trip)
    M = O.meson_blocks(phi_t, L, mom)
    dt = time.perf_counter() - t0
    return B, M, dt, 8.0 * 3 * V * (nt + N * N) * P, O.num_threads()


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, bounded samples per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    L, T, N, _ = WORKLOADS[args.workload]
    mom = momenta_for(args.workload)
    phi = synth.random_phi(L, N, T=1, instance=0)[0]
    n_sample = args.ref_triples
    times, flops = [], 0.0
    threads = 1
    for step in range(args.warmup + args.steps):
        _, _, dt, fl, threads = oracle_sample(phi, L, mom, n_trip_sample=n_sample, seed=step)
        if step >= args.warmup:
            times.append(dt)
            flops = fl
    ms = 1e3 * statistics.mean(times)
    value = flops / (ms / 1e3) / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"L={L},T={T},N={N},P={len(mom)} (oracle timed on a sample)", "L": L, "T": T, "N": N,
                   "P": int(len(mom))},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": f"1 timeslice: {n_sample} random i<j<k triples x {len(mom)} momenta + all N^2 "
                                   f"meson entries, per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def triplet_flops_per_timeslice(L, N, P):
    """Algorithmic flops of the dense three-field triplets: 3V complex MACs per output entry."""
    return 8.0 * 3 * L ** 3 * N ** 3 * P


def measure_triplets(laph, L, T, N, mom, mode, steps, warmup, n_sample=0, timed_oracle=False, tune=False):
    """Three-field triplets B3 (dense) through a LAPH_PLAN_FIELDS plan: device time per step, contraction
    kernel time, and (n_sample > 0) the relative error of sampled (i, j, k) of timeslice 0 against the
    oracle, with the oracle's own rate when timed_oracle."""
    import torch
    P = mom.shape[0]
    V = L ** 3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.SEED_BASE + 7)
    fields = []
    for _ in range(3):
        z = torch.randn((T, N, V, 3, 2), generator=gen, device="cuda", dtype=torch.float32)
        fields.append(torch.view_as_complex(z).contiguous() / math.sqrt(3 * V))
    plan = laph.Plan([(L, T, N, mom)], mode=mode,
                     flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_M | laph.PLAN_TIMING | (laph.PLAN_AUTOTUNE if tune else 0))
    sched = schedule_of(plan, tune)
    Bs, _ = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.execute_fields([fields], Bs, ws, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.execute_fields([fields], Bs, ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    status = plan.device_status()
    ms = e0.elapsed_time(e1) / steps
    n_con = plan.contraction_launches()
    k_ms = sum(plan.kernel_times(steps * n_con)) / steps
    o_ms = sum(plan.operand_times(steps * n_con)) / steps
    flops = T * triplet_flops_per_timeslice(L, N, P)
    out = {"ms_per_step": ms, "kernel_ms": k_ms, "operand_ms": o_ms, "flops_per_step": flops,
           "value": flops / (ms / 1e3) / 1e12, "kernel_tflops": flops / (k_ms / 1e3) / 1e12,
           "launches": plan.launches_per_execute() * steps, "device_status": status, "schedule": sched}
    if n_sample:
        from oracle import oracle as O
        rng = np.random.default_rng(5)
        ijk = rng.integers(0, N, size=(n_sample, 3))
        f0 = [f[0].cpu().numpy() for f in fields]
        t0 = time.perf_counter()
        ref = O.triplet_triples(f0[0], f0[1], f0[2], L, mom, ijk)
        dt = time.perf_counter() - t0
        got = Bs[0][0][:, ijk[:, 0], ijk[:, 1], ijk[:, 2]].cpu().numpy().T
        out["rel_err"] = {"B3": rel_frob(got, ref), "sample": f"{n_sample} random (i,j,k) x {P} momenta, timeslice 0"}
        if timed_oracle:
            out["cpu_baseline"] = {"value": 8.0 * 3 * V * n_sample * P / dt / 1e12, "unit": "TFLOP/s",
                                   "cores": O.num_threads(), "kind": "oracle",
                                   "sample": f"{n_sample} random (i,j,k) triples x {P} momenta of timeslice 0 "
                                             f"({dt:.1f} s)"}
    plan.close()
    del Bs, ws, fields
    torch.cuda.empty_cache()
    return out


LARGE = dict(L=48, T=96, N=128, n2=4)   # 33 momenta: |n|^2 <= 4


def measure_large(laph, L, T, N, mom, mode, steps, warmup, n_sample=0, timed_oracle=False, tune=False):
    """The large streamed form: T timeslices of N complex64 vectors on L^3 sites flow through HBM one at a time.  The
    vectors of timeslice t+1 are drawn on the device (torch's generator, seeded per timeslice, entries complex
    Gaussian / sqrt(3V)) on a side stream into the other half of a double buffer while timeslice t is contracted by a
    one-timeslice plan; B and M of every timeslice land in [T]-sized outputs.  Returns the device time per pass over
    the T timeslices, the kernel times and, with n_sample > 0, the relative errors of sampled baryon triples and of the
    meson blocks of 12 vectors, for the first and the last timeslice, against the FP64 oracle."""
    import torch
    P = mom.shape[0]
    V = L ** 3
    plan = laph.Plan([(L, 1, N, mom)], mode=mode, flags=laph.PLAN_TIMING | (laph.PLAN_AUTOTUNE if tune else 0))
    sched = schedule_of(plan, tune)
    ws = plan.alloc_workspace()
    B = torch.empty((T, P, math.comb(N, 3)), dtype=torch.complex128, device="cuda")
    M = torch.empty((T, P, N, N), dtype=torch.complex128, device="cuda")
    bufs = [torch.empty((1, N, V, 3), dtype=torch.complex64, device="cuda") for _ in range(2)]
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    gen = torch.Generator(device="cuda")
    ev_gen = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    for e in ev_used:
        e.record(main)
    sd = 1.0 / math.sqrt(2 * 3 * V)        # re and im each N(0, 1/(6V)): E|phi|^2 = 1 per vector

    def generate(t, out, stream):
        with torch.cuda.stream(stream):
            gen.manual_seed(synth.SEED_BASE + 31 + t)
            torch.view_as_real(out).normal_(0.0, sd, generator=gen)

    def one_pass():
        slot = 0
        side.wait_event(ev_used[0])
        generate(0, bufs[0], side)
        ev_gen[0].record(side)
        for t in range(T):
            slot = t % 2
            if t + 1 < T:
                nxt = (t + 1) % 2
                side.wait_event(ev_used[nxt])
                generate(t + 1, bufs[nxt], side)
                ev_gen[nxt].record(side)
            main.wait_event(ev_gen[slot])
            plan.execute([bufs[slot]], [B[t:t + 1]], [M[t:t + 1]], ws, stream=main)
            ev_used[slot].record(main)

    for _ in range(warmup):
        one_pass()
    torch.cuda.synchronize()
    if plan.device_status() != laph.LAPH_OK:
        raise RuntimeError("device status not OK after warm-up (large workload)")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for _ in range(steps):
        one_pass()
    e1.record(main)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    n = steps * T * plan.contraction_launches()
    k_ms = sum(plan.kernel_times(min(n, 256))) * (n / min(n, 256)) / steps
    flops = T * flops_per_timeslice(L, N, P)
    out = {"ms_per_step": ms, "kernel_ms": k_ms, "flops_per_step": flops, "value": flops / (ms / 1e3) / 1e12,
           "kernel_tflops": flops / (k_ms / 1e3) / 1e12, "device_status": plan.device_status(),
           "launches": plan.launches_per_execute() * T * steps, "schedule": sched}
    if n_sample:
        from oracle import oracle as O
        rng = np.random.default_rng(12)
        trip = sorted({tuple(int(v) for v in sorted(rng.choice(N, 3, replace=False))) for _ in range(n_sample)})
        idx = [math.comb(k, 3) + math.comb(j, 2) + i for (i, j, k) in trip]
        sub = np.sort(rng.choice(N, 12, replace=False))
        errs = {}
        dt = 0.0
        for t in (0, T - 1):
            phi = torch.empty((1, N, V, 3), dtype=torch.complex64, device="cuda")
            generate(t, phi, main)
            ph = phi[0].cpu().numpy()
            t0 = time.perf_counter()
            ref = O.baryon_triples(ph, L, mom, trip)
            rM = O.meson_blocks(ph[sub], L, mom)
            dt += time.perf_counter() - t0
            errs[f"t{t}"] = {"B": rel_frob(B[t][:, idx].cpu().numpy().T, ref),
                             "M": rel_frob(M[t].cpu().numpy()[:, sub][:, :, sub], rM)}
        out["rel_err"] = dict(errs, sample=f"{len(trip)} random i<j<k triples x {P} momenta and the meson blocks of "
                                           f"12 random vectors, timeslices 0 and {T - 1}")
        if timed_oracle:
            fl = 2 * 8.0 * 3 * V * (len(trip) + 144) * P
            out["cpu_baseline"] = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": O.num_threads(),
                                   "kind": "oracle", "sample": out["rel_err"]["sample"] + f" ({dt:.1f} s)"}
    plan.close()
    del B, M, bufs, ws
    torch.cuda.empty_cache()
    return out


def run_large(args):
    """--workload large: L=48 (110,592 sites), T=96, N=128, 33 momenta, streamed timeslice by timeslice with the
    next timeslice's vectors generated on the device beside the current contraction."""
    import torch
    from paper_2510_26313_gb300 import binding as laph
    torch.cuda.set_device(0)
    L, T, N = LARGE["L"], LARGE["T"], LARGE["N"]
    mom = synth.momentum_shell(LARGE["n2"])
    clocks = ClockSampler(0)
    clocks.start()
    r = measure_large(laph, L, T, N, mom, args.mode, args.steps, args.warmup,
                      n_sample=0 if args.no_cpu_baseline else 200, timed_oracle=not args.no_cpu_baseline,
                      tune=not args.no_autotune)
    clk = clocks.stop()
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    line = {
        "metric": f"baryon+meson block complex TFLOP/s at L={L},N={N},Np={mom.shape[0]} (streamed)",
        "value": r["value"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.mode}->f32/f64", "data": "synthetic (seeded complex Gaussian generated on the device)",
        "config": {"workload": f"L={L},T={T},N={N},P={mom.shape[0]} (large, streamed)", "L": L, "T": T, "N": N,
                   "P": int(mom.shape[0]), "mode": args.mode,
                   "l2": "inputs larger than L2 (phi %.2f GB per timeslice)" % (N * L ** 3 * 24 / 1e9)},
        "roofline": {"bound": "tensor", "achieved": r["kernel_tflops"], "peak": peak, "unit": "TFLOP/s",
                     "frac": r["kernel_tflops"] / peak, "traffic": None, "peak_source": src},
        "cpu_baseline": r.get("cpu_baseline"), "e2e": None, "gpu_launches": r["launches"], "clocks": clk,
        "rel_err": r.get("rel_err"), "kernel_ms": r["kernel_ms"], "device_status": r["device_status"],
        "schedule": r["schedule"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_triplets(args):
    """--workload triplets: three-field triplets (the next row of the hot path: stochastic-LapH quark
    sinks, no antisymmetry) at L=32, T=8, N=64, P=19."""
    import torch
    from paper_2510_26313_gb300 import binding as laph
    torch.cuda.set_device(0)
    L, T, N = 32, 8, 64
    mom = synth.momentum_shell(2)
    clocks = ClockSampler(0)
    clocks.start()
    r = measure_triplets(laph, L, T, N, mom, args.mode, args.steps, args.warmup,
                         n_sample=0 if args.no_cpu_baseline else 150000, timed_oracle=not args.no_cpu_baseline,
                         tune=not args.no_autotune)
    clk = clocks.stop()
    peaks, _ = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    line = {
        "metric": "three-field triplet complex TFLOP/s at L=32,N=64,Np=19 (dense N^3)", "value": r["value"],
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"{args.mode}->f32/f64",
        "data": "synthetic (seeded complex Gaussian fields phi, psi, chi)",
        "config": {"workload": f"L={L},T={T},N={N},P={mom.shape[0]} (triplets)", "L": L, "T": T, "N": N,
                   "P": int(mom.shape[0]), "mode": args.mode, "schedule": r["schedule"]},
        "roofline": {"bound": "tensor", "achieved": r["kernel_tflops"], "peak": peak, "unit": "TFLOP/s",
                     "frac": r["kernel_tflops"] / peak, "traffic": None,
                     "note": "achieved counts algorithmic flops; the 3-term split executes 3x that"},
        "cpu_baseline": r.get("cpu_baseline"), "e2e": None, "gpu_launches": r["launches"], "clocks": clk,
        "rel_err": r.get("rel_err"), "kernel_ms": r["kernel_ms"], "operand_ms": r["operand_ms"],
        "device_status": r["device_status"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_projection(args):
    """--workload projection: the projection of solution vectors onto LapH eigenvectors (the inner
    products <v_i, s_j> per timeslice, n = 0) at L=32, T=16, Nv=128 eigenvectors, Ns=512 columns."""
    import torch
    from paper_2510_26313_gb300 import binding as laph
    from oracle import oracle as O
    torch.cuda.set_device(0)
    L, T, Nv, Ns = 32, 16, 128, 512
    V = L ** 3
    mom = np.zeros((1, 3), dtype=np.int32)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.SEED_BASE + 11)
    fields = []
    for n in (Nv, Ns):
        z = torch.randn((T, n, V, 3, 2), generator=gen, device="cuda", dtype=torch.float32)
        fields.append(torch.view_as_complex(z).contiguous() / math.sqrt(3 * V))
    tune = not args.no_autotune
    plan = laph.Plan([(L, T, Nv, mom, Ns)], mode=args.mode,
                     flags=laph.PLAN_FIELDS | laph.PLAN_SKIP_B | laph.PLAN_TIMING | (laph.PLAN_AUTOTUNE if tune else 0))
    sched = schedule_of(plan, tune)
    _, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.execute_fields([fields], Ms, ws, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.execute_fields([fields], Ms, ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    n_con = plan.contraction_launches()
    k_ms = sum(plan.kernel_times(args.steps * n_con)) / args.steps
    o_ms = sum(plan.operand_times(args.steps * n_con)) / args.steps
    flops = 8.0 * 3 * V * Nv * Ns * T
    in_bytes = (Nv + Ns) * T * V * 3 * 8
    rel = cpu = None
    if not args.no_cpu_baseline:
        v0, s0 = fields[0][0].cpu().numpy(), fields[1][0].cpu().numpy()
        t0 = time.perf_counter()
        ref = O.projection(v0, s0, L, mom)
        dt = time.perf_counter() - t0
        rel = {"P": rel_frob(Ms[0][0].cpu().numpy(), ref), "timeslice": 0}
        cpu = {"value": 8.0 * 3 * V * Nv * Ns / dt / 1e12, "unit": "TFLOP/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"timeslice 0: all {Nv} x {Ns} inner products ({dt:.1f} s)"}
    peaks, _ = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    line = {
        "metric": "eigenvector projection complex TFLOP/s at L=32, Nv=128 x Ns=512 (n = 0)",
        "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.mode}->f32/f64", "data": "synthetic (seeded complex Gaussian v and s)",
        "config": {"workload": f"L={L},T={T},Nv={Nv},Ns={Ns},P=1 (projection)", "L": L, "T": T, "Nv": Nv, "Ns": Ns,
                   "mode": args.mode, "schedule": sched},
        "roofline": {"bound": "tensor", "achieved": flops / (k_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / (k_ms / 1e3) / 1e12 / peak, "traffic": None,
                     "note": "achieved counts algorithmic flops; the 3-term split executes 3x that",
                     "input_gbs": in_bytes / (ms / 1e3) / 1e9, "hbm_peak": hbm},
        "cpu_baseline": cpu, "e2e": None, "gpu_launches": plan.launches_per_execute() * args.steps, "clocks": clk,
        "rel_err": rel, "kernel_ms": k_ms, "operand_ms": o_ms, "device_status": plan.device_status(),
    }
    print(json.dumps(line), flush=True)
    return 0


LANCZOS = {
    # the LapH eigenvectors of the L=32, T=64, N=64 workload
    "lanczos": dict(L=32, T=64, n_ev=64, m=128, degree=48, lo=0.95, eps=0.6),
    # a small case of the same kernels for profiler captures (one group of 8 timeslices)
    "lanczos-small": dict(L=32, T=8, n_ev=16, m=24, degree=8, lo=0.95, eps=0.6),
}


# DRAM bytes (read + write) of one lap_soa_kernel launch on a group of 8 timeslices at L=32 with links read as three
# rows, from the ncu capture summarised in profiles/lap_soa_kernel_L32_T8_group8_full.md (warm L2, the launch shape of
# every filter launch of the L=32, T=64 workload); to be retaken whenever the kernel changes
LAP_SOA_TRAFFIC = 12.7e6


def laplacian_bytes_per_site(with_z: bool, link_rows: int = 3) -> int:
    """Algorithmic bytes of one application of -Delta (or one Chebyshev step) per site and vector: the three links
    leaving the site counted once each (3 x 72 B, or 3 x 48 B when read as two rows), the input vector, the output
    and, for a Chebyshev step, the vector y_{k-1} (24 B each)."""
    return 3 * 24 * link_rows + 24 + 24 + (24 if with_z else 0)


def run_lanczos(args):
    """--workload lanczos: the LapH eigenvectors, the 64 lowest eigenpairs of the 3-d gauge-covariant Laplacian
    on every timeslice of an L=32, T=64 lattice (batched Lanczos, 128 Krylov steps on a degree-48 Chebyshev
    filter), smoothed synthetic links.  Under torchrun every rank solves its own seeded batch of T timeslices on
    its own GPU (the timeslices are independent problems: no collective on the data path); the time is the
    slowest rank's and the value counts the timeslices of all ranks."""
    import torch
    import torch.distributed as dist
    from paper_2510_26313_gb300 import binding as laph
    from oracle import oracle as O
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c = LANCZOS[args.workload]
    L, T, n_ev, m, d, lo = c["L"], c["T"], c["n_ev"], c["m"], c["degree"], c["lo"]
    V = L ** 3
    U = synth.random_links_device(L, T, c["eps"], synth.SEED_BASE + 21 + 1000 * rank)
    evecs = torch.empty((T, n_ev, V, 3), dtype=torch.complex64, device="cuda")
    ws = torch.empty(laph.lanczos_workspace_size(L, T, n_ev, m, d, lo), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        laph.lanczos(U, L, n_ev, m, cheb_degree=d, cheb_lo=lo, out=evecs, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        st = {}
        _, ev, res = laph.lanczos(U, L, n_ev, m, cheb_degree=d, cheb_lo=lo, out=evecs, workspace=ws, stream=stream,
                                  stats=st)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, "cuda")
    apply_ms = sum(s["apply_ms"] for s in stats) / args.steps
    orth_ms = sum(s["orth_ms"] for s in stats) / args.steps
    n_apply = stats[0]["apply_launches"]
    rows = 2 if stats[0]["links_two_rows"] else 3
    tg = stats[0]["ts_group"]
    # algorithmic bytes: Laplacian launches (the first step of each filter without y_{k-1})
    per_iter = laplacian_bytes_per_site(False, rows) + (d - 1) * laplacian_bytes_per_site(True, rows)
    apply_bytes = m * per_iter * V * T
    # orthogonalisation of step j: two passes over the j + 1 basis vectors, each reading them once for the
    # inner products (with w) and once for the update (reading and writing w; the second update also sums |w|^2)
    K8 = 3 * V * 8
    orth_bytes = sum(2 * ((j + 2) + (j + 3)) for j in range(m)) * K8 * T
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    apply_gbs = apply_bytes / (apply_ms / 1e3) / 1e9
    orth_gbs = orth_bytes / (orth_ms / 1e3) / 1e9
    dominant = "apply" if apply_ms >= orth_ms else "orth"
    ach = apply_gbs if dominant == "apply" else orth_gbs
    # the public laph_laplacian (caller's layouts, no workspace) on one vector of every timeslice, timed alone
    f1 = evecs[:, :1].contiguous()
    g1 = torch.empty_like(f1)
    for _ in range(3):
        laph.laplacian(U, f1, L, out=g1, stream=stream)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(20):
        laph.laplacian(U, f1, L, out=g1, stream=stream)
    eb.record(stream)
    torch.cuda.synchronize()
    lap_ms = ea.elapsed_time(eb) / 20
    lap_api = {"ms": lap_ms, "gbs": laplacian_bytes_per_site(False) * V * T / (lap_ms / 1e3) / 1e9,
               "note": "laph_laplacian on [T][1][V][3] with the caller's [T][3][V][3][3] links, algorithmic bytes"}
    e2e = None
    if not args.no_e2e:
        # through the public API with host buffers: links copied in from pinned memory, eigenvectors and
        # eigenvalues copied back, every step
        U_host = U.cpu().pin_memory()
        out_host = torch.empty((T, n_ev, V, 3), dtype=torch.complex64).pin_memory()
        Ud = torch.empty_like(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            Ud.copy_(U_host, non_blocking=True)
            laph.lanczos(Ud, L, n_ev, m, cheb_degree=d, cheb_lo=lo, out=evecs, workspace=ws, stream=stream)
            out_host.copy_(evecs, non_blocking=True)
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        dt = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.e2e_steps, "cuda") / 1e3
        e2e = {"value": world * T / dt, "unit": "timeslices/s", "h2d_bytes_per_step": U_host.numel() * 8,
               "d2h_bytes_per_step": out_host.numel() * 8 + T * n_ev * 16}
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's plain FP64 Lanczos (same m, filter degree and bound, two Gram-Schmidt passes per step, its own
        # FP64 stencil) solves timeslice 0 of the same links: the timed CPU baseline, and a full-size check of the GPU's
        # eigenvalues of that timeslice
        U0 = U[0].cpu().numpy()
        t0 = time.perf_counter()
        lam, rcpu = O.lanczos_eigenpairs(U0, L, n_ev, m, d, lo)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "timeslices/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"timeslice 0: one whole FP64 Lanczos solve (m={m}, degree {d}, {n_ev} eigenpairs) "
                         f"({dt:.1f} s)"}
        parity = {"max_abs_dlambda_t0": float(np.abs(ev[0] - lam).max()), "oracle_max_resid": float(rcpu.max()),
                  "note": "GPU eigenvalues of timeslice 0 against the oracle's FP64 Lanczos on the same links"}
    line = {
        "metric": f"LapH eigenvectors: timeslices/s for the {n_ev} lowest eigenpairs of the 3-d Laplacian at L={L}",
        "value": world * T / (ms / 1e3), "unit": "timeslices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors, f64 inner products",
        "data": f"synthetic smoothed SU(3) links (polar part of 1 + i {c['eps']} H, H Hermitian Gaussian)",
        "config": {"workload": f"L={L},T={T},n_ev={n_ev} (lanczos: m={m}, Chebyshev degree {d}, lo={lo})",
                   "L": L, "T": T, "n_ev": n_ev, "n_krylov": m, "cheb_degree": d, "cheb_lo": lo,
                   "ts_group": tg, "link_rows": rows,
                   "parallelism": f"replicas x{world} (independent timeslice batches)",
                   "l2": f"inputs larger than L2: links {U.numel() * 8 / 1e9:.2f} GB, basis "
                         f"{T * (m + 1) * 3 * V * 8 / 1e9:.1f} GB"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": LAP_SOA_TRAFFIC if (dominant == "apply" and (L, tg, rows) == (32, 8, 3)) else None,
                     "kernel": "lap_soa_kernel (Chebyshev steps)" if dominant == "apply" else
                     "dots_kernel + update_kernel (orthogonalisation)", "peak_source": src,
                     "bytes_per_launch": apply_bytes / n_apply if dominant == "apply" else None,
                     "note": (f"the filter runs in groups of {tg} timeslices whose links and vectors stay in L2 "
                              f"across its {d} steps, so its algorithmic bytes are mostly served from L2 and the "
                              "fraction of the HBM copy peak can exceed 1") if dominant == "apply" and tg < T else
                             None},
        "phases": {"apply_ms": apply_ms, "apply_gbs": apply_gbs, "apply_launches": n_apply,
                   "orth_ms": orth_ms, "orth_gbs": orth_gbs,
                   "setup_ms": sum(s["setup_ms"] for s in stats) / args.steps,
                   "ritz_ms": sum(s["ritz_ms"] for s in stats) / args.steps,
                   "other_ms": ms - apply_ms - orth_ms, "host_steps": max(s["host_steps"] for s in stats)},
        "convergence": {"max_resid": float(res.max()), "median_resid": float(np.median(res)),
                        "ev_min": float(ev.min()), "ev_max": float(ev.max())},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(sum(s["launches"] for s in stats)), "clocks": clk,
        "laplacian_api": lap_api, "parity": parity,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_ragged(laph, count, mode, chunk_sites, steps, warmup, check=True):
    """`count` seeded ragged instances (L in {16,24,32}, N in [24,96], P in {1,7,19,33}, T in 1..8) in one plan,
    then the same instances as one plan each; with `check`, the FP64 oracle on timeslice 0 of the three smallest."""
    import torch
    insts = synth.ragged_instances(count)
    specs = [(i.L, i.T, i.N, i.momenta) for i in insts]
    flops_step = sum(i.T * flops_per_timeslice(i.L, i.N, i.P) for i in insts)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.SEED_BASE)
    phis = []
    for i in insts:
        z = torch.randn((i.T, i.N, i.V, 3, 2), generator=gen, device="cuda", dtype=torch.float32)
        phis.append(torch.view_as_complex(z).contiguous() / math.sqrt(3 * i.V))
    plan = laph.Plan(specs, mode=mode, flags=laph.PLAN_TIMING, chunk_sites=chunk_sites)
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.execute(phis, Bs, Ms, ws, stream=stream)
    torch.cuda.synchronize()
    if plan.device_status() != laph.LAPH_OK:
        raise RuntimeError("device status not OK after warm-up")
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.execute(phis, Bs, Ms, ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    n_con = plan.contraction_launches()
    k_ms = sum(plan.kernel_times(steps * n_con)) / steps
    rel = []
    if check:
        small = sorted(range(len(insts)), key=lambda n: insts[n].T * flops_per_timeslice(insts[n].L, insts[n].N, insts[n].P))[:3]
        for n in small:
            B0, M0, _, _, _ = oracle_sample(phis[n][0].cpu().numpy().astype(np.complex64), insts[n].L, insts[n].momenta)
            rel.append({"instance": n, "B": rel_frob(Bs[n][0].cpu().numpy(), B0), "M": rel_frob(Ms[n][0].cpu().numpy(), M0)})
    # the same instances, one plan each, executed back to back
    del ws
    torch.cuda.empty_cache()
    single = [laph.Plan([sp], mode=mode, chunk_sites=chunk_sites) for sp in specs]
    sws = torch.empty(max(pl.workspace_size() for pl in single), dtype=torch.uint8, device="cuda")  # shared, stream-ordered
    for n, pl in enumerate(single):
        pl.execute([phis[n]], [Bs[n]], [Ms[n]], sws, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for n, pl in enumerate(single):
        pl.execute([phis[n]], [Bs[n]], [Ms[n]], sws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    out = {"value": flops_step / (ms / 1e3) / 1e12, "ms_per_step": ms, "kernel_ms": k_ms,
           "kernel_tflops": flops_step / (k_ms / 1e3) / 1e12, "flops_step": flops_step,
           "timeslices": sum(i.T for i in insts), "per_instance_plans": {"ms_per_step": ms_single,
                                                                          "value": flops_step / (ms_single / 1e3) / 1e12},
           "rel_err": rel, "clocks": clk, "contraction_launches": n_con,
           "gpu_launches": plan.launches_per_execute() * steps, "schedule": schedule_of(plan, False),
           "device_status": plan.device_status()}
    for pl in single:
        pl.close()
    plan.close()
    return out


def run_ragged(args):
    """--workload ragged: 200 ragged instances (L in {16,24,32}, N in [24,96], P in {1,7,19,33},
    T in 1..8) in one plan; the same instances as 200 separate plans for comparison."""
    import torch
    from paper_2510_26313_gb300 import binding as laph
    torch.cuda.set_device(0)
    r = measure_ragged(laph, 200, args.mode, args.chunk_sites, args.steps, args.warmup, not args.no_cpu_baseline)
    peaks, _ = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    line = {
        "metric": "ragged batch complex TFLOP/s (200 instances, one plan)", "value": r["value"],
        "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"{args.mode}->f32/f64",
        "data": "synthetic (seeded complex Gaussian, not orthonormalised)",
        "config": {"workload": "200 ragged instances: L in {16,24,32}, N in [24,96], P in {1,7,19,33}, T in 1..8",
                   "timeslices": r["timeslices"], "mode": args.mode},
        "roofline": {"bound": "tensor", "achieved": r["kernel_tflops"], "peak": peak, "unit": "TFLOP/s",
                     "frac": r["kernel_tflops"] / peak, "traffic": None},
        "per_instance_plans": r["per_instance_plans"],
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "rel_err": r["rel_err"],
        "contraction_launches": r["contraction_launches"], "kernel_ms": r["kernel_ms"], "schedule": r["schedule"],
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_medium_fp32(laph, steps, warmup, check=True):
    """The FP32 CUDA-core path (the plain FP32 GPU path) at the medium configuration (L=24, T=48, N=32, 7 momenta);
    with `check`, the FP64 oracle on timeslice 0."""
    import torch
    L, T, N, _ = WORKLOADS["medium"]
    mom = momenta_for("medium")
    P = int(mom.shape[0])
    phi_h = synth.random_phi(L, N, T=T, instance=0)
    phi = torch.from_numpy(phi_h).cuda()
    plan = laph.Plan([(L, T, N, mom)], mode="fp32")
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.execute([phi], Bs, Ms, ws, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        plan.execute([phi], Bs, Ms, ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"value": T * flops_per_timeslice(L, N, P) / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
           "workload": f"L={L},T={T},N={N},P={P}", "device_status": plan.device_status()}
    if check:
        B0, M0, _, _, _ = oracle_sample(phi_h[0], L, mom)
        out["rel_err"] = {"B": rel_frob(Bs[0][0].cpu().numpy(), B0), "M": rel_frob(Ms[0][0].cpu().numpy(), M0),
                          "timeslice": 0}
    plan.close()
    return out


def measure_lanczos(laph, cfg, steps, warmup, seed):
    """One batched Lanczos solve of configuration `cfg` (see LANCZOS) on seeded smoothed links, timed: timeslices
    per second, the phases, the eigenvalue range and the largest residual norm."""
    import torch
    L, T, n_ev, m, d, lo = cfg["L"], cfg["T"], cfg["n_ev"], cfg["m"], cfg["degree"], cfg["lo"]
    V = L ** 3
    U = synth.random_links_device(L, T, cfg["eps"], seed)
    evecs = torch.empty((T, n_ev, V, 3), dtype=torch.complex64, device="cuda")
    ws = torch.empty(laph.lanczos_workspace_size(L, T, n_ev, m, d, lo), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        laph.lanczos(U, L, n_ev, m, cheb_degree=d, cheb_lo=lo, out=evecs, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(steps):
        st = {}
        _, ev, res = laph.lanczos(U, L, n_ev, m, cheb_degree=d, cheb_lo=lo, out=evecs, workspace=ws, stream=stream,
                                  stats=st)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ev = ev.cpu().numpy() if hasattr(ev, "cpu") else np.asarray(ev)
    res = res.cpu().numpy() if hasattr(res, "cpu") else np.asarray(res)
    out = {"value": T / (ms / 1e3), "unit": "timeslices/s", "ms_per_solve": ms,
           "filter_ms": sum(s["apply_ms"] for s in stats) / steps, "orth_ms": sum(s["orth_ms"] for s in stats) / steps,
           "ritz_ms": sum(s["ritz_ms"] for s in stats) / steps, "host_steps": max(s["host_steps"] for s in stats),
           "eigenvalues": [float(ev.min()), float(ev.max())], "max_residual": float(res.max()),
           "config": {k: cfg[k] for k in ("L", "T", "n_ev", "m", "degree", "lo")}}
    del ws, evecs, U
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="f16x3")
    ap.add_argument("--workload", default="metric", choices=sorted(WORKLOADS) + ["ragged", "triplets", "projection", "large"] + sorted(LANCZOS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-extra-aux", action="store_true",
                    help="skip the ragged-batch, eigensolver and FP32 medium-configuration side measurements "
                         "(thousands of launches: keep them out of profiler launch lists)")
    ap.add_argument("--ref-triples", type=int, default=6000)
    ap.add_argument("--chunk-sites", type=int, default=0)
    ap.add_argument("--sum-sites", type=int, default=0)
    ap.add_argument("--tile-cols", type=int, default=0)
    ap.add_argument("--layout", type=int, default=0, help="tensor-core layout of the complex product (0 or 1)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="metric workload: the default schedule instead of the autotuned one")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ragged":
        return run_ragged(args)
    if args.workload == "triplets":
        return run_triplets(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "projection":
        return run_projection(args)
    if args.workload in LANCZOS:
        return run_lanczos(args)

    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2510_26313_gb300 import binding as laph

    L, T, N, _ = WORKLOADS[args.workload]
    mom = momenta_for(args.workload)
    P = int(mom.shape[0])
    V = L ** 3

    # ---- inputs: seeded per rank (weak scaling), host generation, then resident in HBM
    phi_h = synth.random_phi(L, N, T=T, instance=rank)
    phi = torch.from_numpy(phi_h).cuda()
    tune = args.mode != "fp32" and not args.no_autotune
    t_plan = time.perf_counter()
    plan = laph.Plan([(L, T, N, mom)], mode=args.mode,
                     flags=laph.PLAN_TIMING | (laph.PLAN_AUTOTUNE if tune else 0), chunk_sites=args.chunk_sites,
                     sum_sites=args.sum_sites, tile_cols=args.tile_cols, layout=args.layout)
    t_plan = time.perf_counter() - t_plan
    desc = plan.describe()
    schedule = dict(schedule_of(plan, tune), plan_create_s=t_plan)
    Bs, Ms = plan.alloc_outputs()
    ws = plan.alloc_workspace()
    stream = torch.cuda.current_stream()

    def step():
        plan.execute([phi], Bs, Ms, ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if plan.device_status() != laph.LAPH_OK:
        raise RuntimeError("device status not OK after warm-up")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    n_con = plan.contraction_launches()
    kernel_ms = plan.kernel_times(args.steps * n_con)
    operand_ms = plan.operand_times(args.steps * n_con) if args.mode != "fp32" else []
    reduce_ms = plan.reduce_times(args.steps * n_con) if args.mode != "fp32" else []
    ms = max_over_ranks(ms, "cuda")
    status = plan.device_status()

    flops_step = T * flops_per_timeslice(L, N, P)
    value = weak_scaling_value(flops_step, ms, world)
    k_avg = sum(kernel_ms) / args.steps          # contraction kernel time per step (all chunks)
    achieved = flops_step / (k_avg / 1e3) / 1e12
    peaks, peak_src = measured_peaks()
    tc = args.mode != "fp32"
    if tc:
        peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        nc = desc["tile_cols"]
        n_ct = -(-(N * P) // nc)
        img_b = 192 * nc if desc["tile_rows"] == 64 else 384 * nc  # one stage image (layout 1: one B row per column)
        images = T * n_ct * (-(-(3 * V) // 24)) * img_b            # stage images read per step
        shape = (desc["tile_rows"], nc)
        ratio = TC_DRAM_PER_IMAGE_BYTE.get(shape)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": ratio * images / n_con if ratio else None,
                "traffic_source": (f"per tc_kernel launch: DRAM bytes per stage-image byte from the ncu capture at "
                                   f"L=24, T=2 ({TC_PROFILE[shape]}) x this launch's image bytes"
                                   if ratio else "no capture of this tile shape"),
                "peak_source": f"{peak_src} bf16 dense sustained (cuBLAS); FP16 runs at the bf16 rate",
                "note": "achieved counts algorithmic flops; the 3-term split executes 3x that on the tensor pipe"}
        # B-operand stage images: HBM-bound, algorithmic bytes = images written + phi read once
        psi_bytes = images + T * N * V * 3 * 8
        o_avg = sum(operand_ms) / args.steps
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        # the step's own algorithmic bytes: phi in, B and M out (complex128)
        step_bytes = T * (N * V * 3 * 8 + P * (math.comb(N, 3) + N * N) * 16)
        roof["operand_kernel"] = {"name": "psi_kernel", "ms_per_step": o_avg, "bound": "hbm",
                                  "achieved": psi_bytes / (o_avg / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": psi_bytes / (o_avg / 1e3) / 1e9 / hbm,
                                  "image_bytes_per_step": psi_bytes, "step_algorithmic_bytes": step_bytes,
                                  "images_over_step_bytes": psi_bytes / step_bytes,
                                  "note": "bytes = stage images written + phi read; the images are an intermediate "
                                          "of this design, written once and read back by the contraction"}
        # FP64 site reduction: FP32 partials of every site block read, complex128 outputs written
        r_avg = sum(reduce_ms) / args.steps
        sum_sites, n_sc = plan.sum_sites()
        n_out = P * (math.comb(N, 3) + N * N)
        red_bytes = T * n_out * (n_sc * 8 + 16)
        roof["reduce_kernel"] = {"name": "reduce_kernel", "event_ms_per_step": r_avg, "site_blocks": n_sc,
                                 "sum_sites": sum_sites, "bytes_per_step": red_bytes,
                                 "note": "runs on a side stream beside the next chunk's B-operand pass, so its event "
                                         "time includes that overlap; bound by FP64 additions (2 (blocks - 1) per "
                                         "complex output), not by HBM"}
        # executed tensor work: every MMA of every tile (3 split terms, padding, triangle waste)
        mma = plan.tensor_flops()
        executed = mma / (k_avg / 1e3) / 1e12
        sm_mhz = (clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0)))
        clock_peak = 152 * 8192 * sm_mhz * 1e6 / 1e12
        roof["tensor_pipe"] = {"executed_tflops": executed, "executed_over_algorithmic": mma / flops_step,
                               "frac_of_sustained_peak": executed / peak,
                               "issue_peak_at_median_clock": clock_peak, "frac_of_issue_peak": executed / clock_peak,
                               "note": "tensor-pipe utilisation estimated from the MMAs issued: executed flops / "
                                       "kernel time / (152 SMs x 8192 flops per cycle x median SM clock)"}
    else:
        # FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock
        smax = float(peaks.get("sm_max_mhz", 2070.0))
        peak = 152 * 128 * 2 * smax * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": "152 SMs x 128 FP32 FMA lanes x 2 x max SM clock"}

    # ---- the memory-bound stages on their own (outside the timed region):
    # materialised diquarks D (K-b) on 4 timeslices and the dense sign fill (K-g)
    aux = None
    if rank == 0:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        Td = min(4, T)
        npair = N * (N - 1) // 2
        D = torch.empty((Td, npair, V, 3), dtype=torch.complex64, device="cuda")
        dense = torch.empty((Td, P, N, N, N), dtype=torch.complex128, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        laph.diquarks(phi[:Td], L, out=D)
        laph.baryon_dense(Bs[0][:Td], N, out=dense)
        torch.cuda.synchronize()
        reps = 3
        ev[0].record(stream)
        for _ in range(reps):
            laph.diquarks(phi[:Td], L, out=D)
        ev[1].record(stream)
        for _ in range(reps):
            laph.baryon_dense(Bs[0][:Td], N, out=dense)
        ev[2].record(stream)
        torch.cuda.synchronize()
        dq_ms = ev[0].elapsed_time(ev[1]) / reps
        df_ms = ev[1].elapsed_time(ev[2]) / reps
        dq_bytes = Td * N * V * 3 * 8 + D.numel() * 8
        df_bytes = Td * P * (N * (N - 1) * (N - 2) // 6) * 16 + dense.numel() * 16
        aux = {
            "diquark_kernel": {"timeslices": Td, "ms": dq_ms, "bytes": dq_bytes, "achieved": dq_bytes / (dq_ms / 1e3) / 1e9,
                               "peak": hbm, "unit": "GB/s", "frac": dq_bytes / (dq_ms / 1e3) / 1e9 / hbm},
            "dense_fill_kernel": {"timeslices": Td, "ms": df_ms, "bytes": df_bytes,
                                  "achieved": df_bytes / (df_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": df_bytes / (df_ms / 1e3) / 1e9 / hbm},
        }
        del D, dense
        # the large streamed form (L=48, N=128, 33 momenta), two timeslices
        if args.mode in ("f16x3", "bf16x3"):
            lg = measure_large(laph, LARGE["L"], 2, LARGE["N"], synth.momentum_shell(LARGE["n2"]), args.mode, 1, 1,
                               n_sample=0 if args.no_cpu_baseline else 200)
            aux["large_streamed"] = {"workload": f"L={LARGE['L']},T=2,N={LARGE['N']},P=33 (streamed)",
                                     "ms": lg["ms_per_step"], "kernel_ms": lg["kernel_ms"], "value": lg["value"],
                                     "kernel_tflops": lg["kernel_tflops"], "unit": "TFLOP/s",
                                     "rel_err": lg.get("rel_err"), "device_status": lg["device_status"]}
        # the next row of the path: three-field triplets at the workload's shape, 4 timeslices
        if args.mode in ("f16x3", "bf16x3"):
            tr = measure_triplets(laph, L, min(4, T), N, mom, args.mode, 2, 1,
                                  n_sample=0 if args.no_cpu_baseline else 24)
            aux["triplets"] = {"timeslices": min(4, T), "ms": tr["ms_per_step"], "kernel_ms": tr["kernel_ms"],
                               "value": tr["value"], "kernel_tflops": tr["kernel_tflops"], "unit": "TFLOP/s",
                               "rel_err": tr.get("rel_err"), "device_status": tr["device_status"]}
        # the ragged batch (200 instances in one plan, and as 200 plans) and the LapH eigensolver at its benchmark
        # configuration, so that the default run records them too
        if args.mode in ("f16x3", "bf16x3") and args.workload == "metric" and not args.no_extra_aux:
            rg = measure_ragged(laph, 200, args.mode, args.chunk_sites, 2, 1, check=not args.no_cpu_baseline)
            aux["ragged_200"] = {k: rg[k] for k in ("value", "ms_per_step", "kernel_tflops", "timeslices",
                                                      "per_instance_plans", "rel_err", "device_status")}
            aux["ragged_200"]["unit"] = "TFLOP/s"
            aux["lanczos"] = measure_lanczos(laph, LANCZOS["lanczos"], 2, 1, synth.SEED_BASE + 21)
            aux["medium_fp32"] = measure_medium_fp32(laph, 3, 2, check=not args.no_cpu_baseline)

    # ---- accuracy and CPU baseline on timeslice 0 (rank 0 only)
    rel = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        B0, M0, dt, fl, threads = oracle_sample(phi_h[0], L, mom)
        gB = Bs[0][0].cpu().numpy()
        gM = Ms[0][0].cpu().numpy()
        rel = {"B": rel_frob(gB, B0), "M": rel_frob(gM, M0), "timeslice": 0}
        cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
               "sample": f"timeslice 0 of the workload: all C(N,3) baryon and N^2 meson entries x {P} momenta "
                         f"({dt:.1f} s)"}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        phi_pin = torch.from_numpy(phi_h).pin_memory()
        Bh = [torch.empty(tuple(Bs[0].shape), dtype=torch.complex128).pin_memory()]
        Mh = [torch.empty(tuple(Ms[0].shape), dtype=torch.complex128).pin_memory()]
        hws = torch.empty(plan.host_workspace_size(), dtype=torch.uint8, device="cuda")
        del phi
        plan.execute_host([phi_pin], Bh, Mh, hws, stream=stream)   # warm-up
        if world > 1:
            dist.barrier()
        clocks_e2e = ClockSampler(local)
        clocks_e2e.start()
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            plan.execute_host([phi_pin], Bh, Mh, hws, stream=stream)   # returns after its copies out
            step_ms.append(1e3 * (time.perf_counter() - t1))
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        clk_e2e = clocks_e2e.stop()
        e2e_s = max_over_ranks(e2e_s, "cuda")
        e2e = {"value": weak_scaling_value(flops_step, 1e3 * e2e_s, world), "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(phi_pin.numel() * 8),
               "d2h_bytes_per_step": int(Bh[0].numel() * 16 + Mh[0].numel() * 16),
               "ms_per_step": 1e3 * e2e_s, "step_ms": [round(x, 2) for x in step_ms],
               "median_step_ms": statistics.median(step_ms), "clocks": clk_e2e,
               "pinned_copy_rates": pinned_copy_rates()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "f16x3": "f16x3->f32/f64", "bf16x3": "bf16x3->f32/f64",
                                           "f16": "f16->f32/f64", "bf16": "bf16->f32/f64"}[args.mode],
            "data": "synthetic",
            "config": {"workload": f"L={L},T={T},N={N},P={P} ({args.workload})", "L": L, "T": T, "N": N, "P": P,
                       "mode": args.mode, "l2": "inputs larger than L2 (phi %.2f GB)" % (phi_h.nbytes / 1e9),
                       "parallelism": f"replicas x{world} (independent timeslice batches)",
                       "schedule": schedule},
            "roofline": roof,
            "aux_kernels": aux,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": plan.launches_per_execute() * args.steps,
            "clocks": clk,
            "rel_err": rel,
            "kernel_ms": k_avg,
            "device_status": status,
            "blocks_per_s": world * T * P * 2 / (ms / 1e3),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
