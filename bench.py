"""Benchmark of the operator apply on GB300 (one JSON line on rank 0).

Default workload (``n64_bumps8``): n = 64 grid (262,144 points, 786,432 complex
unknowns), k = 16 pi (8 wavelengths at about 8 points per wavelength), eps = 1 +
tapered sum of 8 seeded Gaussian bumps, one incident plane wave, complex64.
One step = one application of the operator on the hot path: ``--op QA``
(default) applies A (contrast multiply, zero-padded FFTs, Fourier-side product
with the four kernel spectra, inverse FFTs, +x) and then the sparsifying row
combination Q; ``--op A`` applies A alone.

``solve`` (same JSON line): time to a true relative residual of 1e-6 for the
workload's incident field with the S^-1 Q preconditioned GMRES(20), complex64
operator and factor inside the FP64 outer loop (``mixed``) and plain complex128
throughout (``fp64``, the default ``--solve both``; ``--solve mixed`` skips the
complex128 factor), with their ratio ``fp64_over_mixed``.  Set-up (stencils,
factor) is timed apart from the solve, as the paper reports T_setup apart from
T_solve.  ``solve_block64`` does the same for the 64 plane waves of the n = 64
medium as one block right-hand side (mixed vs FP64 batched time-to-solution).
``apply_n256`` times the n = 256 apply of A (L = 512), where the pass
intermediates stream through HBM, against the measured HBM and FP32 peaks.

Roofline denominators: HBM from MEASURED_PEAKS.json (copy bandwidth); FP32 and
FP64 measured in the same process by the library's FMA micro-benchmark
(``spm_measure_peak``).

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
launch stream, with an L2 flush (a 512 MiB buffer write) between steps, barrier
and synchronize around the timed region, max over ranks.  ``e2e`` repeats the
measurement through the public API with the input copied from pinned host
memory and the result read back every step.  ``cpu_baseline`` times the FP64
CPU oracle's FFT apply on a bounded sample on the host cores.

``--impl reference``: the CPU oracle timed as it stands (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import spm_inputs as si  # noqa: E402

METRIC = "operator applies/s + HBM GB/s frac; time-to-1e-6 solve, cx64-mixed vs FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n64_bumps8")
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--op", default="QA", choices=["A", "QA"])
    ap.add_argument("--solve", default="both", choices=["none", "mixed", "both"])
    ap.add_argument("--no-block-solve", action="store_true",
                    help="skip the 64-RHS block solve (config 3) in the default n = 64 run")
    ap.add_argument("--no-2d", action="store_true", help="skip the 2-D variant's apply and solve measurements")
    ap.add_argument("--no-n256", action="store_true",
                    help="skip the n = 256 apply sub-measurement of the default run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--uneven-solve-all", action="store_true",
                    help="uneven32: also solve the n = 96 problems, one after another")
    ap.add_argument("--uneven-n96-factor", default="c64", choices=["c64", "c64h"],
                    help="uneven32 --uneven-solve-all: factor of the n = 96 problems (complex64 or half storage)")
    ap.add_argument("--profile-case", default=None, choices=["qa64", "a128", "a256", "2d959", "2d959c128", "2d119"],
                    help="small fixed case for ncu captures: a few applies (Q A at n = 64 with seeded random "
                         "stencil tables, no factor; or A at n = 128 / 256) with the z-pass plan --zplan, no timing")
    ap.add_argument("--zplan", type=int, default=0, help="apply-plan variant for --profile-case")
    ap.add_argument("--applies", type=int, default=3, help="applies for --profile-case")
    return ap.parse_args()


def run_profile_case(args):
    """A small fixed workload for ncu (a few GB on the device at most): the apply
    of the bench's medium, one right-hand side, complex64, a fixed z-pass plan.
    For Q A the stencil tables are seeded random numbers installed with
    spm_set_stencils (S is assembled, not factored): Q's cost does not depend on
    their values, and the 26 GB factor of the full bench stays out of the capture."""
    import torch
    import paper_1804_02297_gb300 as spm
    if args.profile_case.startswith("2d"):
        # the 2-D variant's apply of A: lens medium at n = 959 (L = 2048) or 119 (L = 256), one RHS
        n = 119 if args.profile_case == "2d119" else 959
        wl = si.workload_2d(f"lens2d_n{n}")
        P = spm.Problem2D(n, wl["omega"], wl["eps"], wl["grad"])
        dt = torch.complex128 if args.profile_case.endswith("c128") else torch.complex64
        x = torch.from_numpy(wl["einc"]).to(dt).to("cuda").contiguous()
        y = torch.zeros_like(x)
        for _ in range(args.applies):
            P.apply_A(x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "workload": f"lens2d_n{n}", "applies": args.applies,
                          "device_gb": torch.cuda.max_memory_allocated() / 1e9}))
        return
    name = {"qa64": "n64_bumps8", "a128": "n128_bumps32_rhs8", "a256": "n256_bumps32"}[args.profile_case]
    wl = si.workload(name)
    n = wl["n"]
    P = spm.Problem(n, wl["omega"], wl["eps"], wl["grad"])
    spm.set_apply_plan(spm.SPM_C64, 2 * n, args.zplan)
    x = torch.from_numpy(wl["einc"][:1]).to(torch.complex64).to("cuda").contiguous()
    y = torch.zeros_like(x)
    if args.profile_case == "qa64":
        rng = np.random.default_rng(1)
        P.set_stencils(rng.standard_normal((27, 81, 3)) + 1j * rng.standard_normal((27, 81, 3)),
                       rng.standard_normal((27, 108, 3)) + 1j * rng.standard_normal((27, 108, 3)))
        fn = P.apply_QA
    else:
        fn = P.apply_A
    for _ in range(args.applies):
        fn(x, y)
    torch.cuda.synchronize()
    P.device_status()
    print(json.dumps({"profile_case": args.profile_case, "workload": name, "zplan": args.zplan,
                      "applies": args.applies, "device_gb": torch.cuda.max_memory_allocated() / 1e9}))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def compulsory_bytes(n, prec, nrhs=1):
    """Algorithmic bytes of one apply: read x, m, p (complex) and the 4 octant
    spectra, write y.  Each complex element is 8 (c64) or 16 (c128) bytes."""
    el = 8 if prec == "c64" else 16
    N = n ** 3
    return el * (nrhs * 3 * N + N + 3 * N + 4 * (n + 1) ** 3 + nrhs * 3 * N)


def alu_peaks(spm, torch):
    """FP32 and FP64 peaks of this GPU, measured in this process by the library's
    FMA micro-benchmark (spm_measure_peak: independent register FMA chains on
    every SM, best of five launches of a few ms).  The FP32 peak is the larger of
    the scalar FFMA and the packed FP32x2 FFMA rates.  The SM count comes from
    the device; the derived figure (SMs x 128 FP32 lanes x 2 x max SM clock) is
    reported beside the measurement."""
    f1, m1 = spm.measure_peak(spm.PEAK_FFMA)
    f2, m2 = spm.measure_peak(spm.PEAK_FFMA2)
    d1, m3 = spm.measure_peak(spm.PEAK_DFMA)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    return {"fp32": max(f1, f2), "fp64": d1, "fp32_ffma": f1, "fp32_ffma2": f2, "fp64_dfma": d1,
            "sms": sms, "fp32_derived_at_2070MHz": sms * 128 * 2 * 2.070e9 / 1e12,
            "source": "measured: spm_measure_peak FMA micro-benchmark, this run"}


def algorithmic_flops(n, op, nrhs=1):
    """Flops of one apply by the usual count: 7 zero-padded 3-D FFTs of L^3
    points at 5 L^3 log2(L^3) each, times 7/12 for the pruned zero half and the
    cropped outputs, 48 L^3 for the Fourier-side product (6 complex MACs per
    frequency), and 1944 n^3 for Q (243 complex MACs per point)."""
    import math
    L = 2 * n
    L3 = float(L) ** 3
    f = 7 * 5 * L3 * math.log2(L3) * 7.0 / 12.0 + 48 * L3
    if op == "QA":
        f += 1944.0 * n ** 3
    return f * nrhs


def zpass_name(spm, prec, L):
    """The z-pass kernel the library's timed plan chose for FFT length L."""
    z = spm.get_apply_plan(spm.SPM_C64 if prec == "c64" else spm.SPM_C128, L)
    if z < 0:
        return "not chosen"
    name = {0: "four-line", 1: "one-field prefetch", 2: "TMA-fed persistent", 3: "16 per thread",
            4: "staged spectra", 5: "even/odd split"}.get(z & 7, "?")
    return name + (" + fused x/y plane passes" if z & 8 else "")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=10.0):
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)

    def mark(self):
        return len(self.lines)

    def stop(self, begin=0, end=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines[begin:end]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(wl, seconds, op, max_steps=None, warmup=1, single_thread_seconds=0.0):
    """FP64 oracle apply (A, then Q for op QA) on a bounded sample: `warmup`
    untimed applies, then whole timed applies until about `seconds` have passed
    (or `max_steps` applies).  For Q the stencil tables are seeded random
    numbers: the oracle's cost does not depend on their values."""
    import oracle
    n, k = wl["n"], wl["omega"]
    m, p = oracle.medium(wl["eps"], wl["grad"])
    x = wl["einc"][0]
    F = oracle.FFTOperator(n, k)
    alpha = si.random_field(1, 99, 27 * 81).reshape(-1)[: 27 * 81 * 3].reshape(27, 81, 3)

    def one():
        y = F.apply(m, p, x)
        if op == "QA":
            y = oracle.apply_Q(n, alpha, y)
        return y

    for _ in range(max(1, warmup)):
        one()
    t0 = time.perf_counter()
    count = 0
    while max_steps is None or count < max_steps:
        one()
        count += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    what = "A then Q" if op == "QA" else "A"
    out = {"value": count / dt, "unit": "applies/s", "cores": cores, "kind": "oracle", "steps_run": count,
           "sample": f"{count} FP64 oracle applies of {what} at n={n} (kernel spectra precomputed), "
                     f"{dt:.1f} s on {cores} host threads"}
    if single_thread_seconds > 0:
        oracle.set_threads(1)
        t0 = time.perf_counter()
        c1 = 0
        while True:
            one()
            c1 += 1
            if time.perf_counter() - t0 > single_thread_seconds:
                break
        d1 = time.perf_counter() - t0
        oracle.set_threads(cores)
        out["single_thread"] = {"value": c1 / d1, "unit": "applies/s", "cores": 1,
                                "sample": f"{c1} applies, {d1:.1f} s on one host thread"}
    F.close()
    return out


def run_reference(args):
    """The reference arm: the CPU oracle as it stands.  One step is one whole
    oracle apply; the run stops after --steps steps or --cpu-seconds of timed
    work, whichever comes first (a full oracle apply at n = 64 takes about
    0.2 s on 16 host threads), and reports the steps it ran."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = si.workload(args.workload)
    cb = cpu_baseline(wl, args.cpu_seconds, args.op, max_steps=args.steps, warmup=min(args.warmup, 3))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "applies/s",
            "n_gpus": args.gpus, "steps": cb["steps_run"], "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "n": wl["n"], "nrhs": 1, "op": args.op,
                       "parallelism": "replicas1"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate_timing(total_ms, steps, units_per_step, world, dist=None, device="cpu"):
    """Max of the timed region over ranks; value = units of all ranks per second.

    With world > 1 every rank runs an independent replica (no data-path
    collective); only this timing reduction crosses ranks."""
    if world > 1 and dist is not None:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    value = world * units_per_step * steps / (total_ms / 1000.0)
    return ms_per_step, value


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("apply.cu", "fft_reg.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1804_02297_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, prec, op):
    """DRAM bytes per apply (read + write, all launches of one apply) from the
    committed ncu summary profiles/apply_dram_traffic.md, or None when the
    kernel sources changed since the counters were taken (hash mismatch)."""
    path = os.path.join(ROOT, "profiles", "apply_dram_traffic.md")
    if not os.path.exists(path):
        return None
    want = f"{workload}/{prec}/{op}"
    for line in open(path):
        f = line.strip().strip("|").split("|")
        f = [x.strip().strip("`") for x in f]
        if len(f) >= 3 and f[0] == want and f[2] == kernel_source_hash():
            try:
                return int(f[1])
            except ValueError:
                return None
    return None


def chunk_of(P, n, prec):
    """Right-hand sides per pass chunk inside the library: up to 4 GiB of
    intermediates (24 n^3 complex per right-hand side), at most 64."""
    el = 8 if prec == "c64" else 16
    per = 24.0 * n ** 3 * el
    budget = 4096 * 2 ** 20
    return 1 if per >= budget else min(64, int(budget // per))


def run_uneven(args, torch, spm, rank, world, local):
    """32 independent problems (n in {32, 48, 64, 96}): batched apply (one CUDA
    graph launch per step) and the batched mixed-precision solve to 1e-6."""
    probs = si.uneven_batch(32)
    B = spm.Batch([q["n"] for q in probs], [q["omega"] for q in probs], [q["eps"] for q in probs],
                  [q["grad"] for q in probs])
    dtype = torch.complex64 if args.prec == "c64" else torch.complex128
    xs = [torch.from_numpy(q["einc"]).to(dtype).to("cuda") for q in probs]
    ys = [torch.zeros_like(x) for x in xs]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        B.apply_A(xs, ys)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_first()
    mark0 = sampler.mark()
    ev = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.apply_A(xs, ys)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    mark1 = sampler.mark()
    time.sleep(0.25)
    clocks = sampler.stop(max(0, mark0 - 1), mark1 + 1)
    total_ms = float(np.sum([a.elapsed_time(b) for a, b in ev]))
    dist = torch.distributed if world > 1 else None
    ms_per_step, value = aggregate_timing(total_ms, args.steps, len(probs), world, dist, "cuda")
    alg = sum(compulsory_bytes(q["n"], args.prec) for q in probs)
    peak, peak_kind = peaks()
    achieved = alg / (ms_per_step / 1000.0) / 1e9
    flops = sum(algorithmic_flops(q["n"], "A") for q in probs)
    apk = alu_peaks(spm, torch)
    fpeak = apk["fp32"] if args.prec == "c64" else apk["fp64"]
    tflops = flops / (ms_per_step / 1000.0) / 1e12
    line = {"metric": METRIC, "value": value, "unit": "problem applies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": "uneven32", "sizes": sorted(set(q["n"] for q in probs)), "problems": len(probs),
                       "op": "A", "graph": "one CUDA graph launch per step", "l2": "flushed between steps",
                       "zpass": {str(2 * m): zpass_name(spm, args.prec, 2 * m) for m in sorted(set(q["n"] for q in probs))},
                       "parallelism": f"replicas{world}"},
            "roofline": {"bound": "alu", "kernel": "batched apply_A (graph)", "achieved": tflops, "peak": fpeak,
                         "unit": "TFLOP/s", "frac": tflops / fpeak, "algorithmic_flops": flops, "traffic": None,
                         "peak_source": apk["source"], "peaks": apk,
                         "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                 "peak_source": peak_kind, "algorithmic_bytes": alg}},
            "gpu_launches": 5 * len(probs) * args.steps, "clocks": clocks}
    if args.solve != "none":
        # solves: the problems with n <= 64 (the nested-dissection factor of one
        # n = 96 problem alone needs 65-131 GB, so six of them cannot stay resident)
        sub = [q for q in probs if q["n"] <= 64]
        B2 = spm.Batch([q["n"] for q in sub], [q["omega"] for q in sub], [q["eps"] for q in sub],
                       [q["grad"] for q in sub])
        t0 = time.perf_counter()
        B2.build_stencils(spm.SPM_C64H)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        gs = []
        for i, q in enumerate(sub):
            e = torch.from_numpy(q["einc"]).to("cuda")
            g = torch.zeros_like(e)
            B2.problems[i].rhs_from_incident(e, g)
            gs.append(g)
        xs2 = [torch.zeros_like(g) for g in gs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos, st = B2.solve(gs, xs2, prec=spm.SPM_MIXED, tol=1e-6, maxit=400, check=False)
        torch.cuda.synchronize()
        line["solve"] = {"problems": len(sub), "sizes": sorted(set(q["n"] for q in sub)),
                         "mixed_half_factor_batch_time_s": time.perf_counter() - t0, "status": st,
                         "max_iterations": max(i.iterations for i in infos),
                         "max_true_relres": max(i.true_relres for i in infos),
                         "setup_stencils_factor_c64_half_storage_s": setup_s}
        big = [q for q in probs if q["n"] > 64]
        if args.uneven_solve_all and big:
            # the n = 96 problems one after another: set-up, solve, release
            B2.close()
            del B2, gs, xs2
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            line["solve"]["free_gb_after_batch_release"] = torch.cuda.mem_get_info()[0] / 1e9
            rows = []
            for q in big:
                free_gb = torch.cuda.mem_get_info()[0] / 1e9
                Pq = spm.Problem(q["n"], q["omega"], q["eps"], q["grad"])
                t0 = time.perf_counter()
                try:
                    Pq.build_stencils(spm.SPM_C64 if args.uneven_n96_factor == "c64" else spm.SPM_C64H)
                except spm.SpmError as err:
                    rows.append({"status": err.status, "error": str(err), "free_gb_before": free_gb})
                    Pq.close()
                    del Pq
                    torch.cuda.empty_cache()
                    continue
                torch.cuda.synchronize()
                su = time.perf_counter() - t0
                e = torch.from_numpy(q["einc"]).to("cuda")
                g = torch.zeros_like(e)
                Pq.rhs_from_incident(e, g)
                xq = torch.zeros_like(g)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info, stq = Pq.solve(g, xq, prec=spm.SPM_MIXED, tol=1e-6, maxit=400, check=False)
                torch.cuda.synchronize()
                variant, attempts, _, probe, _ = Pq.factor_info(spm.SPM_C64)
                rows.append({"free_gb_before": free_gb, "setup_s": su, "solve_s": time.perf_counter() - t0,
                             "iterations": info.iterations,
                             "true_relres": info.true_relres, "status": stq, "tree_variant": variant,
                             "factorisations": attempts, "probe": probe})
                Pq.close()
                del Pq, e, g, xq
                torch.cuda.empty_cache()
            line["solve"]["n96_one_at_a_time"] = rows
        elif big:
            line["solve"]["excluded"] = ("n = 96 problems: apply only here (factor 65-131 GB each; "
                                         "--uneven-solve-all solves them one after another)")
    if rank == 0:
        print(json.dumps(line), flush=True)


def time_solve_S(spm, torch, P, prec_factor, nrhs=1, reps=10):
    """Device time of one S^-1 (forward and backward sweep of the factor) and
    the bandwidth it reaches reading the stored blocks once."""
    n = P.n
    x = torch.randn(nrhs, 3, n, n, n, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    stream = torch.cuda.current_stream()
    P.solve_S(x, y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        P.solve_S(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = P.factor_bytes(prec_factor)
    peak, _ = peaks()
    gbs = nbytes / (ms / 1000.0) / 1e9
    return {"ms": ms, "factor_bytes": nbytes, "achieved_gbs": gbs, "frac_of_hbm_peak": gbs / peak}


def measure_solve(spm, torch, P, wl, args, have_c64_factor):
    """Time-to-1e-6 of the preconditioned solve (set-up reported separately)."""
    out = {"tol": 1e-6, "restart": 20, "nrhs": int(wl["einc"].shape[0])}
    n = wl["n"]
    t0 = time.perf_counter()
    if not have_c64_factor:
        P.build_stencils(spm.SPM_C64)
    torch.cuda.synchronize()
    e = torch.from_numpy(wl["einc"]).to("cuda")  # every incident field of the workload, one block solve
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    modes = [("mixed", spm.SPM_MIXED)]
    if args.solve == "both":
        t1 = time.perf_counter()
        P.factor_S(spm.SPM_C128)
        out["setup_factor_c128_s"] = time.perf_counter() - t1
        modes.append(("fp64", spm.SPM_C128))
    for name, prec in modes:
        times = []
        for _ in range(3):
            x = torch.zeros_like(g)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            info, st = P.solve(g, x, prec=prec, tol=1e-6, maxit=400, restart=20, check=False)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        out[name] = {"time_s": float(np.median(times)), "iterations": info.iterations,
                     "outer_steps": info.outer_steps, "true_relres": info.true_relres, "status": st}
    out["s_inverse_c64"] = time_solve_S(spm, torch, P, spm.SPM_C64)
    # the same mixed solve with the factor's blocks stored as scaled binary16
    t1 = time.perf_counter()
    P.factor_S(spm.SPM_C64H)
    torch.cuda.synchronize()
    out["setup_factor_c64_half_storage_s"] = time.perf_counter() - t1
    times = []
    for _ in range(3):
        x = torch.zeros_like(g)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        info, st = P.solve(g, x, prec=spm.SPM_MIXED, tol=1e-6, maxit=400, restart=20, check=False)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t1)
    out["mixed_half_factor"] = {"time_s": float(np.median(times)), "iterations": info.iterations,
                                "outer_steps": info.outer_steps, "true_relres": info.true_relres, "status": st}
    out["s_inverse_c64_half"] = time_solve_S(spm, torch, P, spm.SPM_C64)
    if "fp64" in out:
        out["fp64_over_mixed"] = out["fp64"]["time_s"] / out["mixed"]["time_s"]
        out["fp64_over_mixed_half_factor"] = out["fp64"]["time_s"] / out["mixed_half_factor"]["time_s"]
    return out


def time_apply(torch, fn, x, y, steps, warmup=3):
    """Median device time (ms) of fn(x, y) with the L2 flushed before each call."""
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        fn(x, y)
    torch.cuda.synchronize()
    ev = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(x, y)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


def measure_n256(spm, torch, apk, hbm_peak, hbm_kind, steps=12, warmup=3):
    """The n = 256 apply of A (L = 512, 32 bumps, k = 64 pi, one right-hand side,
    complex64), where the pass intermediates (24 n^3 complex = 3.2 GB) stream
    through HBM: device time per apply (CUDA events, L2 flushed between applies),
    its algorithmic bytes and flops against the measured peaks, and the DRAM
    bytes ncu recorded for one apply (profiles/apply_dram_traffic.md, while the
    apply sources are unchanged)."""
    wl = si.workload("n256_bumps32")
    n = wl["n"]
    P = spm.Problem(n, wl["omega"], wl["eps"], wl["grad"])
    x = torch.from_numpy(wl["einc"]).to(torch.complex64).to("cuda").contiguous()
    y = torch.zeros_like(x)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        P.apply_A(x, y)
    torch.cuda.synchronize()
    ev = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.apply_A(x, y)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    alg = compulsory_bytes(n, "c64")
    flops = algorithmic_flops(n, "A")
    traffic = recorded_traffic("n256_bumps32", "c64", "A")
    out = {"workload": "n256_bumps32", "op": "A", "dtype": "c64", "steps": steps, "ms_per_apply": ms,
           "applies_per_s": 1000.0 / ms, "zpass": zpass_name(spm, "c64", 2 * n),
           "algorithmic_bytes": alg, "hbm_frac_algorithmic": alg / (ms / 1000.0) / 1e9 / hbm_peak,
           "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_kind,
           "algorithmic_flops": flops, "tflops": flops / (ms / 1000.0) / 1e12,
           "fp32_frac": flops / (ms / 1000.0) / 1e12 / apk["fp32"], "fp32_peak_tflops": apk["fp32"],
           "traffic": traffic}
    if traffic is not None:
        out["dram_gbs"] = traffic / (ms / 1000.0) / 1e9
        out["dram_frac"] = out["dram_gbs"] / hbm_peak
    # the cuFFT comparison apply (full padded 3-D transforms) on the same input
    out["cufft_ms_per_apply"] = time_apply(torch, P.apply_A_cufft, x, y, steps)
    out["ours_over_cufft_speedup"] = out["cufft_ms_per_apply"] / ms
    P.close()
    del P, x, y, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


# Section 4, Tables 1-3 (2-D, MATLAB on four Xeon E7-4830 v3): per k/2pi (n =
# 119, 239, 479, 959) the set-up, apply (one application of the preconditioner
# S^-1) and solve seconds and iteration counts of the Gaussian lens (Table 1),
# context for the 2-D numbers (another machine).
PAPER_2D_LENS = {119: (1.25, 5.58e-2, 6, 9.13e-1), 239: (5.52, 3.27e-1, 6, 2.51), 479: (21.7, 1.40, 6, 8.93),
                 959: (98.7, 5.03, 6, 41.3)}


def measure_2d(spm, torch, apk, hbm_peak, hbm_kind, sizes=(119, 239, 479, 959), steps=20):
    """The 2-D variant (include/spm2d.h) at the four sizes of the paper's 2-D
    tables (N = 2 n^2, six points per wavelength): device time of the apply of A
    (one right-hand side, complex64 and complex128, L2 flushed between applies)
    with its algorithmic bytes and flops against the measured peaks; then the
    Gaussian-lens solve to 1e-6 in FP64 as the paper's (stencils fitted on the
    device, complex128 nested-dissection factor, GMRES(20)), set-up and solve wall
    times and iterations.  (A complex64 factor of these 2-D S loses accuracy from
    n = 479 on: its probe residual reaches 0.1-0.5 and GMRES needs 30-70 steps.)"""
    out = {"sizes": list(sizes), "apply": [], "solve": [],
           "paper_table1_lens_s": {str(n): {"setup": v[0], "apply": v[1], "iterations": v[2], "solve": v[3]}
                                   for n, v in PAPER_2D_LENS.items()}}
    for n in sizes:
        wl = si.workload_2d(f"lens2d_n{n}")
        t0 = time.perf_counter()
        P = spm.Problem2D(n, wl["omega"], wl["eps"], wl["grad"])
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        L = P.info()[1]
        N, H = n * n, L // 2 + 1
        flops = 5.0 * L * np.log2(L) * (3 * n + 5 * L + 2 * n) + 32.0 * L * L
        for prec, dt, el in (("c64", torch.complex64, 8), ("c128", torch.complex128, 16)):
            x = torch.from_numpy(wl["einc"]).to(dt).to("cuda").contiguous()
            y = torch.zeros_like(x)
            ms = time_apply(torch, P.apply_A, x, y, steps)
            alg = el * (7 * N + 3 * H * H)
            fpk = apk["fp32"] if prec == "c64" else apk["fp64"]
            out["apply"].append({"n": n, "L": L, "dtype": prec, "ms": ms, "algorithmic_bytes": alg,
                                 "hbm_frac": alg / (ms / 1000.0) / 1e9 / hbm_peak, "algorithmic_flops": flops,
                                 "alu_frac": flops / (ms / 1000.0) / 1e12 / fpk,
                                 "alu_peak": "fp32" if prec == "c64" else "fp64"})
            del x, y
        t1 = time.perf_counter()
        P.build_stencils(spm.SPM_C128)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t1
        e = torch.from_numpy(wl["einc"]).to("cuda")
        g = torch.zeros_like(e)
        P.rhs_from_incident(e, g)
        x = torch.zeros_like(g)
        # one S^-1 (the paper's T_apply), complex128 factor, device time
        s_inv_ms = time_apply(torch, P.solve_S, g, x, 5)
        x.zero_()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        info, st = P.solve(g, x, prec=spm.SPM_C128, tol=1e-6, maxit=200, restart=20, check=False)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t2
        ref = PAPER_2D_LENS.get(n)
        out["solve"].append({"n": n, "unknowns": 2 * N, "k_over_2pi": wl["omega"] / (2 * np.pi), "dtype": "c128",
                             "create_s": t_create, "stencils_and_factor_s": t_setup, "setup_s": t_create + t_setup,
                             "solve_s": t_solve, "iterations": info.iterations,
                             "true_relres": info.true_relres, "status": st,
                             "factor_probe": P.factor_info(spm.SPM_C128)[3], "s_inverse_ms": s_inv_ms,
                             "paper_s_inverse_over_ours": ref[1] / (s_inv_ms / 1000.0) if ref else None,
                             "paper_setup_over_ours": ref[0] / (t_create + t_setup) if ref else None,
                             "paper_solve_over_ours": ref[3] / t_solve if ref else None})
        P.close()
        del P, e, g, x
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    out["hbm_peak_gbs"] = hbm_peak
    out["hbm_peak_source"] = hbm_kind
    return out


def measure_block_solve(spm, torch, P, args):
    """Config 3: the 64 incident plane waves (32 Fibonacci directions x 2
    polarisations) of the n = 64 medium as one block right-hand side, solved to a
    true relative residual of 1e-6, complex64 operator and factor inside the FP64
    outer loop (mixed) and plain complex128 (fp64, when --solve both built its
    factor).  Set-up is shared with the single-RHS solve and not counted."""
    wl = si.workload("n64_bumps8_rhs64")
    e = torch.from_numpy(wl["einc"]).to("cuda")
    g = torch.zeros_like(e)
    P.rhs_from_incident(e, g)
    del e
    out = {"nrhs": int(g.shape[0]), "tol": 1e-6, "restart": 20}
    modes = [("mixed", spm.SPM_MIXED)] + ([("fp64", spm.SPM_C128)] if args.solve == "both" else [])
    # the mixed solve with the complex64 factor (the half-storage one was built last)
    P.factor_S(spm.SPM_C64)
    for name, prec in modes:
        x = torch.zeros_like(g)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        info, st = P.solve(g, x, prec=prec, tol=1e-6, maxit=400, restart=20, check=False)
        torch.cuda.synchronize()
        out[name] = {"time_s": time.perf_counter() - t1, "iterations": info.iterations,
                     "outer_steps": info.outer_steps, "true_relres": info.true_relres, "status": st,
                     "field_solves_per_s": g.shape[0] / (time.perf_counter() - t1)}
        del x
    if "fp64" in out:
        out["fp64_over_mixed"] = out["fp64"]["time_s"] / out["mixed"]["time_s"]
    del g
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1804_02297_gb300 as spm

    if args.workload == "uneven32":
        return run_uneven(args, torch, spm, rank, world, local)
    wl = si.workload(args.workload)
    n = wl["n"]
    P = spm.Problem(n, wl["omega"], wl["eps"], wl["grad"])
    dtype = torch.complex64 if args.prec == "c64" else torch.complex128
    nrhs = wl["einc"].shape[0]
    x = torch.from_numpy(wl["einc"]).to(dtype).to("cuda").contiguous()
    y = torch.zeros_like(x)
    setup = {}
    if n > 64:
        args.solve = "none"  # the nested-dissection factor does not fit in one GPU above n = 64
        if args.op == "QA":
            args.op = "A"
    if args.op == "QA" or args.solve != "none":
        t0 = time.perf_counter()
        P.build_stencils(spm.SPM_C64)  # device stencil fit, S assembly, complex64 factor
        torch.cuda.synchronize()
        setup["stencils_assembly_factor_c64_s"] = time.perf_counter() - t0
    fn = P.apply_QA if args.op == "QA" else P.apply_A
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.warmup):
        fn(x, y)
    torch.cuda.synchronize()
    # launches of one apply chunk, per the plan the first apply chose: five FFT
    # passes (three when the x/y plane passes are fused), plus Q for Q A (its
    # interior, face and edge blocks share one launch)
    zv = spm.get_apply_plan(spm.SPM_C64 if args.prec == "c64" else spm.SPM_C128, 2 * n)
    launches_per_step = (3 if zv >= 0 and zv & 8 else 5) + (1 if args.op == "QA" else 0)
    sampler.wait_first()
    if world > 1:
        torch.distributed.barrier()
    mark0 = sampler.mark()
    times = []
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(x, y)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    mark1 = sampler.mark()
    time.sleep(0.25)
    clocks = sampler.stop(max(0, mark0 - 1), mark1 + 1)
    step_ms = [a.elapsed_time(b) for a, b in times]
    total_ms = float(np.sum(step_ms))
    dist = torch.distributed if world > 1 else None
    ms_per_step, value = aggregate_timing(total_ms, args.steps, nrhs, world, dist, "cuda")

    # e2e: the host-buffer C-ABI call (spm_apply_QA_host / spm_apply_A_host): every
    # step's fields start in page-locked host memory and its results end there;
    # the library overlaps the copies of one field with the apply of the previous
    # one.  Calls of up to 32 steps each, the K steps timed as a whole.
    per_call = max(1, 32 // nrhs)
    x0 = torch.from_numpy(wl["einc"]).to(dtype)
    xh = x0.repeat(per_call, 1, 1, 1, 1).contiguous().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    host_fn = P.apply_QA_host if args.op == "QA" else P.apply_A_host
    host_fn(xh[:nrhs], yh[:nrhs])
    host_fn(xh, yh)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    done = 0
    while done < args.steps:
        cnt = min(per_call, args.steps - done)
        host_fn(xh[: cnt * nrhs], yh[: cnt * nrhs])
        done += cnt
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    _, e2e_value = aggregate_timing(e2e_ms, args.steps, nrhs, world, dist, "cuda")
    # the host result equals the device result of the same input
    ref = torch.empty_like(x)
    fn(x, ref)
    torch.cuda.synchronize()
    e2e_check = float((yh[:nrhs].to("cuda") - ref).abs().max() / ref.abs().max())
    nbytes = x0.numel() * x0.element_size()  # one step's fields (copied in, and the results out)

    peak, peak_kind = peaks()
    alg = compulsory_bytes(n, args.prec, nrhs)
    achieved = alg / (ms_per_step / 1000.0) / 1e9
    flops = algorithmic_flops(n, args.op, nrhs)
    tflops = flops / (ms_per_step / 1000.0) / 1e12
    apk = alu_peaks(spm, torch)
    fpeak = apk["fp32"] if args.prec == "c64" else apk["fp64"]
    # roofline: the bound whose minimum time is longer (flops at the ALU peak vs
    # compulsory bytes at the measured HBM bandwidth) is the one reported
    alu_bound = flops / (fpeak * 1e12) > alg / (peak * 1e9)
    traffic = recorded_traffic(args.workload, args.prec, args.op)
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
           "algorithmic_bytes": alg, "traffic": traffic}
    if traffic is not None and nrhs == 1:
        # DRAM bytes the passes actually move (ncu, committed profile) over the measured step time
        hbm["dram_achieved"] = traffic / (ms_per_step / 1000.0) / 1e9
        hbm["dram_frac"] = hbm["dram_achieved"] / peak
    alu = {"achieved": tflops, "peak": fpeak, "unit": "TFLOP/s", "frac": tflops / fpeak,
           "peak_source": apk["source"] + (" (FP32)" if args.prec == "c64" else " (FP64)"),
           "algorithmic_flops": flops, "peaks": apk}
    roof = dict(alu if alu_bound else hbm)
    roof["bound"] = "alu" if alu_bound else "hbm"
    roof["kernel"] = f"apply_{args.op} ({launches_per_step} launches)"
    roof["traffic"] = hbm["traffic"]
    roof["hbm"] = hbm
    roof["alu"] = alu
    line = {"metric": METRIC, "value": value, "unit": "field applies/s" if nrhs > 1 else "applies/s",
            "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nrhs": nrhs, "op": args.op,
                       "zpass": zpass_name(spm, args.prec, 2 * n),
                       "l2": "flushed (512 MiB write) between steps",
                       "parallelism": f"replicas{world}"},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "field applies/s" if nrhs > 1 else "applies/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "api": "spm_apply_QA_host" if args.op == "QA" else "spm_apply_A_host",
                    "steps_per_call": per_call, "max_rel_diff_vs_device_call": e2e_check},
            "gpu_launches": launches_per_step * args.steps * max(1, -(-nrhs // chunk_of(P, n, args.prec))),
            "clocks": clocks,
            "step_ms_min": float(np.min(step_ms)), "step_ms_median": float(np.median(step_ms))}
    if nrhs == 1:
        # every pass of one apply timed with CUDA events on the launch stream
        # (serialised: an event between passes), and the dominant pass's own
        # roofline: its algorithmic flops over its measured time
        pass_ms = P.profile_apply(x, y, with_q=(args.op == "QA"), reps=50 if n <= 64 else 5)
        zv = spm.get_apply_plan(spm.SPM_C64 if args.prec == "c64" else spm.SPM_C128, 2 * n)
        names = (["xy-forward (fused)", "z-pass", "yx-inverse (fused)"] if zv >= 0 and zv & 8
                 else ["x-forward", "y-forward", "z-pass", "y-inverse", "x-inverse"])
        if args.op == "QA":
            names = names + ["Q"]
        L = 2 * n
        # z-pass: 7 full-length line transforms per column (4 forward, 3 inverse) over L^2
        # columns at 5 L log2 L each, plus 6 complex MACs (48 flops) per frequency
        z_flops = 7.0 * L * L * 5.0 * L * np.log2(L) + 48.0 * L ** 3
        q_flops = 1944.0 * n ** 3
        tot = sum(pass_ms)
        line["passes"] = {"names": names, "ms": pass_ms, "share": [v / tot for v in pass_ms],
                          "note": "serialised by an event between passes; the pipelined step is shorter"}
        iz = names.index("z-pass")
        fpk = fpeak * 1e12
        line["roofline"]["z_pass"] = {"kernel": "z-pass (" + zpass_name(spm, args.prec, L) + ")", "bound": "alu",
                                      "ms": pass_ms[iz], "algorithmic_flops": z_flops,
                                      "achieved": z_flops / (pass_ms[iz] / 1000.0) / 1e12, "peak": fpeak,
                                      "unit": "TFLOP/s", "frac": z_flops / (pass_ms[iz] / 1000.0) / fpk,
                                      "traffic": recorded_traffic(args.workload, args.prec,
                                                                  "zpass-" + zpass_name(spm, args.prec, L))}
        if args.op == "QA":
            line["roofline"]["q_gather"] = {"kernel": "k_q", "bound": "alu", "ms": pass_ms[-1],
                                            "algorithmic_flops": q_flops,
                                            "achieved": q_flops / (pass_ms[-1] / 1000.0) / 1e12, "peak": fpeak,
                                            "unit": "TFLOP/s", "frac": q_flops / (pass_ms[-1] / 1000.0) / fpk,
                                            "traffic": recorded_traffic(args.workload, args.prec, "q")}
    if args.prec == "c64" and nrhs == 1:
        # the apply of A alone, hand-written passes against the cuFFT comparison apply
        a_ms = time_apply(torch, P.apply_A, x, y, 200 if n <= 64 else 20)
        c_ms = time_apply(torch, P.apply_A_cufft, x, y, 200 if n <= 64 else 20)
        line["cufft_compare"] = {"op": "A", "n": n, "ours_ms": a_ms, "cufft_ms": c_ms, "speedup": c_ms / a_ms,
                                 "note": "cuFFT: zero-padded (2n)^3 arrays, batched 3-D C2C plans, same product kernel"}
    if args.solve != "none" and n <= 64:
        line["solve"] = measure_solve(spm, torch, P, wl, args, True)
        line["solve"]["setup"] = setup
        if args.workload == "n64_bumps8" and not args.no_block_solve:
            line["solve_block64"] = measure_block_solve(spm, torch, P, args)
    if args.workload == "n64_bumps8" and not args.no_n256:
        fn = None
        P.close()  # release the n = 64 factors before the n = 256 problem
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["apply_n256"] = measure_n256(spm, torch, apk, peak, peak_kind)
    if args.workload == "n64_bumps8" and not args.no_2d:
        line["twod"] = measure_2d(spm, torch, apk, peak, peak_kind)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds, args.op, single_thread_seconds=5.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
