"""Benchmark: staggered-grid Fourier pseudo-spectral elastic solver on GB300.

Workload (default): 256^3 synthetic marine model (water column over five
sediment layers, cp 1800-4000 m/s with depth gradient, cs = cp/1.8, Gardner
rho, 5% Gaussian-correlated perturbation of correlation length 8 cells,
seed 1), 12-cell PML, one random strike/dip/rake double couple in the
reservoir box a third of the way down (seed 2), Ricker 30 Hz, dt from
CFL 0.3, 3000 time steps, 64 x 64 seabed 4C receivers; every step of the
benchmark also superposes 300 log-normal-amplitude events (origin times
uniform in 2 s) of the step's traces into a 4C gather.

One benchmark step = one es_run of all 3000 time steps (three velocity and
three stress FFT-derivative passes, injection and recording per time step)
plus the superposition.  value = nx ny nz nt / device time (Mcell-steps/s),
summed over ranks.  Inputs (fields, materials: ~1.3 GB) exceed the 129 MB
L2, so no flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the paper ships no code of its own).
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

from paper_1705_04874_gb300 import synth  # noqa: E402

PASS_SOURCE = os.path.join(ROOT, "paper_1705_04874_gb300", "csrc", "fft_pass.cuh")


def kernel_code_hash(path: str = PASS_SOURCE) -> str:
    """sha256 of the pass kernels' code with comments and blank lines removed
    (the key under which profiles/traffic.json records its ncu DRAM bytes)."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()
from paper_1705_04874_gb300.replicas import max_over_ranks, sum_over_ranks  # noqa: E402

# algorithmic bytes per cell for one launch of each pass kernel (FP32), the
# lean pass model: a velocity pass reads its 3 source fields, reads and writes
# its 3 targets and reads rho (the buoyancies follow from it): 10 arrays; a
# stress pass reads 3 sources, reads and writes 5 targets and reads lambda and
# mu: 15 arrays.  300 B per cell-step over the six passes.
VEL_BYTES_CELL = 4 * (3 + 2 * 3 + 1)
STR_BYTES_CELL = 4 * (3 + 2 * 5 + 2)


def workload(name):
    if name == "256":
        return dict(n=256, pml=12, nt=3000, rx=64, f0=30.0, seed=1, src_seed=2,
                    desc="256^3 marine, PML 12, random DC in reservoir box, Ricker 30 Hz, "
                         "3000 steps, 64x64 seabed 4C receivers, + superpose 300 events")
    if name == "128":
        return dict(n=128, pml=10, nt=2000, rx=32, f0=30.0, seed=1, src_seed=2,
                    desc="128^3 marine, PML 10, DC strike 30 dip 60 rake 90, Ricker 30 Hz, "
                         "2000 steps, 32x32 seabed 4C receivers, + superpose 300 events")
    raise ValueError(name)


def build_inputs(w, rank=0):
    n = w["n"]
    rho, cp, cs = synth.marine_model(n, seed=w["seed"])
    dt = 0.3 * 10.0 / float(cp.max())  # CFL 0.3 (Eq. (5))
    box = synth.reservoir_box((n, n, n), w["pml"])
    rng = synth.SplitMix64(w["src_seed"] + 1000 * rank)
    if n == 128:
        mt = synth.double_couple_sdr(30, 60, 90)
        pos = tuple((lo + hi) // 2 for lo, hi in box)
    else:
        mt = synth.random_dc(rng)
        pos = tuple(int(v) for v in synth.random_positions(rng, box, 1)[0]) if rank else \
            tuple((lo + hi) // 2 for lo, hi in box)
    wav = synth.ricker(w["nt"], dt, w["f0"])
    ev = synth.events(synth.SplitMix64(3), 300, 1, t_span=2.0)
    n_out = w["nt"] + int(np.ceil(2.0 / dt))
    return dict(rho=rho, cp=cp, cs=cs, dt=dt, mt=mt, pos=pos, wav=wav, ev=ev, n_out=n_out)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(gpus):
    if gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    return rank, world, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def oracle_sample(w, inp, steps, nthreads=0):
    """Time the FP64 oracle on `steps` time steps of the workload."""
    import oracle
    oracle.build()
    n = w["n"]
    t0 = time.perf_counter()
    rcv = oracle.seabed_receivers(inp["cs"], w["pml"], w["rx"], w["rx"])
    oracle.simulate(inp["rho"], inp["cp"], inp["cs"], dx=10.0, dt=inp["dt"], nt=steps, pml=w["pml"],
                    sources=[dict(kind="moment", pos=inp["pos"], m=inp["mt"], w=inp["wav"][:steps])],
                    receivers=rcv, nthreads=nthreads)
    el = time.perf_counter() - t0
    cores = nthreads or oracle.default_threads()
    return n ** 3 * steps / el / 1e6, el, cores


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    inp = build_inputs(w)
    steps = 2
    for _ in range(args.warmup):
        oracle_sample(w, inp, 1)
    vals, els = [], []
    cores = 0
    for _ in range(args.steps):
        v, el, cores = oracle_sample(w, inp, steps)
        vals.append(v)
        els.append(el)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": "Mcell-steps/s", "value": value, "unit": "Mcell-steps/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(els)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["desc"], "grid": [w["n"]] * 3, "sample": f"{steps} time steps per step"},
            "cpu_baseline": {"value": value, "unit": "Mcell-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} time steps of the {w['n']}^3 workload per step"},
            "e2e": {"value": value, "unit": "Mcell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="256", choices=["256", "128", "surrogate", "configs", "gemm", "serve", "train", "paper"])
    ap.add_argument("--gemm-small", action="store_true", help="gemm workload: the decoder shape only")
    ap.add_argument("--sur-locations", type=int, default=682)
    ap.add_argument("--sur-epochs", type=int, default=150)
    ap.add_argument("--sur-hidden", type=int, default=768)
    ap.add_argument("--sur-latent", type=int, default=768)
    ap.add_argument("--sur-nfreq", type=int, default=9)
    ap.add_argument("--sur-lr", type=float, default=3e-3)
    ap.add_argument("--sur-random", type=int, default=10000, help="surrogate workload: sources at random cells")
    ap.add_argument("--nt", type=int, default=0, help="override time steps per es_run (diagnostics)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the reduced surrogate measurement")
    ap.add_argument("--batched-nt", type=int, default=2000, help="time steps of the batched measurement")
    args = ap.parse_args()
    if args.workload == "surrogate":
        return measure_surrogate(args)
    if args.workload == "configs":
        return measure_configs(args)
    if args.workload == "gemm":
        return measure_gemm(args)
    if args.workload == "serve":
        return measure_serve(args)
    if args.workload == "train":
        return measure_train(args)
    if args.workload == "paper":
        return measure_paper(args)
    w = workload(args.workload)
    if args.nt:
        w["nt"] = args.nt
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    from paper_1705_04874_gb300 import es

    rank, world, dist = dist_setup(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    inp = build_inputs(w, rank)
    n, nt = w["n"], w["nt"]
    stream = torch.cuda.current_stream()

    m = es.Model(inp["rho"], inp["cp"], inp["cs"], dx=10.0, pml=w["pml"], stream=stream)
    rcv = torch.from_numpy(m.seabed_receivers(w["rx"], w["rx"])).cuda()
    n_rcv = rcv.shape[0]
    m.source_set(inp["pos"], inp["mt"], torch.from_numpy(inp["wav"]).cuda())
    traces = torch.empty((1, 4, n_rcv, nt), device="cuda")
    gather = torch.empty((4, n_rcv, inp["n_out"]), device="cuda")
    ev_src, ev_amp, ev_t0 = (torch.from_numpy(a).cuda() for a in inp["ev"])

    def step():
        m.state_reset()
        m.run(nt, inp["dt"], rcv, traces[0])
        es.es_superpose(traces, ev_src, ev_amp, ev_t0, inp["dt"], inp["n_out"], gather=gather, stream=stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    kern = []
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
        kern.append(m.last_step_kernel_ms())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    ms = max_over_ranks(dist, ms)
    cells = float(n) ** 3 * nt
    total_cells = sum_over_ranks(dist, cells)
    value = total_cells / (ms * 1e-3) / 1e6

    # per-kernel time of a time step (CUDA events around each launch of the
    # last time step of every es_run in the timed region)
    kern = np.array(kern)
    kmean = kern.mean(axis=0)
    names = list(es.KERNEL_NAMES[:len(kmean)])
    bytes_cell = {k: VEL_BYTES_CELL for k in names if k.startswith("vel")}
    bytes_cell.update({k: STR_BYTES_CELL for k in names if k.startswith("str")})
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    passes = {k: kmean[i] for i, k in enumerate(names) if k in bytes_cell}
    dom = max(passes, key=passes.get)
    achieved = bytes_cell[dom] * n ** 3 / (passes[dom] * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        # ncu DRAM bytes per launch, valid only for the kernel code they were taken on
        try:
            rec = json.load(open(prof))
            if kernel_code_hash().startswith(rec.get("kernel_code_sha256_prefix", "-")):
                traffic = rec.get(f"{args.workload}:{dom}")
        except (OSError, ValueError):
            traffic = None
    kernels = {k: {"ms": round(float(kmean[i]), 5),
                   "GBps": round(bytes_cell[k] * n ** 3 / (kmean[i] * 1e-3) / 1e9, 1) if k in bytes_cell else None}
               for i, k in enumerate(names)}
    step_bytes = sum(bytes_cell[k] for k in bytes_cell) * float(n) ** 3 * nt
    kps = m.kernels_per_step()
    launches = args.steps * (kps * nt + 3)

    line = {"metric": "Mcell-steps/s", "value": value, "unit": "Mcell-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["desc"], "grid": [n] * 3, "time_steps": nt, "receivers": n_rcv,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (fields+materials ~%.1f GB)" % (17 * 4 * n ** 3 / 1e9)},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": peak_src,
                         "bytes_per_cell": round(bytes_cell[dom], 2)},
            "useful_hbm_frac": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4),
            "kernels": kernels, "gpu_launches": launches}
    if clk:
        line["clocks"] = clk

    if not args.no_e2e and rank == 0:
        line["e2e"] = e2e(es, w, inp, stream)
    if not args.no_batched and rank == 0:
        m.close()
        line["batched"] = measure_batched(es, args.batched_nt, 1, stream)
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        v, el, cores = oracle_sample(w, inp, 3)
        line["cpu_baseline"] = {"value": v, "unit": "Mcell-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"3 time steps of the {n}^3 workload ({el:.1f} s)"}
    m.close()
    if not args.no_surrogate and rank == 0 and world == 1:
        # the surrogate half of the metric on a reduced catalog (bench.py --workload surrogate
        # runs the full 682-location, 4092-run one)
        sur_out, _ = surrogate_pipeline(128, 400, args.sur_lr, args.sur_hidden, args.sur_latent, args.sur_nfreq,
                                        gemm=False)
        line["surrogate"] = {"value": sur_out["random_positions"]["pipeline_seismograms_per_s"],
                             "value_is": "sources at random cells of the reservoir box (network where the gate "
                                         "trusts it, solver elsewhere)",
                             "unit": "4C seismogram sets/s",
                             "gate": "relative L2 <= 5 % (held-out, 0.8 margin); served sources checked",
                             **sur_out}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_batched(es, nt, reps, stream):
    """Batched workload (C4): 64 sources (uniform in the reservoir box, random
    double couples) on the 128^3 marine model plus 16 on a 96^3 and 8 on a
    160^3 model, nt steps each (full length: 2000), all advanced in one graph
    (one branch per model), then 300 events (log-normal amplitudes, sigma 1;
    origin times uniform in 2 s; sources drawn from the 64) superposed into a
    4C gather -- both inside the timed region.  The plain rate runs the same
    sources one per es_run on each grid size (timed per size on one source and
    weighted by the batch's source counts), plus the same superposition."""
    import torch
    specs = [(128, 10, 64), (96, 8, 16), (160, 10, 8)]
    models, rcvs, dts, cells, inputs = [], [], [], 0.0, []
    for i, (n, pml, nb) in enumerate(specs):
        rho, cp, cs = synth.marine_model(n, seed=1)
        dt = 0.3 * 10.0 / float(cp.max())
        rng = synth.SplitMix64(40 + i)
        box = synth.reservoir_box((n, n, n), pml)
        pos = synth.random_positions(rng, box, nb)
        mts = np.array([synth.random_dc(rng) for _ in range(nb)])
        wav = np.stack([synth.ricker(nt, dt, 30.0)] * nb)
        m = es.Model(rho, cp, cs, dx=10.0, pml=pml, stream=stream)
        rcv = m.seabed_receivers(32, 32)
        m.batch_set(pos, mts, wav)
        m.autotune(reps=3)  # FFT plans for this batched model, before the timed region
        models.append(m)
        rcvs.append(torch.from_numpy(rcv).cuda())
        dts.append(dt)
        inputs.append((rho, cp, cs, pml, pos, mts, wav))
        cells += float(n) ** 3 * nb * nt
    outs = [torch.empty((m.nsim, 4, r.shape[0], nt), device="cuda") for m, r in zip(models, rcvs)]
    ev_src, ev_amp, ev_t0 = (torch.from_numpy(a).cuda() for a in synth.events(synth.SplitMix64(3), 300, 64, t_span=2.0))
    n_out = nt + int(np.ceil(2.0 / dts[0]))
    gather = torch.empty((4, rcvs[0].shape[0], n_out), device="cuda")

    def superpose(traces):
        es.es_superpose(traces, ev_src, ev_amp, ev_t0, dts[0], n_out, gather=gather, stream=stream)

    def group():
        for m in models:
            m.state_reset()
        es.es_run_group(models, nt, dts, rcvs, outs)
        superpose(outs[0])

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ms = timed(group, reps)
    ms_sup = timed(lambda: superpose(outs[0]), 3)
    # plain: one source per es_run, on each grid size
    plain_ms, per_size = 0.0, {}
    for (n, pml, nb), (rho, cp, cs, pml_, pos, mts, wav), dt in zip(specs, inputs, dts):
        single = es.Model(rho, cp, cs, dx=10.0, pml=pml, stream=stream)
        rc = single.seabed_receivers(32, 32)
        single.source_set(pos[0], mts[0], torch.from_numpy(wav[0]).cuda())
        rct = torch.from_numpy(rc).cuda()
        tr = torch.empty((4, rct.shape[0], nt), device="cuda")

        def one():
            single.state_reset()
            single.run(nt, dt, rct, tr)
        t1 = timed(one, 2)
        single.close()
        per_size[f"{n}^3"] = {"ms_per_source": round(t1, 2), "Mcell_steps_per_s": round(n ** 3 * nt / (t1 * 1e-3) / 1e6, 1)}
        plain_ms += nb * t1
    plain_ms += ms_sup
    plain = cells / (plain_ms * 1e-3) / 1e6
    value = cells / (ms * 1e-3) / 1e6
    for m in models:
        m.close()
    plans = {f"{'x' if k == 0 else 'yz'}{n}": "x".join(map(str, es.es_fft_plan(k, n)))
             for n in (96, 128, 160) for k in (0, 1)}
    return {"value": round(value, 1), "unit": "Mcell-steps/s", "plain_value": round(plain, 1), "plans": plans,
            "speedup_vs_plain": round(value / plain, 3), "time_steps": nt, "ms_per_run": round(ms, 2),
            "superpose_ms": round(ms_sup, 3), "plain_per_size": per_size,
            "workload": "64 sources on 128^3 + 16 on 96^3 + 8 on 160^3 marine models, one graph, 32x32 receivers, "
                        f"{nt} steps; then 300 events superposed (included)"}


def gemm_tflops(sur, M, N, K, b_nk, reps=5):
    """TFLOP/s of es_gemm_bf16 on random BF16 operands (A [M][K]; B [N][K] when b_nk -- the
    tcgen05 path -- else [K][N], the mma.sync path), CUDA events on the current stream."""
    import torch
    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16) if b_nk else \
        torch.randn(K, N, device="cuda").to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda")
    sur.es_gemm_bf16(A, B, C, b_nk=b_nk)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        sur.es_gemm_bf16(A, B, C, b_nk=b_nk)
    e1.record()
    torch.cuda.synchronize()
    sur.es_gemm_status()
    return 2.0 * M * N * K * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12


def measure_gemm(args):
    """The surrogate's GEMM alone: the decoder product of 256 and of 1024 sources (M x 262,144 x
    4,608, tcgen05), and 8192^3 on the tcgen05 and mma.sync paths (--gemm-small: the first only)."""
    import torch
    from paper_1705_04874_gb300 import surrogate as sur
    torch.cuda.set_device(0)
    shapes = [("tcgen05_decoder_256x262144x4608", 256, 262144, 4608, True),
              ("tcgen05_decoder_1024x262144x4608", 1024, 262144, 4608, True),
              ("tcgen05_8192", 8192, 8192, 8192, True), ("mma_sync_8192", 8192, 8192, 8192, False)]
    if args.gemm_small:
        shapes = shapes[:1]
    res = {name: round(gemm_tflops(sur, M, N, K, b, reps=args.steps), 1) for name, M, N, K, b in shapes}
    print(json.dumps({"metric": "TFLOP/s", "gemm": res, "unit": "TFLOP/s", "dtype": "bf16/f32"}))
    return 0


def measure_serve(args):
    """Serving cost of the surrogate network alone: the C5 network shape (64 receivers x 1024
    samples, 3 -> 768 -> 768 -> 768 latent, 9 positional frequencies; 1.21 G parameters) with
    its initial weights (the cost does not depend on the values), 10,000 random sources in
    batches of 1024 (the serving batch) through es_sur_predict.  Metric: seismogram sets per second."""
    import torch
    from paper_1705_04874_gb300 import surrogate as sur
    torch.cuda.set_device(0)
    s = sur.Surrogate(64, 1024, nfreq=9, hidden=768, latent=768, max_batch=1024, seed=1)
    rng = np.random.default_rng(3)
    n_src, B = 10000, 1024
    pos = torch.from_numpy(rng.uniform(-1, 1, (n_src + B, 3)).astype(np.float32)).cuda()
    mt = torch.from_numpy(rng.standard_normal((n_src + B, 6)).astype(np.float32)).cuda()
    out = torch.empty((B, s.D), device="cuda")

    def serve_all():
        for b in range(0, n_src, B):
            s.predict(pos[b:b + B], mt[b:b + B], out)
    serve_all()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        serve_all()
    e1.record()
    torch.cuda.synchronize()
    sur.es_gemm_status()
    ms = e0.elapsed_time(e1) / args.steps
    s.close()
    n_batches = (n_src + B - 1) // B
    print(json.dumps({"metric": "seismograms/s", "value": round(n_src / (ms * 1e-3), 1),
                      "unit": "4C seismogram sets/s (network only)", "ms_per_10k": round(ms, 2),
                      "batches": n_batches, "dtype": "bf16/f32", "data": "synthetic"}))
    return 0


def measure_train(args):
    """Training cost of the surrogate network alone: the C5 network shape (as --workload serve)
    with its initial weights, a batch of 256 sources with synthetic targets of the C5 trace shape
    (the cost does not depend on the values); --warmup then --steps Adam steps through
    es_sur_train_step, timed with CUDA events.  Metric: milliseconds per Adam step."""
    import torch
    from paper_1705_04874_gb300 import surrogate as sur
    torch.cuda.set_device(0)
    s = sur.Surrogate(64, 1024, nfreq=9, hidden=768, latent=768, max_batch=256, seed=1)
    rng = np.random.default_rng(4)
    B = 256
    pos = torch.from_numpy(rng.uniform(-1, 1, (B, 3)).astype(np.float32)).cuda()
    mt = torch.from_numpy(rng.standard_normal((B, 6)).astype(np.float32)).cuda()
    tgt = torch.from_numpy((1e-3 * rng.standard_normal((B, s.D))).astype(np.float32)).cuda()
    s.set_output_scale([1e-3] * 4)
    for _ in range(max(args.warmup, 0)):
        s.train_step(pos, mt, tgt, 1e-4, want_loss=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        s.train_step(pos, mt, tgt, 1e-4, want_loss=False)
    e1.record()
    torch.cuda.synchronize()
    sur.es_gemm_status()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    n_par = s.num_params()
    s.close()
    print(json.dumps({"metric": "ms per Adam step", "value": round(ms, 3), "unit": "ms", "higher_is_better": False,
                      "batch": B, "params": n_par, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "bf16/f32", "data": "synthetic"}))
    return 0


def measure_paper(args):
    """The paper's own workload shape: 125 x 75 x 301 cells (12.5 / 12.5 / 10 m), PML 10, a double
    couple in the reservoir box, Ricker 30 Hz, 2000 steps (--nt overrides), 105 x 55 seabed receivers
    (every interior x-y point).  No axis length has an FFT plan, so every pass is a circulant pass.
    Device time of whole es_run calls, --steps timed after --warmup."""
    import torch
    from paper_1705_04874_gb300 import es
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    shape, d, pml = (301, 75, 125), (12.5, 12.5, 10.0), 10
    nt = args.nt or 2000
    rho, cp, cs = synth.marine_model(shape=shape, seed=1)
    dt = 0.3 * min(d) / float(cp.max())
    box = synth.reservoir_box(shape, pml)
    pos = tuple((lo + hi) // 2 for lo, hi in box)
    cells = 125 * 75 * 301
    out = {}
    # the default path (every pass on the CUDA cores), then the opt-in tensor-core passes for
    # the 301-cell axis (ES_PREC_FP32_TC, outside the paper's design)
    for label, prec in (("cuda_cores", es.ES_PREC_FP32), ("tensor_cores_opt_in", es.ES_PREC_FP32_TC)):
        with es.Model(rho, cp, cs, dx=d[0], pml=pml, stream=stream) as m:
            m.set_spacing(*d)
            m.set_precision(prec)
            rcv = torch.from_numpy(m.seabed_receivers(105, 55)).cuda()
            m.source_set(pos, synth.double_couple_sdr(30, 60, 90), torch.from_numpy(synth.ricker(nt, dt, 30.0)).cuda())
            tr = torch.empty((4, rcv.shape[0], nt), device="cuda")

            def run():
                m.state_reset()
                m.run(nt, dt, rcv, tr)
            for _ in range(max(args.warmup, 0)):
                run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            out[label] = {"value": round(cells * nt / (ms * 1e-3) / 1e6, 1), "ms_per_run": round(ms, 3),
                          "kernels_ms": [round(float(k), 4) for k in m.last_step_kernel_ms()]}
    ms = out["cuda_cores"]["ms_per_run"]
    print(json.dumps({"metric": "Mcell-steps/s", "value": out["cuda_cores"]["value"],
                      "unit": "Mcell-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "s_per_source": round(ms * 1e-3, 3), "dtype": "f32",
                      "data": "synthetic",
                      "config": {"workload": "the paper's grid 125x75x301, 12.5/12.5/10 m, PML 10, "
                                             f"{nt} steps, 105x55 seabed receivers; x (125 = 5x5x5) and y (75 = 5x15) "
                                             "through the FFT passes, z (301 = 7x43) through the circulant "
                                             "passes"},
                      "paths": out}))
    return 0


def measure_configs(args):
    """Per-configuration numbers: the solver on C1 (32^3 two-layer, explosive, 300 steps, 4x4
    receivers), C2 (128^3 marine, DC 30/60/90, 2000 steps, 32x32 receivers), 96^3 / 160^3 marine
    models (1000 steps, 16x16 receivers) and the paper's own grid (125 x 75 x 301 cells, 12.5 /
    12.5 / 10 m, PML 10, 2000 steps, 105 x 55 seabed receivers = every interior x-y point),
    device time of whole es_run calls; the FP64 oracle on C1
    in full, on the first 100 steps of C2 (extrapolated) and on 2 steps of C3 with 1 core and with
    every core; and the timed comparison with
    cuFFT: one time step's 18 staggered derivatives of 256^3 fields by torch.fft R2C / C2R with the
    multiplier and a PyTorch axpy update (no PML), against the solver's six fused pass kernels."""
    import torch
    import oracle
    from paper_1705_04874_gb300 import es
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    cfgs = [("C1", (32, 32, 32), 6, 300, (4, 4), "two"), ("C2", (128, 128, 128), 10, 2000, (32, 32), "marine"),
            ("96^3", (96, 96, 96), 10, 1000, (16, 16), "marine"),
            ("160^3", (160, 160, 160), 10, 1000, (16, 16), "marine"),
            ("paper grid 125x75x301", (301, 75, 125), 10, 2000, (105, 55), "paper")]
    out = {"solver": {}}
    oracle.build()
    for name, shape, pml, nt, (rx, ry), kind in cfgs:
        d = (12.5, 12.5, 10.0) if kind == "paper" else (10.0, 10.0, 10.0)
        if kind == "two":
            rho, cp, cs = synth.two_layer_model(shape[0], water_cells=8)
            mt, pos, f0 = synth.explosive(), (16, 16, 16), 25.0
        else:
            rho, cp, cs = synth.marine_model(shape=shape, seed=1)
            box = synth.reservoir_box(shape, pml)
            mt, pos, f0 = synth.double_couple_sdr(30, 60, 90), tuple((lo + hi) // 2 for lo, hi in box), 30.0
        dt = 0.3 * min(d) / float(cp.max())
        wav = synth.ricker(nt, dt, f0)
        n = shape[0] * shape[1] * shape[2]
        with es.Model(rho, cp, cs, dx=d[0], pml=pml, stream=stream) as m:
            if kind == "paper":
                m.set_spacing(*d)
            rcv = m.seabed_receivers(rx, ry)
            m.source_set(pos, mt, torch.from_numpy(wav).cuda())
            rcv_d = torch.from_numpy(rcv).cuda()
            tr = torch.empty((4, len(rcv), nt), device="cuda")

            def run():
                m.state_reset()
                m.run(nt, dt, rcv_d, tr)
            ms = timed(run, 3)
        rec = {"grid": list(shape[::-1]), "time_steps": nt, "receivers": len(rcv), "ms_per_run": round(ms, 3),
               "Mcell_steps_per_s": round(float(n) * nt / (ms * 1e-3) / 1e6, 1)}
        if kind == "paper":
            # the paper's per-source times on this grid (2000 samples): K20 ~1313 s, C2075 ~2091 s
            rec["passes"] = "x 125 (5x5x5) and y 75 (5x15) FFT, z 301 = 7 x 43 circulant"
            rec["s_per_source"] = round(ms * 1e-3, 3)
            rec["vs_paper_k20_s_per_source"] = round(1313.0 / (ms * 1e-3), 1)
        if name == "C1":
            t0 = time.perf_counter()
            oracle.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=nt, pml=pml,
                            sources=[dict(kind="moment", pos=pos, m=mt, w=wav)], receivers=rcv)
            el = time.perf_counter() - t0
            rec["oracle_full_run_s"] = round(el, 2)
            rec["oracle_Mcell_steps_per_s"] = round(float(n) * nt / el / 1e6, 2)
            rec["oracle_cores"] = oracle.default_threads()
        if name == "C2":
            # a bounded sample: the first 100 of the 2000 steps, all cores
            k = 100
            t0 = time.perf_counter()
            oracle.simulate(rho, cp, cs, dx=10.0, dt=dt, nt=k, pml=pml,
                            sources=[dict(kind="moment", pos=pos, m=mt, w=wav[:k])], receivers=rcv)
            el = time.perf_counter() - t0
            rec["oracle_sample"] = f"first {k} of {nt} steps, timed and extrapolated per step"
            rec["oracle_Mcell_steps_per_s"] = round(float(n) * k / el / 1e6, 2)
            rec["oracle_full_run_s_extrapolated"] = round(el * nt / k, 1)
            rec["oracle_cores"] = oracle.default_threads()
        out["solver"][name] = rec
    w = workload("256")
    inp = build_inputs(w)
    v1, el1, _ = oracle_sample(w, inp, 2, nthreads=1)
    va, ela, ca = oracle_sample(w, inp, 2)
    out["oracle_C3"] = {"1_core": round(v1, 3), "all_cores": round(va, 3), "cores": ca, "unit": "Mcell-steps/s",
                        "sample": "2 time steps of the 256^3 workload"}
    # cuFFT comparison at 256^3
    n, d = 256, 10.0
    g = torch.Generator(device="cuda").manual_seed(5)
    f = torch.randn((n, n, n), device="cuda", generator=g)
    tgt = torch.zeros_like(f)
    kap = 2 * np.pi * np.arange(n // 2 + 1) / (n * d)
    mult = {sh: torch.from_numpy((1j * kap * np.exp(sh * 1j * kap * d / 2)).astype(np.complex64)).cuda()
            for sh in (1, -1)}

    def cufft_deriv(x, axis, sh):
        dim = 2 - axis  # axis 0 = x = the last array dimension
        shp = [1, 1, 1]
        shp[dim] = n // 2 + 1
        return torch.fft.irfft(torch.fft.rfft(x, dim=dim) * mult[sh].view(shp), n=n, dim=dim)

    ref = torch.empty_like(f)
    es.es_derivative(f, 0, d, 1, ref, stream=stream)
    diff = float((cufft_deriv(f, 0, 1) - ref).norm() / ref.norm())

    def cufft_step():
        for k in range(18):
            tgt.add_(cufft_deriv(f, k % 3, 1 if k % 2 else -1), alpha=1e-3)
    ms_cufft = timed(cufft_step, 5)
    rho, cp, cs = synth.marine_model(n, seed=1)
    with es.Model(rho, cp, cs, dx=d, pml=12, stream=stream) as m:
        m.source_set(inp["pos"], inp["mt"], torch.from_numpy(inp["wav"][:50]).cuda())
        m.run(50, inp["dt"])
        ks = m.last_step_kernel_ms()
    ms_ours = float(sum(ks[:6]))
    out["cufft_comparison_256"] = {"cufft_18_derivatives_ms": round(ms_cufft, 3), "fused_6_passes_ms": round(ms_ours, 3),
                                   "speedup": round(ms_cufft / ms_ours, 2), "derivative_rel_diff": float(f"{diff:.2e}"),
                                   "note": "cuFFT side: R2C, multiply, C2R, axpy per derivative, no PML, no material "
                                           "coefficients; fused side: the full velocity and stress update with PML"}
    print(json.dumps({"metric": "Mcell-steps/s", "configs": out, "n_gpus": 1, "dtype": "f32", "data": "synthetic"}))
    return 0


def surrogate_pipeline(n_loc, epochs, lr, hidden, latent, nfreq, n_src=10000, gemm=True, serve_batch=1024,
                       train_batch=256, n_rand=1000, n_held=128):
    """The surrogate workflow on the 96^3 marine model (PML 10, 8 x 8 seabed
    receivers, 1024 samples, Ricker 30 Hz): a catalog of n_loc Latin-hypercube
    locations in the reservoir box whose 6 unit-moment responses come from
    6 n_loc batched solver runs; training on the GPU; the gate; n_src random
    sources (catalog location, random double couple) served by the surrogate
    where the gate trusts the location and by the solver elsewhere, each
    checked against its exact reference.  Training takes batches of
    train_batch sources, serving batches of serve_batch: the decoder product
    reads its 2.4 GB of weights once per batch, so a wide serving batch turns
    it from HBM-bound (256) to tensor-bound (1024).  Returns (summary dict,
    decoder roofline dict or None)."""
    import torch
    from paper_1705_04874_gb300 import es, surrogate as sur
    torch.cuda.set_device(0)
    n, pml, nt, f0 = 96, 10, 1024, 30.0
    rho, cp, cs = synth.marine_model(n, seed=1)
    dt = 0.3 * 10.0 / float(cp.max())
    wav = synth.ricker(nt, dt, f0)
    box = synth.reservoir_box((n, n, n), pml)
    locations = synth.latin_hypercube_positions(synth.SplitMix64(4), box, n_loc)
    m = es.Model(rho, cp, cs, dx=10.0, pml=pml)
    rcv = m.seabed_receivers(8, 8)
    out = {"workload": f"96^3 marine, 64 receivers x 1024 samples, {n_loc} catalog locations x 6 unit moment "
                       f"tensors ({6 * n_loc} solver runs), {n_src} served sources"}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G = sur.green_catalog(m, locations, nt, dt, rcv, wav, per_batch=16)
    torch.cuda.synchronize()
    t_cat = time.perf_counter() - t0
    out["catalog_s"] = round(t_cat, 2)
    solver_rate = 6 * n_loc / t_cat  # seismogram sets per second, batched solver
    pos_n = sur.normalize_positions(locations, box)
    s = sur.Surrogate(len(rcv), nt, nfreq=nfreq, hidden=hidden, latent=latent, max_batch=serve_batch, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = sur.train(s, pos_n, G, epochs=epochs, lr=lr, batch=train_batch)
    torch.cuda.synchronize()
    out["train_s"] = round(time.perf_counter() - t0, 2)
    out["train_loss"] = [float(f"{hist[0]:.3e}"), float(f"{hist[-1]:.3e}")]
    trusted, errs = sur.calibrate_gate(s, pos_n, G, n_val=4)
    out["trusted_locations"] = round(float(trusted.mean()), 4)
    e_loc = errs.max(axis=1)
    out["gate_err_median"] = float(f"{np.median(e_loc):.3e}")
    out["gate_err_max"] = float(f"{e_loc.max():.3e}")
    rng = synth.SplitMix64(11)
    loc = np.minimum(np.floor(rng.uniform(n_src) * n_loc).astype(int), n_loc - 1)
    mts = np.array([synth.random_dc(rng) for _ in range(n_src)])
    # surrogate alone on all sources (rate of the network)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    SB = s.max_batch
    res = torch.empty((SB, 4 * len(rcv) * nt), device="cuda")
    for b in range(0, n_src, SB):
        idx = np.arange(b, min(n_src, b + SB))
        k = (len(idx) + 7) // 8 * 8
        idx = np.concatenate([idx, np.repeat(idx[:1], k - len(idx))])
        s.predict(torch.from_numpy(pos_n[loc[idx]]).cuda(), torch.from_numpy(mts[idx].astype(np.float32)).cuda(),
                  res[:k])
    torch.cuda.synchronize()
    sur_rate = n_src / (time.perf_counter() - t0)
    # served pipeline (surrogate where trusted, solver elsewhere) on all the sources, or on
    # the first 1000 when the gate sends more than 2 % of the locations to the solver
    n_pipe = n_src if trusted.mean() >= 0.98 else min(n_src, 1000)
    del res
    served = torch.empty((n_pipe, 4, len(rcv), nt), device="cuda")  # the serving buffer, reused across requests
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    served, used_solver = sur.serve(s, pos_n, trusted, loc[:n_pipe], mts[:n_pipe], m, locations, nt, dt, rcv, wav,
                                    batch_solver=32, out=served)
    torch.cuda.synchronize()
    pipe_rate = n_pipe / (time.perf_counter() - t0)
    # every served seismogram against the exact solver reference (linear combination of
    # the solver's unit responses), in chunks
    sc = G.permute(2, 0, 1, 3, 4).reshape(4, -1).pow(2).mean(dim=1).sqrt().view(1, 4, 1, 1)
    d = torch.empty(n_pipe, device="cuda")
    for b in range(0, n_pipe, 500):
        e = min(n_pipe, b + 500)
        ref = sur.combine(G, loc[b:e], mts[b:e])
        d[b:e] = ((served[b:e] - ref) / sc).reshape(e - b, -1).norm(dim=1) / (ref / sc).reshape(e - b, -1).norm(dim=1)
        del ref
    out["pipeline_sources"] = n_pipe
    # sources away from the catalog: n_held held-out cells (not catalog locations) with exact
    # solver references, the network against the two baselines, the position gate; then
    # n_rand sources at random cells of the box served with the solver as the fallback
    rng = synth.SplitMix64(21)
    cand = synth.random_positions(rng, box, 4 * n_held)
    _, dcand = sur.nearest_locations(locations, cand)
    held = cand[dcand[:, 0] > 0][:n_held]
    hmt = np.array([synth.random_dc(rng) for _ in held])
    truth = sur.solver_references(m, held, hmt, nt, dt, rcv, wav, per_batch=64)
    _, hd = sur.nearest_locations(locations, held)
    hd = hd[:, 0]
    e_net = sur.scaled_rel_l2(sur.predict_at(s, box, held, hmt), truth, sc)
    e_near = sur.scaled_rel_l2(sur.baseline_nearest(G, locations, held, hmt), truth, sc)
    e_idw = sur.scaled_rel_l2(sur.baseline_idw(G, locations, held, hmt), truth, sc)
    del truth
    d_star = sur.calibrate_position_gate(hd, e_net)
    near1 = hd <= 1.5
    out["off_catalog"] = {
        "held_out_sources": int(len(held)), "median_distance_cells": round(float(np.median(hd)), 2),
        "network_median_rel_l2": round(float(np.median(e_net)), 4),
        "nearest_location_median_rel_l2": round(float(np.median(e_near)), 4),
        "idw8_median_rel_l2": round(float(np.median(e_idw)), 4),
        "within_1.5_cells": {"n": int(near1.sum()),
                             "network": round(float(np.median(e_net[near1])), 4) if near1.any() else None,
                             "nearest": round(float(np.median(e_near[near1])), 4) if near1.any() else None},
        "network_within_5pct": round(float((e_net < 0.05).mean()), 4),
        "network_beats_nearest": round(float((e_net < e_near).mean()), 4),
        "network_beats_idw8": round(float((e_net < e_idw).mean()), 4),
        "position_gate_d_star": d_star}
    rnd = synth.random_positions(synth.SplitMix64(31), box, n_rand)
    rmt = np.array([synth.random_dc(rng) for _ in rnd])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    served_r, used_r = sur.serve_positions(s, box, trusted, d_star, locations, rnd, rmt, m, nt, dt, rcv, wav,
                                           batch_solver=64)
    torch.cuda.synchronize()
    t_r = time.perf_counter() - t0
    del served_r
    out["random_positions"] = {"sources": int(n_rand), "pipeline_seismograms_per_s": round(n_rand / t_r, 2),
                               "pipeline_solver_fraction": round(float(used_r.mean()), 4),
                               "network_fraction": round(float(1 - used_r.mean()), 4),
                               "speedup_vs_solver": round(n_rand / t_r / solver_rate, 3)}
    out.update({"solver_seismograms_per_s": round(solver_rate, 2), "surrogate_seismograms_per_s": round(sur_rate, 1),
                "pipeline_seismograms_per_s": round(pipe_rate, 1),
                "pipeline_solver_fraction": round(float(used_solver.mean()), 4),
                "served_max_rel_l2": float(f"{float(d.max()):.3e}"),
                "served_over_5pct": int((d > 0.05).sum()),
                "speedup_surrogate_vs_solver": round(sur_rate / solver_rate, 1),
                "speedup_pipeline_vs_solver": round(pipe_rate / solver_rate, 1),
                "network": {"hidden": hidden, "latent": latent, "nfreq": nfreq, "params": s.num_params(),
                            "epochs": epochs, "lr": lr, "train_batch": train_batch, "serve_batch": SB}})
    roof = None
    if gemm:
        # throughput of the network's GEMMs: tcgen05 (both operands K-major: inference decoder,
        # dZ), mma.sync (the other storage orders), and the decoder product at the served shape
        K6 = 6 * latent
        dec_name = f"tcgen05_decoder_{SB}x{s.D}x{K6}"
        g = {"tcgen05_8192": round(gemm_tflops(sur, 8192, 8192, 8192, True), 1),
             "mma_sync_8192": round(gemm_tflops(sur, 8192, 8192, 8192, False), 1),
             f"tcgen05_decoder_256x{s.D}x{K6}": round(gemm_tflops(sur, 256, s.D, K6, True), 1),
             dec_name: round(gemm_tflops(sur, SB, s.D, K6, True), 1)}
        out["gemm_tflops"] = g
        roof = decoder_roofline(g[dec_name], SB, s.D, K6)
    s.close()
    m.close()
    del G
    torch.cuda.empty_cache()
    return out, roof


def decoder_roofline(tflops, M, N, K):
    """Roofline object of the decoder product C[M][N] = A[M][K] B[N][K]^T (BF16 in, FP32 out): it
    reads its weights once (N K 2 bytes), the codes (M K 2) and writes the output (M N 4).  Below the
    bf16 ridge (measured peak flop/s over measured HBM bytes/s) HBM bounds it, above it the tensor
    cores do; the kernel is timed alone, so the burst bf16 peak applies."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    flop = 2.0 * M * N * K
    nbytes = 2.0 * N * K + 2.0 * M * K + 4.0 * M * N
    gbs = nbytes / (flop / (tflops * 1e12)) / 1e9
    tensor = flop / nbytes > peak * 1e12 / (hbm * 1e9)
    r = {"bound": "tensor" if tensor else "hbm", "kernel": f"gemm_tc_kernel (decoder product, {M} sources)",
         "achieved": round(tflops if tensor else gbs, 1), "peak": peak if tensor else hbm,
         "unit": "TFLOP/s" if tensor else "GB/s", "frac": round((tflops / peak) if tensor else (gbs / hbm), 4),
         "traffic": None, "algorithmic_bytes": nbytes, "flop": flop, "flop_per_byte": round(flop / nbytes, 1),
         "tflops": tflops, "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4), "tensor_frac": round(tflops / peak, 4),
         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    return r


def measure_surrogate(args):
    """Surrogate workload (C5): 682 catalog locations x 6 unit moment tensors
    (4092 solver runs), training, the gates, 10,000 sources at catalog
    locations and 10,000 at random cells of the reservoir box served (the
    latter mostly by the solver fallback).  Metric: seismograms/s of the served
    pipeline on the random cells."""
    out, roof = surrogate_pipeline(args.sur_locations, args.sur_epochs, args.sur_lr, args.sur_hidden,
                                   args.sur_latent, args.sur_nfreq, n_rand=args.sur_random)
    print(json.dumps({"metric": "seismograms/s", "value": out["random_positions"]["pipeline_seismograms_per_s"],
                      "unit": "4C seismogram sets/s", "n_gpus": 1, "higher_is_better": True, "dtype": "bf16/f32",
                      "data": "synthetic", "config": {"workload": out["workload"]}, "roofline": roof,
                      "surrogate": out}))
    return 0


def e2e(es, w, inp, stream):
    """Same metric through the C ABI with host buffers: model creation from
    host arrays, source from host memory, traces and gather back to host
    memory, every step (host<->device copies inside the timed region)."""
    import torch
    n, nt = w["n"], w["nt"]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    rho, cp, cs = pin(inp["rho"]), pin(inp["cp"]), pin(inp["cs"])
    wav = pin(inp["wav"])
    ev = [pin(a) for a in inp["ev"]]
    host_tr = None
    rcv_host = None

    def step():
        nonlocal host_tr, rcv_host
        m = es.Model(rho, cp, cs, dx=10.0, pml=w["pml"], stream=stream)
        if rcv_host is None:
            rcv_host = pin(m.seabed_receivers(w["rx"], w["rx"]))
            host_tr = torch.empty((1, 4, rcv_host.shape[0], nt)).pin_memory()
        m.source_set(inp["pos"], inp["mt"], wav)
        m.run(nt, inp["dt"], rcv_host, host_tr[0])
        g = es.es_superpose(host_tr, ev[0], ev[1], ev[2], inp["dt"], inp["n_out"], stream=stream)
        m.close()
        return g

    step()
    torch.cuda.synchronize()
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        g = step()
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / reps
    n_rcv = rcv_host.shape[0]
    h2d = 3 * 4 * n ** 3 + 4 * nt + 12 * n_rcv + host_tr.numel() * 4 + 300 * 12
    d2h = host_tr.numel() * 4 + g.size * 4
    return {"value": float(n) ** 3 * nt / el / 1e6, "unit": "Mcell-steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * el}


if __name__ == "__main__":
    sys.exit(main())
