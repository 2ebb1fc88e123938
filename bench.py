#!/usr/bin/env python3
"""Throughput of batched (ab|cd) evaluation on GB300: (ii|ii) quartets/s.

Default workload: 4096 (ii|ii) shell quartets (all l = 6, K = 1), centers uniform in a
20-bohr cube, exponents log-uniform in [0.05, 20], real solid-harmonic output (13^4 per
quartet); the Cartesian output (28^4) of the same batch is timed beside it.  One step is
one lx_eri_batch call over the whole batch: normalisation, pair/H build, Boys + [r]^(0),
GEMM1 and GEMM2 (every row of the hot path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU under torchrun, each evaluating its own replica of the
batch (quartets are independent: weak scaling, no data-path collective); the timing is
the max over ranks.  Rank 0 prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "(ii|ii) quartets/s & FP64-equiv TFLOP/s; split vs FP64 path at ≤1e-10 max err"
UNIT = "quartets/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--nquartet", type=int, default=4096)
    p.add_argument("--no-cart", action="store_true", help="skip the Cartesian-output measurement")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-split", action="store_true", help="skip the split-precision measurement")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-class graph measurement")
    p.add_argument("--mixed-quartets", type=int, default=200_000,
                   help="quartets of the mixed-class workload (one graph launch on the split path)")
    p.add_argument("--mixed-fp64-sample", type=int, default=2000,
                   help="leading quartets of the mixed workload timed on the FP64 path")
    p.add_argument("--no-split-config", action="store_true",
                   help="skip the (hh|hh)+(ii|ii) K=1..3 split-path workload")
    p.add_argument("--no-routed", action="store_true", help="skip the routed-workload sample")
    p.add_argument("--no-pairs", action="store_true", help="skip the bra-list x ket-list (engine form) workload")
    p.add_argument("--pairs", type=int, default=64, help="bra pairs = ket pairs of the engine-form and J/K workloads")
    p.add_argument("--routed-quartets", type=int, default=200_000)
    p.add_argument("--routed-fp64-sample", type=int, default=4000,
                   help="leading quartets of the routed workload timed on the FP64 path")
    p.add_argument("--no-sweep-rows", action="store_true", help="skip the small class x K table")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    p.add_argument("--sweep", action="store_true",
                   help="instead of the benchmark line: one JSON line per integral class (dd|dd)..(kk|kk) "
                        "and total contraction degree 1, 5, 25, both paths, with per-stage shares")
    return p.parse_args(argv)


# ------------------------------------------------------------------ model of the work

def pyr(n):
    return (n + 1) * (n + 2) * (n + 3) // 6


def nfun(l, solid):
    return 2 * l + 1 if solid else (l + 1) * (l + 2) // 2


# DRAM bytes per quartet of one launch, from single ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum) of these kernels on 256 solid (ii|ii) K = 1 quartets; a launch's
# traffic grows with its quartet count.  Each figure holds for that workload and for the
# kernel source it was captured on, named with its sha256: once that file changes, the
# traffic is reported as unknown (null) until it is captured again.
NCU_TRAFFIC = {
    "gemm1": (311.383296e6 / 256, "paper_2307_03452_gb300/csrc/lx_gemm.cu",
              "2e31e62d4b0eb5d2d87ec27d9d5e2bf675e0e8eec6d9707d1c2f2df1cb75f841"),
    "split_gemm1": ((957.045504e6 + 145.702656e6) / 256, "paper_2307_03452_gb300/csrc/lx_split.cu",
                    "559aa480485e877e1e889fde8c826245b58238bb6559e839d3fb8fb2230d99a4"),
}


def ncu_traffic(kernel, nquartet):
    """DRAM bytes of one launch of `kernel` over nquartet (ii|ii) quartets, or None when its
    source has changed since the capture."""
    import hashlib
    per, path, sha = NCU_TRAFFIC[kernel]
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != sha:
                return None
    except OSError:
        return None
    return per * nquartet


def gemm_flops(basis, quartets, solid):
    """Algorithmic FLOPs of the two transforms (paper, Eq. make-abq and Eq. make-abcd):
    2 N_ab (K_bra N_p)(K_ket N_q) and 2 N_ab (K_ket N_q) N_cd per quartet."""
    import numpy as np
    l, K = np.asarray(basis["l"]), np.asarray(basis["nprim"])
    q = np.asarray(quartets)
    la, lb, lc, ld = (l[q[:, i]] for i in range(4))
    kbra = K[q[:, 0]] * K[q[:, 1]]
    kket = K[q[:, 2]] * K[q[:, 3]]
    f = (lambda x: 2 * x + 1) if solid else (lambda x: (x + 1) * (x + 2) // 2)
    nab, ncd = f(la) * f(lb), f(lc) * f(ld)
    npp = (la + lb + 1) * (la + lb + 2) * (la + lb + 3) // 6
    nq = (lc + ld + 1) * (lc + ld + 2) * (lc + ld + 3) // 6
    g1 = 2.0 * nab * (kbra * npp) * (kket * nq)
    g2 = 2.0 * nab * (kket * nq) * ncd
    return float(g1.sum()), float(g2.sum()), float((nab * ncd).sum())


# ------------------------------------------------------------------ distributed

def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("LX_BENCH_BACKEND", "nccl")
        dist.init_process_group(backend=backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(value: float, world: int) -> float:
    """Max of a float over ranks (timing only; no data-path collective)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=5)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ measurements

def fp64_peak_tflops(torch):
    """cuBLAS DGEMM 4096^3, best of 5 (a measured FP64 rate of this GPU)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def time_steps(torch, lx, batch, out, ws, steps, warmup, flush_buf, world):
    """Warm up, then time exactly `steps` calls with per-step CUDA events on the launching
    stream (L2 flushed before each step, outside the events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        batch.run(out, ws, stream)
    lx.sync_status(stream)
    lx.stage_times(stream)  # clear
    evs = []
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(steps):
        flush_buf.add_(1)  # write > L2 between timed steps
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        batch.run(out, ws, stream, time_stages=True)
        e.record(stream)
        evs.append((s, e))
    torch.cuda.synchronize()
    barrier(world)
    lx.sync_status(stream)
    step_ms = [s.elapsed_time(e) for s, e in evs]
    stage_ms, launches = lx.stage_times(stream)
    return step_ms, stage_ms, launches


def _bf16_peak_and_source():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"  # fallback figure for a GB300 when the measured file is absent


# nominal dense rates of a GB300 (TFLOP/s): the FP64 peak is the measured BF16 peak scaled by
# their ratio (no FP64 figure is measured for the pool)
NOMINAL_FP64_TFLOPS, NOMINAL_BF16_TFLOPS = 1.25, 2250.0


def cpu_baseline(basis, quartets, solid, seconds):
    """The oracle as it stands, on the host cores, on a bounded prefix of the workload."""
    import numpy as np

    import oracle
    from paper_2307_03452_gb300 import inputs
    oracle.build()
    cores = oracle.max_threads()
    chunk = max(1, cores)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < len(quartets):
        idx = np.arange(done, min(done + chunk, len(quartets)))
        sb, sq = inputs.subset(basis, quartets, idx)
        oracle.eri(sb, sq, solid=solid)
        done += len(idx)
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of the {len(quartets)} quartets, {'solid' if solid else 'Cartesian'} output, "
                      f"{dt:.1f} s of CPU work (plain McMurchie-Davidson in C, FP64, OpenMP)"}


def workload_name(nq):
    """The headline workload, as both arms name it in their config."""
    return (f"(ii|ii) K=1 x{nq} quartets, 20-bohr cube, exponents log-uniform [0.05, 20], "
            "real solid-harmonic output (13^4 per quartet); Cartesian (28^4) beside")


# ------------------------------------------------------------------ oracle samples

CLASS_LETTERS = "spdfghik"


def class_name(basis, q):
    l = basis["l"]
    a, b, c, d = (CLASS_LETTERS[int(l[s])] for s in q)
    return f"({a}{b}|{c}{d})"


def oracle_seconds(basis, q):
    """Rough single-core cost of one quartet in the oracle: proportional to its primitive
    quartets times the Cartesian size of its first transform (about 0.2 s for one (ii|ii)
    primitive quartet)."""
    l, K = basis["l"], basis["nprim"]
    la, lb, lc, ld = (int(l[s]) for s in q)
    nc = lambda x: (x + 1) * (x + 2) // 2  # noqa: E731
    work = pyr(la + lb) * pyr(lc + ld) * nc(la) * nc(lb)
    for s in q:
        work *= int(K[s])
    return 0.2 * work / (455 * 455 * 784)


def pick_sample(basis, quartets, per_class=2, cheap_s=2.0, heavy_s=0.0, limit=None):
    """Indices of a small per-class sample: the first `per_class` quartets of each class whose
    oracle cost is at most cheap_s, plus (heavy_s > 0) the one with the most primitive quartets
    whose cost is at most heavy_s."""
    n = len(quartets) if limit is None else min(limit, len(quartets))
    K = basis["nprim"]
    cheap, heavy = {}, {}
    for i in range(n):
        q = quartets[i]
        c = class_name(basis, q)
        cost = oracle_seconds(basis, q)
        if cost <= cheap_s and len(cheap.setdefault(c, [])) < per_class:
            cheap[c].append(i)
        elif heavy_s > 0 and cost <= heavy_s:
            kp = int(np.prod([K[x] for x in q]))
            if c not in heavy or kp > heavy[c][0]:
                heavy[c] = (kp, i)
    idx = [i for v in cheap.values() for i in v] + [v[1] for v in heavy.values()]
    return sorted(set(idx))


def gather_blocks(out, offsets, sizes, idx):
    """Host copy of the output blocks of quartets idx (concatenated)."""
    return np.concatenate([out[int(offsets[i]):int(offsets[i]) + int(sizes[i])].cpu().numpy() for i in idx])


class OracleChecks:
    """GPU results kept for a seeded sample of each workload, compared with the CPU oracle
    after every GPU leg (rank 0, one process): per class, the largest |error| of each path and
    the largest |integral|."""

    def __init__(self):
        self.items = []  # (target dict, key, sample basis, sample quartets, {path: host blocks})

    def add(self, target, key, basis, quartets, idx, results):
        sb, sq = inputs_subset(basis, quartets, idx)
        self.items.append((target, key, sb, sq, results))

    def run(self):
        import oracle
        from paper_2307_03452_gb300 import inputs
        if not self.items:
            return 0.0
        oracle.build()
        t0 = time.perf_counter()
        basis, quartets = inputs.concat([(sb, sq) for _, _, sb, sq, _ in self.items])
        ref, off = oracle.eri(basis, quartets, solid=True)
        pos = 0
        for target, key, sb, sq, results in self.items:
            nq = len(sq)
            sizes = [int(np.prod([2 * int(sb["l"][x]) + 1 for x in q])) for q in sq]
            start = int(off[pos])
            per = {}
            o = 0
            for j, q in enumerate(sq):
                c = class_name(sb, q)
                r = ref[start + o:start + o + sizes[j]]
                e = per.setdefault(c, {"n": 0, "max_abs_integral": 0.0})
                e["n"] += 1
                e["max_abs_integral"] = max(e["max_abs_integral"], float(np.abs(r).max()))
                for path, got in results.items():
                    k = f"max_abs_err_{path}"
                    e[k] = max(e.get(k, 0.0), float(np.abs(got[o:o + sizes[j]] - r).max()))
                o += sizes[j]
            for e in per.values():
                if "max_abs_err_fp64" in e and e["max_abs_integral"] > 0:
                    e["rel_err_fp64"] = e["max_abs_err_fp64"] / e["max_abs_integral"]
            target[key] = per
            pos += nq
        return time.perf_counter() - t0


def inputs_subset(basis, quartets, idx):
    from paper_2307_03452_gb300 import inputs
    return inputs.subset(basis, quartets, idx)


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload and metric (bounded samples)."""
    import numpy as np

    import oracle
    from paper_2307_03452_gb300 import inputs
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    basis, quartets = inputs.iiii_fp64(args.nquartet)
    oracle.build()
    cores = oracle.max_threads()
    per_step = max(1, cores)  # quartets per step: one per thread
    times = []
    for k in range(args.warmup + args.steps):
        idx = np.arange(k * per_step, (k + 1) * per_step) % len(quartets)
        sb, sq = inputs.subset(basis, quartets, idx)
        t0 = time.perf_counter()
        oracle.eri(sb, sq, solid=True)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.nquartet),
                       "path": "CPU oracle (plain FP64 McMurchie-Davidson in C, OpenMP); each step a sample of "
                               f"{per_step} quartets of the workload, solid output",
                       "parallelism": f"{cores} host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} quartets per step, {args.steps} timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


SWEEP_CLASSES = [(2, 2, 2, 2), (3, 3, 3, 3), (4, 4, 4, 4), (5, 5, 5, 5), (6, 6, 6, 6), (7, 7, 7, 7)]
# total contraction degree K_bra K_ket -> per-shell degrees (a, b, c, d)
SWEEP_K = {1: (1, 1, 1, 1), 5: (5, 1, 1, 1), 25: (5, 1, 5, 1)}


def run_sweep(args):
    """Per class and total contraction degree: quartets/s, FP64-equivalent TFLOP/s and the
    share of each stage, on both paths (the paper's class x K table and stage breakdown)."""
    import torch

    from paper_2307_03452_gb300 import inputs, lx
    torch.cuda.set_device(0)
    lx.load(build_if_missing=True)
    flush_buf = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    names = "spdfghik"
    for cls in SWEEP_CLASSES:
        for ktot, ks in SWEEP_K.items():
            la, lb, lc, ld = cls
            # about 0.25 s of FP64-path GEMM work at 1 TFLOP/s, between 64 and 65536 quartets
            b1, q1 = inputs.class_sweep(cls, 1, ks, 1)
            g1, g2, _ = gemm_flops(b1, q1, True)
            nq = int(min(65536, max(64, 0.25e12 / (g1 + g2))))
            basis, quartets = inputs.class_sweep(cls, nq, ks, 4100 + 10 * la + ktot)
            g1, g2, nint = gemm_flops(basis, quartets, True)
            line = {"class": "(" + names[la] + names[lb] + "|" + names[lc] + names[ld] + ")", "K_total": ktot,
                    "K_per_shell": list(ks), "nquartet": nq, "solid": True}
            ref = None
            for path in ("fp64", "split"):
                b = lx.Batch(basis, quartets, solid=True, path=path)
                out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
                ws = lx.alloc_workspace(max(b.workspace_min(), min(b.workspace_size(), 64 << 30)))
                ms, stage, _ = time_steps(torch, lx, b, out, ws, 3, 2, flush_buf, 1)
                t = sum(ms) / len(ms)
                tot = sum(stage.values())
                line[path] = {"quartets_per_s": nq / (t * 1e-3), "integrals_per_s": nint / (t * 1e-3),
                              "ms_per_step": t, "fp64_equiv_tflops": (g1 + g2) / (t * 1e-3) / 1e12,
                              "stage_share": {k: v / tot for k, v in stage.items() if v > 0}}
                if path == "fp64":
                    ref = out.clone()
                else:
                    line[path]["max_abs_diff_vs_fp64_path"] = float((out - ref).abs().max())
                del b, out, ws
                torch.cuda.empty_cache()
            print(json.dumps(line), flush=True)
    return 0


def _graph_time_ms(torch, g, flush_buf):
    """Device time of one replay of a captured batch (L2 written before it, outside the events)."""
    flush_buf.add_(1)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    g.launch()
    s1.record()
    torch.cuda.synchronize()
    return s0.elapsed_time(s1)


def run_mixed(args, torch, lx, inputs, flush_buf, world, checks):
    """Mixed classes (gg|gg), (hh|hh), (ii|ii), (gh|ii), (gi|hh) with K = 1..5 per shell: the
    whole batch as one CUDA graph on the split path; the FP64 path (tiles autotuned per class
    and K) on the leading quartets of the same batch, also as a graph."""
    nq = args.mixed_quartets
    mb, mq = inputs.mixed_fp64(nquartet=nq, seed=2309)
    g1, g2, nint = gemm_flops(mb, mq, True)
    ns = min(args.mixed_fp64_sample, nq)
    sb, sq = inputs.subset(mb, mq, np.arange(ns))
    sg1, sg2, _ = gemm_flops(sb, sq, True)
    res = {"workload": f"{nq} quartets drawn uniformly over (gg|gg),(hh|hh),(ii|ii),(gh|ii),(gi|hh), K = 1..5 "
                       "per shell, exponents log-uniform [0.05, 50], raw coefficients uniform (0, 1], 20-bohr cube, "
                       "solid harmonics",
           "fp64_equiv_gflop_per_step": (g1 + g2) / 1e9}
    ws_cap = 64 << 30
    # split path, whole batch: warm up on the leading sample (same kernels), then one replay
    bw = lx.Batch(sb, sq, True, path="split")
    b = lx.Batch(mb, mq, True, path="split")
    ws = lx.alloc_workspace(max(b.workspace_min(), min(b.workspace_size(), ws_cap)))
    outw = torch.empty(bw.out_size, dtype=torch.float64, device="cuda")
    gw = lx.Graph(bw, outw, ws)
    gw.launch()
    torch.cuda.synchronize()
    gw.close()
    del outw
    out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    g = lx.Graph(b, out, ws)
    create_s = time.perf_counter() - t0
    ms = reduce_max(_graph_time_ms(torch, g, flush_buf), world)
    lx.sync_status()
    g.close()
    res["split"] = {"quartets_per_s": world * nq / (ms * 1e-3), "ms_per_step": ms, "steps": 1,
                    "fp64_equiv_tflops": world * (g1 + g2) / (ms * 1e-3) / 1e12,
                    "integrals_per_s": world * nint / (ms * 1e-3), "graph_launches_per_step": 1,
                    "graph_create_s": create_s,
                    "timing": "one replay of the whole batch captured as one CUDA graph, after a warm-up replay "
                              "of its leading sample"}
    # FP64 path on the leading sample: tiles tuned per (class, K), captured, warm-up + timed replay
    t0 = time.perf_counter()
    rows = lx.autotune(lx.Batch(sb, sq, True), max_keys=24, samples=4)
    res["autotune_s"] = time.perf_counter() - t0
    res["tuned_keys"] = int(len(rows))
    bf = lx.Batch(sb, sq, True)
    outf = torch.empty(bf.out_size, dtype=torch.float64, device="cuda")
    del ws
    torch.cuda.empty_cache()
    wsf = lx.alloc_workspace(max(bf.workspace_min(), min(bf.workspace_size(), ws_cap)))
    gf = lx.Graph(bf, outf, wsf)
    gf.launch()
    torch.cuda.synchronize()
    fms = reduce_max(_graph_time_ms(torch, gf, flush_buf), world)
    lx.sync_status()
    gf.close()
    res["fp64"] = {"quartets_per_s": world * ns / (fms * 1e-3), "ms_per_step": fms, "steps": 1,
                   "sample_quartets": ns, "fp64_equiv_tflops": world * (sg1 + sg2) / (fms * 1e-3) / 1e12,
                   "graph_launches_per_step": 1,
                   "timing": f"one replay of the leading {ns} quartets captured as one CUDA graph, after a "
                             "warm-up replay"}
    res["split_speedup_vs_fp64"] = res["split"]["quartets_per_s"] / res["fp64"]["quartets_per_s"]
    nout = int(bf.out_size)  # the sample's blocks lead the whole batch's output
    res["split_max_abs_diff_vs_fp64_on_sample"] = float((out[:nout] - outf).abs().max())
    oidx = pick_sample(sb, sq, per_class=2, cheap_s=2.0, heavy_s=15.0)
    offs, sizes = bf.quartets["out_offset"], bf.sizes
    checks.add(res, "oracle_err_per_class", sb, sq, oidx,
               {"split": gather_blocks(out, offs, sizes, oidx), "fp64": gather_blocks(outf, offs, sizes, oidx)})
    del out, outf, wsf
    torch.cuda.empty_cache()
    return res


def run_routed(args, torch, lx, inputs, world, checks):
    """The routed workload (l = 4..6, K = 1..5, bra-ket separations 0..30 bohr): one routed
    library call over the whole batch, the split path alone on the same batch, and the FP64
    path alone on its leading quartets; the error of each against the FP64 path there."""
    from paper_2307_03452_gb300 import router as rtr
    if not os.path.exists(rtr.WEIGHTS):
        return None
    r = rtr.Router.load()
    nq = args.routed_quartets
    rb, rq = inputs.routed(nquartet=nq, seed=2311 + 7)
    g1, g2, _ = gemm_flops(rb, rq, True)
    ns = min(args.routed_fp64_sample, nq)
    sb, sq = inputs.subset(rb, rq, np.arange(ns))
    ws_limit = 32 << 30
    # warm-up of both arms on the leading sample
    rtr.routed_eri(sb, sq, r, return_tiers=False, workspace_limit=ws_limit)
    lx.eri(sb, sq, solid=True, path="split", workspace_limit=ws_limit)
    torch.cuda.synchronize()
    barrier(world)
    # the FP64 arm first: its sample's blocks lead the batch's output, so each other arm keeps
    # only that leading part once timed and the whole batch's output is held once at a time
    t0 = time.perf_counter()
    fout, foff = lx.eri(sb, sq, solid=True, path="fp64", workspace_limit=ws_limit)
    torch.cuda.synchronize()
    t_fp64 = reduce_max(time.perf_counter() - t0, world)
    nout = fout.numel()
    t0 = time.perf_counter()
    rout, roff = rtr.routed_eri(rb, rq, r, return_tiers=False, workspace_limit=ws_limit)  # one library call
    torch.cuda.synchronize()
    t_routed = reduce_max(time.perf_counter() - t0, world)
    rout = rout[:nout].clone()
    torch.cuda.empty_cache()
    dest = r.tiers(lx.route_features(rb, rq), rb, rq)  # destination per quartet, for the report only
    t0 = time.perf_counter()
    sout, _ = lx.eri(rb, rq, solid=True, path="split", workspace_limit=ws_limit)
    torch.cuda.synchronize()
    t_split = reduce_max(time.perf_counter() - t0, world)
    sout = sout[:nout].clone()
    torch.cuda.empty_cache()
    res = {"workload": f"{nq} quartets, l = 4..6 and K = 1..5 per shell, pair centers within 3 bohr, bra-ket "
                       "separations 0..30 bohr, exponents log-uniform [0.05, 50], solid harmonics",
           "fp64_equiv_gflop_per_step": (g1 + g2) / 1e9,
           "routed_quartets_per_s": world * nq / t_routed, "split_only_quartets_per_s": world * nq / t_split,
           "fp64_only_quartets_per_s": world * ns / t_fp64, "fp64_only_sample_quartets": ns,
           "routed_fp64_equiv_tflops": world * (g1 + g2) / t_routed / 1e12,
           "speedup_vs_fp64": (nq / t_routed) / (ns / t_fp64),
           "routed_vs_split_only": t_split / t_routed,
           "tier_fraction": {("fp64" if d == 0 else f"split{d}"): float((dest == d).mean()) for d in (0, 4, 5, 6)},
           "digit_products_per_quartet": float(sum((dest == d).mean() * d * (d + 1) / 2 for d in (4, 5, 6))),
           "routed_max_abs_err_vs_fp64_on_sample": float((rout - fout).abs().max()),
           "split_only_max_abs_err_vs_fp64_on_sample": float((sout - fout).abs().max()),
           "tau": r.tau, "router_val_rmse_log10": r.meta.get("val_rmse_log10"),
           "baseline_rmse_log10": r.meta.get("baseline_rmse_log10"),
           "timing": "wall clock of one library call per arm (routed: features, MLP inference, host planning of "
                     "both sub-batches, kernels; split and FP64: host planning and kernels)"}
    b = lx.Batch(sb, sq, True)
    oidx = pick_sample(sb, sq, per_class=1, cheap_s=1.5, limit=ns)[:24]
    checks.add(res, "oracle_err_per_class", sb, sq, oidx,
               {"routed": gather_blocks(rout, b.quartets["out_offset"], b.sizes, oidx),
                "split": gather_blocks(sout, b.quartets["out_offset"], b.sizes, oidx),
                "fp64": gather_blocks(fout, b.quartets["out_offset"], b.sizes, oidx)})
    del rout, sout, fout
    torch.cuda.empty_cache()
    return res


# the small class x K table of the default run: class, total contraction degree
SWEEP_ROWS = [((2, 2, 2, 2), 1), ((2, 2, 2, 2), 25), ((3, 3, 3, 3), 1), ((3, 3, 3, 3), 25), ((6, 6, 6, 6), 1),
              ((6, 6, 6, 6), 25)]


def run_sweep_rows(torch, lx, inputs, flush_buf, checks):
    """Per row (class, total contraction degree): quartets/s, FP64-equivalent TFLOP/s and the
    share of each stage on both paths, about 0.1 s of FP64 work per step, 3 timed steps."""
    rows = []
    for cls, ktot in SWEEP_ROWS:
        ks = SWEEP_K[ktot]
        b1, q1 = inputs.class_sweep(cls, 1, ks, 1)
        f1, f2, _ = gemm_flops(b1, q1, True)
        nq = int(min(65536, max(64, 0.1e12 / (f1 + f2))))
        la = cls[0]
        basis, quartets = inputs.class_sweep(cls, nq, ks, 4100 + 10 * la + ktot)
        g1, g2, nint = gemm_flops(basis, quartets, True)
        row = {"class": class_name(basis, quartets[0]), "K_total": ktot, "K_per_shell": list(ks), "nquartet": nq}
        kept = {}
        oidx = [0, nq - 1]
        for path in ("fp64", "split"):
            b = lx.Batch(basis, quartets, True, path=path)
            out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
            ws = lx.alloc_workspace(max(b.workspace_min(), min(b.workspace_size(), 32 << 30)))
            ms, stage, _ = time_steps(torch, lx, b, out, ws, 3, 1, flush_buf, 1)
            t = sum(ms) / len(ms)
            tot = sum(stage.values())
            row[path] = {"quartets_per_s": nq / (t * 1e-3), "ms_per_step": t,
                         "fp64_equiv_tflops": (g1 + g2) / (t * 1e-3) / 1e12,
                         "stage_share": {k: round(v / tot, 4) for k, v in stage.items() if v > 0}}
            kept[path] = gather_blocks(out, b.quartets["out_offset"], b.sizes, oidx)
            if path == "fp64":
                ref = out
            else:
                row["split"]["max_abs_diff_vs_fp64_path"] = float((out - ref).abs().max())
                row["split_speedup"] = row["fp64"]["ms_per_step"] / t
            del ws
        del out, ref
        torch.cuda.empty_cache()
        checks.add(row, "oracle_err", basis, quartets, oidx, kept)
        rows.append(row)
    return rows


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    import numpy as np
    import torch

    from paper_2307_03452_gb300 import inputs, lx

    rank, local, world = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    lx.load(build_if_missing=True)
    basis, quartets = inputs.iiii_fp64(args.nquartet)
    nq = len(quartets)
    default_workload = True  # solid (ii|ii) K = 1 at any count: the class NCU_TRAFFIC was taken on

    checks = OracleChecks()
    peak64 = fp64_peak_tflops(torch)
    flush_buf = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # ---- solid-harmonic output: the headline
    b = lx.Batch(basis, quartets, solid=True)
    out = torch.empty(b.out_size, dtype=torch.float64, device="cuda")
    ws = lx.alloc_workspace(b.workspace_size())
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if \
        os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    sampler = ClockSampler(gpu_index)
    sampler.start()
    step_ms, stage_ms, launches = time_steps(torch, lx, b, out, ws, args.steps, args.warmup, flush_buf, world)
    clocks = sampler.stop()
    total_ms = reduce_max(sum(step_ms), world)
    value = world * nq * args.steps / (total_ms * 1e-3)
    g1, g2, nint = gemm_flops(basis, quartets, True)
    fp64_tf = world * (g1 + g2) * args.steps / (total_ms * 1e-3) / 1e12
    dominant = max(("gemm1", "gemm2", "pair_h", "boys_r"), key=lambda s: stage_ms[s])
    dom_flops = {"gemm1": g1, "gemm2": g2}.get(dominant)
    per_launch_ms = stage_ms[dominant] / max(1, launches[dominant])
    # the FP64 GEMMs are contractions on the FP64 mma.sync path.  Their peak: the measured BF16
    # tensor peak times the nominal FP64 / BF16 ratio, or the FP64 rate cuBLAS DGEMM reaches in
    # this run if that is higher (a measured rate is a lower bound of the true peak, so the
    # fraction cannot pass 1 on a figure the chip was seen to beat)
    bf16_peak, bf16_src = _bf16_peak_and_source()
    fp64_derived = bf16_peak * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
    fp64_peak = max(fp64_derived, peak64)
    roofline = {"bound": "tensor", "kernel": dominant, "unit": "TFLOP/s",
                "achieved": (dom_flops / (per_launch_ms * 1e-3) / 1e12) if dom_flops else None,
                "peak": fp64_peak,
                "peak_source": f"max of MEASURED_PEAKS.json bf16_tflops x nominal FP64/BF16 dense ratio "
                               f"({NOMINAL_FP64_TFLOPS} / {NOMINAL_BF16_TFLOPS} TFLOP/s) = {fp64_derived:.4f} "
                               f"(of {bf16_src}) and cuBLAS DGEMM 4096^3 measured in this run = {peak64:.4f}",
                "cublas_dgemm_tflops": peak64, "dtype": "f64",
                "traffic": (ncu_traffic("gemm1", nq) if dominant == "gemm1" and default_workload else None),
                "traffic_source": "ncu capture on 256 quartets scaled by quartet count; null if the kernel source "
                                  "changed since"}
    roofline["frac"] = roofline["achieved"] / fp64_peak if roofline["achieved"] else None
    roofline["frac_of_cublas_dgemm"] = roofline["achieved"] / peak64 if roofline["achieved"] else None
    roofline["frac_le_1"] = bool(roofline["frac"] is not None and roofline["frac"] <= 1.0)
    del ws
    torch.cuda.empty_cache()

    # ---- split-precision path on the same batch (BF16 slices on the tensor cores)
    split = None
    if not args.no_split:
        bsp = lx.Batch(basis, quartets, solid=True, path="split")
        outs = torch.empty(bsp.out_size, dtype=torch.float64, device="cuda")
        wss = lx.alloc_workspace(bsp.workspace_size())
        sms, sstage, slaunch = time_steps(torch, lx, bsp, outs, wss, args.steps, args.warmup, flush_buf, world)
        stot = reduce_max(sum(sms), world)
        maxdiff = float((outs - out).abs().max())
        # roofline of the dominant tensor-core kernel of the split path
        sdom = max(("gemm1", "gemm2"), key=lambda k: sstage[k])
        # tensor work asked of the tensor cores: 21 digit products of the useful sizes
        tens = {"gemm1": 21 * g1, "gemm2": 21 * g2}.get(sdom)
        sper = sstage[sdom] / max(1, slaunch[sdom])
        sroof = {"bound": "tensor", "kernel": f"split_{sdom}", "unit": "TFLOP/s",
                 "achieved": (tens / (sper * 1e-3) / 1e12) if tens else None, "peak": bf16_peak,
                 "peak_source": f"MEASURED_PEAKS.json bf16_tflops (burst), of {bf16_src}",
                 "traffic": (ncu_traffic("split_gemm1", nq) if sdom == "gemm1" and default_workload else None),
                 "traffic_source": "ncu capture on 256 quartets scaled by quartet count; null if the kernel source "
                                   "changed since"}
        sroof["frac"] = sroof["achieved"] / bf16_peak if sroof["achieved"] and bf16_peak else None
        split = {"quartets_per_s": world * nq * args.steps / (stot * 1e-3), "ms_per_step": stot / args.steps,
                 "fp64_equiv_tflops": world * (g1 + g2) * args.steps / (stot * 1e-3) / 1e12,
                 "max_abs_diff_vs_fp64_path": maxdiff, "speedup_vs_fp64_path": (total_ms / stot),
                 "stage_ms_per_step": {k: v / args.steps for k, v in sstage.items()},
                 "gpu_launches": int(sum(slaunch.values())), "roofline": sroof,
                 "scheme": "6 BF16 digits of 8 bits per FP64 value, per-row powers of two, H columns scaled "
                           "into (-1, 1) by powers of two folded into the other operand, 21 digit products, "
                           "int64 recombination"}
        del wss, outs
        torch.cuda.empty_cache()

    # ---- end to end through the public API: pinned host descriptors in, result out to pinned host
    e2e = None
    if not args.no_e2e:
        be = lx.Batch(basis, quartets, solid=True)
        be.pin()
        ws = lx.alloc_workspace(be.workspace_size())
        # two device outputs: the result of step i is copied to the host on a second stream
        # while step i + 1 computes into the other buffer (step i + 2 waits for that copy)
        dev_outs = [torch.empty(be.out_size, dtype=torch.float64, device="cuda") for _ in range(2)]
        host_out = torch.empty(be.out_size, dtype=torch.float64, pin_memory=True)
        stream = torch.cuda.current_stream()
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_step(i):
            o = dev_outs[i % 2]
            if i >= 2:
                stream.wait_event(copied[i % 2])
            be.run(o, ws, stream)  # descriptors from pinned host memory, uploaded in the call
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                host_out.copy_(o, non_blocking=True)
            copied[i % 2].record(copy_stream)

        for i in range(args.warmup):
            e2e_step(i)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for i in range(args.steps):
            e2e_step(i)
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, world)
        barrier(world)
        lx.sync_status(stream)
        h2d = be.host_bytes()
        e2e = {"value": world * nq * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": be.out_size * 8,
               "note": "wall clock per step: host planning, descriptor upload from pinned memory, kernels, "
                       "result copy to pinned host memory (on a second stream, overlapping the next "
                       "step's kernels; two device output buffers)"}
        del ws, dev_outs, host_out
        torch.cuda.empty_cache()

    # ---- Cartesian output of the same batch
    cart = None
    if not args.no_cart:
        bc = lx.Batch(basis, quartets, solid=False)
        outc = torch.empty(bc.out_size, dtype=torch.float64, device="cuda")
        wsc = lx.alloc_workspace(bc.workspace_size())
        csteps = max(1, min(args.steps, 5))
        cms, cstage, _ = time_steps(torch, lx, bc, outc, wsc, csteps, 1, flush_buf, world)
        ctot = reduce_max(sum(cms), world)
        cg1, cg2, _ = gemm_flops(basis, quartets, False)
        cart = {"quartets_per_s": world * nq * csteps / (ctot * 1e-3), "ms_per_step": ctot / csteps,
                "fp64_tflops": world * (cg1 + cg2) * csteps / (ctot * 1e-3) / 1e12, "steps": csteps,
                "stage_ms_per_step": {k: v / csteps for k, v in cstage.items()}}
        del wsc, outc
        torch.cuda.empty_cache()

    # ---- mixed classes, K = 1..5: the whole batch as one CUDA graph (split path), autotuned FP64
    # tiles on a leading sample of it
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, torch, lx, inputs, flush_buf, world, checks)

    # ---- split path at full size: 16384 (hh|hh) + 16384 (ii|ii), K = 1..3 per shell
    split_cfg = None
    if not args.no_split_config:
        sb_, sq_ = inputs.split_hhhh_iiii()
        sg1, sg2, _ = gemm_flops(sb_, sq_, True)
        bsc = lx.Batch(sb_, sq_, solid=True, path="split")
        outc = torch.empty(bsc.out_size, dtype=torch.float64, device="cuda")
        wsc = lx.alloc_workspace(max(bsc.workspace_min(), min(bsc.workspace_size(), 64 << 30)))
        cms, cstage, _ = time_steps(torch, lx, bsc, outc, wsc, 2, 1, flush_buf, world)
        ctot = reduce_max(sum(cms), world)
        # FP64 path and error on a 1024-quartet sample (512 of each class)
        samp = np.concatenate([np.arange(512), len(sq_) // 2 + np.arange(512)])
        ssb, ssq = inputs.subset(sb_, sq_, samp)
        bsf = lx.Batch(ssb, ssq, solid=True)
        outf = torch.empty(bsf.out_size, dtype=torch.float64, device="cuda")
        fms, _, _ = time_steps(torch, lx, bsf, outf, lx.alloc_workspace(bsf.workspace_size()), 1, 1, flush_buf, 1)
        offs = bsc.quartets["out_offset"]
        gathered = torch.cat([outc[int(offs[i]):int(offs[i]) + int(bsc.sizes[i])] for i in samp])
        split_cfg = {"workload": f"{len(sq_)} quartets: (hh|hh) and (ii|ii) halves, K = 1..3 per shell, 20-bohr cube, "
                                 "exponents log-uniform [0.05, 20], solid harmonics, split path",
                     "quartets_per_s": world * len(sq_) * 2 / (ctot * 1e-3), "ms_per_step": ctot / 2,
                     "fp64_equiv_tflops": world * (sg1 + sg2) * 2 / (ctot * 1e-3) / 1e12,
                     "stage_ms_per_step": {k: v / 2 for k, v in cstage.items()},
                     "fp64_path_sample_quartets_per_s": len(samp) / (fms[0] * 1e-3),
                     "max_abs_err_vs_fp64_path_on_sample": float((gathered - outf).abs().max())}
        oidx = pick_sample(sb_, sq_, per_class=3, cheap_s=2.0, heavy_s=12.0, limit=256) + \
            [len(sq_) // 2 + i for i in pick_sample(*inputs.subset(sb_, sq_, np.arange(len(sq_) // 2, len(sq_))),
                                                   per_class=3, cheap_s=2.0, heavy_s=12.0, limit=256)]
        checks.add(split_cfg, "oracle_err_per_class", sb_, sq_, oidx,
                   {"split": gather_blocks(outc, offs, bsc.sizes, oidx)})
        del wsc, outc, outf, gathered
        torch.cuda.empty_cache()

    # ---- routed workload: l = 4..6, K = 1..5, separations 0..30 bohr; routed, split-only and
    # FP64-only arms on the same batch
    routed = None
    if not args.no_routed:
        routed = run_routed(args, torch, lx, inputs, world, checks)

    # ---- engine form: 64 (ii) bra pairs x 64 (ii) ket pairs, each pair's H (and digit planes)
    # built once and shared by its 64 quartets
    pairs = None
    if not args.no_pairs:
        pbas, pbra, pket = inputs.iiii_pairs(args.pairs, args.pairs)
        pq = [(a, b, c, d) for (a, b) in pbra for (c, d) in pket]
        pg1, pg2, _ = gemm_flops(pbas, pq, True)
        pairs = {"workload": f"{len(pbra)} (ii) bra pairs x {len(pket)} (ii) ket pairs = {len(pq)} quartets, K = 1, "
                             "20-bohr cube, exponents log-uniform [0.05, 20], solid harmonics (lx_eri_pairs)"}
        for path in ("fp64", "split"):
            pb = lx.PairBatch(pbas, pbra, pket, True, path=path)
            outp = torch.empty(pb.out_size, dtype=torch.float64, device="cuda")
            wsp = lx.alloc_workspace(pb.workspace_size())
            pms, pstage, _ = time_steps(torch, lx, pb, outp, wsp, max(2, min(args.steps, 3)), 2, flush_buf, world)
            ptot = reduce_max(sum(pms), world)
            nst = len(pms)
            pairs[path] = {"quartets_per_s": world * len(pq) * nst / (ptot * 1e-3), "ms_per_step": ptot / nst,
                           "fp64_equiv_tflops": world * (pg1 + pg2) * nst / (ptot * 1e-3) / 1e12,
                           "stage_ms_per_step": {k: v / nst for k, v in pstage.items()}}
            if path == "fp64":
                ref_p = outp
            else:
                pairs["split"]["max_abs_diff_vs_fp64_path"] = float((outp - ref_p).abs().max())
            del wsp
        del ref_p, outp
        torch.cuda.empty_cache()

    # ---- J/K digestion of the same pair-list workload (nbf 3,328): each quartet's block is
    # digested from the workspace into J and K instead of being returned
    jk = None
    if not args.no_pairs:
        pbas, pbra, pket = inputs.iiii_pairs(args.pairs, args.pairs)
        pq = np.array([(a, b, c, d) for (a, b) in pbra for (c, d) in pket], np.int32)
        jb_ = {p_: lx.JKBatch(pbas, pq, True, path=p_) for p_ in ("fp64", "split")}
        nbf = jb_["fp64"].nbf
        Dd = torch.randn(nbf, nbf, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
        Dd = Dd + Dd.T
        Jd, Kd = torch.zeros_like(Dd), torch.zeros_like(Dd)
        jk = {"workload": f"J and K of {len(pq)} (ii|ii) quartets ({len(pbra)} x {len(pket)} pair lists, K = 1) "
                          f"against a dense symmetric density, nbf = {nbf} (lx_eri_jk)"}

        class _JKRun:  # time_steps drives .run(out, ws, stream, time_stages)
            def __init__(self, b):
                self.b = b

            def run(self, out, ws_, stream=None, time_stages=False):
                self.b.run_jk(Dd, Jd, Kd, ws_, stream, time_stages)

        for path in ("fp64", "split"):
            wsj = lx.alloc_workspace(jb_[path].workspace_size())
            jms, jstage, _ = time_steps(torch, lx, _JKRun(jb_[path]), None, wsj, max(2, min(args.steps, 3)), 2,
                                        flush_buf, world)
            jtot = reduce_max(sum(jms), world)
            nst = len(jms)
            blk_bytes = 8 * 169 * 169 * len(pq)
            jk[path] = {"quartets_per_s": world * len(pq) * nst / (jtot * 1e-3), "ms_per_step": jtot / nst,
                        "stage_ms_per_step": {k: v / nst for k, v in jstage.items()},
                        "digest_gbs": blk_bytes / (jstage["digest"] / nst * 1e-3) / 1e9 if jstage["digest"] else None}
            del wsj
        del Dd, Jd, Kd
        torch.cuda.empty_cache()

    # ---- a small class x K table (the paper's Tables 1 and 2 on this GPU)
    sweep = None
    if not args.no_sweep_rows:
        sweep = run_sweep_rows(torch, lx, inputs, flush_buf, checks)

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        cpu = cpu_baseline(basis, quartets, True, args.cpu_seconds)
        # the kept GPU results of every leg against the oracle (after every timed region)
        cpu["oracle_checks_s"] = checks.run()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(nq),
                       "path": "plain FP64", "l2": "512 MB buffer written between timed steps",
                       "parallelism": f"replicas x{world}"},
            "fp64_equiv_tflops": fp64_tf, "integrals_per_s": world * nint * args.steps / (total_ms * 1e-3),
            "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
            "roofline": roofline, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "cartesian": cart,
            "split": split, "mixed": mixed, "split_config": split_cfg, "routed": routed, "pairs": pairs, "jk": jk,
            "sweep": sweep,
            "gpu_launches": int(sum(launches.values())),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
