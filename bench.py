"""Benchmark of prox_{lambda R} on GB300: one JSON line on stdout.

Workload (the single-large-vector configuration): d = 2^26 FP32 weights,
w_i ~ N(0, 1) with 10% of positions overwritten by exact duplicates, seeded;
each step is one prox (the whole hot path: sort, shift, exact merge, cluster
values, lookup back to the caller's order) with lambda cycling through
{1e-2, 1, 1e2}.  The input (256 MiB) is larger than L2 and resident in HBM
before the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica (the single-vector
path does not shard), value = all ranks' elements / max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores instead (rank 0
only), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "prox_R elements/s and HBM-roofline fraction, FP32-comp vs FP64 at stated error"
LAMBDAS = (1e-2, 1.0, 1e2)
WORKLOAD = "single vector d=2^26 FP32 N(0,1) + 10% exact duplicates, lambda cycling {1e-2, 1, 1e2}"

# Algorithmic HBM bytes per element for each kernel kind of the device-wide
# path (FP32 storage): what a launch must read and write at the least.
ALGO_BYTES_PER_ELEM_F32 = {
    "onesweep": 8,    # read key (pass 0: the value) + write key
    "hist": 4,        # read the value
    "tile_hull": 4,   # read the sorted key (hull vertices are data dependent, not counted)
    "lookup": 12,     # read w, write out and cluster id (I/O floor)
}

# Whole-step byte models per element (FP32 storage), fixed before tuning:
# the I/O floor (read w, write out and cluster id), this library's key-only
# sort pipeline (histogram read 4 + four 8-bit passes x (read + write key) 32 +
# merge read of the sorted keys 4 + lookup 12) and the sort-with-index-payload
# pipeline of the design survey (80 B).  One-CTA segments of a batch move the
# I/O floor only.
IO_FLOOR_B = 12
ONE_CTA_MAX_F32 = 4096   # FP32 segments up to this length run one CTA each
MODEL_B = {"key_only_52B": 52, "index_payload_80B": 80}

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the bench's own workload, and the hash of the source files the
# kernel is built from when the counters were taken; reported as null once any
# of them changes (see profiles/).
NCU_SOURCES = {"onesweep": ["ws_sort.cu", "ws_kernels.cuh", "ws_block.cuh", "ws_common.cuh"]}
NCU_TRAFFIC = {"onesweep": 511.8e6}   # d = 2^26, mean of the 4 passes (1 ncu pass each)
NCU_SOURCE_HASH = {"onesweep": "bb6a5940a12a3213"}


def source_hash(files=None) -> str:
    """Hash of the kernel sources (all of csrc/, or the listed files of it)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_03096_gb300", "csrc")
    for f in sorted(files if files is not None else os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def byte_fracs(elems_small: int, elems_large: int, ms: float, peak_gbs: float) -> dict:
    """Fractions of the measured HBM peak that the byte models above reach in `ms`."""
    def frac(b_large, b_small):
        return (b_large * elems_large + b_small * elems_small) / (ms / 1e3) / (peak_gbs * 1e9)

    return {"model_bytes_frac": {k: frac(b, IO_FLOOR_B) for k, b in MODEL_B.items()},
            "io_floor_frac": frac(IO_FLOOR_B, IO_FLOOR_B)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling (200 ms) during the benchmark; lines are timestamped."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        inwin = [p for (t, p) in self.samples if t0 - 0.25 <= t <= t1 + 0.25]
        use = inwin if len(inwin) >= 1 else [p for (_, p) in self.samples]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[2]) for p in use if num(p[2]) is not None]
        mx = [num(p[3]) for p in use if num(p[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in use for i in range(4) if "Active" in p[6 + i] and "Not" not in p[6 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "in_window": len(inwin)}


def oracle_rate(w_sample: np.ndarray, steps: int):
    """Time the FP64 oracle on a sample, cycling lambda; returns elements/s."""
    import oracle

    t = time.perf_counter()
    for k in range(steps):
        oracle.prox(w_sample, LAMBDAS[k % len(LAMBDAS)])
    dt = time.perf_counter() - t
    return w_sample.shape[0] * steps / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_2311_03096_gb300 import inputs

    oracle.build()
    w = inputs.normal_with_duplicates(args.d, seed=args.seed, dtype=np.float32)
    # size the per-step sample so that warmup + steps finish in about two minutes
    probe = w[: 1 << 17]
    rate, _ = oracle_rate(probe, 3)
    budget = 120.0 / max(1, args.steps + args.warmup)
    # the oracle's rate falls slowly with n (the sort), so stay a power of two below the estimate
    n = int(min(args.d, 1 << 22, max(1 << 14, 2 ** (int(np.log2(max(1.0, rate * budget))) - 1))))
    sample = w[:n]
    for k in range(args.warmup):
        oracle.prox(sample, LAMBDAS[k % 3])
    value, dt = oracle_rate(sample, args.steps)
    cfg = config_dict(args, world)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": f"first {n} elements of the workload vector per step (lambda cycling)"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_calls(fn, stream, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _oracle_segments(args):
    import oracle

    vals, off, lam = args
    for s in range(len(lam)):
        oracle.prox(vals[off[s]:off[s + 1]], float(lam[s]))
    return int(off[-1])


def bench_batched(ws, ctx, stream, peak, reps=5):
    """Batched MLP layout (rows, whole layers, 4096 log-uniform extras): elements/s
    of each set and of all of them in one call (eager and CUDA-graph replay),
    errors against the oracle on sampled segments, and the oracle run
    segment-parallel over the host cores on a bounded sample."""
    import multiprocessing as mp
    import os

    import torch

    import oracle
    from paper_2311_03096_gb300 import inputs

    vals, off, lam, kinds = inputs.batched_segments(seed=0)
    kinds = np.asarray(kinds)
    res = {"elements": int(off[-1]), "segments": int(len(lam))}
    dev = torch.device("cuda", torch.cuda.current_device())
    for name, sel in (("rows", kinds == "row"), ("layers", kinds == "layer"), ("extras", kinds == "extra"),
                      ("all", np.ones(len(kinds), bool))):
        idx = np.nonzero(sel)[0]
        lens = np.diff(off)[idx]
        sub_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        sub_vals = vals if name == "all" else np.concatenate([vals[off[s]:off[s + 1]] for s in idx])
        plan = ws.Plan(sub_off, torch.float32, ctx=ctx)
        v = torch.from_numpy(sub_vals).to(dev)
        lt = torch.from_numpy(lam[idx]).to(dev)
        out = torch.empty_like(v)
        ids = torch.empty(v.shape[0], dtype=torch.int32, device=dev)
        nc = torch.zeros(len(idx), dtype=torch.int64, device=dev)
        run = lambda: plan.forward(v, lt, "fp32comp", out=out, id_out=ids, n_clusters=nc, stream=stream)  # noqa: E731
        ms = _time_calls(run, stream, reps)
        e_small = int(lens[lens <= ONE_CTA_MAX_F32].sum())
        e_large = int(sub_off[-1]) - e_small
        entry = {"elements": int(sub_off[-1]), "segments": int(len(idx)), "ms": ms,
                 "elements_per_s": sub_off[-1] / (ms / 1e3), "elements_one_cta": e_small,
                 **byte_fracs(e_small, e_large, ms, peak)}
        if name == "rows":
            g_r = torch.from_numpy(inputs.normal(int(sub_off[-1]), seed=5, dtype=np.float32)).to(dev)
            gin_r = torch.empty_like(g_r)
            entry["backward_ms"] = _time_calls(lambda: plan.backward(g_r, ids, grad_in=gin_r, stream=stream), stream,
                                               reps)
            del g_r, gin_r
        if name == "all":
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                run_g = lambda: plan.forward(v, lt, "fp32comp", out=out, id_out=ids, n_clusters=nc)  # noqa: E731
                run_g()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                run_g()
            msg = _time_calls(g.replay, stream, reps)
            entry["graph_ms"] = msg
            entry["graph_elements_per_s"] = sub_off[-1] / (msg / 1e3)
            entry["graph"] = byte_fracs(e_small, e_large, msg, peak)
            tuned = ws.Plan.autotuned(sub_off, v, lt, "fp32comp", thresholds=[0, 1024, 2048, 4096], reps=2, ctx=ctx)
            entry["autotune"] = {"threshold": tuned.threshold, "ic_cap": tuned.ic_cap,
                                 "ms_by_threshold": dict(zip(["0", "1024", "2048", "4096"], tuned.times_ms)),
                                 "tuned": "one-CTA length threshold, then the Imminent Collisions round cap "
                                          "(8/16/32/64) on the chosen plan"}
            del tuned
            ctx.check(what="bench batched")
            out_h, ids_h = out.cpu().numpy(), ids.cpu().numpy()
            rng = np.random.default_rng(7)
            pick = list(np.nonzero(kinds == "layer")[0]) + list(rng.choice(np.nonzero(kinds == "row")[0], 8)) + \
                list(rng.choice(np.nonzero(kinds == "extra")[0], 8))
            worst, same = 0.0, True
            for s in pick:
                a, b = off[s], off[s + 1]
                ref, rid, _ = oracle.prox(vals[a:b], float(lam[s]))
                scale = float(np.abs(vals[a:b]).max()) + float(lam[s])
                worst = max(worst, float(np.abs(out_h[a:b].astype(np.float64) - ref).max()) / scale)
                same &= bool(np.array_equal(ids_h[a:b], rid))
            entry["error_vs_oracle_sampled"] = {"segments": len(pick), "max_err_rel_to_max_w_plus_lambda": worst,
                                                "partition_equal": same}
        res[name] = entry
        del plan, v, lt, out, ids, nc
        torch.cuda.empty_cache()
    ctx.check(what="bench batched")
    # the oracle over all host cores (one segment per task), on rows + layers + the first extras
    cores = os.cpu_count() or 1
    extra_idx = np.nonzero(kinds == "extra")[0]
    take = [s for s in range(len(lam)) if kinds[s] != "extra"] + list(extra_idx[:256])
    chunks = [[] for _ in range(cores)]
    for j, s in enumerate(sorted(take, key=lambda s: -(off[s + 1] - off[s]))):
        chunks[j % cores].append(s)
    tasks = []
    for c in chunks:
        if not c:
            continue
        lens = np.array([off[s + 1] - off[s] for s in c], np.int64)
        sub_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        tasks.append((np.concatenate([vals[off[s]:off[s + 1]] for s in c]), sub_off, lam[c]))
    t0 = time.time()
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        n = sum(pool.map(_oracle_segments, tasks))
    dt = time.time() - t0
    res["oracle_parallel"] = {"value": n / dt, "unit": "elements/s", "cores": len(tasks), "cpu_model": cpu_model(),
                              "kind": "oracle",
                              "sample": f"{len(take)} segments (all rows, all layers, 256 extras; {n} elements), "
                                        f"{dt:.1f} s including process start"}
    return res


def bench_configs(ws, ctx, stream):
    """Timings of the other single-vector configurations: d = 4096 FP64 N(0,1)
    (lambda in {0, 0.1, 1, 1000}, FP64 arithmetic) and the adversarial cascade
    and mirror at d = 2^24 (sorted and shuffled)."""
    import torch

    from paper_2311_03096_gb300 import inputs

    dev = torch.device("cuda", torch.cuda.current_device())
    res = {}
    w = torch.from_numpy(inputs.normal(4096, seed=0, dtype=np.float64)).to(dev)
    out = torch.empty_like(w)
    ids = torch.empty(4096, dtype=torch.int32, device=dev)
    nc = torch.zeros(1, dtype=torch.int64, device=dev)
    for lam in (0.0, 0.1, 1.0, 1000.0):
        run = lambda: ws.prox(w, lam, "fp64", ctx=ctx, out=out, id_out=ids, n_clusters=nc, stream=stream)  # noqa
        ms = _time_calls(run, stream, 200)
        res[f"d4096_f64_lam{lam:g}"] = {"us_per_call": 1e3 * ms, "elements_per_s": 4096 / (ms / 1e3),
                                        "clusters": int(nc.item())}
    d = 1 << 24
    for name, gen in (("cascade", inputs.cascade), ("mirror", inputs.mirror)):
        for shuffle in (False, True):
            w_np, lam = gen(d, seed=0, shuffle=shuffle)
            w = torch.from_numpy(w_np).to(dev)
            out = torch.empty_like(w)
            ids = torch.empty(d, dtype=torch.int32, device=dev)
            run = lambda: ws.prox(w, lam, "fp32comp", ctx=ctx, out=out, id_out=ids, n_clusters=nc, stream=stream)  # noqa
            ms = _time_calls(run, stream, 10)
            res[f"{name}_2^24_{'shuffled' if shuffle else 'sorted'}"] = {
                "ms": ms, "elements_per_s": d / (ms / 1e3), "clusters": int(nc.item()), "merges": d - int(nc.item())}
    ctx.check(what="bench configs")
    return res


def bench_train(ws, ctx, stream, steps=10):
    """Proximal SGD step on the MLP (batch 256 of 32x32x3): ms per step and the
    prox share, cold and with the warm start from the previous step's clusters."""
    import torch

    from paper_2311_03096_gb300 import inputs
    from paper_2311_03096_gb300.train import ProxMLP

    x_np, y_np = inputs.images(batch=256, seed=0)
    x, y = torch.from_numpy(x_np).cuda(), torch.from_numpy(y_np).cuda()
    res = {}
    for warm in (False, True):
        m = ProxMLP(seed=0, warm=warm)
        for _ in range(3):
            m.step(x, y)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * steps)]
        for k in range(steps):
            ev[3 * k].record(stream)
            m.sgd(x, y)
            ev[3 * k + 1].record(stream)
            m.prox(stream=stream)
            ev[3 * k + 2].record(stream)
        torch.cuda.synchronize()
        ctx.check(what="bench train")
        step = sum(ev[3 * k].elapsed_time(ev[3 * k + 2]) for k in range(steps)) / steps
        prox = sum(ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(steps)) / steps
        r = {"ms_per_step": step, "prox_ms": prox, "prox_share": prox / step}
        if not warm:
            res.update(r)
            res.update({"rows": int(m.offsets.shape[0] - 1), "weights": int(m.flat.shape[0]), "batch": 256,
                        "lr": m.lr, "alpha": m.alpha})
        else:
            res["warm_start"] = r
    return res


def run_rows_case(args):
    """The batched MLP rows (8202 segments of 3072/4096, one-CTA kernel) alone:
    warm-up + steps forward calls, CUDA-event time of the steps."""
    import torch

    import __graft_entry__
    from paper_2311_03096_gb300 import inputs, ws

    __graft_entry__.build()
    ctx = ws.Context.get(0)
    stream = torch.cuda.current_stream()
    vals, off, lam, kinds = inputs.batched_segments(seed=args.seed, layers=False, extra=0)
    plan = ws.Plan(off, torch.float32, ctx=ctx)
    v = torch.from_numpy(vals).cuda()
    lt = torch.from_numpy(lam).cuda()
    out = torch.empty_like(v)
    ids = torch.empty(v.shape[0], dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        plan.forward(v, lt, args.prec, out=out, id_out=ids, stream=stream)
    ms = _time_calls(lambda: plan.forward(v, lt, args.prec, out=out, id_out=ids, stream=stream), stream,
                     max(args.steps, 1))
    ctx.check(what="rows case")
    print(json.dumps({"case": "rows", "segments": int(len(lam)), "elements": int(off[-1]), "ms_per_call": ms}))


def run_backward_case(args):
    """The device-wide backward alone at d (FP32, lambda --lam): one forward for
    the cluster ids, then warm-up + steps backward calls, CUDA-event time of the
    steps -- the launches that the backward's profiles capture."""
    import torch

    import __graft_entry__
    from paper_2311_03096_gb300 import inputs, ws

    __graft_entry__.build()
    ctx = ws.Context.get(0)
    stream = torch.cuda.current_stream()
    w = torch.from_numpy(inputs.normal_with_duplicates(args.d, seed=args.seed, dtype=np.float32)).cuda()
    g = torch.from_numpy(inputs.normal(args.d, seed=args.seed + 1, dtype=np.float32)).cuda()
    gin = torch.empty_like(g)
    _, ids, nc = ws.prox(w, args.lam, args.prec, ctx=ctx)
    for _ in range(args.warmup):
        ws.prox_backward(g, ids, ctx=ctx, grad_in=gin)
    ms = _time_calls(lambda: ws.prox_backward(g, ids, ctx=ctx, grad_in=gin), stream, max(args.steps, 1))
    ctx.check(what="backward case")
    print(json.dumps({"case": "backward", "d": args.d, "lambda": args.lam, "clusters": int(nc.item()),
                      "ms_per_call": ms}))


def config_dict(args, world):
    return {"workload": WORKLOAD, "d": args.d, "lambdas": list(LAMBDAS), "storage": "f32", "prec": args.prec,
            "arithmetic": "merge decisions exact in 64/128-bit fixed point; cluster values in "
                          + ("FP32" if args.prec == "fp32comp" else "FP64"),
            "seed": args.seed, "l2": "inputs larger than L2 (256 MiB vector per step)",
            "parallelism": f"replicas x{world}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--d", type=int, default=1 << 26)
    ap.add_argument("--prec", default="fp32comp", choices=["fp32comp", "fp64"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--case", default="single", choices=["single", "rows", "backward"],
                    help="rows: only run the batched MLP rows forward (warm-up + steps calls) and print its "
                         "ms per call -- the launch that the one-CTA kernel's profiles capture; backward: "
                         "only the device-wide backward at --d and --lam")
    ap.add_argument("--lam", type=float, default=1e-2, help="lambda of --case backward")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case == "rows":
        run_rows_case(args)
        return
    if args.case == "backward":
        run_backward_case(args)
        return

    import torch

    import __graft_entry__
    from paper_2311_03096_gb300 import inputs, replicas, ws

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = ws.Context.get(local)
    stream = torch.cuda.current_stream()

    w_np = inputs.normal_with_duplicates(args.d, seed=args.seed, dtype=np.float32)
    w = torch.from_numpy(w_np).to(dev)
    out = torch.empty_like(w)
    ids = torch.empty(args.d, dtype=torch.int32, device=dev)
    nc = torch.zeros(1, dtype=torch.int64, device=dev)

    # first call plans (allocates) and is excluded from everything below
    ws.prox(w, 1.0, args.prec, ctx=ctx, out=out, n_clusters=nc)
    ctx.check(what="bench warm-up")

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    time.sleep(0.5)
    for k in range(args.warmup):
        ws.prox(w, LAMBDAS[k % 3], args.prec, ctx=ctx, out=out, n_clusters=nc)
    torch.cuda.synchronize()
    ctx.check(what="bench warm-up")

    # ---- timed region: K steps, inputs resident in HBM, no per-kernel events
    launches0 = ctx.launch_count()
    replicas.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    for k in range(args.steps):
        ws.prox(w, LAMBDAS[k % 3], args.prec, ctx=ctx, out=out, n_clusters=nc)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    replicas.barrier()
    launches = ctx.launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    ctx.check(what="bench timed region")
    ms_max = replicas.max_over_ranks(ms_total, dev)
    value = replicas.job_rate(args.d * args.steps, world, ms_max)
    ms_per_step = ms_max / args.steps

    # ---- kernel timing: the same steps again with a CUDA event pair recorded
    # around every launch on the launching stream (kept out of the value above)
    ctx.profile(True)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for k in range(args.steps):
        ws.prox(w, LAMBDAS[k % 3], args.prec, ctx=ctx, out=out, n_clusters=nc)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    kern = ctx.profile_read()
    ctx.profile(False)
    ctx.check(what="bench kernel timing")

    # ---- dominant kernel roofline (live CUDA-event durations from the timed region)
    peak, peak_kind = load_peaks()
    shares = {k: {"ms_total": v[0], "launches": v[1], "ms_per_launch": v[0] / v[1], "share": v[0] / ms_prof}
              for k, v in kern.items()}
    dom = max(kern.items(), key=lambda kv: kv[1][0])[0] if kern else None
    roofline = None
    if dom is not None:
        ms_avg = kern[dom][0] / kern[dom][1]
        per_launch = ALGO_BYTES_PER_ELEM_F32.get(dom)
        traffic = None
        if dom in NCU_TRAFFIC and NCU_SOURCE_HASH.get(dom) == source_hash(NCU_SOURCES.get(dom)):
            traffic = NCU_TRAFFIC[dom]
        if per_launch is not None:
            achieved = per_launch * args.d / (ms_avg / 1e3) / 1e9
            roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                        "bytes_per_launch": per_launch * args.d, "ms_per_launch": ms_avg, "traffic": traffic,
                        "timing": "CUDA events around every launch on the launching stream, in a second run "
                                  "of the timed loop (same steps and inputs; the value comes from the first, "
                                  "unprofiled run)"}
        else:
            roofline = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                        "ms_per_launch": ms_avg, "traffic": traffic}

    # ---- end to end through the public API with host buffers (pinned).  Every step
    # copies its input in and its result (values + ids) out; the copies of one step
    # overlap the prox of the neighbouring steps (two buffers, copy engines on their
    # own streams), as a pipelined caller would run it.
    e2e = None
    if not args.no_e2e:
        h_w = torch.from_numpy(w_np).pin_memory()
        h_out = [torch.empty(args.d, dtype=torch.float32).pin_memory() for _ in range(2)]
        h_ids = [torch.empty(args.d, dtype=torch.int32).pin_memory() for _ in range(2)]
        d_w = [torch.empty_like(w) for _ in range(2)]
        d_out = [out, torch.empty_like(w)]
        d_ids = [ids, torch.empty_like(ids)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        n_e2e = max(3, min(args.steps, 50))

        def e2e_steps(count):
            s_in.wait_stream(stream)    # nothing of these steps starts before the timer
            s_out.wait_stream(stream)
            done = [None, None]
            for k in range(count):
                b = k % 2
                ev_free = torch.cuda.Event()
                if done[b] is not None:
                    s_in.wait_event(done[b])          # the buffer's previous step has been copied out
                with torch.cuda.stream(s_in):
                    d_w[b].copy_(h_w, non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(s_in)
                stream.wait_event(ev_in)
                ws.prox(d_w[b], LAMBDAS[k % 3], args.prec, ctx=ctx, out=d_out[b], n_clusters=nc, stream=stream,
                        id_out=d_ids[b])
                ev_c = torch.cuda.Event()
                ev_c.record(stream)
                s_out.wait_event(ev_c)
                with torch.cuda.stream(s_out):
                    h_out[b].copy_(d_out[b], non_blocking=True)
                    h_ids[b].copy_(d_ids[b], non_blocking=True)
                ev_free.record(s_out)
                done[b] = ev_free
            stream.wait_stream(s_out)

        e2e_steps(2)
        torch.cuda.synchronize()
        replicas.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        e2e_steps(n_e2e)
        f1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = replicas.max_over_ranks(f0.elapsed_time(f1), dev)
        e2e = {"value": replicas.job_rate(args.d * n_e2e, world, ms_e2e), "unit": "elements/s",
               "h2d_bytes_per_step": 4 * args.d, "d2h_bytes_per_step": 8 * args.d, "steps": n_e2e,
               "pipelined": "copies of one step overlap the prox of the neighbouring steps (2 buffers)"}
        ctx.check(what="bench e2e")

    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)

    # ---- variants: per-lambda and FP64 arithmetic / FP64 storage throughput, error at 2^20
    variants = None
    if not args.no_variants and rank == 0:
        variants = {}
        reps = 20
        for lam in LAMBDAS:
            for prec in ("fp32comp", "fp64"):
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    ws.prox(w, lam, prec, ctx=ctx, out=out, n_clusters=nc)
                b.record(stream)
                torch.cuda.synchronize()
                variants[f"f32_{prec}_lam{lam:g}"] = {"elements_per_s": args.d * reps / (a.elapsed_time(b) / 1e3),
                                                      "clusters": int(nc.item())}
        # the cluster merge path of each lambda: in-tile Imminent Collisions
        # rounds (default round cap) against the tree of bridge merges alone
        # (cap 0), and which path every hull tile took
        merge_paths = {}
        for lam in LAMBDAS:
            entry = {}
            for name, cap in (("ic_rounds", -1), ("merges_only", 0)):
                ctx.set_ic_cap(cap)
                ws.prox(w, lam, args.prec, ctx=ctx, out=out, n_clusters=nc)
                ms = _time_calls(lambda: ws.prox(w, lam, args.prec, ctx=ctx, out=out, n_clusters=nc), stream, 10)
                hs = ctx.hull_stats(args.d)
                entry[name] = {"ms_per_step": ms, "tiles_general_kernel": hs["general"],
                               "tiles_capped_to_merges": hs["capped"],
                               "tiles_converged_by_rounds": {str(r): c for r, c in enumerate(hs["rounds"]) if r and c}}
            ctx.set_ic_cap(-1)
            merge_paths[f"lam{lam:g}"] = entry
        variants["merge_paths"] = merge_paths
        # backward (cluster-mean Jacobian), exact fixed-point sums
        g_t = torch.from_numpy(inputs.normal(args.d, seed=args.seed + 1, dtype=np.float32)).to(dev)
        gin_t = torch.empty_like(g_t)
        bwd = {}
        for lam in LAMBDAS:
            _, ids_l, _ = ws.prox(w, lam, args.prec, ctx=ctx)
            ms = _time_calls(lambda: ws.prox_backward(g_t, ids_l, ctx=ctx, grad_in=gin_t), stream, 5)
            bwd[f"lam{lam:g}"] = {"ms": ms, "elements_per_s": args.d / (ms / 1e3)}
            del ids_l
        variants["backward_single_vector"] = bwd
        del g_t, gin_t
        ctx.check(what="bench merge paths")
        w64 = w.double()
        out64 = torch.empty_like(w64)
        for lam in LAMBDAS:
            ws.prox(w64, lam, "fp64", ctx=ctx, out=out64, n_clusters=nc)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                ws.prox(w64, lam, "fp64", ctx=ctx, out=out64, n_clusters=nc)
            b.record(stream)
            torch.cuda.synchronize()
            variants[f"f64_fp64_lam{lam:g}"] = {"elements_per_s": args.d * reps / (a.elapsed_time(b) / 1e3)}
        del w64, out64
        ctx.check(what="bench variants")
        # error against the oracle on a 2^20 prefix (full comparison; oracle on host)
        import oracle

        n = 1 << 20
        ws_np = w_np[:n]
        xs = torch.from_numpy(ws_np).to(dev)
        errs = {}
        for lam in LAMBDAS:
            ref, ref_ids, _ = oracle.prox(ws_np, lam)
            scale = float(np.abs(ws_np).max()) + lam
            for prec in ("fp32comp", "fp64"):
                o, i, _ = ws.prox(xs, lam, prec, ctx=ctx)
                err = float(np.abs(o.cpu().numpy().astype(np.float64) - ref).max()) / scale
                same = bool(np.array_equal(i.cpu().numpy(), ref_ids))
                errs[f"{prec}_lam{lam:g}"] = {"max_err_rel_to_max_w_plus_lambda": err, "partition_equal": same}
        variants["error_vs_oracle_2^20"] = errs
        variants["batched_mlp"] = bench_batched(ws, ctx, stream, peak)
        variants["configs"] = bench_configs(ws, ctx, stream)
        variants["train_step"] = bench_train(ws, ctx, stream)

    # ---- CPU baseline: the oracle on the host cores, bounded sample
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle

        oracle.build()
        n = 1 << 22
        rate, dt = oracle_rate(w_np[:n], 6)
        cpu = {"value": rate, "unit": "elements/s", "cores": 1, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"first {n} elements of the workload vector, 6 calls cycling lambda ({dt:.1f} s)"}

    fracs = byte_fracs(0, args.d, ms_per_step, peak)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32comp" else "f64", "data": "synthetic",
            "config": config_dict(args, world), "roofline": roofline, **fracs, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "kernels": shares, "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
