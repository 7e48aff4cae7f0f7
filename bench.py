#!/usr/bin/env python
"""Benchmark of the Squint learner on GB300: SAC updates/s at batch 512, UTD-4 graph.

A step is one squint_update(k=4) call: four full SAC updates (minibatch draw,
shift + squint, encoder, target, critic/encoder step, temperature step, actor
step, polyak) replayed as one CUDA graph, on the training-shape workload: a
100k-slot ring of 3x128x128 uint8 frames (4.9 GB, uniform random slots, so the
gathered inputs are larger than L2), batch 512, 4 conv layers of 32 channels,
256-d projections, critics 512-512 x2 with 101 atoms, actor 512-512.

Prints one JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle
instead (rank 0 only), on the same workload and metric.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "train_b512"
UTD_K = 4
METRIC = "SAC updates/s at B=512 (BF16 vs FP32 plain); act p50/p99 latency on 1 GB300"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
N_SM = 152
FP32_LANES_PER_SM = 128
# act floor per query at the training shape: the 3x128x128 uint8 frame read once, and the
# encoder + actor projection + actor MLP contractions
ACT_BYTES = 3 * 128 * 128
ACT_FLOPS = 9.37e6
# update floor at the training shape (B = 512): HBM bytes (gather, Adam, polyak) and
# contraction FLOPs of one update
UPDATE_BYTES = 50.33e6 + 74.9e6 + 18.9e6
UPDATE_FLOPS = 27.96e9

# DRAM traffic per launch of the dominant kernel class from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the class's launches
# in one update; ncu replays each launch with cold caches), keyed by (class,
# precision).  Set back to nothing when the kernel changes.
NCU_TRAFFIC = {
    # train_b512: the five fused head launches of one BF16 update (the actor's two halves
    # apart), 8.98 MB read, 0 written (ncu dram__bytes_read.sum + dram__bytes_write.sum,
    # third update of the small-ring run)
    ("mlp_tc_fwd", "bf16", "train_b512"): 1796506,
}


WORKLOAD_TEXT = {
    "train_b512": ("train_b512: 100k x 3x128x128 uint8 ring (4.9 GB), batch 512, UTD 4 per step, shift pad 8, "
                   "squint 4x to 32x32, 4 conv x 32ch, proj 256 + LN, critics 512-512 x2 (101 atoms), actor 512-512",
                   "inputs larger than L2: 4.9 GB ring, 50 MB of uniformly random frames per update; "
                   "weights and activations stay L2-resident between updates as in training"),
    "stored_b512": ("stored_b512: squint at insert, 1M x 3x32x32 uint8 ring (3.1 GB) filled from 3x128x128 "
                    "renders by the insert kernel, batch 512, UTD 4 per step, shift pad 2 at 32x32, 4 conv x "
                    "32ch, proj 256 + LN, critics 512-512 x2 (101 atoms), actor 512-512",
                    "inputs larger than L2: 3.1 GB ring, 3.1 MB of uniformly random frames per update; "
                    "weights and activations stay L2-resident between updates as in training"),
    "state_b512": ("state_b512: state-based SAC (no encoder), 1M x 48-d state ring (0.2 GB with actions, "
                   "rewards, dones), batch 512, UTD 4 per step, critics 512-512 x2 (101 atoms), actor 512-512",
                   "inputs larger than L2: 0.2 GB ring, 0.2 MB of uniformly random rows per update; "
                   "weights and activations stay L2-resident between updates as in training"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8", "mxfp8"], default="bf16")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the plain FP32 path beside the BF16 one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", choices=["train_b512", "stored_b512", "state_b512"], default=WORKLOAD,
                    help="stored_b512: squint at insert, a 1M-slot ring of 3x32x32 frames filled by the insert "
                         "kernel; state_b512: state-based SAC, no encoder, a 1M-slot ring of 48-d states")
    ap.add_argument("--ring-slots", type=int, default=None,
                    help="replay-ring slots (default: the workload's 100k; smaller only for profiler captures)")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
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
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
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
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed plumbing
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def oracle_updates_per_s(cfg, ring, budget_s, max_updates=3):
    """Time the FP64 oracle on a bounded sample: whole updates (or a batch slice) within ~budget_s."""
    import numpy as np
    from oracle import squint_sac as o
    state = o.init_state(cfg)
    t0 = time.perf_counter()
    o.update(state, ring, cfg)
    one = time.perf_counter() - t0
    n = max(1, min(max_updates, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(n):
        o.update(state, ring, cfg)
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        n = [d.get("num_threads") for d in info if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


class LazyRows:
    def __init__(self, t):
        self.t = t
        self.shape = tuple(t.shape)

    def __getitem__(self, idx):
        import numpy as np
        import torch
        ii = torch.as_tensor(np.asarray(idx), device=self.t.device, dtype=torch.long)
        return self.t.index_select(0, ii).cpu().numpy()


def workload_config(workload, world):
    """The bench line's `config`, the same for both arms (each arm's arithmetic is its `dtype`)."""
    return {"workload": WORKLOAD_TEXT[workload][0], "updates_per_step": UTD_K,
            "l2": WORKLOAD_TEXT[workload][1], "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the same workload, rank 0 only.

    Every timed oracle update is a whole update of the batch-512 workload, as in our
    arm.  A step holds UTD_K of them when the K + W steps fit in about three minutes,
    else fewer (at least one): the rate in updates/s does not depend on how many
    updates a step groups, so the sample is bounded without scaling a smaller batch.
    """
    import torch
    from paper_2602_21203_gb300 import synth
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    cfg = synth.make_config(WORKLOAD)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    ring = {k: LazyRows(v) for k, v in synth.make_ring(cfg, args.seed, device=dev).items()}
    from oracle import squint_sac as o
    state = o.init_state(cfg)
    t0 = time.perf_counter()
    o.update(state, ring, cfg)                       # also the first warm-up update
    one = time.perf_counter() - t0
    per_step = max(1, min(UTD_K, int(180.0 / max(one * (args.steps + args.warmup), 1e-9))))
    for _ in range(args.warmup * per_step - 1):
        o.update(state, ring, cfg)
    t0 = time.perf_counter()
    for _ in range(args.steps * per_step):
        o.update(state, ring, cfg)
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    cores = blas_threads()
    sample = (f"{args.steps} steps of {per_step} whole FP64 oracle update(s) of the batch-512 workload "
              f"({args.steps * per_step} updates in {dt:.1f} s)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(WORKLOAD, world),
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch
    from paper_2602_21203_gb300 import lib, synth

    world, rank, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the learner has no CPU path)")
    peaks, peaks_src = load_peaks()
    cfg = synth.make_config(args.workload)
    if args.ring_slots:
        cfg["ring_size"] = int(args.ring_slots)
    stored = "render_f" in cfg
    prec = {"fp32": lib.PREC_FP32, "bf16": lib.PREC_BF16, "fp8": lib.PREC_FP8, "mxfp8": lib.PREC_MXFP8}[args.precision]
    ring = synth.make_ring(cfg, args.seed + rank, device="cuda")
    if stored:   # squint at insert: the ring's frames come from 3x128x128 renders through the insert kernel
        from paper_2602_21203_gb300 import ops
        for c0 in range(0, cfg["ring_size"], 8192):
            n = min(8192, cfg["ring_size"] - c0)
            ops.squint_store(synth.render_frames(n, cfg, 1000 + c0, device="cuda"), ring["obs"], c0, cfg["render_f"])
        torch.cuda.synchronize()
    learner = lib.Learner(cfg, ring, precision=prec, max_k=8)
    stream = torch.cuda.Stream()
    K = args.steps
    W = max(3, args.warmup)

    with torch.cuda.stream(stream):
        for _ in range(W):
            learner.update(UTD_K, stats=False, stream=stream)
    stream.synchronize()

    # ---- timed region: K graph replays of UTD_K updates, inputs already resident in HBM
    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(K):
        learner.update(UTD_K, stats=False, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world)
    updates = world * K * UTD_K
    value = updates / (ms / 1000.0)

    # ---- end to end through the public API with host buffers: per step, insert the
    # transitions one environment step adds at UTD 0.25 (4 updates <- 16 transitions)
    # from pinned host memory into the ring, run the UTD-4 call, read its statistics back.
    # The loop is pipelined as a training loop runs it: step j's statistics are copied to
    # pinned memory by the stream (squint_update_async) and read on the host while step
    # j + 1 is queued behind them; every step's copies and statistics are inside the timed
    # region, the last step's read before the clock stops.
    n_new = int(UTD_K / 0.25)
    host = {k: v[:n_new].cpu().pin_memory() for k, v in ring.items()}
    if stored:   # renders arrive at full resolution and are squinted on insert
        host["obs"] = synth.render_frames(n_new, cfg, 7, device="cpu").pin_memory()
        staging = torch.empty_like(host["obs"], device="cuda")
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = UTD_K * 32
    head = 0
    bufs = [lib.PinnedStats(UTD_K), lib.PinnedStats(UTD_K)]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    seen = []
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(K):
        with torch.cuda.stream(stream):
            sl = slice(head, head + n_new)
            for k2, v in host.items():
                if stored and k2 == "obs":
                    staging.copy_(v, non_blocking=True)
                    ops.squint_store(staging, ring["obs"], head, cfg["render_f"])
                else:
                    ring[k2][sl].copy_(v, non_blocking=True)
            head = (head + n_new) % (cfg["ring_size"] - n_new)
        learner.update_async(UTD_K, bufs[i % 2], stream=stream)   # the stream copies the statistics back
        done[i % 2].record(stream)
        if i > 0:                                                # the previous step's statistics, read
            done[(i - 1) % 2].synchronize()
            seen.append(bufs[(i - 1) % 2].read()[-1]["critic_loss"])
    done[(K - 1) % 2].synchronize()
    seen.append(bufs[(K - 1) % 2].read()[-1]["critic_loss"])
    learner.update_check(stream=stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if len(seen) != K or not all(math.isfinite(x) for x in seen):
        raise SystemExit("bench.py: end-to-end statistics missing or not finite")
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": world * K * UTD_K / e2e_s, "unit": "updates/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # ---- per-kernel device times: one in-order eager update on the timed stream, every
    # launch bracketed by CUDA events; the roofline is the class with the most device time
    kprof = {}
    for _ in range(5):
        for name, (nl, kms, work, unit) in learner.profile_kernels(stream=stream).items():
            e = kprof.setdefault(name, [nl, [], work, unit])
            e[1].append(kms)
    kernels = {}
    for name, (nl, times, work, unit) in kprof.items():
        t = statistics.median(times)
        kernels[name] = {"launches": nl, "ms": round(t, 5), "work": work, "unit": unit}
    phase_ms = {}
    for _ in range(3):
        for name, t in learner.profile_update(stream=stream).items():
            phase_ms.setdefault(name, []).append(t)
    phase_ms = {k: round(statistics.median(v), 4) for k, v in phase_ms.items()}
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12

    def class_roof(name, k):
        secs = k["ms"] / 1000.0
        if k["work"] <= 0 or secs <= 0:
            return None
        if k["unit"] == "B":
            ach = k["work"] / secs / 1e9
            return {"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peaks["hbm_gbs"],
                    "peak_source": f"{peaks_src} copy bandwidth"}
        ach = k["work"] / secs / 1e12
        if name == "tc_gemm_fwd" and args.precision in ("fp8", "mxfp8"):   # e4m3 operands: FP8 peak
            return {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": 2.0 * peaks["bf16_tflops"],
                    "peak_source": f"{peaks_src} bf16 burst x 2 (nominal fp8/bf16 dense ratio 4.5/2.25)"}
        if name.startswith(("tc_", "conv_tc", "mlp_tc")):
            return {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": peaks["bf16_tflops"],
                    "peak_source": f"{peaks_src} bf16 burst (kernel timed alone)"}
        return {"bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": fp32_peak,
                "peak_source": f"FP32 FMA {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz"}

    ranked = sorted((n for n in kernels if class_roof(n, kernels[n])), key=lambda n: -kernels[n]["ms"])
    dom = ranked[0]
    roof = class_roof(dom, kernels[dom])
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = NCU_TRAFFIC.get((dom, args.precision, args.workload))
    roof["kernel"] = dom
    roof["launches_per_update"] = kernels[dom]["launches"]
    roof["work_per_launch"] = kernels[dom]["work"] / kernels[dom]["launches"]
    roof["avg_launch_us"] = 1000.0 * kernels[dom]["ms"] / kernels[dom]["launches"]
    for n in kernels:
        cr = class_roof(n, kernels[n])
        if cr:
            kernels[n]["achieved"] = round(cr["achieved"], 3)
            kernels[n]["frac"] = round(cr["achieved"] / cr["peak"], 5)
    roof["kernels_per_update"] = kernels
    roof["phase_ms"] = phase_ms
    # the whole update against its floor at the measured peaks (training shape): HBM bytes
    # and contraction FLOPs overlapped (the larger time) or serial (the sum)
    if args.workload == "train_b512":
        t_h = UPDATE_BYTES / (peaks["hbm_gbs"] * 1e9) * 1e6
        t_t = UPDATE_FLOPS / (peaks["bf16_tflops_sustained"] * 1e12) * 1e6
        us = 1e6 / value
        roof["update"] = {"us_per_update": us, "floor_us_overlapped": max(t_h, t_t), "floor_us_serial": t_h + t_t,
                          "frac_overlapped": max(t_h, t_t) / us, "frac_serial": (t_h + t_t) / us,
                          "floor": "HBM: gather 50.3 MB + Adam 74.9 MB + polyak 18.9 MB; tensor: 27.96 GFLOP at "
                                   "the sustained bf16 peak"}

    # ---- serving: continuous batching beside the UTD-4 update stream
    serving = None
    if not args.no_serving and rank == 0:
        serving = measure_serving(lib, learner, cfg, stream)
    gpu_launches = learner.graph_kernel_count(UTD_K) * K
    pflat = learner.params()
    learner.close()

    # ---- the plain FP32 path on the same ring and schedule, for the BF16-vs-FP32 comparison
    fp32_plain = None
    if prec != lib.PREC_FP32 and not args.no_fp32_compare:
        plain = lib.Learner(cfg, ring, precision=lib.PREC_FP32, max_k=8)
        with torch.cuda.stream(stream):
            for _ in range(W):
                plain.update(UTD_K, stats=False, stream=stream)
        stream.synchronize()
        Kp = min(K, 30)
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(Kp):
            plain.update(UTD_K, stats=False, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        pms = max_over_ranks(ev0.elapsed_time(ev1), world)
        fp32_plain = {"value": world * Kp * UTD_K / (pms / 1000.0), "unit": "updates/s", "steps": Kp,
                      "ms_per_step": pms / Kp, "dtype": "f32",
                      "path": "same kernels' FP32 variants: CUDA-core GEMMs and convolutions, no BF16 casts"}
        fp32_plain["bf16_speedup"] = value / fp32_plain["value"]
        plain.close()

    # ---- CPU baseline: the oracle on this workload, rank 0 at N=1
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        lazy = {k: LazyRows(v) for k, v in ring.items()}
        ups, n, dt = oracle_updates_per_s(cfg, lazy, budget_s=15.0, max_updates=12)
        cpu = {"value": ups, "unit": "updates/s", "cores": blas_threads(), "kind": "oracle",
               "sample": f"{n} FP64 oracle update(s) of the full batch-512 workload in {dt:.1f} s"}
        if serving and cfg.get("conv_layers", 0) > 0:
            # the oracle's inference on the same policy: 512 queries (one group of the serving mix)
            from oracle import squint_sac as o
            P, off = {}, 0
            for name, shape, _, _ in o.param_spec(cfg):
                k = int(np.prod(shape))
                P[name] = np.asarray(pflat[off:off + k], dtype=np.float64).reshape(shape)
                off += k
            obs_c, prop_c = synth.make_obs_batch(512, cfg, 5, device="cpu")
            t0 = time.perf_counter()
            o.act(P, obs_c.numpy(), prop_c.numpy(), 1, True, cfg)
            adt = time.perf_counter() - t0
            serving["cpu_baseline"] = {"value": 512 / adt, "unit": "queries/s", "cores": blas_threads(),
                                       "kind": "oracle", "sample": f"512 FP64 oracle queries in {adt:.2f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3+bf16", "mxfp8": "e4m3(mx)+bf16"}[args.precision],
            "data": "synthetic",
            "config": workload_config(args.workload, world),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": gpu_launches, "clocks": clk,
        }
        if fp32_plain:
            line["fp32_plain"] = fp32_plain
        if serving:
            line["serving"] = serving
        print(json.dumps(line), flush=True)


def measure_serving(lib, learner, cfg, upd_stream, seconds=4.0, n_envs=4096, mean_step_us=200.0):
    """Actor queries for n_envs environments in groups of U{1..512}, beside UTD-4 updates.

    Closed loop: each group submits its query, and after its actions come back
    waits an exponential environment-step time (mean mean_step_us) before the next
    one, so arrivals are Poisson-like and about n_envs queries stay in flight.
    The update thread runs UTD-4 calls and refreshes the policy snapshot after each.
    """
    import numpy as np
    import torch
    from paper_2602_21203_gb300 import synth
    rng = np.random.default_rng(1)
    sizes, left = [], n_envs
    while left > 0:
        n = min(int(rng.integers(1, 513)), left)
        sizes.append(n)
        left -= n
    offs = np.concatenate([[0], np.cumsum(sizes)])
    obs, prop = synth.make_obs_batch(n_envs, cfg, 3, device="cuda")
    out = torch.empty(n_envs, cfg["action_dim"], device="cuda")
    learner.serve_start(max_rows=n_envs, mem_budget_bytes=16 << 30)
    stop = threading.Event()
    counter = {"updates": 0}

    def updater():
        with torch.cuda.stream(upd_stream):
            while not stop.is_set():
                learner.update(UTD_K, stats=False, stream=upd_stream)
                learner.refresh_policy(stream=upd_stream)
                upd_stream.synchronize()
                counter["updates"] += UTD_K

    th = threading.Thread(target=updater)
    th.start()
    time.sleep(0.2)
    t_start = time.perf_counter()
    tickets = [None] * len(sizes)
    next_t = [t_start] * len(sizes)
    lats, rows_done, key = [], 0, 0
    u0 = counter["updates"]
    while time.perf_counter() - t_start < seconds:
        now = time.perf_counter()
        for g, n in enumerate(sizes):
            if tickets[g] is None:
                if now >= next_t[g]:
                    a, b = int(offs[g]), int(offs[g + 1])
                    req = lib.Learner.request(None if obs is None else obs[a:b], prop[a:b], out[a:b], key=key,
                                              group_id=g)
                    tickets[g] = learner.serve_submit(req)
                    key += 1
            else:
                r = learner.serve_poll(tickets[g], 0)
                if r is not None:
                    lats.append(r[0])
                    rows_done += n
                    tickets[g] = None
                    next_t[g] = time.perf_counter() + rng.exponential(mean_step_us * 1e-6)
    elapsed = time.perf_counter() - t_start
    u1 = counter["updates"]
    for g in range(len(sizes)):
        if tickets[g] is not None:
            learner.serve_poll(tickets[g], 5_000_000)
    stop.set()
    th.join()
    info = learner.serve_info()
    learner.serve_stop()
    if not lats:
        return None
    qps = rows_done / elapsed
    # act floor per query: 49,152 B of observation read (HBM) and 9.37 MFLOP (tensor), at the
    # measured peaks; overlapped (the larger) and serial (the sum)
    peaks, _ = load_peaks()
    t_hbm = ACT_BYTES / (peaks["hbm_gbs"] * 1e9)
    t_ten = ACT_FLOPS / (peaks["bf16_tflops"] * 1e12)
    return {"envs": n_envs, "groups": len(sizes), "requests_completed": len(lats),
            "queries_per_s": qps, "p50_us": float(np.percentile(lats, 50)),
            "p99_us": float(np.percentile(lats, 99)), "updates_per_s_concurrent": (u1 - u0) / elapsed,
            "slots": info["slots"], "slot_rows": info["slot_rows"], "arena_bytes": info["arena_bytes"],
            "floor": {"bytes_per_query": ACT_BYTES, "flops_per_query": ACT_FLOPS,
                      "queries_per_s_overlapped": 1.0 / max(t_hbm, t_ten), "queries_per_s_serial": 1.0 / (t_hbm + t_ten),
                      "frac_of_serial_floor": qps * (t_hbm + t_ten), "frac_of_overlapped_floor": qps * max(t_hbm, t_ten),
                      "peaks": "measured HBM copy and bf16 burst"},
            "group_sizes": "U{1..512}", "arrivals": f"closed loop, exponential env step mean {mean_step_us:.0f} us",
            "latency": "host queueing until the batch's launch plus the batch's device time (launch marker to "
                       "completion event)"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
