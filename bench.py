"""Benchmark: whole MUSTER registrations of the realistic series on GB300.

Workload (one "step" = one complete registration, every row of the hot path):
10 sessions of a 160x192x160 float32 brain-like phantom, 4-level pyramid,
flow grid 2x coarser than each level, 7 squarings, 7^3 window, SiLNCC,
100 Adam steps per level. Metric: Gvoxel-iters/s = sum over levels of
steps x N(N-1) x voxels of the level, divided by the wall time of the
registration (forward, adjoint and update included; ordered-pair voxels).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun) every rank registers its own subject (independent
replicas, no collective on the data path); value = all ranks' units / max time.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # tiny: 3 x 48^3 blob phantoms, 1 level x 20 steps, K=6, w=5
    "c1": dict(kind="plain", generator="blob_series", shape=(48, 48, 48), n_sessions=3, n_levels=1, steps=[20], K=6,
               window=5, name="c1 tiny: 3 x 48^3 blob phantoms, 1 level x 20 steps, K=6, w=5, SiLNCC"),
    # the metric's configuration: 10 x 160x192x160, 4 levels x 100 steps, K=7, w=7, SiLNCC
    "c2": dict(kind="plain", generator="brain_series", shape=(160, 192, 160), n_sessions=10, n_levels=4,
               steps=[100, 100, 100, 100], K=7, window=7,
               name="c2 realistic: 10 x 160x192x160, 4 levels x 100 steps, K=7, w=7, SiLNCC"),
    # served: Poisson stream of subjects with uneven session counts and shapes
    "c4": dict(kind="serve", generator="brain_series", n_jobs=64, rate=2.0, n_min=2, n_max=12,
               shapes=[(128, 128, 128), (160, 192, 160), (192, 224, 192)], n_levels=4, steps=[100, 100, 100, 100],
               K=7, window=7, shape=(160, 192, 160), n_sessions=12,
               name="c4 served: Poisson 2 jobs/s, 64 subjects, N 2..12, shapes {128^3, 160x192x160, 192x224x192}, "
                    "4 levels x 100 steps, K=7, w=7, SiLNCC"),
    # large series: 16 x 256^3, K=8, w=9, squaring intermediates recomputed
    "c5": dict(kind="plain", generator="brain_series", shape=(256, 256, 256), n_sessions=16, n_levels=4,
               steps=[100, 100, 100, 100], K=8, window=9, recompute=1,
               name="c5 large: 16 x 256^3, 4 levels x 100 steps, K=8, w=9, SiLNCC, recomputed squarings"),
    # Jacobian determinant maps and deformation metrics of the 9 session displacements of a
    # 10 x 160x192x160 series (the phantom's ground truth against a perturbed estimate)
    "jacobian": dict(kind="jacobian", generator="brain_series", shape=(160, 192, 160), n_sessions=10, n_levels=1,
                     steps=[1], K=7, window=7,
                     name="jacobian maps + metrics: 9 displacement fields of 160x192x160 (c2 series)"),
    # session-count sweep: the first N sessions of one 12-session series, N = 2, 4, ..., 12,
    # registration throughput and accuracy against the phantom's ground truth
    "sweep": dict(kind="sweep", generator="brain_series", shape=(160, 192, 160), n_sessions=12, n_levels=4,
                  steps=[100, 100, 100, 100], K=7, window=7, counts=[2, 4, 6, 8, 10, 12],
                  name="session-count sweep: N = 2..12 of a 12 x 160x192x160 series, c2 schedule"),
    # small case for ncu captures (128^3 volumes): 6 x 128^3, 1 level x 2 steps, K=7, w=7
    "profile": dict(kind="plain", generator="brain_series", shape=(128, 128, 128), n_sessions=6, n_levels=1,
                    steps=[2], K=7, window=7, name="profile: 6 x 128^3, 1 level x 2 steps, K=7, w=7, SiLNCC"),
}
WORKLOAD = WORKLOADS["c2"]
PARAMS = dict(n_levels=4, steps_per_level=[100, 100, 100, 100], n_squarings=7, window=7, similarity=0,
              alpha_ss=0.05, alpha_l2=0.005, alpha_ts=0.0, lr=0.05)


def select_workload(name):
    global WORKLOAD, PARAMS
    WORKLOAD = WORKLOADS[name]
    PARAMS = dict(PARAMS, n_levels=WORKLOAD["n_levels"], steps_per_level=list(WORKLOAD["steps"]),
                  n_squarings=WORKLOAD["K"], window=WORKLOAD["window"],
                  recompute_squaring=WORKLOAD.get("recompute", 0))


def load_series(seed):
    from paper_2412_14671_gb300 import phantom

    return phantom.cached(WORKLOAD["generator"], shape=WORKLOAD["shape"], n_sessions=WORKLOAD["n_sessions"],
                          seed=seed)


METRIC = "Gvoxel-iters/s fwd+adjoint (ordered-pair voxels x gradient steps / s, whole registration)"
UNIT = "Gvoxel-iters/s"
FALLBACK_HBM_GBS = 6800.0


def level_dims(shape, n_levels):
    dims = [tuple(shape)]
    for _ in range(n_levels - 1):
        dims.append(tuple((a + 1) // 2 for a in dims[-1]))
    return dims[::-1]


def units_per_registration(shape=None, n_sessions=None):
    N = n_sessions or WORKLOAD["n_sessions"]
    P = N * (N - 1)
    dims = level_dims(shape or WORKLOAD["shape"], WORKLOAD["n_levels"])
    return sum(s * P * int(np.prod(d)) for s, d in zip(WORKLOAD["steps"], dims))


L2_BYTES = 129 * 2**20


def resident_bytes(reg):
    """Images of every level plus the velocity-sized state the step reads and writes."""
    N = reg.n_sessions
    img = sum(N * int(np.prod(reg.level_dims(l)[0])) for l in range(reg.params.n_levels))
    top = reg.params.n_levels - 1
    flow = int(np.prod(reg.level_dims(top)[1]))
    return 4 * img + 4 * 4 * (N - 1) * flow * 6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def max_over_ranks(x, ws, device):
    """Largest value of x over the ranks (the whole job ends with its slowest replica)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, steps, ms_max, ws):
    """Whole-job Gvoxel-iters/s: every rank registers its own subject (replicas), so the
    job does ws x units x steps in the slowest rank's time."""
    return ws * units_per_rank * steps / (ms_max / 1e3) / 1e9


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
                except ValueError:
                    continue
                for name, val in zip(names, f[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_text(src, name):
    """Source text of the kernel template `name` in file `src`: from the template line
    before its definition to the matching closing brace."""
    text = open(src).read()
    i = text.index(" " + name + "(")
    start = text.rfind("template", 0, i)
    depth, k = 0, text.index("{", i)
    for p in range(k, len(text)):
        if text[p] == "{":
            depth += 1
        elif text[p] == "}":
            depth -= 1
            if depth == 0:
                return text[start:p + 1]
    raise ValueError("unbalanced braces in " + src)


def traffic_record():
    """DRAM bytes per unit of the top kernel from the committed ncu summary
    (profiles/traffic.txt, "key: value" lines), if the kernel's own source text has not
    changed since the capture (function_sha1: SHA-1 of kernel_text)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        rec = {}
        with open(path) as fh:
            for line in fh:
                k, sep, v = line.partition(":")
                if sep and k.strip() and not k.startswith("#"):
                    rec[k.strip()] = v.strip()
        for k in ("dram_bytes_per_unit", "algorithmic_bytes_per_unit"):
            rec[k] = float(rec[k])
        src = os.path.join(ROOT, "paper_2412_14671_gb300", "csrc", rec["source"])
        h = hashlib.sha1(kernel_text(src, rec["function"]).encode()).hexdigest()[:12]
        return rec if h == rec.get("function_sha1") else None
    except Exception:
        return None


# ----------------------------------------------------------------------------- oracle (CPU) legs
def oracle_sample(imgs, level_index, n_levels=4):
    """One fwd+adjoint+update step of the FP64 oracle at one pyramid level, all pairs.
    Returns (seconds, pair-voxel-iters)."""
    import oracle

    lv = imgs.astype(np.float64)
    dims = level_dims(imgs.shape[1:], n_levels)
    for _ in range(n_levels - 1 - level_index):
        lv = np.stack([oracle.downsample2(x) for x in lv])
    N = lv.shape[0]
    ni = lv.shape[1:]
    assert tuple(ni) == tuple(dims[level_index])
    nf = tuple((a + 1) // 2 for a in ni)
    p = oracle.params(n_levels=1, steps=(1,), K=PARAMS["n_squarings"], window=PARAMS["window"],
                      alpha_ss=PARAMS["alpha_ss"], alpha_l2=PARAMS["alpha_l2"], alpha_ts=0.0, lr=PARAMS["lr"])
    theta = np.zeros((N - 1, 3) + nf)
    m1, v1 = np.zeros_like(theta), np.zeros_like(theta)
    t0 = time.perf_counter()
    _, _, g = oracle.loss_grad(lv, theta, p)
    oracle.adam_step(theta, m1, v1, g, 1, oracle.lr_at(1, 100, PARAMS["lr"]))
    dt = time.perf_counter() - t0
    return dt, N * (N - 1) * int(np.prod(ni))


def method_bytes():
    """Bytes per registration of the method's own compulsory traffic (no intermediate is
    stored): per step 11 B per ordered pair-voxel (fixed image, warped gather, the pair
    displacement and its gradient on the flow grid), 108 B per flow voxel per squaring per
    exponential field (forward and adjoint), 144 B per flow voxel per composed map and
    120 B per flow voxel per velocity field (regulariser and Adam), summed over the
    schedule. Returns (all steps, the pair part)."""
    N, K = WORKLOAD["n_sessions"], WORKLOAD["K"]
    P, C = N * (N - 1), (N - 1) * (N - 2)
    tot = pair = 0.0
    for T, ni in zip(WORKLOAD["steps"], level_dims(WORKLOAD["shape"], WORKLOAD["n_levels"])):
        V = float(np.prod(ni))
        v = float(np.prod([(a + 1) // 2 for a in ni]))
        pb = 11.0 * P * V
        tot += T * (pb + 108.0 * 2 * (N - 1) * K * v + 144.0 * C * v + 120.0 * (N - 1) * v)
        pair += T * pb
    return tot, pair


PAIR_KERNELS = ("warp", "sim_fwd", "sim_bwd", "warp_bwd")


def sample_level(max_pair_voxels):
    """Finest pyramid level whose one oracle step covers at most max_pair_voxels."""
    N = WORKLOAD["n_sessions"]
    dims = level_dims(WORKLOAD["shape"], WORKLOAD["n_levels"])
    ok = [l for l, d in enumerate(dims) if N * (N - 1) * int(np.prod(d)) <= max_pair_voxels]
    return ok[-1] if ok else 0


def cores_used():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def run_reference(args):
    rank, _, ws = dist_env()
    if rank != 0:
        return 0
    imgs = load_series(0)["images"]
    level = sample_level(1e7)  # c2: 40x48x40 images, a bounded sample per step
    for _ in range(args.warmup):
        oracle_sample(imgs, level, WORKLOAD["n_levels"])
    tot_t, tot_u = 0.0, 0
    for _ in range(args.steps):
        dt, u = oracle_sample(imgs, level, WORKLOAD["n_levels"])
        tot_t += dt
        tot_u += u
    value = tot_u / tot_t / 1e9
    dims = level_dims(WORKLOAD["shape"], WORKLOAD["n_levels"])[level]
    N = WORKLOAD["n_sessions"]
    sample = "one FP64 fwd+adjoint+Adam step per timed step at pyramid level %d of %d (%dx%dx%d images), all %d pairs" % (
        (level + 1, WORKLOAD["n_levels"]) + dims + (N * (N - 1),))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores_used(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU leg
def run_gpu(args):
    import torch

    rank, local_rank, ws = dist_env()
    torch.cuda.set_device(local_rank)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import paper_2412_14671_gb300 as m

    series = load_series(rank)
    imgs_host = torch.from_numpy(series["images"]).pin_memory()
    imgs_dev = imgs_host.cuda()
    N = WORKLOAD["n_sessions"]
    tuning = autotune_problem(WORKLOAD["shape"], N, imgs_dev, args)
    reg = m.Muster(WORKLOAD["shape"], N, **PARAMS)
    reg.set_images(imgs_dev)
    stream = torch.cuda.current_stream()
    units = units_per_registration()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up (untimed)
    warm_ms = []
    for _ in range(args.warmup):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        reg.run()
        b.record(stream)
        torch.cuda.synchronize()
        warm_ms.append(a.elapsed_time(b))
    # Timed region: K whole registrations, each bracketed by CUDA events on the launching
    # stream. When the images and fields of a step fit in L2 a >129 MB buffer is
    # written between steps, outside the bracketed intervals.
    flush = None
    if resident_bytes(reg) < 2 * L2_BYTES:
        flush = torch.empty(L2_BYTES // 2, dtype=torch.float32, device="cuda")

    def timed_steps(k):
        evs, out = [], None
        for _ in range(k):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = reg.run()
            b.record(stream)
            evs.append((a, b))
            if flush is not None:
                flush.fill_(1.0)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs), out

    clocks = Clocks(local_rank)
    barrier()
    clocks.start()
    reg.profile_begin()
    ms, final = timed_steps(args.steps)
    barrier()
    stats = reg.profile_end()
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws, "cuda")
    value = replica_throughput(units, args.steps, ms, ws)
    # the same steps without per-launch events (CUDA-graph replays), for context
    barrier()
    ms_np, _ = timed_steps(args.steps)
    value_unprofiled = units * args.steps / (ms_np / 1e3) / 1e9
    # and, for context, the other adjoint mode (reproducible or atomic) on two registrations
    other = None
    if WORKLOAD["kind"] == "plain":
        alt = m.Muster(WORKLOAD["shape"], N, **dict(PARAMS, deterministic=1 - PARAMS.get("deterministic", 0)))
        alt.set_images(imgs_dev)
        alt.run()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(2):
            alt.run()
        b.record(stream)
        barrier()
        other = {"deterministic": 1 - PARAMS.get("deterministic", 0),
                 "value": units * 2 / (a.elapsed_time(b) / 1e3) / 1e9, "registrations": 2}
        alt.close()

    # end to end through the public API with host buffers: H2D images, registration, D2H velocities
    e2e_steps = max(1, min(args.steps, 3))
    top = WORKLOAD["n_levels"] - 1
    vel_host = torch.empty((N - 1, 3) + reg.level_dims(top)[1], dtype=torch.float32).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        reg.set_images(imgs_host.numpy())
        reg.run()
        for k in range(N - 1):
            vel_host[k].copy_(torch.from_numpy(reg.get_field(m.VELOCITY, k, level=top, device=False)))
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, ws, "cuda")
    e2e_value = replica_throughput(units, e2e_steps, e2e_ms, ws)

    if rank == 0:
        hbm, src = peaks()
        top = max(stats, key=lambda s: s["ms"])
        launches = sum(s["all_launches"] for s in stats)
        per_launch_bytes = top["bytes"] / max(top["launches"], 1)
        achieved = top["bytes"] / (top["ms"] / 1e3) / 1e9 if top["ms"] > 0 else 0.0
        tr = traffic_record()
        traffic = None
        if tr and tr.get("kernel") == top["name"]:
            # captured on a smaller case: DRAM bytes per unit x the units of the mean launch here
            traffic = tr["dram_bytes_per_unit"] * per_launch_bytes / tr["algorithmic_bytes_per_unit"]
        total_ms = sum(s["ms"] for s in stats)
        kernels = {s["name"]: {"launches": s["all_launches"], "timed_launches": s["launches"],
                               "ms": round(s["ms"], 3),
                               "share": round(s["ms"] / total_ms, 4) if total_ms else 0.0,
                               "GBps": round(s["bytes"] / (s["ms"] / 1e3) / 1e9, 1) if s["ms"] > 0 else None}
                   for s in stats if s["all_launches"]}
        # CPU baseline: the oracle on a bounded sample (one step at a level of about 7e7 pair-voxels at
        # most), in single-GPU runs only
        lvl = sample_level(7e7)
        cpu = None
        if not args.no_cpu and ws == 1:
            dt, u = oracle_sample(series["images"], lvl, WORKLOAD["n_levels"])
            dims = level_dims(WORKLOAD["shape"], WORKLOAD["n_levels"])[lvl]
            cpu = {"value": u / dt / 1e9, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                   "sample": "one FP64 fwd+adjoint+Adam step at pyramid level %d of %d (%dx%dx%d images), "
                             "all %d pairs, %.1f s" % ((lvl + 1, WORKLOAD["n_levels"]) + dims + (N * (N - 1), dt))}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded brain-like phantom series)",
            "config": {"workload": WORKLOAD["name"], "deterministic": PARAMS.get("deterministic", 0),
                       "units_per_step": units, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": ("L2 flushed between timed steps (%.0f MB resident)" if flush is not None else
                              "inputs larger than L2 (%.0f MB of images and fields resident)") % (resident_bytes(reg) / 1e6),
                       "value_unprofiled": value_unprofiled,
                       "other_adjoint_mode": other,
                       "autotune": tuning,
                       "final_loss": final, "warmup_ms": [round(w, 1) for w in warm_ms],
                       "profiled": "CUDA events around every kernel of one graph-replayed step in %d and "
                                   "of the eager steps, during the timed region; roofline and shares "
                                   "from the timed launches" % 8},
            "roofline": {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": hbm,
                         "peak_source": src, "unit": "GB/s", "frac": achieved / hbm,
                         "algorithmic_bytes_per_launch": per_launch_bytes,
                         "avg_launch_ms": top["ms"] / max(top["launches"], 1), "traffic": traffic,
                         "method_basis": method_basis(stats, ms / args.steps, hbm)},
            "kernels": kernels,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(imgs_host.numel() * 4),
                    "d2h_bytes_per_step": int(vel_host.numel() * 4), "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line))
    reg.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def method_basis(stats, ms_per_registration, hbm):
    """The method's own bytes (method_bytes) over the measured time: for the whole
    registration, and for the pair path over the share of device time its four kernels
    took in the timed launches."""
    tot, pair = method_bytes()
    total_ms = sum(s["ms"] for s in stats) or 1.0
    pair_share = sum(s["ms"] for s in stats if s["name"] in PAIR_KERNELS) / total_ms
    step_gbs = tot / (ms_per_registration / 1e3) / 1e9
    pair_gbs = pair / (pair_share * ms_per_registration / 1e3) / 1e9 if pair_share > 0 else 0.0
    return {"bytes_per_registration": tot, "achieved": step_gbs, "frac": step_gbs / hbm,
            "pair_path_bytes_per_registration": pair, "pair_path_share": pair_share,
            "pair_path_achieved": pair_gbs, "pair_path_frac": pair_gbs / hbm,
            "basis": "11 B per pair-voxel, 108 B per flow voxel per squaring per field, 144 B per flow "
                     "voxel per composed map, 120 B per flow voxel per velocity field, per step"}


def autotune_problem(shape, n, images, args):
    """Chooses the launch configuration of the problem (paper_2412_14671_gb300.autotune:
    short registrations of the problem timed on the device, before any timed step) and
    applies it to PARAMS. Returns what the bench line reports about it."""
    if args.no_tune:
        return None
    from paper_2412_14671_gb300 import autotune

    t0 = time.perf_counter()
    res = autotune.tune(shape, n, PARAMS, images=images)
    PARAMS.update(autotune.knob_params(res["choice"], n))
    return {"choice": res["choice"], "cached": res["cached"], "seconds": round(time.perf_counter() - t0, 2),
            "trials_ms": [[k, v, round(ms, 3)] for k, v, ms in res["trials"]],
            "how": "coordinate search from the defaults over flow_nf, chunk_pct, pair_batch; short "
                   "registrations of the problem (4 steps per level), best of 2 after one untimed run"}


# ----------------------------------------------------------------------------- served workload
def _series_for_shape(args):
    shape, n, seed = args
    from paper_2412_14671_gb300 import phantom

    phantom.cached("brain_series", shape=shape, n_sessions=n, seed=seed)
    return shape


def serve_jobs(n_jobs, seed):
    """The subjects of the served workload: arrival times (Poisson), session counts
    (uniform), shapes (uniform over the set) and images. Each shape has one seeded
    brain-like series of n_max sessions; a subject takes N consecutive sessions of it
    from a random start. Phantoms are generated in spawned processes (no CUDA yet)."""
    import multiprocessing as mp

    from paper_2412_14671_gb300 import phantom
    from paper_2412_14671_gb300.serve import Job, poisson_arrivals

    W = WORKLOAD
    rng = np.random.default_rng([20241219, 5, seed])
    arrivals = poisson_arrivals(n_jobs, W["rate"], seed=seed)
    Ns = rng.integers(W["n_min"], W["n_max"] + 1, size=n_jobs)
    shape_idx = rng.integers(0, len(W["shapes"]), size=n_jobs)
    starts = [int(rng.integers(0, W["n_max"] - n + 1)) for n in Ns]
    todo = [(tuple(W["shapes"][k]), W["n_max"], 100 * seed + k) for k in sorted(set(shape_idx.tolist()))]
    with mp.get_context("spawn").Pool(len(todo)) as pool:
        pool.map(_series_for_shape, todo)
    series = {k: phantom.cached("brain_series", shape=tuple(W["shapes"][k]), n_sessions=W["n_max"],
                                seed=100 * seed + k)["images"] for k in set(shape_idx.tolist())}
    jobs = []
    for i in range(n_jobs):
        imgs = np.ascontiguousarray(series[int(shape_idx[i])][starts[i]:starts[i] + int(Ns[i])])
        jobs.append(Job(i, imgs, dict(PARAMS), arrival=float(arrivals[i])))
    return jobs


def run_serve(args):
    """Served subjects per hour and p50/p99 latency of a Poisson stream of subjects, with
    continuous batching (args.max_active concurrent jobs) and, on the same stream, the
    plain one-subject-at-a-time path; the two must agree on every subject's result."""
    rank, local_rank, ws = dist_env()
    n_jobs = args.jobs or WORKLOAD["n_jobs"]
    jobs = serve_jobs(n_jobs, seed=rank)  # CPU work before the first CUDA call
    import torch

    torch.cuda.set_device(local_rank)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2412_14671_gb300.serve import EngineBackend, Job, MusterServer, serve_plain, summary

    # launch configuration per shape: tuned on the subject of that shape whose session count
    # is nearest the middle of the range, applied to every subject of the shape
    tuning = {}
    if not args.no_tune:
        from paper_2412_14671_gb300 import autotune

        mid = (WORKLOAD["n_min"] + WORKLOAD["n_max"]) / 2.0
        t0 = time.perf_counter()
        for shape in sorted({tuple(j.images.shape[1:]) for j in jobs}):
            rep = min((j for j in jobs if tuple(j.images.shape[1:]) == shape),
                      key=lambda j: (abs(j.images.shape[0] - mid), j.id))
            res = autotune.tune(shape, rep.images.shape[0], PARAMS, images=rep.images)
            tuning["x".join(map(str, shape))] = {"sessions": int(rep.images.shape[0]), "choice": res["choice"]}
        for j in jobs:
            j.params = autotune.tuned_params(j.images.shape[1:], j.images.shape[0], j.params)
        tuning["seconds"] = round(time.perf_counter() - t0, 1)
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(args.budget_gb * 2**30, free - 8 * 2**30))
    units = {j.id: units_per_registration(j.images.shape[1:], j.images.shape[0]) for j in jobs}
    total_units = sum(units.values())

    def serve(max_active, quantum, stream_jobs):
        srv = MusterServer(EngineBackend(local_rank, max_active=max_active), budget, max_active=max_active,
                           quantum=quantum)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = srv.run(stream_jobs)
        torch.cuda.synchronize()
        makespan = time.perf_counter() - t0
        info = dict(created=srv.created, reused=srv.reused, evicted=srv.evicted, peak_active=srv.peak_active,
                    peak_in_use_gb=round(srv.peak_in_use / 2**30, 2))
        srv.close()
        return res, makespan, info

    # warm-up: one small subject per shape through a server (library load, kernel set-up)
    warm = [Job(-1 - k, j.images[:2].copy(), dict(PARAMS, steps_per_level=[3] * WORKLOAD["n_levels"]))
            for k, j in enumerate({tuple(j.images.shape[1:]): j for j in jobs}.values())]
    for _ in range(max(1, args.warmup)):
        serve(2, 4, warm)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_1 = serve_plain(jobs)  # the plain path: one subject at a time, a new context each
    torch.cuda.synchronize()
    span_1 = time.perf_counter() - t0
    info_1 = {}
    barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    res_b, span_b, info_b = serve(args.max_active, args.quantum, jobs)
    clk = clocks.stop()
    barrier()
    # the same subject gives the same result alone and in the mix
    dv = max(float(np.abs(a.velocities - b.velocities).max()) for a, b in zip(res_1, res_b))
    dl = max(abs(a.final_loss - b.final_loss) / max(abs(a.final_loss), 1e-30) for a, b in zip(res_1, res_b))
    s1, sb = summary(res_1, span_1), summary(res_b, span_b)
    tot = [sb["subjects"], span_b, s1["subjects"], span_1]
    if ws > 1:
        tot = [sb["subjects"] * ws, max_over_ranks(span_b, ws, "cuda"), s1["subjects"] * ws,
               max_over_ranks(span_1, ws, "cuda")]
    if rank == 0:
        value = 3600.0 * tot[0] / tot[1]
        h2d = sum(j.images.nbytes for j in jobs) / len(jobs)
        d2h = sum(r.velocities.nbytes for r in res_b) / len(res_b)
        line = {
            "metric": "served subjects/hr (continuous batching), p50/p99 latency", "value": value,
            "unit": "subjects/hr", "n_gpus": ws, "steps": 1, "warmup": max(1, args.warmup),
            "ms_per_step": 1e3 * tot[1], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded brain-like phantom series)",
            "config": {"workload": WORKLOAD["name"], "subjects": n_jobs, "max_active": args.max_active,
                       "deterministic": PARAMS.get("deterministic", 0),
                       "quantum_steps": args.quantum, "budget_gb": round(budget / 2**30, 1),
                       "autotune": tuning or None,
                       "l2": "inputs larger than L2 (every subject >= 33 MB of images plus its fields)"},
            "serving": {
                "batched": dict(sb, **info_b, gvoxel_iters_per_s=total_units / span_b / 1e9),
                "plain_one_at_a_time": dict(s1, **info_1, gvoxel_iters_per_s=total_units / span_1 / 1e9),
                "speedup_subjects_per_hour": (3600.0 * tot[0] / tot[1]) / (3600.0 * tot[2] / tot[3]),
                "max_abs_velocity_diff_vox": dv, "max_rel_loss_diff": dl,
            },
            "e2e": {"value": value, "unit": "subjects/hr", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "note": "each subject: host images in, registration, host velocities out"},
            "clocks": clk,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- session-count sweep
def run_sweep(args):
    """Registration of the first N sessions of one series for each N: Gvoxel-iters/s and
    the Sec. Evaluation Metrics of every session's displacement (pair k -> 0 pulled onto
    grid k) against the phantom's ground truth over the head (intensity > 0.1), averaged
    over the sessions."""
    rank, local_rank, ws = dist_env()
    from paper_2412_14671_gb300 import phantom

    s = phantom.cached("brain_series", shape=WORKLOAD["shape"], n_sessions=WORKLOAD["n_sessions"], seed=rank,
                       return_truth=True)
    import torch

    torch.cuda.set_device(local_rank)
    import paper_2412_14671_gb300 as m

    imgs_all, truth = s["images"], s["truth_disp"]
    top = WORKLOAD["n_levels"] - 1
    rows = []
    stream = torch.cuda.current_stream()
    clocks = Clocks(local_rank)
    clocks.start()
    for N in WORKLOAD["counts"]:
        imgs = torch.from_numpy(np.ascontiguousarray(imgs_all[:N])).cuda()
        with m.Muster(WORKLOAD["shape"], N, **PARAMS) as reg:
            reg.set_images(imgs)
            for _ in range(max(1, args.warmup)):
                reg.run()
            ms = []
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                reg.run()
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            acc = []
            # ROI: the head in session k (the background carries no information on the motion)
            for k in range(1, N):
                est = reg.get_field(m.PAIR_DISP, k, 0, level=top)  # pulls session 0 onto grid k
                roi = torch.from_numpy(imgs_all[k] > 0.1).cuda()
                acc.append(m.op_deformation_metrics(torch.from_numpy(truth[k]).cuda(), est, roi))
        units = units_per_registration(WORKLOAD["shape"], N)
        t = statistics.median(ms)
        rows.append({"N": N, "Gvoxel_iters_per_s": units / (t / 1e3) / 1e9, "registration_s": t / 1e3,
                     "Eu": float(np.mean([a["Eu"] for a in acc])), "PCC": float(np.mean([a["PCC"] for a in acc])),
                     "B": float(np.mean([a["B"] for a in acc]))})
    clk = clocks.stop()
    if rank == 0:
        tot_units = sum(units_per_registration(WORKLOAD["shape"], r["N"]) for r in rows)
        tot_s = sum(r["registration_s"] for r in rows)
        line = {
            "metric": "Gvoxel-iters/s over a session-count sweep (and accuracy vs ground truth)", "unit": "Gvoxel-iters/s",
            "value": tot_units / tot_s / 1e9, "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup),
            "ms_per_step": 1e3 * tot_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded brain-like phantom series with ground-truth displacements)",
            "config": {"workload": WORKLOAD["name"], "l2": "inputs larger than L2 (39 MB or more of images per N)",
                       "per_N": rows},
            "clocks": clk,
        }
        print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- Jacobian maps
def run_jacobian(args):
    """Jacobian determinant maps (det(I + grad u), 12 B read + 4 B written per voxel) and the
    deformation metrics of every session displacement of the series, fields resident."""
    rank, local_rank, ws = dist_env()
    from paper_2412_14671_gb300 import phantom

    s = phantom.cached("brain_series", shape=WORKLOAD["shape"], n_sessions=WORKLOAD["n_sessions"], seed=rank,
                       return_truth=True)
    truth = s["truth_disp"][1:]  # (N-1, 3, D, H, W): session k -> session 0
    rng = np.random.default_rng([20241219, 6, rank])
    est = (0.9 * truth + 0.05 * rng.standard_normal(truth.shape, dtype=np.float32)).astype(np.float32)
    import torch

    torch.cuda.set_device(local_rank)
    import paper_2412_14671_gb300 as m

    ut, ue = torch.from_numpy(truth).cuda(), torch.from_numpy(est).cuda()
    F = ut.shape[0]
    V = int(np.prod(ut.shape[2:]))
    J = torch.empty((F,) + tuple(ut.shape[2:]), device="cuda")
    stream = torch.cuda.current_stream()

    def one_step(evj, evm):
        for f in range(F):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m.op_jacobian_det(ue[f], out=J[f])
            b.record(stream)
            evj.append((a, b))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = [m.op_deformation_metrics(ut[f], ue[f]) for f in range(F)]
        b.record(stream)
        evm.append((a, b))
        return res

    for _ in range(args.warmup):
        one_step([], [])
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.start()
    evj, evm = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = one_step(evj, evm)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    # end to end: the estimate fields from pinned host memory, the maps back to pinned host memory
    est_h = torch.from_numpy(est).pin_memory()
    J_h = torch.empty(J.shape, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(args.steps):
        dev = est_h.to("cuda", non_blocking=True)
        for f in range(F):
            m.op_jacobian_det(dev[f], out=J[f])
        J_h.copy_(J, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(h0.elapsed_time(h1), ws, "cuda")
    jac_ms = sum(a.elapsed_time(b) for a, b in evj) / len(evj)
    met_ms = sum(a.elapsed_time(b) for a, b in evm) / len(evm)
    if rank == 0:
        hbm, src = peaks()
        cpu = None
        if not args.no_cpu and ws == 1:
            import oracle

            t0 = time.perf_counter()
            oracle.jacobian_det(est[0])
            dt = time.perf_counter() - t0
            cpu = {"value": V / dt / 1e9, "unit": "Gvoxel/s", "cores": cores_used(), "kind": "oracle",
                   "sample": "one FP64 Jacobian determinant map of a 160x192x160 field, %.2f s" % dt}
        bytes_per_launch = 16.0 * V
        line = {
            "metric": "Jacobian determinant maps (Gvoxel/s) and deformation metrics", "unit": "Gvoxel/s",
            "value": ws * F * V * args.steps / (total_ms / 1e3) / 1e9, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (metric sums: double-float per thread, f64 across CTAs)",
            "data": "synthetic (ground-truth displacements of the seeded brain-like phantom series)",
            "config": {"workload": WORKLOAD["name"], "fields": F,
                       "l2": "inputs larger than L2 (%d fields of 59 MB resident)" % (2 * F),
                       "jacobian_ms_per_field": jac_ms, "metrics_ms_per_field": met_ms / F,
                       "metrics_example": {k: (float(v) if np.isscalar(v) else None) for k, v in res[-1].items()}},
            "roofline": {"bound": "hbm", "kernel": "jacobian_det", "achieved": bytes_per_launch / (jac_ms / 1e3) / 1e9,
                         "peak": hbm, "peak_source": src, "unit": "GB/s",
                         "frac": bytes_per_launch / (jac_ms / 1e3) / 1e9 / hbm,
                         "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": jac_ms, "traffic": None},
            "cpu_baseline": cpu,
            "e2e": {"value": ws * F * V * args.steps / (e2e_ms / 1e3) / 1e9, "unit": "Gvoxel/s",
                    "h2d_bytes_per_step": int(est_h.numel() * 4), "d2h_bytes_per_step": int(J_h.numel() * 4),
                    "note": "Jacobian maps only: fields in from pinned host memory, maps out"},
            "gpu_launches": args.steps * F * 5,
            "clocks": clk,
        }
        print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--max-active", type=int, default=3, help="served workload: concurrent jobs")
    ap.add_argument("--quantum", type=int, default=25, help="served workload: steps issued per job per pump")
    ap.add_argument("--budget-gb", type=float, default=200.0, help="served workload: HBM budget for contexts")
    ap.add_argument("--jobs", type=int, default=0, help="served workload: number of subjects (0 = workload's)")
    ap.add_argument("--deterministic", action="store_true",
                    help="exact fixed-point sums in the scatter adjoints: bit-reproducible (the served default)")
    ap.add_argument("--atomic", action="store_true", help="floating-point reductions in the scatter adjoints")
    ap.add_argument("--no-tune", action="store_true", help="library default launch configuration (no autotuner)")
    args = ap.parse_args()
    select_workload(args.workload)
    # the served workload compares each subject alone and in the mix: reproducible by default
    det = WORKLOAD["kind"] == "serve"
    if args.deterministic:
        det = True
    if args.atomic:
        det = False
    PARAMS["deterministic"] = int(det)
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOAD["kind"] == "serve":
        return run_serve(args)
    if WORKLOAD["kind"] == "jacobian":
        return run_jacobian(args)
    if WORKLOAD["kind"] == "sweep":
        return run_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
