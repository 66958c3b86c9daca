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
    # config 2 (the metric's configuration): 10 x 160x192x160, 4 levels x 100 steps, K=7, w=7, SiLNCC
    "c2": dict(shape=(160, 192, 160), n_sessions=10, n_levels=4, steps=[100, 100, 100, 100], K=7, window=7,
               name="c2 realistic: 10 x 160x192x160, 4 levels x 100 steps, K=7, w=7, SiLNCC"),
    # small case for ncu captures (config-3 volume): 6 x 128^3, 1 level x 2 steps, K=7, w=7
    "profile": dict(shape=(128, 128, 128), n_sessions=6, n_levels=1, steps=[2], K=7, window=7,
                    name="profile: 6 x 128^3, 1 level x 2 steps, K=7, w=7, SiLNCC"),
}
WORKLOAD = WORKLOADS["c2"]
PARAMS = dict(n_levels=4, steps_per_level=[100, 100, 100, 100], n_squarings=7, window=7, similarity=0,
              alpha_ss=0.05, alpha_l2=0.005, alpha_ts=0.0, lr=0.05)


def select_workload(name):
    global WORKLOAD, PARAMS
    WORKLOAD = WORKLOADS[name]
    PARAMS = dict(PARAMS, n_levels=WORKLOAD["n_levels"], steps_per_level=list(WORKLOAD["steps"]),
                  n_squarings=WORKLOAD["K"], window=WORKLOAD["window"])
METRIC = "Gvoxel-iters/s fwd+adjoint (ordered-pair voxels x gradient steps / s, whole registration)"
UNIT = "Gvoxel-iters/s"
FALLBACK_HBM_GBS = 6800.0


def level_dims(shape, n_levels):
    dims = [tuple(shape)]
    for _ in range(n_levels - 1):
        dims.append(tuple((a + 1) // 2 for a in dims[-1]))
    return dims[::-1]


def units_per_registration():
    N = WORKLOAD["n_sessions"]
    P = N * (N - 1)
    return sum(s * P * int(np.prod(d)) for s, d in zip(WORKLOAD["steps"], level_dims(WORKLOAD["shape"], WORKLOAD["n_levels"])))


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


def traffic_record():
    """DRAM bytes per launch from the committed ncu summary, if it still matches the kernels."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        src = os.path.join(ROOT, "paper_2412_14671_gb300", "csrc", rec["source"])
        h = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
        return rec if h == rec.get("source_sha1") else None
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


def cores_used():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def run_reference(args):
    rank, _, ws = dist_env()
    if rank != 0:
        return 0
    from paper_2412_14671_gb300 import phantom

    s = phantom.cached("brain_series", shape=WORKLOAD["shape"], n_sessions=WORKLOAD["n_sessions"], seed=0)
    imgs = s["images"]
    level = max(0, WORKLOAD["n_levels"] - 3)  # c2: 40x48x40 images, a bounded sample per step
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
    from paper_2412_14671_gb300 import phantom

    series = phantom.cached("brain_series", shape=WORKLOAD["shape"], n_sessions=WORKLOAD["n_sessions"], seed=rank)
    imgs_host = torch.from_numpy(series["images"]).pin_memory()
    imgs_dev = imgs_host.cuda()
    N = WORKLOAD["n_sessions"]
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
    # timed region: inputs resident in HBM (197 MB of images > 129 MB L2)
    clocks = Clocks(local_rank)
    barrier()
    clocks.start()
    reg.profile_begin()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    final = None
    for _ in range(args.steps):
        final = reg.run()
    ev1.record(stream)
    barrier()
    stats = reg.profile_end()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * units * args.steps / (ms / 1e3) / 1e9

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
    if ws > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = ws * units * e2e_steps / (e2e_ms / 1e3) / 1e9

    if rank == 0:
        hbm, src = peaks()
        top = max(stats, key=lambda s: s["ms"])
        launches = sum(s["launches"] for s in stats)
        per_launch_bytes = top["bytes"] / max(top["launches"], 1)
        achieved = top["bytes"] / (top["ms"] / 1e3) / 1e9 if top["ms"] > 0 else 0.0
        tr = traffic_record()
        traffic = tr["dram_bytes_per_launch"] if tr and tr.get("kernel") == top["name"] else None
        total_ms = sum(s["ms"] for s in stats)
        kernels = {s["name"]: {"launches": s["launches"], "ms": round(s["ms"], 3),
                               "share": round(s["ms"] / total_ms, 4) if total_ms else 0.0,
                               "GBps": round(s["bytes"] / (s["ms"] / 1e3) / 1e9, 1) if s["ms"] > 0 else None}
                   for s in stats if s["launches"]}
        # CPU baseline: the oracle on a bounded sample (one step at the level with 1/8 of the voxels)
        lvl = max(0, WORKLOAD["n_levels"] - 2)
        cpu = None
        if not args.no_cpu:
            dt, u = oracle_sample(series["images"], lvl, WORKLOAD["n_levels"])
            dims = level_dims(WORKLOAD["shape"], WORKLOAD["n_levels"])[lvl]
            cpu = {"value": u / dt / 1e9, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                   "sample": "one FP64 fwd+adjoint+Adam step at pyramid level %d of %d (%dx%dx%d images), "
                             "all %d pairs, %.1f s" % ((lvl + 1, WORKLOAD["n_levels"]) + dims + (N * (N - 1), dt))}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded brain-like phantom series)",
            "config": {"workload": WORKLOAD["name"],
                       "units_per_step": units, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (197 MB of images, 1.3 GB of fields per step)",
                       "final_loss": final, "warmup_ms": [round(w, 1) for w in warm_ms],
                       "profiled": "per-launch CUDA events during the timed region"},
            "roofline": {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": hbm,
                         "peak_source": src, "unit": "GB/s", "frac": achieved / hbm,
                         "algorithmic_bytes_per_launch": per_launch_bytes,
                         "avg_launch_ms": top["ms"] / max(top["launches"], 1), "traffic": traffic},
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    args = ap.parse_args()
    select_workload(args.workload)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
