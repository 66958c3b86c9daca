"""Autotuner of the engine's launch configuration.

For a problem (image shape, sessions, window, squarings, similarity, adjoint mode, and the
device) it chooses three knobs of muster_params by timing short registrations of the problem
on the device, one knob at a time from the library defaults:

  flow_nf      fields per thread of the flow-grid gather kernels (2, 1): the results do not
               depend on it;
  chunk_pct    the D-chunk rule of the image-grid kernels, in percent of its default CTA target
               (100, 50, 200, 400): chunks change where the window sums restart and the order
               of the loss partial sums, so results differ in their last bits between values;
  pair_batch   ordered pairs per image-grid launch (all, half).

A candidate is kept only if it is at least `min_gain` faster than the current choice. The
choice is cached in a JSON file (``$MUSTER_TUNE_CACHE``, else ``~/.cache/muster/tune.json``)
under the problem's key, so later contexts of the problem, and later processes that share the
file, take it without measuring again: with the same cache, a problem gets the same
configuration, hence the same bits, in every run. Entries are also kept per shape (without
the session count), which a lookup for an untuned session count falls back to.
"""
from __future__ import annotations

import json
import os
import tempfile
import time
from typing import Callable, Dict, Optional, Sequence, Tuple

import numpy as np

KNOBS: Tuple[Tuple[str, Tuple], ...] = (
    ("flow_nf", (2, 1)),
    ("chunk_pct", (100, 50, 200, 400)),
    ("pair_batch", ("all", "half")),
)
_KEY_PARAMS = ("window", "n_squarings", "similarity", "deterministic", "recompute_squaring", "rigid")


def cache_path() -> str:
    p = os.environ.get("MUSTER_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "muster", "tune.json")


def device_name() -> str:
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except Exception:
        pass
    return "cpu"


def problem_key(shape: Sequence[int], n_sessions: Optional[int], params: Dict, device: str) -> str:
    """Cache key of a problem; n_sessions None gives the shape-level key."""
    p = {k: int(params.get(k, 0)) for k in _KEY_PARAMS}
    n = "any" if n_sessions is None else str(int(n_sessions))
    return "%s|%s|N=%s|%s" % (device, "x".join(str(int(a)) for a in shape), n,
                               ",".join("%s=%d" % kv for kv in sorted(p.items())))


def load_cache(path: Optional[str] = None) -> Dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(data: Dict, path: Optional[str] = None) -> None:
    """Writes the cache atomically (a temporary file in the same folder, then a rename)."""
    path = path or cache_path()
    folder = os.path.dirname(os.path.abspath(path))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=folder, suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def knob_params(choice: Dict, n_sessions: int) -> Dict:
    """muster_params fields of a knob choice."""
    out = {}
    if "flow_nf" in choice:
        out["flow_nf"] = int(choice["flow_nf"])
    if "chunk_pct" in choice:
        out["chunk_pct"] = int(choice["chunk_pct"])
    if "pair_batch" in choice:
        P = n_sessions * (n_sessions - 1)
        out["pair_batch"] = 0 if choice["pair_batch"] == "all" else max(1, (P + 1) // 2)
    return out


def lookup(shape: Sequence[int], n_sessions: int, params: Dict, path: Optional[str] = None,
           device: Optional[str] = None) -> Optional[Dict]:
    """The cached knob choice of a problem (or of its shape), or None."""
    cache = load_cache(path)
    dev = device or device_name()
    for key in (problem_key(shape, n_sessions, params, dev), problem_key(shape, None, params, dev)):
        ent = cache.get(key)
        if ent and "choice" in ent:
            return dict(ent["choice"])
    return None


def tuned_params(shape: Sequence[int], n_sessions: int, params: Dict, path: Optional[str] = None) -> Dict:
    """params with the cached launch configuration of the problem applied (unchanged when
    there is none; explicit settings in params win)."""
    choice = lookup(shape, n_sessions, params, path)
    if not choice:
        return dict(params)
    out = knob_params(choice, n_sessions)
    out.update({k: v for k, v in params.items() if k in ("flow_nf", "chunk_pct", "pair_batch") and v})
    return dict(params, **out)


def registration_ms(shape: Sequence[int], n_sessions: int, params: Dict, images, steps: int = 4,
                    trials: int = 2) -> float:
    """Device milliseconds of a short registration (steps per level) of the problem: the
    best of `trials` after one untimed run."""
    import torch

    from .api import Muster

    p = dict(params, steps_per_level=[steps] * int(params.get("n_levels", 1)))
    with Muster(shape, n_sessions, **p) as reg:
        reg.set_images(images)
        reg.run()
        best = float("inf")
        stream = torch.cuda.current_stream()
        for _ in range(trials):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            reg.run()
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
    return best


def tune(shape: Sequence[int], n_sessions: int, params: Dict, images=None, path: Optional[str] = None,
         measure: Optional[Callable[[Dict], float]] = None, min_gain: float = 0.02, also_shape: bool = True,
         force: bool = False) -> Dict:
    """Chooses the knobs of the problem (coordinate search from the defaults) and caches
    the choice. measure(params) -> milliseconds (default: registration_ms on `images`).
    Returns {"choice", "ms", "trials": [(knob, value, ms), ...], "cached": bool}."""
    dev = device_name()
    key = problem_key(shape, n_sessions, params, dev)
    cache = load_cache(path)
    if not force and key in cache and "choice" in cache[key]:
        return dict(cache[key], cached=True)
    if measure is None:
        if images is None:
            raise ValueError("images are needed to time the problem")

        def measure(p):
            return registration_ms(shape, n_sessions, p, images)

    choice = {name: values[0] for name, values in KNOBS}
    base = dict(params)

    def run(ch):
        return float(measure(dict(base, **knob_params(ch, n_sessions))))

    best_ms = run(choice)
    trials = [("default", None, best_ms)]
    for name, values in KNOBS:
        if name == "pair_batch" and n_sessions * (n_sessions - 1) < 2:
            continue
        for v in values[1:]:
            cand = dict(choice, **{name: v})
            ms = run(cand)
            trials.append((name, v, ms))
            if ms < best_ms * (1.0 - min_gain):
                best_ms, choice = ms, cand
    ent = {"choice": choice, "ms": best_ms, "trials": trials, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    cache = load_cache(path)  # re-read: another process may have written meanwhile
    cache[key] = ent
    if also_shape:
        skey = problem_key(shape, None, params, dev)
        cache.setdefault(skey, dict(ent, from_sessions=int(n_sessions)))
    save_cache(cache, path)
    return dict(ent, cached=False)


def phantom_images(shape: Sequence[int], n_sessions: int, seed: int = 0) -> np.ndarray:
    """Seeded brain-like phantom series to time a problem on when the caller has no images."""
    from . import phantom

    return phantom.brain_series(tuple(shape), n_sessions, seed=seed)["images"]
