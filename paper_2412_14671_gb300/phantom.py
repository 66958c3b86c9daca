"""Seeded synthetic longitudinal phantoms (inputs for tests, benchmark and users).

Stands in for the paper's Traveling Brains / ADNI series, which are not
available: every series is generated from a seed, in float64, and returned as
float32. This module holds none of the registration method's arithmetic: the
template is analytic, deformations are integrated with many small Euler steps
and resampled with scipy.ndimage (a library routine), and nothing here calls
the CUDA library or the oracle.

Two generators, after the workloads of the paper's experiments (Sec. Simulated
Deformations, Sec. Sensitivity to clinical outcomes):
  blob_series   3-class tissue map + Gaussian blobs, random smooth deformations
                per consecutive session pair, multiplicative bias, Rician noise;
  brain_series  ellipsoidal head with CSF / GM / WM ordering of T1 intensities,
                ventricles expanding by a set percentage per session plus a
                small random smooth deformation, bias field, Rician noise.
"""
from __future__ import annotations

import numpy as np
import scipy.ndimage as ndi

BASE_SEED = 20241219


def _rng(seed: int, *sub: int) -> np.random.Generator:
    return np.random.default_rng([BASE_SEED, int(seed), *[int(s) for s in sub]])


def _grid(shape):
    return np.stack(np.meshgrid(*[np.arange(a, dtype=np.float64) for a in shape], indexing="ij"))


def smooth_noise(rng, shape, sigma, rms=1.0, components=3):
    """Gaussian-smoothed white noise, scaled to a vector RMS of `rms`. Wide kernels
    are applied on a coarser grid and interpolated back (the result is smooth)."""
    f = max(1, int(sigma // 2))
    small = tuple(max(2, -(-a // f)) for a in shape)
    white = [rng.normal(size=small) for _ in range(components)]

    def one(w):
        x = ndi.gaussian_filter(w, sigma / f, mode="wrap")
        if f > 1:
            x = ndi.zoom(x, [a / b for a, b in zip(shape, small)], order=1, mode="nearest", grid_mode=True)
        return x

    f3 = _per_component(one, white) if components == 3 else np.stack([one(w) for w in white])
    return f3 * (rms / np.sqrt((f3**2).sum(0).mean()))


def _resample(field, pts):
    """field (D,H,W) at points pts (3, ...), linear, edges replicated."""
    return ndi.map_coordinates(field, pts, order=1, mode="nearest")


_POOL = None


def _per_component(fn, *arrays):
    """np.stack([fn(a[0], ...), fn(a[1], ...), fn(a[2], ...)]) with the three calls on
    threads (scipy.ndimage releases the GIL); same values as the plain loop."""
    global _POOL
    if _POOL is None:
        import concurrent.futures

        _POOL = concurrent.futures.ThreadPoolExecutor(3)
    return np.stack(list(_POOL.map(fn, *arrays)))


def integrate_velocity(v, steps=16, coarse=1):
    """Displacement of the flow of a stationary velocity v after unit time, by
    forward Euler with `steps` small steps (each step resamples v). With
    coarse = c > 1 the (smooth) velocity is integrated on a grid c times coarser
    and the displacement interpolated back."""
    shape = v.shape[1:]
    if coarse > 1:
        small = tuple(max(2, -(-a // coarse)) for a in shape)
        zf = [b / a for a, b in zip(shape, small)]
        v = _per_component(lambda x: ndi.zoom(x, zf, order=1, mode="nearest", grid_mode=True), v) / coarse
    X = _grid(v.shape[1:])
    d = np.zeros_like(v)
    for _ in range(steps):
        pts = X + d
        d = d + _per_component(lambda x: _resample(x, pts), v) / steps
    if coarse > 1:
        zb = [a / b for a, b in zip(shape, d.shape[1:])]
        d = _per_component(lambda x: ndi.zoom(x, zb, order=1, mode="nearest", grid_mode=True), d) * coarse
    return d


def compose_displacements(D_prev, d):
    """Total displacement of x -> x + d(x) followed by the map with displacement D_prev."""
    X = _grid(d.shape[1:])
    pts = X + d
    return d + _per_component(lambda x: _resample(x, pts), D_prev)


def bias_field(rng, shape, amplitude):
    """Smooth multiplicative field with values in [1 - amplitude, 1 + amplitude]."""
    small = tuple(max(2, a // 8) for a in shape)
    b = ndi.gaussian_filter(rng.normal(size=small), max(small) / 6.0, mode="wrap")
    b = ndi.zoom(b, [a / c for a, c in zip(shape, small)], order=1, mode="nearest", grid_mode=True)
    b = b / np.abs(b).max()
    return 1.0 + amplitude * b


def rician(rng, I, sigma):
    return np.sqrt((I + sigma * rng.normal(size=I.shape)) ** 2 + (sigma * rng.normal(size=I.shape)) ** 2)


def blob_series(shape=(48, 48, 48), n_sessions=3, seed=0, n_blobs=40, vel_sigma=4.0, vel_rms=1.5,
                bias=0.10, noise=0.02, return_truth=False):
    """3-class tissue map + blobs (sigma 2-6 voxels), intensities in [0, 1]."""
    rng = _rng(seed, 1)
    shape = tuple(int(s) for s in shape)
    tissue = ndi.gaussian_filter(rng.normal(size=shape), 5.0, mode="wrap")
    q1, q2 = np.quantile(tissue, [0.33, 0.66])
    classes = np.where(tissue < q1, 0.2, np.where(tissue < q2, 0.5, 0.8))
    T = ndi.gaussian_filter(classes, 0.8)
    X = _grid(shape)
    for _ in range(n_blobs):
        c = rng.uniform(0, np.array(shape) - 1)
        s = rng.uniform(2.0, 6.0)
        a = rng.uniform(-0.2, 0.2)
        T = T + a * np.exp(-((X - c[:, None, None, None]) ** 2).sum(0) / (2 * s * s))
    T = np.clip(T, 0.0, 1.0)
    D = np.zeros((3,) + shape)
    imgs, truth = [], [D.copy()]
    for k in range(n_sessions):
        if k > 0:
            v = smooth_noise(rng, shape, vel_sigma, vel_rms)
            D = compose_displacements(D, integrate_velocity(v))
            truth.append(D.copy())
        I = ndi.map_coordinates(T, X + D, order=3, mode="nearest")
        I = I * bias_field(rng, shape, bias)
        I = rician(rng, np.clip(I, 0.0, None), noise)
        imgs.append(I)
    out = {"images": np.stack(imgs).astype(np.float32), "times": np.arange(n_sessions, dtype=np.float64)}
    if return_truth:
        out["truth_disp"] = np.stack(truth).astype(np.float32)  # session k -> session 0 coordinates
    return out


def _soft(x, width=0.6):
    return 1.0 / (1.0 + np.exp(-x / width))


def _brain_template(P, shape, tex):
    """T1-like intensities at points P (3, ...): scalp, CSF, GM, WM, ventricles."""
    c = (np.array(shape, dtype=np.float64) - 1) / 2
    ax = np.array(shape, dtype=np.float64) * np.array([0.42, 0.44, 0.40])
    R = np.sqrt((((P - c.reshape(3, *([1] * (P.ndim - 1)))) / ax.reshape(3, *([1] * (P.ndim - 1)))) ** 2).sum(0))
    s = min(shape) / 160.0  # about 1 voxel per mm at 160 voxels
    head = _soft((1.0 - R) * ax.min(), 0.8 * s)
    brain = _soft((0.90 - R) * ax.min(), 0.8 * s)
    wm = _soft((0.74 - R) * ax.min(), 1.2 * s)
    I = 0.02 + 0.55 * head * (1 - brain) + brain * (0.25 + 0.30 * _soft((0.86 - R) * ax.min(), 0.8 * s))
    I = I + wm * 0.30
    # two lateral ventricles (CSF) near the centre
    for sgn in (-1.0, 1.0):
        vc = c + np.array([0.0, -0.05, sgn * 0.08]) * np.array(shape)
        va = np.array(shape, dtype=np.float64) * np.array([0.07, 0.16, 0.045])
        rv = np.sqrt((((P - vc.reshape(3, *([1] * (P.ndim - 1)))) / va.reshape(3, *([1] * (P.ndim - 1)))) ** 2).sum(0))
        vent = _soft((1.0 - rv) * va.min(), 0.8 * s)
        I = I * (1 - vent) + 0.25 * vent
    return I + brain * tex


def ventricle_velocity(shape, rate):
    """Radial expansion around the ventricles: volume grows by about `rate` per unit time."""
    c = (np.array(shape, dtype=np.float64) - 1) / 2
    X = _grid(shape)
    v = np.zeros((3,) + tuple(shape))
    for sgn in (-1.0, 1.0):
        vc = c + np.array([0.0, -0.05, sgn * 0.08]) * np.array(shape)
        rho = 0.12 * min(shape)
        d = X - vc[:, None, None, None]
        g = np.exp(-(d**2).sum(0) / (2 * rho * rho))
        v += (rate / 3.0) * d * g  # divergence ~ rate near the centre
    return -v  # pulls from the later session toward the earlier (expanding) anatomy


def _render_brain(D, tex, shape, seed, k, bias, noise):
    """Session k of brain_series: template and texture at x + D(x), bias, Rician noise
    (its own random stream, so sessions can be rendered in any order)."""
    rng = _rng(seed, 4, k)
    P = _grid(shape) + D
    texk = ndi.map_coordinates(tex, P, order=1, mode="nearest")
    I = _brain_template(P, shape, texk)
    I = I * bias_field(rng, shape, bias)
    return rician(rng, np.clip(I, 0.0, None), noise).astype(np.float32)


def brain_series(shape=(160, 192, 160), n_sessions=10, seed=0, atrophy=(0.01, 0.03), vel_sigma=4.0,
                 vel_rms=0.3, bias=0.20, noise=0.03, return_truth=False):
    """Brain-like phantom series; ventricles grow 1-3 % per session. The deformation
    chain is built in order; sessions are rendered on a thread pool meanwhile."""
    import concurrent.futures
    import os

    rng = _rng(seed, 2)
    shape = tuple(int(s) for s in shape)
    tex = ndi.gaussian_filter(rng.normal(size=shape), 1.5, mode="wrap")
    tex = 0.04 * tex / tex.std()
    D = np.zeros((3,) + shape)
    truth = [D.copy()]
    workers = max(1, min(4, (os.cpu_count() or 1) // 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as pool:
        futs = []
        for k in range(n_sessions):
            if k > 0:
                rate = rng.uniform(*atrophy)
                v = ventricle_velocity(shape, rate) + smooth_noise(rng, shape, vel_sigma, vel_rms)
                D = compose_displacements(D, integrate_velocity(v, steps=8, coarse=2))
                truth.append(D)
            futs.append(pool.submit(_render_brain, D, tex, shape, seed, k, bias, noise))
        imgs = [f.result() for f in futs]
    out = {"images": np.stack(imgs), "times": np.arange(n_sessions, dtype=np.float64)}
    if return_truth:
        out["truth_disp"] = np.stack(truth).astype(np.float32)
    return out


def smooth_velocity(shape, n_fields, seed=0, sigma=2.0, rms=0.5):
    """(n_fields, 3, d, h, w) smooth random velocities for tests."""
    rng = _rng(seed, 3)
    return np.stack([smooth_noise(rng, tuple(shape), sigma, rms) for _ in range(n_fields)]).astype(np.float32)


def cached(generator: str, **kwargs):
    """Series from `generator` ('blob_series' or 'brain_series'), memoised on disk
    under $MUSTER_PHANTOM_CACHE (default: the system temp dir) by its arguments."""
    import hashlib
    import json
    import os
    import tempfile

    fn = {"blob_series": blob_series, "brain_series": brain_series}[generator]
    key = hashlib.sha1(json.dumps([generator, kwargs], sort_keys=True, default=str).encode()).hexdigest()[:16]
    root = os.environ.get("MUSTER_PHANTOM_CACHE", os.path.join(tempfile.gettempdir(), "muster_phantoms"))
    path = os.path.join(root, key + ".npz")
    if os.path.exists(path):
        with np.load(path) as z:
            return {k: z[k] for k in z.files}
    out = fn(**kwargs)
    os.makedirs(root, exist_ok=True)
    tmp = path + ".tmp%d.npz" % os.getpid()
    np.savez(tmp, **out)
    os.replace(tmp, path)
    return out
