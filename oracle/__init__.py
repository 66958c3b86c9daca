"""FP64 CPU oracle of MUSTER's registration loop (arXiv 2412.14671).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this package.
The CUDA library never imports, links or calls it, and this package imports
nothing from the CUDA library.

The arithmetic lives in ``muster_oracle.c`` (plain C, FP64, OpenMP over voxel
loops); this module only compiles it and marshals numpy arrays. Arrays are
float64, C-contiguous; a vector field has shape (3, D, H, W) with component c
the displacement along axis c, in voxel units of its own grid.

Pins (tests/test_oracle_*.py, all ``-m "not gpu"``):
  sample        affine functions reproduced exactly; clamp = constant extension;
                derivative equals the affine slope; brute-force trilinear formula
  exp           phi = 0 -> 0 exactly; constant -> exact translation; affine phi ->
                ((I + A/2^K)^(2^K) - I)(x - x0) in the interior and expm(A) within
                O(|A|^2/2^K); Exp(phi) o Exp(-phi) ~ identity, shrinking with K
  compose       constant fields add exactly (pins the chain indexing); affine maps
                compose as the matrix product in the interior, in the right order
  upsample/warp zero -> identity; constant -> f*c; affine -> exact in the interior;
                integer translation -> exact shift
  similarity    window sums vs brute-force Python loops (several sizes, w in 3,5,7);
                identical / affinely related images -> maximal similarity;
                E[LNCC] of Eq. E_lncc and OLS residual variance for SiLNCC (Monte Carlo)
  regulariser   linear field -> |A|_F^2; constant -> |c|^2; proportional-in-time
                flows -> L_ts = 0; constant flows -> closed-form L_ts
  objective     constant whole-voxel velocities: pair maps are exact translations, and the
                similarity total equals a brute-force numpy sum over all ordered pairs of
                shifted copies; weighted regularisers add to it (Eq. reg_sum)
  gradient      FP64 central differences of the total loss on random voxels (both
                similarity kinds, N = 2, 3, 4); adjoint dot-product identities for
                every linear piece
  optimiser     one Adam step vs torch.optim.Adam (float64); schedule closed forms
  pyramid       constants and affine functions through down-sampling / prolongation
  rigid         rho = 0 -> the plain loss; a pure translation = warping by that constant
                displacement; a quarter turn of a cube about its centre permutes voxels exactly;
                rotation matrix vs scipy Rotation; rho gradient by central differences
  smoothing     the Gaussian of Appendix Gaussian Smoothing against numpy.fft; one Fourier mode
                scaled by exactly its response; constants kept; symmetric (its own adjoint);
                smoothed loss gradient by central differences in theta
  jacobian      affine fields -> det(I + A) exactly (every difference is exact for them),
                scaling s x -> (1 + s)^3, random fields vs numpy.gradient + numpy.linalg.det
  metrics       identical fields -> Eu 0, PCC 1, B 1; u_est = A u_true + b without noise ->
                A, b recovered exactly; u_est = -u_true -> PCC -1; Eu of a constant offset;
                ROI masking vs the same sums over the selected voxels
  driver        run (or_run / or_run_rigid): the stage schedule of Sec. Implementation
                Details restated step by step (numpy pyramid, scipy prolongation, closed-form
                schedule per level, a fresh torch.optim.Adam per level, per-level voxel size of
                the Gaussian taps, rigid step sizes); loss history and parameters to 1e-12
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "muster_oracle.c")
_HDR = os.path.join(_HERE, "muster_oracle.h")
_LIB = os.path.join(_HERE, "libmuster_oracle.so")

SILNCC = 0
LNCC = 1
ADAM = 0
SGD = 1


class OrParams(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("steps", ctypes.c_int * 8),
        ("flow_factor", ctypes.c_int),
        ("K", ctypes.c_int),
        ("window", ctypes.c_int),
        ("sim_kind", ctypes.c_int),
        ("optimizer", ctypes.c_int),
        ("pad_", ctypes.c_int),
        ("alpha_ss", ctypes.c_double),
        ("alpha_l2", ctypes.c_double),
        ("alpha_ts", ctypes.c_double),
        ("sim_eps", ctypes.c_double),
        ("lr", ctypes.c_double),
        ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double),
        ("adam_eps", ctypes.c_double),
        ("warmup_frac", ctypes.c_double),
        ("smooth_omega", ctypes.c_double),
        ("spacing", ctypes.c_double * 3),
        ("rigid", ctypes.c_int),
        ("pad2_", ctypes.c_int),
        ("rigid_lr", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags: the same source builds on x86 and Arm)."""
    if not force and os.path.exists(_LIB):
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if os.path.getmtime(_LIB) >= newest:
            return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(ctypes.c_double)
        I3 = ctypes.POINTER(ctypes.c_int)
        d, i = ctypes.c_double, ctypes.c_int
        sig = {
            "or_sample": (d, [P, I3, P, P]),
            "or_exp": (None, [P, I3, i, d, P, P]),
            "or_exp_adjoint": (None, [P, I3, i, d, P, P]),
            "or_compose": (None, [P, P, i, I3, P]),
            "or_compose_adjoint": (None, [P, P, i, I3, P, P, P]),
            "or_upsample": (None, [P, I3, I3, i, P]),
            "or_upsample_adjoint": (None, [P, I3, I3, i, P]),
            "or_warp": (None, [P, I3, P, P]),
            "or_warp_adjoint": (None, [P, I3, P, P, P]),
            "or_similarity": (d, [P, P, I3, i, i, d, P]),
            "or_window_stats": (None, [P, P, I3, i, P, P, P, P, P]),
            "or_regulariser": (None, [P, i, I3, P, d, d, d, P, P]),
            "or_downsample2": (None, [P, I3, P]),
            "or_prolong": (None, [P, I3, I3, P]),
            "or_loss_grad": (d, [P, i, I3, P, I3, ctypes.POINTER(OrParams), P, P, P]),
            "or_lr": (d, [i, i, d, d]),
            "or_adam_step": (None, [P, P, P, P, ctypes.c_size_t, i, d, d, d, d]),
            "or_run": (d, [P, i, I3, ctypes.POINTER(OrParams), P, P, P]),
            "or_level_dims": (None, [I3, i, i, i, I3, I3]),
            "or_jacobian_det": (None, [P, I3, P]),
            "or_smooth": (None, [P, I3, P, d, P]),
            "or_loss_grad_rigid": (d, [P, i, I3, P, I3, ctypes.POINTER(OrParams), P, P, d, P, P, P]),
            "or_rotation": (None, [P, P, P]),
            "or_run_rigid": (d, [P, i, I3, ctypes.POINTER(OrParams), P, P, P, P]),
            "or_deformation_metrics": (None, [P, P, ctypes.c_void_p, I3, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# --------------------------------------------------------------------------- marshalling
def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(n) -> ctypes.Array:
    return (ctypes.c_int * 3)(*[int(v) for v in n])


def _opt(a):
    return None if a is None else _p(a)


def params(
    n_levels=1,
    steps=(20,),
    flow_factor=2,
    K=6,
    window=5,
    sim_kind=SILNCC,
    optimizer=ADAM,
    alpha_ss=1.0,
    alpha_l2=0.01,
    alpha_ts=0.0,
    sim_eps=1e-6,
    lr=0.1,
    beta1=0.9,
    beta2=0.999,
    adam_eps=1e-8,
    warmup_frac=0.2,
    smooth_omega=0.0,
    spacing=(1.0, 1.0, 1.0),
    rigid=0,
    rigid_lr=0.5,
) -> OrParams:
    p = OrParams()
    p.n_levels = n_levels
    st = list(steps) + [0] * (8 - len(steps))
    for k in range(8):
        p.steps[k] = int(st[k])
    p.flow_factor = flow_factor
    p.K = K
    p.window = window
    p.sim_kind = sim_kind
    p.optimizer = optimizer
    p.alpha_ss, p.alpha_l2, p.alpha_ts = alpha_ss, alpha_l2, alpha_ts
    p.sim_eps = sim_eps
    p.lr, p.beta1, p.beta2, p.adam_eps, p.warmup_frac = lr, beta1, beta2, adam_eps, warmup_frac
    p.smooth_omega = smooth_omega
    p.rigid, p.rigid_lr = int(rigid), float(rigid_lr)
    for a in range(3):
        p.spacing[a] = float(spacing[a])
    return p


# --------------------------------------------------------------------------- API
def sample(g, q):
    g = _f64(g)
    q = _f64(q)
    grad = np.zeros(3)
    v = lib().or_sample(_p(g), _dims(g.shape), _p(q), _p(grad))
    return v, grad


def exp(phi, K, sign=1.0, intermediates=False):
    """Alg. 1: displacement of Exp(sign * phi) (and optionally u_0..u_K)."""
    phi = _f64(phi)
    n = phi.shape[1:]
    u = np.zeros_like(phi)
    inter = np.zeros((K + 1,) + phi.shape) if intermediates else None
    lib().or_exp(_p(phi), _dims(n), int(K), float(sign), _p(u), _opt(inter))
    return (u, inter) if intermediates else u


def exp_adjoint(phi, K, sign, g_u):
    phi, g_u = _f64(phi), _f64(g_u)
    g = np.zeros_like(phi)
    lib().or_exp_adjoint(_p(phi), _dims(phi.shape[1:]), int(K), float(sign), _p(g_u), _p(g))
    return g


def compose(up, um):
    """Eq. cum_deformation for all ordered pairs: U[k, i] pulls image k onto grid i."""
    up, um = _f64(up), _f64(um)
    N = up.shape[0] + 1
    n = up.shape[2:]
    U = np.zeros((N, N, 3) + tuple(n))
    lib().or_compose(_p(up), _p(um), N, _dims(n), _p(U))
    return U


def compose_adjoint(up, um, gU):
    up, um, gU = _f64(up), _f64(um), _f64(gU)
    N = up.shape[0] + 1
    g_up, g_um = np.zeros_like(up), np.zeros_like(um)
    lib().or_compose_adjoint(_p(up), _p(um), N, _dims(up.shape[2:]), _p(gU), _p(g_up), _p(g_um))
    return g_up, g_um


def upsample(U, ni, f=2):
    U = _f64(U)
    Ut = np.zeros((3,) + tuple(ni))
    lib().or_upsample(_p(U), _dims(U.shape[1:]), _dims(ni), int(f), _p(Ut))
    return Ut


def upsample_adjoint(gUt, nf, f=2):
    gUt = _f64(gUt)
    gU = np.zeros((3,) + tuple(nf))
    lib().or_upsample_adjoint(_p(gUt), _dims(nf), _dims(gUt.shape[1:]), int(f), _p(gU))
    return gU


def warp(I, Ut):
    I, Ut = _f64(I), _f64(Ut)
    W = np.zeros_like(I)
    lib().or_warp(_p(I), _dims(I.shape), _p(Ut), _p(W))
    return W


def warp_adjoint(I, Ut, gW):
    I, Ut, gW = _f64(I), _f64(Ut), _f64(gW)
    g = np.zeros_like(Ut)
    lib().or_warp_adjoint(_p(I), _dims(I.shape), _p(Ut), _p(gW), _p(g))
    return g


def similarity(F, W, w, kind=SILNCC, eps=1e-6, grad=False):
    """Mean over valid windows of SiLNCC_R (kind=0) or LNCC_R (kind=1); optional dSim/dW."""
    F, W = _f64(F), _f64(W)
    dW = np.zeros_like(W) if grad else None
    s = lib().or_similarity(_p(F), _p(W), _dims(F.shape), int(w), int(kind), float(eps), _opt(dW))
    return (s, dW) if grad else s


def window_stats(F, W, w):
    F, W = _f64(F), _f64(W)
    m = tuple(int(a) - w + 1 for a in F.shape)
    outs = [np.zeros(m) for _ in range(5)]
    lib().or_window_stats(_p(F), _p(W), _dims(F.shape), int(w), *[_p(o) for o in outs])
    return dict(zip(("muF", "muW", "Sff", "Sww", "Sfw"), outs))


def regulariser(phi, t=None, alphas=(1.0, 1.0, 1.0), grad=False):
    """(L_ss, L_L2, L_ts) unweighted, and the gradient of the alpha-weighted sum."""
    phi = _f64(phi)
    N = phi.shape[0] + 1
    t = _f64(np.arange(N) if t is None else t)
    L = np.zeros(3)
    g = np.zeros_like(phi) if grad else None
    lib().or_regulariser(_p(phi), N, _dims(phi.shape[2:]), _p(t), *map(float, alphas), _p(L), _opt(g))
    return (L, g) if grad else L


def downsample2(I):
    I = _f64(I)
    out = np.zeros(tuple((a + 1) // 2 for a in I.shape))
    lib().or_downsample2(_p(I), _dims(I.shape), _p(out))
    return out


def prolong(v, nf):
    v = _f64(v)
    out = np.zeros((3,) + tuple(nf))
    lib().or_prolong(_p(v), _dims(v.shape[1:]), _dims(nf), _p(out))
    return out


def level_dims(n, n_levels, level, flow_factor=2):
    ni, nf = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    lib().or_level_dims(_dims(n), n_levels, level, flow_factor, ni, nf)
    return tuple(ni), tuple(nf)


def loss_grad(imgs, phi, p: OrParams, t=None, grad=True):
    """Total loss at one level (images at that level, phi on its flow grid)."""
    imgs, phi = _f64(imgs), _f64(phi)
    N = imgs.shape[0]
    t = _f64(np.arange(N) if t is None else t)
    split = np.zeros(4)
    g = np.zeros_like(phi) if grad else None
    tot = lib().or_loss_grad(
        _p(imgs), N, _dims(imgs.shape[1:]), _p(phi), _dims(phi.shape[2:]), ctypes.byref(p), _p(t),
        _p(split), _opt(g)
    )
    return tot, split, g


def loss_grad_rigid(imgs, theta, rho, p: OrParams, tscale=1.0, t=None):
    """Loss, theta gradient and rho gradient with the rigid parameters rho ((N-1, 6): angles,
    translation in finest-level voxels; tscale finest voxels per voxel of this level)."""
    imgs, theta, rho = _f64(imgs), _f64(theta), _f64(rho)
    N = imgs.shape[0]
    t = _f64(np.arange(N) if t is None else t)
    split = np.zeros(4)
    g = np.zeros_like(theta)
    gr = np.zeros_like(rho)
    tot = lib().or_loss_grad_rigid(
        _p(imgs), N, _dims(imgs.shape[1:]), _p(theta), _dims(theta.shape[2:]), ctypes.byref(p), _p(t), _p(rho),
        float(tscale), _p(split), _p(g), _p(gr)
    )
    return tot, split, g, gr


def rotation(a):
    """R = R_0(a0) R_1(a1) R_2(a2) and dR/da_k (3, 3, 3)."""
    a = _f64(a)
    R, dR = np.zeros(9), np.zeros(27)
    lib().or_rotation(_p(a), _p(R), _p(dR))
    return R.reshape(3, 3), dR.reshape(3, 3, 3)


def lr_at(step, T, lr, warmup_frac=0.2):
    return lib().or_lr(int(step), int(T), float(lr), float(warmup_frac))


def adam_step(theta, m, v, g, step, lr_t, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().or_adam_step(_p(theta), _p(m), _p(v), _p(g), theta.size, int(step), float(lr_t), b1, b2, eps)


def run(imgs, p: OrParams, t=None, loss_history=False):
    """Whole multi-level registration; returns (final loss, finest-level phi[, losses])."""
    imgs = _f64(imgs)
    N = imgs.shape[0]
    n = imgs.shape[1:]
    t = _f64(np.arange(N) if t is None else t)
    _, nf = level_dims(n, p.n_levels, p.n_levels - 1, p.flow_factor)
    theta = np.zeros((N - 1, 3) + tuple(nf))
    total_steps = sum(p.steps[l] for l in range(p.n_levels))
    hist = np.zeros(max(total_steps, 1)) if loss_history else None
    rho = np.zeros((N - 1, 6))
    loss = lib().or_run_rigid(_p(imgs), N, _dims(n), ctypes.byref(p), _p(t), _p(theta), _opt(hist), _p(rho))
    out = (loss, theta, hist[:total_steps]) if loss_history else (loss, theta)
    return out + (rho,) if p.rigid else out


def jacobian_det(u):
    """det(I + grad u) on u's grid (central differences, one-sided at the edges)."""
    u = _f64(u)
    J = np.zeros(u.shape[1:])
    lib().or_jacobian_det(_p(u), _dims(u.shape[1:]), _p(J))
    return J


def deformation_metrics(u_true, u_est, roi=None):
    """Sec. Evaluation Metrics: dict(Eu, PCC, B, A (3x3), b (3), count) over the ROI."""
    ut, ue = _f64(u_true), _f64(u_est)
    out = np.zeros(16)
    r = None
    if roi is not None:
        r = np.ascontiguousarray(np.asarray(roi, dtype=np.uint8))
    lib().or_deformation_metrics(_p(ut), _p(ue), r.ctypes.data if r is not None else None, _dims(ut.shape[1:]),
                                 _p(out))
    return {"Eu": out[0], "PCC": out[1], "B": out[2], "A": out[3:12].reshape(3, 3), "b": out[12:15],
            "count": int(out[15])}


def smooth(x, omega, h=(1.0, 1.0, 1.0)):
    """Appendix Gaussian Smoothing of one scalar volume (voxel size h mm, periodic grid)."""
    x = _f64(x)
    out = np.zeros_like(x)
    hh = (ctypes.c_double * 3)(*[float(a) for a in h])
    lib().or_smooth(_p(x), _dims(x.shape), ctypes.cast(hh, ctypes.POINTER(ctypes.c_double)), float(omega), _p(out))
    return out
