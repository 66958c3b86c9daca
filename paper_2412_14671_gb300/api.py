"""Python binding of the MUSTER registration engine (include/muster.h).

Thin marshalling over the C ABI: torch supplies device memory and the CUDA
stream; every step of the registration runs in the library's CUDA kernels.
Fields are returned as torch tensors in the layouts of include/muster.h
(volumes (D, H, W), vector fields (3, D, H, W), velocities (N-1, 3, d, h, w)).
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _native as N
from ._native import check, check_op, lib

__all__ = ["Muster", "MusterLoss", "default_params", "footprint", "op_downsample", "op_exp", "op_similarity",
           "op_jacobian_det", "op_deformation_metrics", "torch_allocator"]

_PARAM_KEYS = {name for name, _ in N.MusterParams._fields_} - {"alloc", "free", "alloc_user"}


def default_params(**overrides) -> N.MusterParams:
    p = N.MusterParams()
    lib().muster_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k not in _PARAM_KEYS:
            raise KeyError("unknown parameter %r" % k)
        if k == "steps_per_level":
            st = list(v) + [0] * (8 - len(v))
            for i in range(8):
                p.steps_per_level[i] = int(st[i])
        else:
            setattr(p, k, v)
    return p


def _stream_handle() -> int:
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


def torch_allocator(device: Optional[int] = None):
    """(alloc, free) callbacks for muster_params that take device memory from torch's
    caching allocator, all on the device's default stream: a destroyed context hands its
    blocks back to the cache (no cudaFree, which synchronises the whole device) and the
    next context of a similar size reuses them. A context's memory is only returned
    after the context's work is done (muster_destroy synchronises its stream)."""
    dev = torch.cuda.current_device() if device is None else int(device)
    stream = torch.cuda.default_stream(dev)

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
        except Exception:  # out of memory: the library reports MUSTER_EOOM
            return None

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return N.ALLOC_FN(alloc), N.FREE_FN(free)


def _dev_f32(t: torch.Tensor) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t


def _expect_numel(t, n: int, what: str) -> None:
    """The library reads or writes exactly n floats behind a device pointer: reject a
    tensor of another size here, before its pointer reaches a kernel."""
    if t is not None and t.numel() != n:
        raise ValueError("%s must hold %d elements, got %d (shape %s)" % (what, n, t.numel(), tuple(t.shape)))


def _expect_components(t, what: str) -> None:
    if t.dim() != 4 or t.shape[0] != 3:
        raise ValueError("%s must be a (3, D, H, W) vector field, got shape %s" % (what, tuple(t.shape)))


class Muster:
    """One registration context: N sessions of one (D, H, W) shape.

    Parameters are the fields of ``muster_params`` (include/muster.h), e.g.
    ``Muster((48, 48, 48), 3, n_levels=1, steps_per_level=[20], n_squarings=6, window=5)``.
    """

    def __init__(self, shape: Sequence[int], n_sessions: int, spacing=(1.0, 1.0, 1.0), allocator=None, **params):
        self._lib = lib()
        self.shape = tuple(int(s) for s in shape)
        self.n_sessions = int(n_sessions)
        self.params = default_params(**params)
        self._alloc_cbs = None
        if allocator == "torch":
            self._alloc_cbs = torch_allocator()
        elif allocator is not None:
            self._alloc_cbs = tuple(allocator)  # (ALLOC_FN, FREE_FN) pair
        if self._alloc_cbs:
            self.params.alloc, self.params.free = self._alloc_cbs
        ctx = ctypes.c_void_p()
        shp = (ctypes.c_int64 * 3)(*self.shape)
        sp = (ctypes.c_double * 3)(*[float(s) for s in spacing])
        check(self._lib.muster_create(shp, self.n_sessions, sp, ctypes.byref(self.params), ctypes.byref(ctx)))
        self._ctx = ctx
        self.set_stream(_stream_handle())

    # ------------------------------------------------------------------ lifecycle
    def close(self) -> None:
        if getattr(self, "_ctx", None):
            self._lib.muster_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int) -> None:
        check(rc, self._ctx)

    def set_stream(self, handle: int) -> None:
        self._check(self._lib.muster_set_stream(self._ctx, ctypes.c_void_p(handle or None)))

    # ------------------------------------------------------------------ inputs
    def set_images(self, imgs, times: Optional[Sequence[float]] = None) -> None:
        """imgs: (N, D, H, W) float32, a CUDA tensor (device copy) or host array/tensor."""
        tarr = None
        if times is not None:
            tarr = (ctypes.c_double * self.n_sessions)(*[float(t) for t in times])
        if isinstance(imgs, torch.Tensor) and imgs.is_cuda:
            _expect_numel(imgs, self.n_sessions * self.shape[0] * self.shape[1] * self.shape[2], "imgs")
            x = _dev_f32(imgs)
            self._check(self._lib.muster_set_images(self._ctx, x.data_ptr(), 1, tarr))
        else:
            x = np.ascontiguousarray(np.asarray(imgs, dtype=np.float32))
            if x.shape != (self.n_sessions,) + self.shape:
                raise ValueError("images must have shape %s" % ((self.n_sessions,) + self.shape,))
            self._check(self._lib.muster_set_images(self._ctx, x.ctypes.data, 0, tarr))

    def set_level(self, level: int) -> None:
        self._check(self._lib.muster_set_level(self._ctx, int(level)))

    def set_velocity(self, v) -> None:
        """Parameters of the current level, (N-1, 3, d, h, w): a CUDA tensor or a host array."""
        level, _ = self.level()
        n = None
        if level >= 0:
            _, nf = self.level_dims(level)
            n = (self.n_sessions - 1) * 3 * nf[0] * nf[1] * nf[2]
        if isinstance(v, torch.Tensor) and v.is_cuda:
            if n is not None:
                _expect_numel(v, n, "v")
            self._check(self._lib.muster_set_velocity(self._ctx, _dev_f32(v).data_ptr(), 1))
        else:
            x = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
            if n is not None and x.size != n:
                raise ValueError("v must hold %d elements, got %d (shape %s)" % (n, x.size, x.shape))
            self._check(self._lib.muster_set_velocity(self._ctx, x.ctypes.data, 0))

    def level(self) -> Tuple[int, int]:
        """(current pyramid level or -1, gradient steps issued at it)."""
        lv, st = ctypes.c_int(-1), ctypes.c_int(0)
        self._check(self._lib.muster_get_level(self._ctx, ctypes.byref(lv), ctypes.byref(st)))
        return lv.value, st.value

    # ------------------------------------------------------------------ optimisation
    def step(self, want_loss: bool = True) -> Optional[float]:
        if want_loss:
            out = ctypes.c_double()
            self._check(self._lib.muster_step(self._ctx, ctypes.byref(out)))
            return out.value
        self._check(self._lib.muster_step(self._ctx, None))
        return None

    def run(self) -> float:
        out = ctypes.c_double()
        self._check(self._lib.muster_run(self._ctx, ctypes.byref(out)))
        return out.value

    def advance(self, max_steps: int) -> bool:
        """Issue up to max_steps more steps of the schedule (no host wait); True when done."""
        fin = ctypes.c_int(0)
        self._check(self._lib.muster_advance(self._ctx, int(max_steps), ctypes.byref(fin)))
        return bool(fin.value)

    def eval(self, v: Optional[torch.Tensor], level: int, grad: Optional[torch.Tensor] = None) -> float:
        """Loss (and gradient into `grad`) at velocities v (device, (N-1,3,d,h,w))."""
        out = ctypes.c_double()
        if v is not None or grad is not None:
            _, nf = self.level_dims(level)
            n = (self.n_sessions - 1) * 3 * nf[0] * nf[1] * nf[2]
            _expect_numel(v, n, "v")
            _expect_numel(grad, n, "grad")
        vp = _dev_f32(v).data_ptr() if v is not None else None
        gp = _dev_f32(grad).data_ptr() if grad is not None else None
        self._check(self._lib.muster_eval(self._ctx, vp, int(level), ctypes.byref(out), gp))
        return out.value

    # ------------------------------------------------------------------ outputs
    def level_dims(self, level: int) -> Tuple[Tuple[int, int, int], Tuple[int, int, int]]:
        a, b = (ctypes.c_int64 * 3)(), (ctypes.c_int64 * 3)()
        self._check(self._lib.muster_level_dims(self._ctx, int(level), a, b))
        return tuple(a), tuple(b)

    def get_field(self, kind: int, i: int, j: int = 0, level: Optional[int] = None, device: bool = True):
        """Field of the current level (see MUSTER_* kinds); torch CUDA tensor or numpy array."""
        if level is None:
            raise ValueError("pass the current level (used to size the output)")
        ni, nf = self.level_dims(level)
        shape = {
            N.VELOCITY: (3,) + nf,
            N.GRADIENT: (3,) + nf,
            N.JACOBIAN: ni,
            N.PARAMETERS: (3,) + nf,
            N.PAIR_FLOW: (3,) + nf,
            N.PAIR_DISP: (3,) + ni,
            N.WARPED: ni,
            N.IMAGE: ni,
        }[kind]
        if device:
            out = torch.empty(shape, dtype=torch.float32, device="cuda")
            self._check(self._lib.muster_get_fields(self._ctx, kind, int(i), int(j), out.data_ptr(), 1))
            return out
        out = np.empty(shape, dtype=np.float32)
        self._check(self._lib.muster_get_fields(self._ctx, kind, int(i), int(j), out.ctypes.data, 0))
        return out

    def velocities(self, level: int, device: bool = True):
        outs = [self.get_field(N.VELOCITY, m, level=level, device=device) for m in range(self.n_sessions - 1)]
        return torch.stack(outs) if device else np.stack(outs)

    def rigid(self, grad: bool = False):
        """Rigid parameters (N-1, 6): angles (radians), translation (finest-level voxels);
        with grad=True also their gradient of the last step or eval."""
        F = self.n_sessions - 1
        r, g = np.zeros((F, 6)), np.zeros((F, 6))
        self._check(self._lib.muster_get_rigid(self._ctx, r.ctypes.data_as(N.DP), g.ctypes.data_as(N.DP)))
        return (r, g) if grad else r

    def set_rigid(self, rho) -> None:
        r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.n_sessions - 1, 6))
        self._check(self._lib.muster_set_rigid(self._ctx, r.ctypes.data_as(N.DP)))

    def loss_split(self) -> Dict[str, float]:
        out = (ctypes.c_double * 5)()
        self._check(self._lib.muster_get_loss_split(self._ctx, out))
        return dict(zip(("total", "sim", "L_ss", "L_L2", "L_ts"), list(out)))

    def loss_history(self) -> np.ndarray:
        n = ctypes.c_size_t(0)
        self._check(self._lib.muster_get_loss_history(self._ctx, None, ctypes.byref(n)))
        buf = np.zeros(max(n.value, 1), dtype=np.float64)
        n2 = ctypes.c_size_t(n.value)
        self._check(self._lib.muster_get_loss_history(self._ctx, buf.ctypes.data_as(N.DP), ctypes.byref(n2)))
        return buf[: n2.value]

    def get_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        self._check(self._lib.muster_get_state(self._ctx, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._lib.muster_get_state(self._ctx, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, state: bytes) -> None:
        buf = ctypes.create_string_buffer(state, len(state))
        self._check(self._lib.muster_set_state(self._ctx, buf, len(state)))

    # ------------------------------------------------------------------ profiling
    def profile_begin(self) -> None:
        self._check(self._lib.muster_profile_begin(self._ctx))

    def profile_end(self) -> List[dict]:
        """Per kernel: name, timed launches, every launch ("all_launches"), their device
        milliseconds and algorithmic bytes over the window since profile_begin."""
        self._check(self._lib.muster_profile_end(self._ctx))
        stats = []
        k = 0
        while True:
            name = ctypes.c_char_p()
            n = ctypes.c_int64()
            ms, by = ctypes.c_double(), ctypes.c_double()
            rc = self._lib.muster_kernel_stat(self._ctx, k, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
            if rc != N.OK:
                break
            every = ctypes.c_int64()
            self._check(self._lib.muster_kernel_launches(self._ctx, k, ctypes.byref(every)))
            stats.append({"name": name.value.decode(), "launches": n.value, "all_launches": every.value,
                          "ms": ms.value, "bytes": by.value})
            k += 1
        return stats


def footprint(shape: Sequence[int], n_sessions: int, **params) -> int:
    """Device bytes a Muster context of this problem allocates (no device needed)."""
    p = default_params(**params)
    out = ctypes.c_size_t(0)
    shp = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    check(lib().muster_footprint(shp, int(n_sessions), ctypes.byref(p), ctypes.byref(out)))
    return int(out.value)


class MusterLoss(torch.autograd.Function):
    """L(phi) of a Muster context as a differentiable torch function.

    forward(v, muster, level) -> 0-d float64 tensor; the hand-written adjoint of
    the CUDA library provides dL/dv, scaled by the incoming gradient.
    """

    @staticmethod
    def forward(ctx, v: torch.Tensor, muster: Muster, level: int):
        v = v.detach().contiguous()
        grad = torch.empty_like(v)
        loss = muster.eval(v, level, grad)
        ctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g.to(grad.dtype), None, None


# ---------------------------------------------------------------------- ops
def op_downsample(x: torch.Tensor) -> torch.Tensor:
    """(n, D, H, W) or (D, H, W) -> 2x2x2 means."""
    x = _dev_f32(x)
    sq = x.dim() == 3
    xx = x[None] if sq else x
    n, D, H, W = xx.shape
    out = torch.empty((n, (D + 1) // 2, (H + 1) // 2, (W + 1) // 2), dtype=torch.float32, device=x.device)
    check_op(lib().muster_op_downsample(xx.data_ptr(), n, D, H, W, out.data_ptr(), ctypes.c_void_p(_stream_handle() or None)))
    return out[0] if sq else out


def op_exp(phi: torch.Tensor, K: int, sign: float = 1.0) -> torch.Tensor:
    """(3, D, H, W) velocity -> displacement of Exp(sign * phi)."""
    _expect_components(phi, "phi")
    phi = _dev_f32(phi)
    u = torch.empty_like(phi)
    _, D, H, W = phi.shape
    check_op(lib().muster_op_exp(phi.data_ptr(), D, H, W, int(K), float(sign), u.data_ptr(), ctypes.c_void_p(_stream_handle() or None)))
    return u


def op_similarity(F: torch.Tensor, W: torch.Tensor, window: int, kind: int = N.SILNCC, eps: float = 1e-6,
                  grad: bool = True):
    """Mean windowed SiLNCC / LNCC of (F, W) and dSim/dW."""
    if F.dim() != 3 or W.shape != F.shape:
        raise ValueError("F and W must be (D, H, W) volumes of one shape, got %s and %s"
                         % (tuple(F.shape), tuple(W.shape)))
    F, W = _dev_f32(F), _dev_f32(W)
    D, H, Wd = F.shape
    out = ctypes.c_double()
    g = torch.empty_like(W) if grad else None
    check_op(lib().muster_op_similarity(F.data_ptr(), W.data_ptr(), D, H, Wd, int(window), int(kind), float(eps),
                                        ctypes.byref(out), g.data_ptr() if grad else None,
                                        ctypes.c_void_p(_stream_handle() or None)))
    return (out.value, g) if grad else out.value


def op_jacobian_det(u: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """det(I + grad u) of a (3, D, H, W) displacement (voxels) on its grid (into out if given)."""
    _expect_components(u, "u")
    u = _dev_f32(u)
    _, D, H, W = u.shape
    J = torch.empty((D, H, W), dtype=torch.float32, device=u.device) if out is None else _dev_f32(out)
    if J.shape != (D, H, W):
        raise ValueError("out must have shape %s" % ((D, H, W),))
    check_op(lib().muster_op_jacobian_det(u.data_ptr(), D, H, W, J.data_ptr(), ctypes.c_void_p(_stream_handle() or None)))
    return J


def op_deformation_metrics(u_true: torch.Tensor, u_est: torch.Tensor, roi: Optional[torch.Tensor] = None) -> Dict:
    """Eu, PCC, slope B (and A, b, ROI size) between two (3, D, H, W) displacements."""
    _expect_components(u_true, "u_true")
    ut, ue = _dev_f32(u_true), _dev_f32(u_est)
    if ut.shape != ue.shape:
        raise ValueError("fields must have the same shape")
    _, D, H, W = ut.shape
    rp = None
    if roi is not None:
        if roi.shape != (D, H, W) or roi.dtype not in (torch.uint8, torch.bool) or not roi.is_cuda:
            raise ValueError("roi must be a (D, H, W) uint8/bool CUDA tensor")
        roi = roi.contiguous().to(torch.uint8)
        rp = roi.data_ptr()
    out = (ctypes.c_double * 16)()
    check_op(lib().muster_op_deformation_metrics(ut.data_ptr(), ue.data_ptr(), rp, D, H, W, out,
                                                 ctypes.c_void_p(_stream_handle() or None)))
    o = list(out)
    return {"Eu": o[0], "PCC": o[1], "B": o[2], "A": np.array(o[3:12]).reshape(3, 3), "b": np.array(o[12:15]),
            "count": int(o[15])}
