"""Host-side failure paths of the engine, made on the host without faulting the GPU:
an allocator that runs out (MUSTER_EOOM), a non-finite loss from host-supplied
velocities or a diverging step size (MUSTER_ENUMERIC), and a host wait that runs out
(MUSTER_ETIMEOUT with a tiny MUSTER_SYNC_TIMEOUT_S). After each, the context (or the
next one) is usable and gives the result of an undisturbed run."""
import os

import numpy as np
import pytest
import torch

import paper_2412_14671_gb300 as m
from paper_2412_14671_gb300 import _native, phantom

pytestmark = pytest.mark.gpu

SHAPE, N = (24, 22, 26), 3
KW = dict(n_levels=2, steps_per_level=[6, 8], n_squarings=4, window=3, alpha_ss=0.1, alpha_l2=0.01, lr=0.05,
          deterministic=1)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _imgs():
    return phantom.blob_series(SHAPE, N, seed=31)["images"]


class CountingAllocator:
    """Device memory from torch's caching allocator; returns NULL once `limit` blocks
    are out, and records every block handed out and given back."""

    def __init__(self, limit):
        self.limit, self.live, self.taken, self.freed, self.refused = limit, set(), 0, 0, 0
        self.stream = torch.cuda.default_stream()

        def alloc(nbytes, user):
            if len(self.live) >= self.limit:
                self.refused += 1
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), self.stream)
            self.live.add(p)
            self.taken += 1
            return p

        def free(ptr, user):
            self.live.discard(ptr)
            self.freed += 1
            torch.cuda.caching_allocator_delete(ptr)

        self.fns = (_native.ALLOC_FN(alloc), _native.FREE_FN(free))


@pytest.mark.parametrize("limit", [0, 5, 20])
def test_allocator_that_runs_out_gives_eoom_and_frees_what_it_took(limit):
    a = CountingAllocator(limit)
    with pytest.raises(m.MusterError) as e:
        m.Muster(SHAPE, N, allocator=a.fns, **KW)
    assert e.value.code == _native.EOOM
    assert a.refused >= 1
    assert a.taken == limit and a.freed == a.taken and not a.live  # every block taken was given back
    # a context with an allocator that does not run out works
    b = CountingAllocator(10 ** 6)
    with m.Muster(SHAPE, N, allocator=b.fns, **KW) as reg:
        reg.set_images(cuda(_imgs()))
        assert np.isfinite(reg.run())
    assert not b.live


def test_non_finite_velocity_gives_enumeric_and_the_context_recovers():
    imgs = _imgs()
    with m.Muster(SHAPE, N, **KW) as reg:
        reg.set_images(cuda(imgs))
        reg.set_level(0)
        ni, nf = reg.level_dims(0)
        v = np.zeros((N - 1, 3) + nf, np.float32)
        v[1, 2, 3, 4, 5] = np.nan
        reg.set_velocity(v)
        with pytest.raises(m.MusterError) as e:
            reg.step()
        assert e.value.code == _native.ENUMERIC
        # a new level start resets the velocities; the schedule then runs as usual
        reg.set_level(0)
        assert np.isfinite(reg.step())
        ref = reg.run()
    with m.Muster(SHAPE, N, **KW) as fresh:
        fresh.set_images(cuda(imgs))
        assert fresh.run() == ref


def test_diverging_step_size_gives_enumeric_from_run():
    with m.Muster(SHAPE, N, **dict(KW, optimizer=m.SGD, lr=1e30)) as reg:
        reg.set_images(cuda(_imgs()))
        with pytest.raises(m.MusterError) as e:
            reg.run()
        assert e.value.code == _native.ENUMERIC
        hist = reg.loss_history()
        assert not np.all(np.isfinite(hist))


def test_host_wait_timeout_leaves_a_usable_context(monkeypatch):
    # long enough that the GPU is still busy when the host starts waiting: 240 steps of
    # 4 x 48x44x52 take tens of milliseconds, issuing them about a millisecond
    shape, n = (48, 44, 52), 4
    kw = dict(KW, steps_per_level=[40, 200])
    imgs = phantom.blob_series(shape, n, seed=32)["images"]
    with m.Muster(shape, n, **kw) as ref:
        ref.set_images(cuda(imgs))
        ref_loss = ref.run()
        ref_v = ref.velocities(1, device=False)
    with m.Muster(shape, n, **kw) as reg:
        reg.set_images(cuda(imgs))
        monkeypatch.setenv("MUSTER_SYNC_TIMEOUT_S", "1e-9")
        with pytest.raises(m.MusterError) as e:
            reg.run()  # the whole schedule is issued; the host stops waiting at once
        assert e.value.code == _native.ETIMEOUT
        monkeypatch.delenv("MUSTER_SYNC_TIMEOUT_S")
        # the issued work completes; calls that synchronise see its result
        assert reg.loss_split()["total"] == ref_loss
        assert np.array_equal(reg.velocities(1, device=False), ref_v)
        assert reg.run() == ref_loss
