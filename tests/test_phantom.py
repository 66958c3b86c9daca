"""The seeded input recipe (no GPU): the phantom generators are deterministic per seed and
produce the structure the workloads are described by -- tissue intensities, the requested
velocity RMS, the bias-field range, the Rician noise floor, the ventricle expansion rate
and identity at the first session. Closed forms and invariants, checked on small volumes."""
import numpy as np
import pytest

from paper_2412_14671_gb300 import phantom


def test_blob_series_is_seeded():
    a = phantom.blob_series((20, 18, 16), 3, seed=5, return_truth=True)
    b = phantom.blob_series((20, 18, 16), 3, seed=5, return_truth=True)
    c = phantom.blob_series((20, 18, 16), 3, seed=6)
    assert a["images"].dtype == np.float32 and a["images"].shape == (3, 20, 18, 16)
    assert np.array_equal(a["images"], b["images"]) and np.array_equal(a["truth_disp"], b["truth_disp"])
    assert not np.array_equal(a["images"], c["images"])
    assert np.array_equal(a["times"], [0.0, 1.0, 2.0])
    # session 0 is the reference: its deformation is the identity
    assert a["truth_disp"].shape == (3, 3, 20, 18, 16) and not a["truth_disp"][0].any()


def test_smooth_noise_has_the_requested_vector_rms():
    for sigma, rms in ((1.0, 0.5), (4.0, 1.5), (6.5, 0.3)):
        f = phantom.smooth_noise(np.random.default_rng(1), (24, 20, 28), sigma, rms)
        assert f.shape == (3, 24, 20, 28)
        assert np.sqrt((f**2).sum(0).mean()) == pytest.approx(rms, rel=1e-12)


def test_integrated_displacement_of_a_constant_velocity_is_that_velocity():
    # Euler steps of a constant field sum to the field itself (unit time)
    v = np.zeros((3, 10, 12, 14))
    v[0], v[1], v[2] = 0.7, -1.2, 0.25
    d = phantom.integrate_velocity(v, steps=16)
    assert np.allclose(d, v, atol=1e-12)


def test_composed_constant_displacements_add():
    a = np.zeros((3, 9, 9, 9))
    b = np.zeros((3, 9, 9, 9))
    a[0], b[2] = 1.0, -0.5
    tot = phantom.compose_displacements(a, b)
    # interior points stay in the grid, so the resampled constant is exact there
    assert np.allclose(tot[:, 2:-2, 2:-2, 2:-2][0], 1.0) and np.allclose(tot[:, 2:-2, 2:-2, 2:-2][2], -0.5)


def test_bias_field_spans_exactly_its_amplitude():
    for amp in (0.1, 0.2):
        b = phantom.bias_field(np.random.default_rng(3), (32, 24, 40), amp)
        assert b.min() >= 1 - amp - 1e-12 and b.max() <= 1 + amp + 1e-12
        # normalised by its largest magnitude: one end of the range is reached
        assert max(b.max() - 1, 1 - b.min()) == pytest.approx(amp, rel=1e-12)


def test_rician_noise_floor_is_the_rayleigh_mean():
    # |0 + n1 + i n2| with n ~ N(0, sigma^2) is Rayleigh: mean sigma sqrt(pi/2), mean square 2 sigma^2
    sigma = 0.03
    x = phantom.rician(np.random.default_rng(7), np.zeros(2_000_000), sigma)
    assert x.mean() == pytest.approx(sigma * np.sqrt(np.pi / 2), rel=3e-3)
    assert (x**2).mean() == pytest.approx(2 * sigma**2, rel=3e-3)


def test_brain_template_orders_t1_intensities():
    shape = (80, 96, 80)
    c = (np.array(shape, dtype=np.float64) - 1) / 2
    ax = np.array(shape) * np.array([0.42, 0.44, 0.40])

    def at(offset_r, direction=(1.0, 0.0, 0.0)):
        d = np.asarray(direction) / np.linalg.norm(direction)
        p = c + offset_r * ax * d
        return float(phantom._brain_template(p.reshape(3, 1), shape, 0.0)[0])

    vent = c + np.array([0.0, -0.05, 0.08]) * np.array(shape)
    csf = float(phantom._brain_template(vent.reshape(3, 1), shape, 0.0)[0])
    wm, gm, outside = at(0.5), at(0.82), at(1.3)
    assert csf == pytest.approx(0.25, abs=0.01)
    assert wm == pytest.approx(0.87, abs=0.02)
    assert outside == pytest.approx(0.02, abs=0.005)
    assert outside < csf < gm < wm


def test_ventricle_velocity_divergence_is_the_expansion_rate():
    # each ventricle adds (rate/3) d exp(-|d|^2 / 2 rho^2), d the offset from its centre, whose
    # divergence is (rate/3) g (3 - |d|^2 / rho^2): rate at its own centre; the field is the
    # negated sum of the two, so its divergence at a ventricle is -rate plus the other's tail
    shape, rate = (64, 72, 64), 0.02
    v = phantom.ventricle_velocity(shape, rate)
    c = (np.array(shape, dtype=np.float64) - 1) / 2
    centres = [c + np.array([0.0, -0.05, s * 0.08]) * np.array(shape) for s in (-1.0, 1.0)]
    rho = 0.12 * min(shape)

    def div_closed_form(p):
        out = 0.0
        for vc in centres:
            r2 = ((p - vc) ** 2).sum()
            out += (rate / 3.0) * np.exp(-r2 / (2 * rho * rho)) * (3.0 - r2 / (rho * rho))
        return -out

    for vc in centres:
        i = np.rint(vc).astype(int)  # nearest grid point
        div = sum((v[a][tuple(i + e)] - v[a][tuple(i - e)]) / 2.0 for a, e in enumerate(np.eye(3, dtype=int)))
        assert div == pytest.approx(div_closed_form(i.astype(np.float64)), rel=2e-2)  # O(h^2 / rho^2) differences
        assert div == pytest.approx(-rate, rel=0.2)  # the expansion rate, up to the other tail


def test_brain_series_is_seeded_and_sessions_differ():
    a = phantom.brain_series((24, 28, 24), 3, seed=2)
    b = phantom.brain_series((24, 28, 24), 3, seed=2)
    assert a["images"].dtype == np.float32 and a["images"].shape == (3, 24, 28, 24)
    assert np.array_equal(a["images"], b["images"])
    assert np.isfinite(a["images"]).all() and a["images"].min() >= 0.0
    assert not np.array_equal(a["images"][0], a["images"][1])
