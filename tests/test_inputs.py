"""Seeded input generators (CPU): the workloads' geometry and request streams have the
properties the measurements rely on."""
import math

import numpy as np
import pytest

from paper_2310_14746_gb300 import inputs


def test_regular_sphere_field_periodic_and_bounded():
    """The regular matrix repeats with its period along every axis, stays in [0, 1], is 0 at
    a sphere centre and 1 at the corner between spheres."""
    f = inputs.regular_sphere_field(64, period=32, radius_ratio=0.3)
    assert f.shape == (64, 64, 64) and f.dtype == np.float32
    assert f.min() >= 0.0 and f.max() <= 1.0
    np.testing.assert_array_equal(f[:, :, :32], f[:, :, 32:])
    np.testing.assert_array_equal(f[:, :32, :], f[:, 32:, :])
    np.testing.assert_array_equal(f[:32], f[32:])
    assert f[16, 16, 16] == 0.0 and f[0, 0, 0] == 1.0


@pytest.mark.parametrize("ratio", [0.15, 0.3, 0.4])
def test_smoothed_field_keeps_the_sphere_volume(ratio):
    """The smoothing profile is odd about the sphere surface, so the mean of the smoothed
    field matches the void fraction 1 - 4/3 pi r^3 of the sharp sphere to O(w^2 / r^2)."""
    f = inputs.regular_sphere_field(64, period=64, radius_ratio=ratio)
    phi = inputs.sphere_matrix_porosity(ratio)
    w, r = inputs.DEFAULT_WIDTH, ratio * 64
    assert abs(float(f.mean()) - phi) < 4.0 * math.pi * r * w * w / 64 ** 3


def test_configuration_porosity_reading():
    """r = 0.3 of the period gives the void fraction 0.8869 of the benchmark matrix."""
    assert abs(inputs.sphere_matrix_porosity(0.3) - 0.8869) < 1e-4


def test_boolean_model_hits_the_target_void_fraction():
    """Over seeds, the rendered Boolean matrix's void fraction averages the target (the
    count is chosen from exp(-n v) = phi)."""
    vals = []
    for seed in range(6):
        centres, radius = inputs.boolean_sphere_geometry(seed, 0.6, 0.08)
        sharp = inputs.render_sphere_geometry(48, centres, radius, width=1e-6)
        vals.append(float((sharp > 0.5).mean()))
    assert abs(np.mean(vals) - 0.6) < 0.03


def test_serving_stream_properties():
    """Edges from the stated set, periods dividing the edge within [16, 64], radius ratios
    within [0.1, 0.45], increasing arrivals with the requested mean rate, reproducible."""
    a = inputs.serving_requests(400, 123, rate_per_s=2.0)
    b = inputs.serving_requests(400, 123, rate_per_s=2.0)
    assert a == b
    t = np.array([r["arrival_s"] for r in a])
    assert np.all(np.diff(t) > 0)
    assert abs(len(a) / t[-1] - 2.0) < 0.3
    for r in a:
        assert r["edge"] in inputs.SERVING_EDGES
        assert r["edge"] % r["period"] == 0 and 16 <= r["period"] <= 64
        assert 0.1 <= r["radius_ratio"] <= 0.45
    assert {r["edge"] for r in a} == set(inputs.SERVING_EDGES)


def test_random_generators_ranges_and_seeds():
    f = inputs.random_populations(19, (3, 4, 5), seed=1, amplitude=0.5)
    assert f.shape == (19, 3, 4, 5) and f.min() > 0.5 / 19 - 1e-15 and f.max() < 1.5 / 19
    np.testing.assert_array_equal(f, inputs.random_populations(19, (3, 4, 5), seed=1, amplitude=0.5))
    v = inputs.random_porosity((4, 5, 6), seed=2, lo=0.3, hi=0.9)
    assert v.dtype == np.float32 and v.min() >= 0.3 and v.max() <= 0.9
