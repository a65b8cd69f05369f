"""The seeded synthetic inputs that the oracle tests, the GPU parity tests and
the benchmark share (no arithmetic of the method lives here).

* Right-hand sides are reproducible from their seed, uniform on [-1, 1), and
  the benchmark's right-hand side is the seed-0 field plus the smooth mode
  sin(2 pi x) cos(2 pi y) zeta.
* Vertical grids: spacings grow by the stated ratio from the bottom, and the
  interfaces span exactly [base, base + thickness]; the panel's levels follow
  r_k = 1 + (k/n_z)^2 H.
* alpha = 1 + 0.5 sin(2 pi x) sin(2 pi y) is sampled at face midpoints.
* The served request stream is reproducible, its arrivals increase, and its
  sizes, anisotropies (10^2..10^5) and lambda^2 (1e-4..1) stay in range.
"""
import math

import numpy as np
import pytest

import workloads as W


def test_rhs_reproducible_and_uniform():
    p = W.box_problem(12, 10, 6, 0.01)
    a = W.rhs_for(p, seed=3)
    assert a.shape == p.shape and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    assert np.array_equal(a, W.rhs_for(p, seed=3))
    assert not np.array_equal(a, W.rhs_for(p, seed=4))
    assert a.min() >= -1.0 and a.max() < 1.0
    big = W.uniform_rhs((200000,), seed=0)
    assert abs(big.mean()) < 0.01 and abs(big.var() - 1.0 / 3.0) < 0.01
    bs = W.batched_rhs(p, [3, 7])
    assert bs.shape == (2,) + p.shape
    assert np.array_equal(bs[0], a) and np.array_equal(bs[1], W.rhs_for(p, seed=7))


def test_benchmark_rhs_is_seed0_plus_smooth_mode():
    p = W.medium_box(scale=16, n_z=8)
    b = W.medium_box_rhs(p)
    mode = b - W.uniform_rhs(p.shape, 0)
    x = (np.arange(p.n_x) + 0.5) / p.n_x
    y = (np.arange(p.n_y) + 0.5) / p.n_y
    zc = 0.5 * (p.z_iface[:-1] + p.z_iface[1:])
    zeta = (zc - p.z_iface[0]) / (p.z_iface[-1] - p.z_iface[0])
    for k in (0, p.n_z - 1):
        for j in (0, 3):
            for i in (1, 5):
                ref = math.sin(2 * math.pi * x[i]) * math.cos(2 * math.pi * y[j]) * zeta[k]
                assert abs(mode[k, j, i] - ref) <= 1e-15
    assert 0.0 < zeta[0] < zeta[-1] < 1.0


@pytest.mark.parametrize("n_z,thickness,ratio,base", [(16, 0.01, 1.05, 0.0), (64, 0.002, 1.05, 1.0), (7, 1.0, 1.0, 0.0)])
def test_graded_interfaces(n_z, thickness, ratio, base):
    z = W.graded_interfaces(n_z, thickness, ratio, base=base)
    assert len(z) == n_z + 1 and z[0] == base and z[-1] == base + thickness
    dz = np.diff(z)
    assert np.all(dz > 0)
    np.testing.assert_allclose(dz[1:] / dz[:-1], ratio, rtol=1e-9)


def test_panel_levels_are_quadratic():
    p = W.panel_problem(8, 8, 10, thickness=0.02)
    k = np.arange(11)
    np.testing.assert_allclose(p.z_iface, 1.0 + (k / 10) ** 2 * 0.02, rtol=0, atol=1e-15)
    assert np.all(p.alpha_e == 6.71e-4) and p.lambda2 == 1.0


def test_sinusoidal_alpha_at_face_midpoints():
    n_x, n_y = 8, 6
    ae, an = W.sinusoidal_alpha(n_x, n_y)
    assert ae.shape == an.shape == (n_y, n_x)
    j, i = 2, 5
    assert abs(ae[j, i] - (1 + 0.5 * math.sin(2 * math.pi * (i + 1) / n_x) * math.sin(2 * math.pi * (j + 0.5) / n_y))) < 1e-15
    assert abs(an[j, i] - (1 + 0.5 * math.sin(2 * math.pi * (i + 0.5) / n_x) * math.sin(2 * math.pi * (j + 1) / n_y))) < 1e-15
    assert ae.min() >= 0.5 and ae.max() <= 1.5


def test_named_workload_shapes():
    assert W.small_box().shape == (16, 32, 32)
    m = W.medium_box()
    assert m.shape == (128, 256, 256) and abs(m.z_iface[-1] - 0.004) < 1e-18
    lb = W.large_box()
    assert lb.shape == (128, 1024, 1024) and lb.alpha_e is not None
    sb = W.shell_band()
    assert sb.shape == (64, 640, 1440) and abs(sb.lat1 - math.radians(80.0)) < 1e-15
    assert abs(sb.z_iface[0] - 1.0) < 1e-15 and abs(sb.z_iface[-1] - 1.002) < 1e-15


def test_request_stream():
    a = W.request_stream(duration_s=1.0, rate_hz=200.0, seed=1)
    b = W.request_stream(duration_s=1.0, rate_hz=200.0, seed=1)
    assert [r.arrival_s for r in a] == [r.arrival_s for r in b]
    assert 150 <= len(a) <= 250                      # Poisson(200): within 3.5 standard deviations
    t = [r.arrival_s for r in a]
    assert all(t1 > t0 for t0, t1 in zip(t, t[1:])) and t[-1] <= 1.0
    for r in a:
        p = r.problem
        assert p.n_x in (64, 128, 256, 512) and p.n_y in (64, 128, 256, 512) and p.n_z in (32, 64, 128)
        h = math.sqrt(1.0 / (p.n_x * p.n_y))
        aniso = (p.n_z * h / (p.z_iface[-1] - p.z_iface[0])) ** 2
        assert 1e2 * (1 - 1e-9) <= aniso <= 1e5 * (1 + 1e-9)
        assert 1e-4 <= p.lambda2 <= 1.0
        assert r.rhs_seed == 1000 + r.index
    assert len(W.request_stream(duration_s=1.0, rate_hz=200.0, seed=1, max_requests=5)) == 5
