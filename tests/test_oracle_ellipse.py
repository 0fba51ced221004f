"""Pins of the oracle's elliptical particles (Sec. 2.6: ellipses of semi-axes
a > b, major axis at angle theta) against closed forms, brute force and
sampling: the deterministic cos/sin, the inside test, the wall fraction q of
a link, the support distance used by the repulsion, the fixed index array,
the moment of inertia, and the zero force and torque on a resting ellipse."""
import math

import numpy as np
import pytest

from paper_2308_16597_gb300 import workloads as W


def ellipse(x, y, a, b, theta, **kw):
    p = np.zeros(1, W.PARTICLE_DTYPE)
    p["x"], p["y"], p["r"], p["b"], p["theta"] = x, y, a, b, theta
    p["rho"] = kw.get("rho", 1.5)
    p["T"] = kw.get("T", 1.0)
    return p


def test_cos_sin_is_accurate(orc):
    rng = np.random.default_rng(1)
    th = np.concatenate([rng.uniform(-50, 50, 2000), [0.0, math.pi / 4, math.pi / 2, -math.pi, 1e4]])
    for t in th:
        c, s = orc.cos_sin(t)
        assert abs(c - math.cos(t)) <= 4e-16 * max(1.0, abs(t) / 100) + 1e-16
        assert abs(s - math.sin(t)) <= 4e-16 * max(1.0, abs(t) / 100) + 1e-16
    assert orc.cos_sin(0.0) == (1.0, 0.0)


def test_inside_test_at_zero_and_right_angles(orc):
    """theta = 0: the axis-aligned formula; theta = pi/2: a and b swap."""
    a, b = 9.3, 4.1
    p0 = ellipse(20.37, 19.61, a, b, 0.0)
    p90 = ellipse(20.37, 19.61, a, b, math.pi / 2)
    for j in range(8, 33):
        for i in range(8, 33):
            dx, dy = i - 20.37, j - 19.61
            f0 = dx * dx / (a * a) + dy * dy / (b * b)
            f90 = dx * dx / (b * b) + dy * dy / (a * a)
            if abs(f0 - 1) > 1e-9:
                assert orc.in_particle(i, j, p0) == (f0 <= 1)
            if abs(f90 - 1) > 1e-6:
                assert orc.in_particle(i, j, p90) == (f90 <= 1)


def test_equal_axes_is_the_disk(orc):
    p = ellipse(20.2, 19.7, 6.5, 6.5, 0.7)  # b == r: the disk path
    q = ellipse(20.2, 19.7, 6.5, 0.0, 0.7)  # b == 0: the disk path
    own1 = orc.raster(41, 41, p)
    own2 = orc.raster(41, 41, q)
    assert np.array_equal(own1, own2)
    d = np.hypot(np.arange(41)[None, :] - 20.2, np.arange(41)[:, None] - 19.7)
    assert np.array_equal(own1 >= 0, d <= 6.5)


@pytest.mark.parametrize("theta", [0.0, 0.4, 1.3, -2.2])
def test_link_q_lands_on_the_ellipse(orc, theta):
    a, b, xc, yc = 10.4, 5.2, 24.3, 23.8
    p = ellipse(xc, yc, a, b, theta)
    own = orc.raster(48, 48, p)
    c, s = math.cos(theta), math.sin(theta)
    n = 0
    for j in range(48):
        for i in range(48):
            if own[j, i] >= 0:
                continue
            for k, (ex, ey) in enumerate(zip(W_EX, W_EY)):
                if k == 0 or not (0 <= i + ex < 48 and 0 <= j + ey < 48) or own[j + ey, i + ex] < 0:
                    continue
                q = orc.link_q_particle(i, j, k, p)
                assert 0.0 < q <= 1.0
                wx, wy = i + q * ex - xc, j + q * ey - yc
                u, v = wx * c + wy * s, wy * c - wx * s
                assert abs(u * u / (a * a) + v * v / (b * b) - 1.0) < 1e-9
                # the first crossing: the segment before it is outside
                for t in (0.25 * q, 0.5 * q, 0.9 * q):
                    px, py = i + t * ex - xc, j + t * ey - yc
                    pu, pv = px * c + py * s, py * c - px * s
                    assert pu * pu / (a * a) + pv * pv / (b * b) > 1.0
                n += 1
    assert n > 50


W_EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
W_EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


def test_support_distance_closed_forms_and_sampling(orc):
    a, b = 8.0, 3.0
    assert orc.support(ellipse(0, 0, a, b, 0.0), 1.0, 0.0) == a
    assert orc.support(ellipse(0, 0, a, b, 0.0), 0.0, 1.0) == b
    assert orc.support(ellipse(0, 0, a, b, math.pi / 2), 1.0, 0.0) == pytest.approx(b, abs=1e-14)
    rng = np.random.default_rng(3)
    for _ in range(20):
        th = rng.uniform(-3, 3)
        ang = rng.uniform(0, 2 * math.pi)
        n = (math.cos(ang), math.sin(ang))
        t = np.linspace(0, 2 * math.pi, 200001)
        px = a * np.cos(t) * math.cos(th) - b * np.sin(t) * math.sin(th)
        py = a * np.cos(t) * math.sin(th) + b * np.sin(t) * math.cos(th)
        h = (px * n[0] + py * n[1]).max()
        assert orc.support(ellipse(0, 0, a, b, th), *n) == pytest.approx(h, abs=1e-8)
    assert orc.support(ellipse(0, 0, 5.0, 0.0, 1.0), 0.6, 0.8) == 5.0  # a disk


@pytest.mark.parametrize("seed", range(6))
def test_fixed_slots_equal_the_brute_force_links_for_ellipses(orc, seed):
    rng = np.random.default_rng(90 + seed)
    nx = ny = 64
    a = rng.uniform(5.0, 12.0)
    b = a * rng.uniform(0.3, 0.9)
    p = ellipse(rng.uniform(a + 3, nx - a - 4), rng.uniform(a + 3, ny - a - 4), a, b, rng.uniform(-4, 4))
    own = orc.raster(nx, ny, p)
    node, q, over = orc.build_slots(nx, ny, own, p)
    assert over == 0  # a convex body crosses each line of the zone once
    bn, bd, bp, bq = orc.links_bruteforce(nx, ny, own, p)
    brute = {(int(n), int(d)): qq for n, d, qq in zip(bn, bd, bq)}
    got = {}
    N = orc.zone_size(a)
    off = 0
    for k in range(1, 9):
        nl = N if k <= 4 else 2 * N - 3
        for line in range(nl):
            if node[off + line] >= 0:
                got[(int(node[off + line]), k)] = float(q[off + line])
        off += nl
    assert set(got) == set(brute)
    for key, qq in got.items():
        assert qq == np.float32(brute[key])


def test_integrator_uses_the_ellipse_inertia(orc):
    """Constant torque: Omega grows by T / I per step with I = M (a^2 + b^2) / 4
    and M = rho pi a b; the centre follows the force with the same M."""
    a, b, rho = 9.0, 4.0, 1.7
    M = rho * math.pi * a * b
    I = M * (a * a + b * b) / 4
    p = ellipse(30.0, 30.0, a, b, 0.3, rho=rho)[0]
    Tz, Fx = 2.5e-3, 1.0e-3
    q = orc.integrate(p, Fx, 0.0, Tz)
    assert q["omega"] == pytest.approx(Tz / I, rel=1e-14)
    assert q["theta"] == pytest.approx(0.3 + 0.5 * Tz / I, rel=1e-14)
    assert q["ux"] == pytest.approx(Fx / M, rel=1e-14)


@pytest.mark.parametrize("theta", [0.0, 0.6, -1.1])
def test_resting_ellipse_in_resting_fluid_feels_no_force_or_torque(orc, theta):
    """Every lattice line through a convex body meets it in one opposed link
    pair with equal populations, and the pair's wall points lie on the line:
    zero force and zero torque for any shape and orientation."""
    nx, ny = 48, 44
    p = ellipse(23.37, 21.81, 9.2, 4.4, theta)
    prm = W.base_params(0.05, 1.0, 0.0, fixed_particles=1)
    o = orc.Oracle(W.cavity(nx, ny), p, prm)
    o.step(1)
    F = o.forces()[0]
    assert np.abs(F).max() < 1e-14
    assert o.counters()[7] > 0
