"""Pins of the oracle's momentum exchange (Sec. 2.4, Eq. force and Eq. torque),
its buoyancy term (Sec. 2.1), the particle weight and the wall repulsion
(Sec. 2.4), against conservation laws and closed forms.

Momentum and angular-momentum balance.  In a fully periodic box streaming
only moves populations, and a collision adds exactly the body force F_b to
the momentum of each fluid node (the moment identity of the Guo forcing,
pinned in test_oracle_pins).  On a link (x_f, e_k) of a fixed particle the
population f_k^+ leaves the fluid into the solid and the bounced-back f_kbar
enters it, so the fluid loses e_k (f_k^+ + f_kbar) of momentum and
(x_f - x_c) x e_k (f_k^+ + f_kbar) of angular momentum about the centre
(streaming keeps the angular momentum of each population, since
(x + e) x e = x x e, away from the periodic seams).  Eq. force and Eq. torque
add the Galilean term -u_w (f_k^+ - f_kbar) to each bracket, so

    F = -(P(t+1) - P(t)) + N_fluid F_b - sum u_w (f_k^+ - f_kbar),
    T = -(L(t+1) - L(t)) + sum (x - x_c) x F_b - sum (x_w - x_c) x u_w (f_k^+ - f_kbar),

with P and L the fluid's momentum and angular momentum before collision.
A sign error in either bracket, a factor, the pre-bounce-back f_kbar in place
of the bounced-back one, or the cross product taken the other way round
breaks one of these identities.
"""
import math

import numpy as np
import pytest

from paper_2308_16597_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def fluid_momentum(f, fluid):
    """Sum over fluid nodes of sum_i e_i f_i (deviations from the rest weights,
    which carry no momentum, to keep the sums small)."""
    d = f - W9[:, None, None]
    px = np.einsum("i,iyx->yx", EX.astype(float), d)
    py = np.einsum("i,iyx->yx", EY.astype(float), d)
    return px[fluid].sum(), py[fluid].sum(), px, py


def fluid_angular_momentum(f, fluid, xc, yc):
    _, _, px, py = fluid_momentum(f, fluid)
    ny, nx = fluid.shape
    X, Y = np.meshgrid(np.arange(nx) - xc, np.arange(ny) - yc)
    return (X * py - Y * px)[fluid].sum()


def one_fixed_disk(x, y, r, ux=0.0, uy=0.0, omega=0.0):
    p = np.zeros(1, W.PARTICLE_DTYPE)
    p["x"], p["y"], p["r"], p["rho"] = x, y, r, 1.5
    p["ux"], p["uy"], p["omega"] = ux, uy, omega
    return p


def galilean_terms(orc, parts, own, f1):
    """sum u_w (f_k^+ - f_kbar) and sum (x_w - x_c) x u_w (f_k^+ - f_kbar) over
    the links of a fixed disk whose fluid starts at rest (f_k^+ = w_k), with
    f_kbar read from the state after the step and the links and wall
    fractions from the oracle's pinned geometry routines."""
    ny, nx = own.shape
    P = parts[0]
    node, d, pid, q = orc.links_bruteforce(nx, ny, own, parts)
    gx = gy = gt = 0.0
    for n, k, qq in zip(node, d, q):
        i, j = int(n) % nx, int(n) // nx
        rx = (i + qq * EX[k]) - P["x"]
        ry = (j + qq * EY[k]) - P["y"]
        uwx = P["ux"] - P["omega"] * ry
        uwy = P["uy"] + P["omega"] * rx
        diff = W9[k] - f1[OPP[k], j, i]
        gx += uwx * diff
        gy += uwy * diff
        gt += (rx * uwy - ry * uwx) * diff
    return gx, gy, gt, len(node)


# ------------------------------------------------------------------ momentum balance
@pytest.mark.parametrize("seed", range(3))
def test_force_equals_the_momentum_the_fluid_loses(orc, seed):
    """Fixed resting disk in a periodic box under a body force, from a random
    state: each step, F = N_fluid F_b - (P(t+1) - P(t)) to rounding."""
    nx, ny = 48, 44
    rng = np.random.default_rng(800 + seed)
    parts = one_fixed_disk(rng.uniform(18, 30), rng.uniform(17, 27), rng.uniform(4.5, 9.0))
    Fb = (2e-5, -7e-6)
    prm = W.base_params(0.05, 1.0, 0.0, body_fx=Fb[0], body_fy=Fb[1], fixed_particles=1)
    o = orc.Oracle(W.cavity(nx, ny, periodic_x=1, periodic_y=1), parts, prm)
    own = o.owner()
    fluid = own < 0
    f, g = W.random_state(nx, ny, 40 + seed, orc.feq(1, 0, 0), orc.geq(1, 0, 0), amp=2e-2)
    f[:, ~fluid] = np.nan
    g[:, ~fluid] = np.nan
    o.set_state(f, g)
    nf = int(fluid.sum())
    for _ in range(4):
        p0x, p0y, _, _ = fluid_momentum(o.state()[0], fluid)
        o.step(1)
        p1x, p1y, _, _ = fluid_momentum(o.state()[0], fluid)
        F = o.forces()[0]
        ex = nf * Fb[0] - (p1x - p0x)
        ey = nf * Fb[1] - (p1y - p0y)
        scale = abs(F[0]) + abs(F[1])
        assert scale > 1e-3  # the random state pushes on the disk
        assert abs(F[0] - ex) < 1e-12 * scale
        assert abs(F[1] - ey) < 1e-12 * scale


def test_steady_drag_balances_the_body_force(orc):
    """At the steady state of flow through a periodic array of fixed disks,
    the fluid's momentum no longer changes, so the drag on the disk equals the
    body force on all fluid nodes, F_x = N_fluid F_b, and F_y = 0."""
    nx, ny = 24, 24
    parts = one_fixed_disk(11.5, 11.5, 4.6)
    Fb = 1e-6
    prm = W.base_params(0.1, 1.0, 0.0, body_fx=Fb, fixed_particles=1)
    o = orc.Oracle(W.cavity(nx, ny, periodic_x=1, periodic_y=1), parts, prm)
    nf = int((o.owner() < 0).sum())
    prev = None
    for _ in range(40):
        o.step(500)
        F = o.forces()[0]
        if prev is not None and abs(F[0] - prev) < 1e-16:
            break
        prev = F[0]
    assert abs(F[0] - nf * Fb) < 1e-9 * nf * Fb
    assert abs(F[1]) < 1e-9 * nf * Fb
    assert abs(F[2]) < 1e-9 * nf * Fb * parts["r"][0]  # symmetric about the flow axis


def test_torque_equals_the_angular_momentum_the_fluid_loses(orc):
    """Fixed resting disk, a random perturbation around it in an otherwise
    resting periodic fluid, no body force: T = -(L(t+1) - L(t)) each step, L
    about the disk centre (the seams carry only rest populations, whose
    crossings cancel)."""
    nx, ny = 72, 68
    xc, yc, r = 35.3, 33.8, 7.4
    parts = one_fixed_disk(xc, yc, r)
    prm = W.base_params(0.05, 1.0, 0.0, fixed_particles=1)
    o = orc.Oracle(W.cavity(nx, ny, periodic_x=1, periodic_y=1), parts, prm)
    own = o.owner()
    fluid = own < 0
    f, g = W.random_state(nx, ny, 77, orc.feq(1, 0, 0), orc.geq(1, 0, 0), amp=2e-2)
    X, Y = np.meshgrid(np.arange(nx) - xc, np.arange(ny) - yc)
    far = np.hypot(X, Y) > r + 12
    f[:, far] = W9[:, None]
    f[:, ~fluid] = np.nan
    g[:, ~fluid] = np.nan
    o.set_state(f, g)
    for _ in range(4):
        L0 = fluid_angular_momentum(o.state()[0], fluid, xc, yc)
        o.step(1)
        L1 = fluid_angular_momentum(o.state()[0], fluid, xc, yc)
        T = o.forces()[0][2]
        assert abs(T) > 1e-3
        assert abs(T + (L1 - L0)) < 1e-11 * abs(T)


@pytest.mark.parametrize("ux,uy,omega", [(0.0, 0.0, 2e-3), (0.0, 0.0, -2e-3), (0.011, -0.004, 1.5e-3)])
def test_moving_wall_force_and_torque_from_the_balance(orc, ux, uy, omega):
    """A fixed disk whose surface moves (translation U, spin Omega) in resting
    periodic fluid: one step's F and T equal the momentum and angular
    momentum the fluid lost plus the Galilean terms of Eq. force / Eq. torque
    (to rounding), and the torque opposes the spin."""
    nx, ny = 64, 60
    xc, yc, r = 31.6, 29.3, 8.2
    parts = one_fixed_disk(xc, yc, r, ux, uy, omega)
    prm = W.base_params(0.05, 1.0, 0.0, fixed_particles=1)
    o = orc.Oracle(W.cavity(nx, ny, periodic_x=1, periodic_y=1), parts, prm)
    own = o.owner()
    fluid = own < 0
    f0 = o.state()[0]
    p0x, p0y, _, _ = fluid_momentum(f0, fluid)
    L0 = fluid_angular_momentum(f0, fluid, xc, yc)
    o.step(1)
    f1 = o.state()[0]
    p1x, p1y, _, _ = fluid_momentum(f1, fluid)
    L1 = fluid_angular_momentum(f1, fluid, xc, yc)
    F = o.forces()[0]
    gx, gy, gt, nlinks = galilean_terms(orc, parts, own, f1)
    assert nlinks == o.counters()[7]
    scale = abs(F[0]) + abs(F[1]) + abs(F[2]) / r
    assert abs(F[0] - (-(p1x - p0x) - gx)) < 1e-12 * scale
    assert abs(F[1] - (-(p1y - p0y) - gy)) < 1e-12 * scale
    assert abs(F[2] - (-(L1 - L0) - gt)) < 1e-12 * scale * r
    if omega != 0.0:
        assert F[2] * omega < 0.0  # the fluid resists the spin
    if ux != 0.0 or uy != 0.0:
        assert F[0] * ux + F[1] * uy < 0.0  # and the translation


# ------------------------------------------------------------------ buoyancy
@pytest.mark.parametrize("T,T0", [(0.7, 0.2), (0.1, 0.6)])
def test_buoyancy_closed_form_in_a_uniform_periodic_box(orc, T, T0):
    """Uniform fluid at rest at temperature T in a periodic box: the force
    density rho g beta (T - T0) y-hat (y up) adds its value to the momentum
    every step, and u = (sum e f + F/2) / rho, so after n steps
    u_y = (n + 1/2) g beta (T - T0), u_x = 0: hot fluid rises, cold sinks."""
    g, beta = 1e-4, 2.0
    prm = W.base_params(0.05, 1.0, g, beta=beta, T0=T0, T_init=T)
    o = orc.Oracle(W.cavity(8, 6, periodic_x=1, periodic_y=1), None, prm)
    Fy = g * beta * (T - T0)
    for n in range(4):
        rho, ux, uy, TT = o.fields()
        assert np.abs(rho - 1.0).max() < 1e-15
        assert np.abs(TT - T).max() < 1e-15
        assert np.abs(ux).max() < 1e-18
        assert np.abs(uy - (n + 0.5) * Fy).max() < 1e-15  # rounding of sums of f ~ 1/9
        o.step(1)


def test_hot_fixed_disk_drives_a_rising_plume(orc):
    """A hot fixed disk in a cold closed cavity: the fluid above it rises and
    warms, the flow at its sides and below goes the other way round."""
    nx = ny = 64
    parts = one_fixed_disk(31.5, 27.5, 6.0)
    parts["T"] = 1.0
    prm = W.base_params(0.05, 0.71, 2e-4, fixed_particles=1)
    o = orc.Oracle(W.cavity(nx, ny), parts, prm)
    o.step(400)
    rho, ux, uy, T = o.fields()
    above = uy[36:44, 28:36]
    below = uy[12:19, 28:36]
    assert np.nanmean(above) > 1e-5
    assert np.nanmean(above) > np.nanmean(below)
    assert np.nanmean(T[36:44, 28:36]) > np.nanmean(T[12:19, 28:36])


# ------------------------------------------------------------------ weight and walls
@pytest.mark.parametrize("rho_p", [1.5, 0.8])
def test_first_step_weight_closed_form(orc, rho_p):
    """A disk at rest in resting isothermal fluid, far from the walls: the
    links give no force (pinned in test_oracle_pins), so the first step
    gives U_y = -(rho_p - rho_f) pi r^2 g / (rho_p pi r^2), U_x = 0 and
    y(1) = y(0) + U_y / 2: heavy disks sink, light ones rise."""
    g, r = 1e-4, 6.3
    p = np.zeros(1, W.PARTICLE_DTYPE)
    p["x"], p["y"], p["r"], p["rho"] = 30.2, 31.7, r, rho_p
    o = orc.Oracle(W.cavity(60, 64), p, W.base_params(0.05, 1.0, g))
    o.step(1)
    assert np.abs(o.forces()).max() < 1e-14
    q = o.particles()[0]
    Uy = -(rho_p - 1.0) * math.pi * r * r * g / (rho_p * math.pi * r * r)
    assert abs(q["uy"] - Uy) < 1e-16
    assert abs(q["ux"]) < 1e-16
    assert abs(q["y"] - (31.7 + 0.5 * Uy)) < 1e-14
    assert q["x"] == 30.2
    assert np.sign(q["uy"]) == (-1.0 if rho_p > 1.0 else 1.0)


def test_wall_repulsion_pushes_away_from_each_wall(orc):
    """Four resting disks, each 1 lattice unit (the gap from the half-way
    wall plane to the surface) from one wall, in resting fluid: the first
    step's velocity is the closed-form spring force (C / eps)((gap - s) / s)^2
    of Sec. 2.4, C = pi r^2 (rho_p - rho_f) g, pointing away from the wall,
    plus the weight; the links give no force."""
    nx = ny = 80
    r, rho_p, g, eps, s, gap = 6.0, 1.5, 1e-4, 1e-3, 3.0, 1.0
    # centres whose surfaces lie `gap` from the wall planes at -1/2 and n - 1/2
    lo, hi = -0.5 + gap + r, (nx - 0.5) - r - gap
    p = np.zeros(4, W.PARTICLE_DTYPE)
    p["x"] = [lo, hi, 40.0, 40.0]
    p["y"] = [40.0, 40.0, lo, hi]
    p["r"], p["rho"] = r, rho_p
    o = orc.Oracle(W.cavity(nx, ny), p, W.base_params(0.05, 1.0, g, eps_w=eps, s_rep=s))
    o.step(1)
    assert np.abs(o.forces()).max() < 1e-14
    q = o.particles()
    C = math.pi * r * r * (rho_p - 1.0) * g
    rep = C / eps * ((gap - s) / s) ** 2
    M = rho_p * math.pi * r * r
    Wt = (rho_p - 1.0) * math.pi * r * r * g
    exp_ux = [rep / M, -rep / M, 0.0, 0.0]
    exp_uy = [-Wt / M, -Wt / M, (rep - Wt) / M, (-rep - Wt) / M]
    assert np.allclose(q["ux"], exp_ux, rtol=1e-13, atol=1e-18)
    assert np.allclose(q["uy"], exp_uy, rtol=1e-13, atol=1e-18)
    assert q["ux"][0] > 0 > q["ux"][1] and q["uy"][2] > 0 > q["uy"][3]
