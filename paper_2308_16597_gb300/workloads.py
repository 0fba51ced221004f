"""Seeded synthetic inputs for the sedimentation workloads.

This module only places particles and states the physical parameters of each
workload; it holds none of the lattice Boltzmann arithmetic, so both the CUDA
path and the FP64 oracle take their inputs from here.

The workloads follow the paper's sedimentation benchmarks (Sec. 2.6.3: hot
disks settling in a cold cavity, all four walls no-slip at the cold
temperature, particles seeded in the upper part).  Particle centres are drawn
by random sequential addition from a PCG64 stream, with a minimum centre
distance of 2r + s + 1 so that no two disks start inside each other's
repulsion range (s = 3 lattice units, Sec. 2.4).  The Rayleigh number
Ra = Pr * Gr with Gr = g beta dT L^3 / nu^2 (Sec. 2.1) fixes the gravity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# r: radius, or semi-major axis of an ellipse; b: semi-minor axis (0 for a disk)
PARTICLE_FIELDS = ("x", "y", "ux", "uy", "theta", "omega", "r", "rho", "T", "b")
PARTICLE_DTYPE = np.dtype([(n, "f8") for n in PARTICLE_FIELDS])

S_REP = 3.0  # repulsion threshold, lattice units (Sec. 2.4)


@dataclass
class Workload:
    name: str
    domain: dict
    particles: np.ndarray
    params: dict
    steps: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.domain["nx"])

    @property
    def ny(self) -> int:
        return int(self.domain["ny"])


def gravity_for_rayleigh(Ra: float, nu: float, alpha: float, H: float, beta: float = 1.0,
                         dT: float = 1.0) -> float:
    """g such that Ra = g beta dT H^3 / (nu alpha)."""
    return Ra * nu * alpha / (beta * dT * H ** 3)


def rsa_disks(rng: np.random.Generator, n: int, radii, xlo, xhi, ylo, yhi,
              min_gap: float, max_tries: int = 2_000_000) -> np.ndarray:
    """Random sequential addition of n disks with centres in [xlo,xhi]x[ylo,yhi]
    and centre distance >= r_a + r_b + min_gap.  radii: scalar or length-n."""
    radii = np.broadcast_to(np.asarray(radii, dtype=np.float64), (n,)).copy()
    rmax = float(radii.max()) if n else 0.0
    cell = 2.0 * rmax + min_gap
    grid: dict = {}
    xs = np.empty(n)
    ys = np.empty(n)
    placed = 0
    tries = 0
    while placed < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition could not place %d disks" % n)
        r = radii[placed]
        x = rng.uniform(xlo, xhi)
        y = rng.uniform(ylo, yhi)
        cx, cy = int(x // cell), int(y // cell)
        ok = True
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                for k in grid.get((gx, gy), ()):
                    if math.hypot(x - xs[k], y - ys[k]) < r + radii[k] + min_gap:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        xs[placed], ys[placed] = x, y
        grid.setdefault((cx, cy), []).append(placed)
        placed += 1
    out = np.zeros(n, PARTICLE_DTYPE)
    out["x"], out["y"], out["r"] = xs, ys, radii
    return out


def base_params(nu: float, Pr: float, g: float, beta: float = 1.0, **kw) -> dict:
    p = dict(nu=nu, alpha=nu / Pr, g=g, beta=beta, T0=0.0, rho_f=1.0, T_init=0.0,
             s_e=0.0, s_eps=0.0, s_q=0.0, q_e=0.0, q_nu=0.0, eps_w=1e-3, s_rep=S_REP,
             body_fx=0.0, body_fy=0.0, fixed_particles=0)
    p.update(kw)
    return p


def cavity(nx: int, ny: int, T_wall=(0.0, 0.0, 0.0, 0.0), periodic_x=0, periodic_y=0) -> dict:
    return dict(nx=nx, ny=ny, periodic_x=periodic_x, periodic_y=periodic_y,
                T_wall=tuple(float(t) for t in T_wall))


def sedimentation(nx, ny, n, radius, rho_ratio, y_frac, seed, nu, Pr, g, T_p=1.0,
                  name="sedimentation", steps=0) -> Workload:
    """Hot disks seeded in the upper (1 - y_frac) part of a cold closed cavity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = float(radius)
    lo = r + S_REP + 1.0
    parts = rsa_disks(rng, n, r, lo, nx - 1 - lo, max(y_frac * ny + r + S_REP, lo),
                      ny - 1 - lo, min_gap=S_REP + 1.0)
    parts["rho"] = rho_ratio
    parts["T"] = T_p
    return Workload(name, cavity(nx, ny), parts, base_params(nu, Pr, g), steps)


def parity_256(seed: int = 2308) -> Workload:
    """256x256 cavity, 8 hot disks r = 10 in the upper half, density ratio 1.5,
    g = 1e-5, Pr = 0.71, nu = 0.02, beta = 1, 1000 steps."""
    return sedimentation(256, 256, 8, 10.0, 1.5, 0.5, seed, nu=0.02, Pr=0.71, g=1e-5,
                         name="cavity256_8disks", steps=1000)


def sedimentation_4000(seed: int = 16597) -> Workload:
    """4000x4000 cavity, 4800 hot disks r = 10 (solid fraction 9.4 %) in the upper
    60 %, density ratio 1.5, Pr = 0.71, nu = 0.02, Ra = 1e8 on H = 4000."""
    nu, Pr = 0.02, 0.71
    g = gravity_for_rayleigh(1e8, nu, nu / Pr, 4000.0)
    return sedimentation(4000, 4000, 4800, 10.0, 1.5, 0.4, seed, nu=nu, Pr=Pr, g=g,
                         name="cavity4000_4800disks_r10", steps=10000)


def paper_4800(spacing: float = 50.0) -> Workload:
    """The paper's own 4800-particle benchmark (Sec. 2.6.3 and its parameter
    table): 4000 x 4000 l.u., 4800 hot disks of diameter 40 l.u. (solid
    fraction 37.7 %) in 60 lines of 80 in the upper part of the cavity,
    rho_p = 1.1, nu = 0.01, alpha = 0.002 (Pr = 5), g = 7.84e-6,
    beta = 1.20e-2, Delta_T = 1.  The line spacing is not given; the disks sit
    on a square lattice of pitch 50 l.u. (80 x 50 = 4000) from the top."""
    n_x, n_y = 80, 60
    parts = np.zeros(n_x * n_y, PARTICLE_DTYPE)
    i, j = np.meshgrid(np.arange(n_x), np.arange(n_y))
    parts["x"] = 0.5 * spacing + spacing * i.ravel()
    parts["y"] = 4000.0 - 0.5 * spacing - spacing * j.ravel()
    parts["r"] = 20.0
    parts["rho"] = 1.1
    parts["T"] = 1.0
    return Workload("cavity4000_4800disks_d40_paper", cavity(4000, 4000), parts,
                    base_params(0.01, 5.0, 7.84e-6, beta=1.2e-2), 6000)


def sedimentation_2000(seed: int = 2000) -> Workload:
    """2000x2000 quarter-area version of sedimentation_4000 (1200 disks, same
    density, Ra = 1e8 on H = 2000): the profiling case, 0.46 GB of state."""
    nu, Pr = 0.02, 0.71
    g = gravity_for_rayleigh(1e8, nu, nu / Pr, 2000.0)
    return sedimentation(2000, 2000, 1200, 10.0, 1.5, 0.4, seed, nu=nu, Pr=Pr, g=g,
                         name="cavity2000_1200disks_r10", steps=1000)


def ellipses_256(seed: int = 1657, n: int = 6, a: float = 12.0, b: float = 6.0) -> Workload:
    """256x256 cavity, n hot ellipses with semi-axes a = 12, b = 6 (the 2:1
    aspect ratio of Sec. 2.6.3), orientations uniform in [0, pi), in the upper
    half; density ratio 1.5, g = 1e-5, Pr = 0.71, nu = 0.02.  Placement keeps
    the circumscribed circles (radius a) apart by the repulsion range."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = a + S_REP + 1.0
    parts = rsa_disks(rng, n, a, lo, 255 - lo, 128.0 + a + S_REP, 255 - lo, min_gap=S_REP + 1.0)
    parts["b"] = b
    parts["theta"] = rng.uniform(0.0, math.pi, n)
    parts["rho"] = 1.5
    parts["T"] = 1.0
    return Workload("cavity256_%dellipses" % n, cavity(256, 256), parts, base_params(0.02, 0.71, 1e-5), 1000)


def ellipse_cluster_129(seed: int = 129, ring_step: float = 56.0) -> Workload:
    """Sec. 2.6.3, elliptical hot particles in a cold cavity (Table of that
    case): 1000 x 2000 l.u., 129 ellipses A x B = 50 x 25 l.u. (semi-axes 25
    and 12.5), density 1.5, nu = 0.01, alpha = 0.002 (Pr = 5),
    g = 9.8e-7, beta = 8.16e-3, Delta_T = 1 (particles hot, walls and fluid
    cold).  The cluster: one particle at (W/2, 3H/4) and rings of 6, 12, 18,
    24, 31 and 37 around it.  The ring spacing is not given; ring m sits at
    radius 56 m, so that the circumscribed circles of neighbours on and
    between rings stay the repulsion range apart.  Each ring starts at a
    seeded angle; orientations are uniform in [0, pi)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W_, H_ = 1000, 2000
    xs, ys = [0.5 * W_], [0.75 * H_]
    for m, count in enumerate((6, 12, 18, 24, 31, 37), start=1):
        phase = rng.uniform(0.0, 2.0 * math.pi)
        ang = phase + 2.0 * math.pi * np.arange(count) / count
        xs.extend(0.5 * W_ + m * ring_step * np.cos(ang))
        ys.extend(0.75 * H_ + m * ring_step * np.sin(ang))
    n = len(xs)
    parts = np.zeros(n, PARTICLE_DTYPE)
    parts["x"], parts["y"] = xs, ys
    parts["r"], parts["b"] = 25.0, 12.5
    parts["theta"] = rng.uniform(0.0, math.pi, n)
    parts["rho"] = 1.5
    parts["T"] = 1.0
    prm = base_params(0.01, 5.0, 9.8e-7, beta=8.16e-3)
    return Workload("cavity1000x2000_129ellipses", cavity(W_, H_), parts, prm, 10000)


def crop_1024(seed: int = 3) -> Workload:
    """1024x1024 crop with 300 disks r = 10 in the upper half (reduced storage)."""
    return sedimentation(1024, 1024, 300, 10.0, 1.5, 0.5, seed, nu=0.02, Pr=0.71, g=1e-5,
                         name="cavity1024_300disks", steps=1000)


def ensemble(count: int = 64, seed: int = 4, sizes=(256, 512, 768, 1024), n_range=(8, 400),
             r_range=(6.0, 12.0), u_range=(0.01, 0.04), nu: float = 0.02, Pr: float = 0.71):
    """Batched ensemble of independent cavities: nx and ny drawn independently
    from `sizes`, a disk count from n_range (capped to what random sequential
    addition fits in the upper half at a 25 % solid fraction), per-disk radii
    uniform in r_range, and g beta from a free-fall velocity
    sqrt(g beta dT H) log-uniform in u_range on H = ny, so that
    Ra = u_ff^2 H^2 Pr / nu^2 runs from 1.2e4 to 3e6.  (Ra drawn from
    [1e6, 1e8] on these cavities at nu = 0.02 means free-fall velocities up
    to 0.8 lattice units, which the lattice cannot carry: such instances
    blow up within a thousand steps.)"""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        nx = int(rng.choice(sizes))
        ny = int(rng.choice(sizes))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        radii = rng.uniform(r_range[0], r_range[1], n)
        upper = (nx - 2 * (r_range[1] + S_REP + 1)) * (ny / 2 - 2 * (r_range[1] + S_REP))
        n = max(1, min(n, int(0.25 * upper / (math.pi * np.mean(radii) ** 2))))
        radii = radii[:n]
        u_ff = float(np.exp(rng.uniform(np.log(u_range[0]), np.log(u_range[1]))))
        g = u_ff ** 2 / ny
        alpha = nu / Pr
        Ra = g * ny ** 3 / (nu * alpha)
        rmax = float(radii.max())
        lo = rmax + S_REP + 1.0
        parts = rsa_disks(rng, n, radii, lo, nx - 1 - lo, max(0.5 * ny + rmax + S_REP, lo), ny - 1 - lo,
                          min_gap=S_REP + 1.0)
        parts["rho"] = 1.5
        parts["T"] = 1.0
        out.append(Workload("ensemble%d_%dx%d_%ddisks" % (k, nx, ny, n), cavity(nx, ny), parts,
                            base_params(nu, Pr, g), 0, dict(Ra=Ra, u_ff=u_ff)))
    return out


def served_stream(count: int = 40, seed: int = 5, rate: float = 20.0, sides=(512, 2048),
                  n_range=(50, 1500), step_range=(2000, 20000), radius: float = 10.0,
                  nu: float = 0.02, Pr: float = 0.71, u_ff: float = 0.04):
    """Served stream of sedimentation requests: Poisson arrivals at `rate` per
    second, square cavities with a side drawn from multiples of 256 in
    `sides`, a disk count from n_range (capped to what fits in the upper 60 %
    at a 25 % solid fraction), radius `radius`, step budgets uniform in
    step_range, and g beta from the free-fall velocity sqrt(g beta dT H) =
    u_ff on H = ny (Ra from 1e6 at 512 to 2e7 at 2048: one fixed Ra would
    make the small cavities' flow too fast for the lattice).
    Returns [(arrival_s, Workload, steps)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    choices = list(range(sides[0], sides[1] + 1, 256))
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        side = int(rng.choice(choices))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        upper = (side - 2 * (radius + S_REP + 1)) * (0.4 * side - 2 * (radius + S_REP))
        n = max(1, min(n, int(0.25 * upper / (math.pi * radius ** 2))))
        steps = int(rng.integers(step_range[0], step_range[1] + 1))
        g = u_ff ** 2 / side
        lo = radius + S_REP + 1.0
        parts = rsa_disks(rng, n, radius, lo, side - 1 - lo, max(0.6 * side + radius + S_REP, lo),
                          side - 1 - lo, min_gap=S_REP + 1.0)
        parts["rho"] = 1.5
        parts["T"] = 1.0
        out.append((t, Workload("request%d_%d_%ddisks" % (k, side, n), cavity(side, side), parts,
                                base_params(nu, Pr, g), steps), steps))
    return out


def random_state(nx: int, ny: int, seed: int, base_f, base_g, amp: float = 1e-3,
                 T_amp: float = 0.5):
    """Seeded perturbation of given per-direction base values (e.g. a rest
    equilibrium): f = base_f (1 + amp N(0,1)), g = base_g T (1 + amp N(0,1)) with
    T uniform in [0, T_amp).  Returned as f[9][ny][nx], g[5][ny][nx] in FP64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bf = np.asarray(base_f, dtype=np.float64)
    bg = np.asarray(base_g, dtype=np.float64)
    f = bf[:, None, None] * (1.0 + amp * rng.standard_normal((9, ny, nx)))
    T = T_amp * rng.uniform(0.0, 1.0, (ny, nx))
    g = bg[:, None, None] * T[None] * (1.0 + amp * rng.standard_normal((5, ny, nx)))
    return f, g
