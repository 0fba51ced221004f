"""GPU momentum exchange (Sec. 2.4, Eq. force / Eq. torque) against the FP64
oracle on the cases whose oracle results are pinned by momentum and
angular-momentum balance (test_oracle_momentum): a fixed disk in a periodic
box under a body force from a random state, a fixed disk whose surface
translates and spins in resting fluid, and the steady drag of flow through a
periodic array of disks, which must equal the body force on the fluid.

Besides matching the oracle's forces (1e-6 relative for the force, 1e-5 for
the torque, each of its own size or of the other's scaled by the radius when
that is larger), the GPU's own fields obey the balance:
with u = (sum e f + F_b / 2) / rho, the fluid momentum before collision is
sum (rho u - F_b / 2) over the fluid nodes, and one step changes it by
N_fluid F_b - F.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402
import oracle.oracle as orc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def one_disk(x, y, r, ux=0.0, uy=0.0, omega=0.0):
    p = np.zeros(1, W.PARTICLE_DTYPE)
    p["x"], p["y"], p["r"], p["rho"] = x, y, r, 1.5
    p["ux"], p["uy"], p["omega"] = ux, uy, omega
    return p


def gpu_momentum(sim, fluid, Fb):
    drho, ux, uy, _ = (a.astype(np.float64) for a in sim.fields())
    rho = 1.0 + drho
    px = (rho * ux)[fluid].sum() - 0.5 * Fb[0] * fluid.sum()
    py = (rho * uy)[fluid].sum() - 0.5 * Fb[1] * fluid.sum()
    return px, py


def same_forces(Fg, Fo, r):
    """Force within 1e-6 of its size or of 0.1 |T| / r, torque within 1e-5
    of its size or of 0.1 r |F|, whichever is larger: both sum link brackets
    whose FP32 roundings scale with the brackets, and on a single disk one of
    them is often a small difference of such terms (the force on a spinning
    disk, the torque on a disk pushed by a flow)."""
    F, T = np.abs(Fo[:2]).max(), abs(Fo[2])
    assert np.abs(Fg[:2] - Fo[:2]).max() <= 1e-6 * max(F, 0.1 * T / r), (Fg, Fo)
    assert abs(Fg[2] - Fo[2]) <= 1e-5 * max(T, 0.1 * r * F), (Fg, Fo)


@pytest.mark.parametrize("seed", range(2))
def test_body_force_balance_and_oracle_forces(seed):
    nx, ny = 48, 44
    rng = np.random.default_rng(800 + seed)
    parts = one_disk(rng.uniform(18, 30), rng.uniform(17, 27), rng.uniform(4.5, 9.0))
    Fb = (2e-5, -7e-6)
    prm = W.base_params(0.05, 1.0, 0.0, body_fx=Fb[0], body_fy=Fb[1], fixed_particles=1)
    dom = W.cavity(nx, ny, periodic_x=1, periodic_y=1)
    sim = lbm.Simulation(dom, parts, prm)
    ref = orc.Oracle(dom, parts, prm)
    fluid = ref.owner() < 0
    assert np.array_equal(sim.owner() < 0, fluid)
    f, g = W.random_state(nx, ny, 40 + seed, orc.feq(1, 0, 0), orc.geq(1, 0, 0), amp=2e-2)
    sim.set_distributions(f, g)
    ref.set_state(f, g)
    nf = int(fluid.sum())
    for _ in range(3):
        p0 = gpu_momentum(sim, fluid, Fb)
        sim.step(1)
        ref.step(1)
        p1 = gpu_momentum(sim, fluid, Fb)
        Fg, Fo = sim.forces()[0], ref.forces()[0]
        same_forces(Fg, Fo, parts['r'][0])
        scale = np.abs(Fg[:2]).max()
        assert abs(Fg[0] - (nf * Fb[0] - (p1[0] - p0[0]))) < 1e-4 * scale
        assert abs(Fg[1] - (nf * Fb[1] - (p1[1] - p0[1]))) < 1e-4 * scale


@pytest.mark.parametrize("ux,uy,omega", [(0.0, 0.0, 2e-3), (0.0, 0.0, -2e-3), (0.011, -0.004, 1.5e-3)])
def test_moving_wall_forces_match_the_oracle(ux, uy, omega):
    nx, ny = 64, 60
    parts = one_disk(31.6, 29.3, 8.2, ux, uy, omega)
    prm = W.base_params(0.05, 1.0, 0.0, fixed_particles=1)
    dom = W.cavity(nx, ny, periodic_x=1, periodic_y=1)
    sim = lbm.Simulation(dom, parts, prm)
    ref = orc.Oracle(dom, parts, prm)
    for _ in range(3):
        sim.step(1)
        ref.step(1)
        Fg, Fo = sim.forces()[0], ref.forces()[0]
        same_forces(Fg, Fo, parts['r'][0])
        if omega != 0.0:
            assert Fg[2] * omega < 0.0
        if ux != 0.0:
            assert Fg[0] * ux + Fg[1] * uy < 0.0


def test_steady_drag_equals_the_body_force_on_the_gpu():
    nx = ny = 24
    parts = one_disk(11.5, 11.5, 4.6)
    Fb = 1e-6
    prm = W.base_params(0.1, 1.0, 0.0, body_fx=Fb, fixed_particles=1)
    sim = lbm.Simulation(W.cavity(nx, ny, periodic_x=1, periodic_y=1), parts, prm)
    nf = int((sim.owner() < 0).sum())
    sim.step(20000)
    F = sim.forces()[0]
    assert abs(F[0] - nf * Fb) < 1e-4 * nf * Fb
    assert abs(F[1]) < 1e-4 * nf * Fb
