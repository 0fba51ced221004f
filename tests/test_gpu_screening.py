"""Pair screening through the cell grid (the 3 x 3 cells around each
particle, filled by the previous update) against screening all pairs
(LBM_FLAG_ALL_PAIRS): the pair forces are summed in exact fixed point, so
the states agree bit for bit; a grid cell that overflows (more than 16
particles) makes the next step scan all pairs, with the same result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402
import oracle.oracle as orc  # noqa: E402
from test_gpu_batch import snapshot, same  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def dense_pack(seed, n=60, nx=160, ny=120, radii=(4.0, 6.0), ellipses=False):
    """Disks (and ellipses) packed 0.5 l.u. apart, so that many pairs are
    inside the repulsion range from the first step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(*radii, n)
    parts = W.rsa_disks(rng, n, r, 8.0, nx - 9.0, 8.0, ny - 9.0, min_gap=0.5)
    if ellipses:
        half = rng.random(n) < 0.5
        parts["b"] = np.where(half, np.maximum(1.0, 0.55 * parts["r"]), 0.0)
        parts["theta"] = rng.uniform(0.0, np.pi, n)
    parts["rho"] = 1.5
    parts["T"] = 1.0
    return W.Workload("dense", W.cavity(nx, ny), parts, W.base_params(0.05, 0.71, 2e-6))


def run(wl, steps, flags=0):
    s = lbm.Simulation(wl.domain, wl.particles, wl.params, flags=flags)
    s.step(steps)
    out = snapshot(s)
    s.close()
    return out


@pytest.mark.parametrize("ellipses", [False, True])
def test_grid_screening_equals_all_pairs(ellipses):
    wl = dense_pack(11, ellipses=ellipses)
    a = run(wl, 150)
    b = run(wl, 150, lbm.LBM_FLAG_ALL_PAIRS)
    same(a, b)
    # the pairs did push: positions moved away from a run without repulsion
    assert np.abs(a["parts"]["x"] - wl.particles["x"]).max() > 1e-4


def test_overflowing_cell_falls_back_to_all_pairs():
    """One disk of radius 24 sets the cell side to 53; 40 disks of radius 2
    packed 1.5 l.u. apart next to it put more than 16 into one cell."""
    rng = np.random.Generator(np.random.PCG64(5))
    big = np.zeros(1, W.PARTICLE_DTYPE)
    big["x"], big["y"], big["r"] = 150.0, 70.0, 24.0
    small = W.rsa_disks(rng, 40, 2.0, 20.0, 60.0, 40.0, 80.0, min_gap=1.5)
    parts = np.concatenate([big, small])
    parts["rho"], parts["T"] = 1.5, 1.0
    wl = W.Workload("overflow", W.cavity(200, 140), parts, W.base_params(0.05, 0.71, 2e-6))
    side = 2 * 24.0 + 3.0 + 2.0
    cx, cy = (small["x"] // side).astype(int), (small["y"] // side).astype(int)
    assert np.bincount(cx * 8 + cy).max() > 16
    a = run(wl, 60)
    b = run(wl, 60, lbm.LBM_FLAG_ALL_PAIRS)
    same(a, b)
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    sim.step(60)
    assert ref.step(60) == 0
    pg, po = sim.particles(), ref.particles()
    err = max(np.abs(pg["x"] - po["x"]).max(), np.abs(pg["y"] - po["y"]).max())
    print("centres vs oracle:", err, "moved:", np.abs(pg["x"] - wl.particles["x"]).max())
    assert err < 1e-4
    sim.close()
