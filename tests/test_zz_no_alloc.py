"""The allocation-free link-force entry point, checked against lbm_step.

Callers that cannot allocate device memory (their memory belongs to an
allocator or pool they cannot grow, or they run where cudaMalloc is not
allowed) compute particle forces with lbm_link_forces_noalloc, whose only
scratch is a static array inside the library.  These tests feed it the exact
state a simulation handle holds before a step and compare its forces with
the ones that step's own link kernel produces, and its bounce-back values and
forces with the FP64 oracle's, each on two calls in a row.  (Its host-side
size and argument checks need no GPU and run in test_abi_cpu.)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402


def _layout(nx, ny):
    pitch = (nx + 31) // 32 * 32
    ps = (pitch * ny + 63) // 64 * 64
    return pitch, ps


@pytest.mark.parametrize("make", [W.parity_256, W.ellipses_256])
def test_noalloc_forces_match_the_step_kernel_on_two_calls(make):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    wl = make()
    nx, ny, n = wl.nx, wl.ny, len(wl.particles)
    pitch, ps = _layout(nx, ny)
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    sim.step(40)
    state = sim.get_state()
    a_bytes = 14 * ps * 4
    own_bytes = nx * ny * 4
    flag_bytes = pitch * ny
    nf = len(lbm.PARTICLE_DTYPE.names)  # particle state: nf arrays of n doubles
    soa = state[a_bytes + own_bytes + flag_bytes:a_bytes + own_bytes + flag_bytes + nf * n * 8]
    soa = soa.view(np.float64).reshape(nf, n)
    parts = np.zeros(n, lbm.PARTICLE_DTYPE)
    for f, name in enumerate(lbm.PARTICLE_DTYPE.names):
        parts[name] = soa[f]
    dev = torch.device("cuda")
    own = torch.from_numpy(state[a_bytes:a_bytes + own_bytes].view(np.int32).copy()).to(dev)
    pdev = torch.from_numpy(parts.view(np.uint8).copy()).to(dev)
    stream = torch.cuda.current_stream()

    sim.step(1)
    ref = sim.forces()
    assert np.isfinite(ref).all() and np.abs(ref).max() > 0

    for call in range(2):
        dist = torch.from_numpy(state[:a_bytes].view(np.float32).copy()).to(dev)
        out = torch.full((3 * n,), 7.0, dtype=torch.float64, device=dev)
        lbm.lbm_link_forces_noalloc(dist.data_ptr(), ps, pitch, own.data_ptr(), nx, ny,
                                    pdev.data_ptr(), n, float(parts["r"].max()), out.data_ptr(),
                                    stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(n, 3)
        scale = np.abs(ref).max(axis=0)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (call, np.abs(got - ref).max(axis=0))


def test_noalloc_bounce_back_values_and_forces_match_the_oracle():
    """From a common random state with moving fixed disks (translation and
    spin enter the wall term): the bounce-back values the call writes into
    the caller's planes equal the oracle's f_kbar(x_f, t+1) and g_kbar(x_f,
    t+1) on every link, and its forces the oracle's, on two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import oracle.oracle as orc
    wl = W.parity_256()
    parts = wl.particles.copy()
    rng = np.random.default_rng(11)
    parts["ux"] = rng.uniform(-0.01, 0.01, len(parts))
    parts["uy"] = rng.uniform(-0.01, 0.01, len(parts))
    parts["omega"] = rng.uniform(-1e-3, 1e-3, len(parts))
    prm = dict(wl.params, fixed_particles=1)
    nx, ny, n = wl.nx, wl.ny, len(parts)
    pitch, ps = _layout(nx, ny)
    sim = lbm.Simulation(wl.domain, parts, prm)
    ref = orc.Oracle(wl.domain, parts, prm)
    f, gg = W.random_state(nx, ny, 5, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), amp=1e-2)
    sim.set_distributions(f, gg)
    ref.set_state(f, gg)
    state = sim.get_state()
    own0 = ref.owner()
    ref.step(1)
    fo, go = ref.state()
    Fo = ref.forces()
    a_bytes = 14 * ps * 4
    dev = torch.device("cuda")
    own = torch.from_numpy(own0.ravel().copy()).to(dev)
    pdev = torch.from_numpy(lbm.pack_particles(parts).view(np.uint8).copy()).to(dev)
    node, kdir, _, _ = orc.links_bruteforce(nx, ny, own0, parts)
    i_f, j_f = node % nx, node // nx
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    opp = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    kb = opp[kdir]
    solid_at = (j_f + ey[kdir]) * pitch + (i_f + ex[kdir])
    exp_f = fo[kb, j_f, i_f]
    ax = kdir <= 4
    exp_g = go[kb[ax], j_f[ax], i_f[ax]]
    for call in range(2):
        dist = torch.from_numpy(state[:a_bytes].view(np.float32).copy()).to(dev)
        out = torch.full((3 * n,), 7.0, dtype=torch.float64, device=dev)
        lbm.lbm_link_forces_noalloc(dist.data_ptr(), ps, pitch, own.data_ptr(), nx, ny, pdev.data_ptr(), n,
                                    float(parts["r"].max()), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        planes = dist.cpu().numpy().reshape(14, ps)
        got_f = planes[kb, solid_at].astype(np.float64) + w9[kb]
        got_g = planes[9 + kb[ax], solid_at[ax]].astype(np.float64)
        tol_f = 1e-5 * np.abs(exp_f - w9[kb]).max()
        tol_g = 1e-5 * np.abs(exp_g).max()
        assert np.abs(got_f - exp_f).max() <= tol_f, (call, np.abs(got_f - exp_f).max(), tol_f)
        assert np.abs(got_g - exp_g).max() <= tol_g, (call, np.abs(got_g - exp_g).max(), tol_g)
        F = out.cpu().numpy().reshape(n, 3)
        assert np.abs(F[:, :2] - Fo[:, :2]).max() <= 1e-6 * np.abs(Fo[:, :2]).max(), call
        assert np.abs(F[:, 2] - Fo[:, 2]).max() <= 1e-5 * np.abs(Fo[:, 2]).max(), call
