"""The allocation-free link-force entry point, checked against lbm_step.

Callers that cannot allocate device memory (their memory belongs to an
allocator or pool they cannot grow, or they run where cudaMalloc is not
allowed) compute particle forces with lbm_link_forces_noalloc, whose only
scratch is a static array inside the library.  This test feeds it the exact
state a simulation handle holds before a step and compares its forces with
the ones that step's own link kernel produces, on two calls in a row.
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


def test_noalloc_rejects_sizes_beyond_its_static_array():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    # 8000 disks of radius 20 need 8000 * (12 * 43 - 12) slots > 2,097,152
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_link_forces_noalloc(16, 1 << 20, 1024, 16, 1000, 1000, 16, 8000, 20.0, 16, 0)
    assert e.value.code == lbm.LBM_ENOSPC
