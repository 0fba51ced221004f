"""The bounds-checked build (-DLBM_CHECK) in place of a memory checker.

That build checks the scattered writes of the particle kernels (fixed index
array, bounce-back values, owner map, flags, screening grid) and every read
and write of the stream-collide fast path (including the reads past the row
ends of the first and last warp of a row, which the buffers' tail pads are
sized for) against the buffer they address; an index outside it is skipped
and reported as LBM_EBOUNDS at the next synchronising call.  The test builds
it beside the default library and runs, in a child process that loads it,
the cases that reach the edges: FP32 disks and ellipses that move, the
largest supported disks, ragged widths in every storage (where the last
block of a row overhangs the pitch, and for 16-bit storage a warp of 64
nodes straddles it), periodic seams, the split stream-collide, and a batch.
"""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import numpy as np
    from paper_2308_16597_gb300 import lbm, workloads as W

    def run(sim, steps):
        sim.step(steps)
        p = sim.particles()          # synchronises: raises on LBM_EBOUNDS
        f = sim.fields()
        assert np.isfinite(p["x"]).all()
        return f

    wl = W.parity_256()
    s = lbm.Simulation(wl.domain, wl.particles, wl.params)
    run(s, 60)
    s.close()
    wl = W.ellipses_256()
    s = lbm.Simulation(wl.domain, wl.particles, wl.params)
    run(s, 60)
    s.close()

    parts = np.zeros(2, W.PARTICLE_DTYPE)
    parts["x"], parts["y"] = [55.3, 140.6], [80.2, 78.9]
    parts["r"] = [28.0, 28.4]
    parts["rho"], parts["T"] = 1.5, 1.0
    s = lbm.Simulation(W.cavity(200, 160), parts, W.base_params(0.05, 0.71, 1e-4))
    run(s, 10)
    s.close()

    w9 = np.array([4/9] + [1/9] * 4 + [1/36] * 4)
    w5 = np.array([0.6] + [0.1] * 4)
    for storage in (lbm.LBM_STORE_FP32, lbm.LBM_STORE_BF16, lbm.LBM_STORE_FP16):
        for (nx, ny), per in (((257, 64), (1, 0)), ((300, 37), (0, 0)), ((70, 50), (0, 1))):
            dom = W.cavity(nx, ny, T_wall=(0.3, 0.8, 1.0, 0.1), periodic_x=per[0], periodic_y=per[1])
            s = lbm.Simulation(dom, None, W.base_params(0.03, 0.71, 3e-3), storage=storage)
            f, g = W.random_state(nx, ny, 7, w9, w5, amp=2e-2)
            s.set_distributions(f, g)
            run(s, 5)
            s.close()

    wl = W.parity_256()
    s = lbm.Simulation(wl.domain, wl.particles, wl.params, flags=lbm.LBM_FLAG_OVERLAP)
    run(s, 20)
    s.close()

    sims = []
    for k, (nx, ny, n) in enumerate(((96, 64, 3), (70, 50, 2), (224, 112, 3))):
        rng = np.random.Generator(np.random.PCG64(70 + k))
        parts = W.rsa_disks(rng, n, 6.0, 16.0, nx - 17.0, 0.4 * ny, ny - 17.0, min_gap=W.S_REP + 1.0)
        parts["rho"], parts["T"] = 1.5, 1.0
        sims.append(lbm.Simulation(W.cavity(nx, ny), parts, W.base_params(0.02, 0.71, 1e-5),
                                   storage=lbm.LBM_STORE_BF16))
    b = lbm.Batch(sims)
    b.step(20)
    b.sync()
    for s in sims:
        s.particles()
    b.close()
    for s in sims:
        s.close()
    print("checked build: no out-of-bounds index")
""")


def test_bounds_checked_build_finds_no_out_of_bounds_index(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16597_gb300 import build as B
    lib = B.build(force=True, extra=["-DLBM_CHECK"], out=str(tmp_path))
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no out-of-bounds index" in r.stdout
