"""Batched instances (lbm_batch_*): several independent simulations of
different sizes, particle counts and radii stepped with one launch per step
kernel over all of them give, for every instance, exactly (bit for bit) the
state that lbm_step gives it alone, in every storage, before and after the
tile autotuner, and match the FP64 oracle's run of that instance (fields
rel-L2 <= 1e-5 in FP32 storage and <= 5u in 16-bit storage, u the format's
unit roundoff, centres within 1e-4 lattice units); mismatched handles are
rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402
import oracle.oracle as orc  # noqa: E402

# per-field rel-L2 bound against the FP64 oracle by storage (test_gpu_parity,
# test_gpu_reduced): FP32 1e-5; 5u with u = 2^-8 (BF16), 2^-11 (FP16)
ORACLE_TOL = {lbm.LBM_STORE_FP32: 1e-5, lbm.LBM_STORE_BF16: 5 * 2.0 ** -8, lbm.LBM_STORE_FP16: 5 * 2.0 ** -11}


def oracle_run(wl, steps):
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    assert ref.step(steps) == 0
    return ref.fields(), ref.particles()


def check_against_oracle(fields, parts, ref, storage):
    """fields: (rho - 1, ux, uy, T) float32 of a GPU run; ref: the oracle's
    (rho, ux, uy, T) and particles after the same steps."""
    exp, eparts = ref
    fluid = ~np.isnan(exp[0]) & ~np.isnan(fields[0])
    assert fluid.mean() > 0.5
    for name, a, b in zip(("rho-1", "ux", "uy", "T"), fields, exp):
        a = a[fluid].astype(np.float64)
        b = b[fluid] - (1.0 if name == "rho-1" else 0.0)
        nb = np.linalg.norm(b)
        if nb < 1e-12 * np.sqrt(b.size):  # a field at rest: exactly zero in every storage
            assert np.abs(a - b).max() < 1e-7, name
            continue
        err = np.linalg.norm(a - b) / nb
        assert err <= ORACLE_TOL[storage], (name, err)
    if len(eparts):
        assert np.abs(parts["x"] - eparts["x"]).max() < 1e-4
        assert np.abs(parts["y"] - eparts["y"]).max() < 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def small_ensemble():
    """Five uneven cavities: sizes 70 x 50 .. 224 x 160, 0 to 12 disks of
    radius 5 to 8 (one instance without particles), settling from rest under
    a gravity of 1e-5."""
    rng = np.random.Generator(np.random.PCG64(77))
    shapes = [(96, 64, 3), (128, 160, 8), (70, 50, 0), (224, 112, 12), (64, 96, 1)]
    out = []
    for k, (nx, ny, n) in enumerate(shapes):
        if n:
            radii = rng.uniform(5.0, 8.0, n)
            lo = 8.0 + W.S_REP + 1.0
            parts = W.rsa_disks(rng, n, radii, lo, nx - 1 - lo, max(0.4 * ny, lo), ny - 1 - lo,
                                min_gap=W.S_REP + 1.0)
            parts["rho"] = 1.5
            parts["T"] = 1.0
        else:
            parts = np.zeros(0, W.PARTICLE_DTYPE)
        out.append(W.Workload("small%d" % k, W.cavity(nx, ny), parts, W.base_params(0.02, 0.71, 1e-5)))
    return out


def snapshot(sim):
    return dict(fields=sim.fields(), parts=sim.particles(), owner=sim.owner(), slots=sim.slots(),
                state=sim.get_state(), counters=sim.counters())


def same(a, b):
    for f, g in zip(a["fields"], b["fields"]):
        assert np.array_equal(f, g, equal_nan=True)
    assert a["parts"].tobytes() == b["parts"].tobytes()
    assert np.array_equal(a["owner"], b["owner"])
    for x, y in zip(a["slots"], b["slots"]):
        assert np.array_equal(x, y)
    assert bytes(a["state"]) == bytes(b["state"])
    assert np.array_equal(a["counters"], b["counters"])


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP32, lbm.LBM_STORE_BF16, lbm.LBM_STORE_FP16])
def test_batch_equals_each_instance_alone(storage):
    wls = small_ensemble()
    steps = 40
    alone = []
    for wl in wls:
        s = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=storage)
        s.step(steps)
        alone.append(snapshot(s))
        s.close()
    sims = [lbm.Simulation(wl.domain, wl.particles, wl.params, storage=storage) for wl in wls]
    b = lbm.Batch(sims)
    b.step(steps // 2)
    choice = b.autotune(2)
    assert choice in ((0, 1, 2) if storage == lbm.LBM_STORE_FP32 else (0, 1, 2, 3))
    b.step(steps - steps // 2)
    b.sync()
    assert b.launch_count() == 5 * steps  # links, particles (+ raster), flags, stream-collide, boundary
    for s, ref in zip(sims, alone):
        same(snapshot(s), ref)
    for s, wl in zip(sims, wls):
        check_against_oracle(s.fields(), s.particles(), oracle_run(wl, steps), storage)
    b.close()
    # the instances keep stepping on their own afterwards
    sims[0].step(1)
    sims[0].sync()
    for s in sims:
        s.close()


def test_batch_rejects_mismatched_handles():
    wls = small_ensemble()[:2]
    a = lbm.Simulation(wls[0].domain, wls[0].particles, wls[0].params)
    b = lbm.Simulation(wls[1].domain, wls[1].particles, wls[1].params, storage=lbm.LBM_STORE_BF16)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Batch([a, b])
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.Batch([a, a])
    for s in (a, b):
        s.close()


def test_batch_of_instances_at_different_steps():
    """A handle that has already taken an odd number of steps joins a batch
    with a fresh one (the serving case); both match their runs alone."""
    wls = small_ensemble()
    w0, w1 = wls[0], wls[3]
    ref0 = lbm.Simulation(w0.domain, w0.particles, w0.params)
    ref0.step(10)
    ref1 = lbm.Simulation(w1.domain, w1.particles, w1.params)
    ref1.step(13)
    a = lbm.Simulation(w0.domain, w0.particles, w0.params)
    c = lbm.Simulation(w1.domain, w1.particles, w1.params)
    c.step(3)
    c.sync()
    bt = lbm.Batch([a, c])
    bt.step(10)
    bt.sync()
    same(snapshot(a), snapshot(ref0))
    same(snapshot(c), snapshot(ref1))
    bt.close()
    for s in (a, c, ref0, ref1):
        s.close()


def test_batch_stops_on_own_step_parity_mismatch():
    wls = small_ensemble()[:2]
    sims = [lbm.Simulation(w.domain, w.particles, w.params) for w in wls]
    bt = lbm.Batch(sims)
    bt.step(2)
    bt.sync()
    sims[1].step(1)
    with pytest.raises(lbm.LbmError) as e:
        bt.step(1)
    assert e.value.code == lbm.LBM_EINVAL
    bt.close()
    for s in sims:
        s.close()


def test_escaping_disk_raises_domain_error_and_is_held():
    """A disk flung at a wall (10 lattice units per step) raises LBM_EDOMAIN;
    it is held inside the cavity, so the handle keeps answering."""
    wl = small_ensemble()[4]
    parts = wl.particles.copy()
    parts["ux"] = 10.0
    s = lbm.Simulation(wl.domain, parts, wl.params)
    s.step(3)
    with pytest.raises(lbm.LbmError) as e:
        s.sync()
    assert e.value.code in (lbm.LBM_EDOMAIN, lbm.LBM_ENUMERIC)
    got = np.zeros(len(parts), lbm.PARTICLE_DTYPE)
    with pytest.raises(lbm.LbmError):
        s.particles(got)  # copies the state, then reports the sticky error
    assert np.all(got["x"] - got["r"] >= -0.5) and np.all(got["x"] + got["r"] <= wl.nx - 0.5)
    torch.cuda.synchronize()  # the context is intact
    s.close()


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_FP32, lbm.LBM_STORE_BF16])
@pytest.mark.parametrize("flags", [lbm.LBM_FLAG_OVERLAP, lbm.LBM_FLAG_OVERLAP | lbm.LBM_FLAG_NO_GRAPH,
                                   lbm.LBM_FLAG_NO_GRAPH])
def test_step_schedules_are_bit_identical(flags, storage):
    """Stream-collide split into a far-tile pass beside the particle kernels
    and a near-tile pass after them (with BF16 storage both through the
    staged kernel) gives exactly the state of the default single pass after
    them, with or without graphs."""
    wl = W.parity_256()
    a = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=storage)
    b = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=storage, flags=flags)
    a.step(60)
    b.step(60)
    same(snapshot(a), snapshot(b))
    a.close()
    b.close()
