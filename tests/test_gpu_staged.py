"""The staged stream-collide kernel of the 16-bit storages (persistent
blocks, row tiles copied into shared memory by bulk asynchronous copies two
tiles ahead) against the one-block-per-tile kernel that reads global memory
directly (LBM_FLAG_SC_UNSTAGED).  Both apply the same pulls and the same
collision arithmetic to every node, so whole states (distributions, owner
map, flags, particles) must agree bit for bit, in BF16 and FP16, on ragged
widths (the last tile of a row overhanging the pitch), periodic seams, side
walls and moving disks with newborn nodes; the fields are also checked
against the FP64 oracle.  Its bounded waits are exercised by a run that
makes them run out: the step reports LBM_ETIMEOUT, and the device stays
usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402
import oracle.oracle as orc  # noqa: E402

STORAGE = {"bf16": lbm.LBM_STORE_BF16, "fp16": lbm.LBM_STORE_FP16}
# unit roundoff of the stored format; per-field rel-L2 bound against the oracle
UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def both(domain, parts, params, storage, flags=0):
    a = lbm.Simulation(domain, parts, params, storage=STORAGE[storage], flags=flags)
    b = lbm.Simulation(domain, parts, params, storage=STORAGE[storage],
                       flags=flags | lbm.LBM_FLAG_SC_UNSTAGED)
    return a, b


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("shape,periodic", [((257, 64), (1, 0)), ((300, 37), (0, 0)), ((70, 50), (0, 1)),
                                            ((600, 40), (1, 1)), ((32, 9), (0, 0)), ((1000, 130), (0, 0))])
def test_staged_equals_unstaged_from_a_random_state(storage, shape, periodic):
    """Random states on widths whose pitch is and is not a multiple of the
    tile (256 nodes), with side walls or seams: every population after 1 and
    4 steps is the same bits."""
    nx, ny = shape
    dom = W.cavity(nx, ny, T_wall=(0.3, 0.8, 1.0, 0.1), periodic_x=periodic[0], periodic_y=periodic[1])
    prm = W.base_params(0.03, 0.71, 3e-3, body_fx=1e-5)
    f, g = W.random_state(nx, ny, 11, orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0), amp=2e-2)
    a, b = both(dom, None, prm, storage)
    a.set_distributions(f, g)
    b.set_distributions(f, g)
    for n in (1, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_staged_equals_unstaged_with_moving_disks(storage):
    """The 256^2 parity cavity with its eight falling hot disks, plus a disk
    spinning and moving at the left wall: newborn nodes, the side columns and
    the first and last rows all change hands over 60 steps; states and
    particles stay bit-identical, and after the first 20 steps every field is
    within 5 unit roundoffs (rel-L2) of the FP64 oracle, the bound of the
    reduced-storage tests."""
    wl = W.parity_256()
    parts = np.concatenate([wl.particles, wl.particles[:1].copy()])
    parts[-1]["x"], parts[-1]["y"] = 11.5, 60.3
    parts[-1]["ux"], parts[-1]["uy"], parts[-1]["omega"] = -0.02, 0.03, 0.01
    a, b = both(wl.domain, parts, wl.params, storage)
    ref = orc.Oracle(wl.domain, parts, wl.params)
    a.step(20)
    b.step(20)
    assert ref.step(20) == 0
    assert np.array_equal(a.get_state(), b.get_state())
    got, exp = a.fields(), ref.fields()
    fluid = ~np.isnan(exp[0]) & ~np.isnan(got[0])
    for name, x, y in zip(("rho-1", "ux", "uy", "T"), got, exp):
        x = x[fluid].astype(np.float64)
        y = y[fluid] - (1.0 if name == "rho-1" else 0.0)
        assert np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-30) < 5.0 * UNIT_ROUNDOFF[storage], name
    for n in (1, 7, 32):
        a.step(n)
        b.step(n)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.particles(), b.particles())
    assert a.counters()[6] == b.counters()[6]
    a.close()
    b.close()


def test_staged_work_counter_is_reset_between_launches():
    """The staged kernel's blocks claim row tiles from a device counter that
    its last block resets: many launches in a row, replayed from graphs and
    launched directly, on a lattice with more tiles than resident blocks and
    on one with fewer, give the same states as the unstaged kernel."""
    for nx, ny in ((2048, 700), (64, 48)):
        dom = W.cavity(nx, ny, T_wall=(0.0, 0.0, 1.0, 0.0))
        prm = W.base_params(0.05, 0.71, 1e-4)
        a, b = both(dom, None, prm, "bf16")
        c = lbm.Simulation(dom, None, prm, storage=lbm.LBM_STORE_BF16, flags=lbm.LBM_FLAG_NO_GRAPH)
        for n in (1, 2, 9, 16):
            a.step(n)
            b.step(n)
            c.step(n)
        assert np.array_equal(a.get_state(), b.get_state())
        assert np.array_equal(a.get_state(), c.get_state())
        for s in (a, b, c):
            s.close()


def test_bounded_wait_reports_timeout_and_the_device_stays_usable():
    """With LBM_FLAG_TEST_WAIT_TIMEOUT the kernel announces one byte more than
    its copies bring, so no stage's barrier completes: every block gives up
    after its bounded wait (about a second), records the timeout and leaves.
    The step reports LBM_ETIMEOUT (held on the handle), and a new simulation
    on the same device then runs normally."""
    dom = W.cavity(96, 40)
    prm = W.base_params(0.05, 0.71, 1e-4)
    sim = lbm.Simulation(dom, None, prm, storage=lbm.LBM_STORE_BF16, flags=lbm.LBM_FLAG_TEST_WAIT_TIMEOUT)
    with pytest.raises(lbm.LbmError) as e:
        sim.step(1)
        sim.sync()
    assert e.value.code == lbm.LBM_ETIMEOUT
    with pytest.raises(lbm.LbmError) as e:
        sim.sync()
    assert e.value.code == lbm.LBM_ETIMEOUT
    sim.close()
    ok = lbm.Simulation(dom, None, prm, storage=lbm.LBM_STORE_BF16)
    ok.step(3)
    ok.sync()
    drho, ux, uy, T = ok.fields()
    assert np.all(drho == 0.0) and np.all(T == 0.0)
    ok.close()


def test_batched_bounded_wait_reports_timeout():
    """The staged kernel over a batch waits the same bounded way: with
    LBM_FLAG_TEST_WAIT_TIMEOUT on its instances every wait runs out, the
    timeout lands in instance 0's error word, and lbm_batch_sync reports
    LBM_ETIMEOUT; a new batch on the same device then runs normally."""
    dom = W.cavity(300, 40)
    prm = W.base_params(0.05, 0.71, 1e-4)
    sims = [lbm.Simulation(dom, None, prm, storage=lbm.LBM_STORE_BF16, flags=lbm.LBM_FLAG_TEST_WAIT_TIMEOUT)
            for _ in range(2)]
    b = lbm.Batch(sims)
    b.step(1)
    with pytest.raises(lbm.LbmError) as e:
        b.sync()
    assert e.value.code == lbm.LBM_ETIMEOUT
    b.close()
    for s in sims:
        s.close()
    sims = [lbm.Simulation(dom, None, prm, storage=lbm.LBM_STORE_BF16) for _ in range(2)]
    b = lbm.Batch(sims)
    b.step(3)
    b.sync()
    for s in sims:
        drho, ux, uy, T = s.fields()
        assert np.all(drho == 0.0) and np.all(T == 0.0)
    b.close()
    for s in sims:
        s.close()
