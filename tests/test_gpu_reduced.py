"""Reduced-precision storage: the 14 planes held as BF16 or scaled FP16
deviations (collision, bounce-back and forces still FP32 / FP64), against
the FP64 oracle on the 1024^2 cavity with 300 hot disks of radius 10.

Every stored population is rounded once per step, with unit roundoff
u = 2^-8 (BF16) or 2^-11 (FP16).  The per-field error after 100 steps is a
few u: the collision relaxes the non-conserved moments, so the roundings do
not accumulate step after step, and the fields inherit about one rounding
of their populations (the measured ratio of the BF16 to the FP16 errors is
8 = 2^3 in every field, as that scaling predicts).  The bound is 5u per
field (measured: at most 1.9u, in rho - 1), and the particle centres stay
within the FP32 bound of 1e-4 lattice units.  The measured errors are
printed (pytest -rP).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402
import oracle.oracle as orc  # noqa: E402

STORAGE = {"bf16": lbm.LBM_STORE_BF16, "fp16": lbm.LBM_STORE_FP16}
# unit roundoff of the stored format; per-field rel-L2 bound after 100 steps
UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}
TOL_FACTOR = 5.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def field_errors(got, exp):
    fluid = ~np.isnan(exp[0]) & ~np.isnan(got[0])
    out = {}
    for name, a, b in zip(("rho-1", "ux", "uy", "T"), got, exp):
        a = a[fluid].astype(np.float64)
        b = b[fluid] - (1.0 if name == "rho-1" else 0.0)
        out[name] = (float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)),
                     float(np.abs(a - b).max()))
    return out


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_rest_state_is_exact_in_reduced_storage(storage):
    dom = W.cavity(133, 70)
    sim = lbm.Simulation(dom, None, W.base_params(0.05, 0.71, 1e-4), storage=STORAGE[storage])
    sim.step(50)
    drho, ux, uy, T = sim.fields()
    assert np.all(drho == 0.0) and np.all(ux == 0.0) and np.all(uy == 0.0) and np.all(T == 0.0)
    sim.close()


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("shape,periodic", [((257, 64), (1, 0)), ((300, 37), (0, 0)), ((70, 50), (0, 1))])
def test_ragged_widths_node_by_node(storage, shape, periodic):
    """With 16-bit storage a thread holds two nodes, so a warp spans 64 nodes;
    where the pitch (nx rounded up to 32) is an odd multiple of 32 the last
    warp of each row runs past it, and the first and last warp of a row read
    past the row's ends.  Node by node, each field stays within a few
    roundings of its populations: |error| <= 8 u S with S the sum of the
    node's |f - w| (rho - 1, ux, uy) or |g| (T) in the oracle's state, after
    1 and 3 steps from a random state.  A single wrongly pulled population
    moves a field by about S / 5, many times the bound."""
    nx, ny = shape
    dom = W.cavity(nx, ny, T_wall=(0.3, 0.8, 1.0, 0.1), periodic_x=periodic[0], periodic_y=periodic[1])
    prm = W.base_params(0.03, 0.71, 3e-3, body_fx=1e-5)
    w9, w5 = orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0)
    f, g = W.random_state(nx, ny, 7, w9, w5, amp=2e-2)
    sim = lbm.Simulation(dom, None, prm, storage=STORAGE[storage])
    ref = orc.Oracle(dom, None, prm)
    sim.set_distributions(f, g)
    ref.set_state(f, g)
    u = UNIT_ROUNDOFF[storage]
    for steps in (1, 3):
        sim.step(steps)
        ref.step(steps)
        fo, go = ref.state()
        Sf = np.abs(fo - w9[:, None, None]).sum(0)
        Sg = np.abs(go).sum(0)
        got, exp = sim.fields(), ref.fields()
        worst = 0.0
        for name, a, b, S in zip(("rho-1", "ux", "uy", "T"), got, exp, (Sf, Sf, Sf, Sg)):
            if name == "rho-1":
                b = b - 1.0
            r = np.abs(a.astype(np.float64) - b) / (u * S)
            worst = max(worst, float(r.max()))
            assert np.all(r <= 8.0), (name, steps, float(r.max()), np.unravel_index(int(r.argmax()), r.shape))
        print(storage, shape, steps, "worst error / (u S):", worst)
    sim.close()


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_state_bytes_halve(storage):
    wl = W.parity_256()
    a = lbm.Simulation(wl.domain, wl.particles, wl.params)
    b = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=STORAGE[storage])
    na, nb = len(a.get_state()), len(b.get_state())
    pitch = (wl.nx + 31) // 32 * 32
    ps = (pitch * wl.ny + 63) // 64 * 64
    assert na - nb == 14 * ps * 2  # 14 planes of 4-byte vs 2-byte elements
    a.close()
    b.close()


_REF = {}


def _oracle_100():
    if "fields" not in _REF:
        wl = W.crop_1024()
        ref = orc.Oracle(wl.domain, wl.particles, wl.params)
        ref.step(100)
        _REF["fields"] = ref.fields()
        _REF["parts"] = ref.particles()
    return _REF["fields"], _REF["parts"]


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp16"])
def test_crop1024_against_oracle_after_100_steps(storage):
    wl = W.crop_1024()
    code = lbm.LBM_STORE_FP32 if storage == "fp32" else STORAGE[storage]
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=code)
    sim.step(100)
    exp, eparts = _oracle_100()
    errs = field_errors(sim.fields(), exp)
    gp = sim.particles()
    dpos = float(max(np.abs(gp["x"] - eparts["x"]).max(), np.abs(gp["y"] - eparts["y"]).max()))
    print("storage %s, 1024^2 x 300 disks, 100 steps: %s; max centre error %.3e lu"
          % (storage, {k: "rel-L2 %.3e max-abs %.3e" % v for k, v in errs.items()}, dpos))
    if storage == "fp32":
        for k, (rl2, _) in errs.items():
            assert rl2 <= 1e-5, (k, rl2)
        assert dpos <= 1e-4
    else:
        for k, (rl2, _) in errs.items():
            assert rl2 <= TOL_FACTOR * UNIT_ROUNDOFF[storage], (storage, k, rl2)
        assert dpos <= 1e-4
    sim.close()


def _oracle_1000():
    if "fields1000" not in _REF:
        wl = W.crop_1024()
        ref = orc.Oracle(wl.domain, wl.particles, wl.params)
        ref.step(1000)
        _REF["fields1000"] = ref.fields()
        _REF["parts1000"] = ref.particles()
    return _REF["fields1000"], _REF["parts1000"]


# rel-L2 per field and centre error bounds after 1000 steps (measured on
# GB300: FP32 1.8e-4 / 1.9e-6, FP16 7.7e-3 / 1.6e-3, BF16 0.25 / 4.8e-2)
BOUND_1000 = {"fp32": (1e-3, 1e-4), "fp16": (2e-2, 1e-2), "bf16": (0.5, 0.2)}


@pytest.mark.slow
@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp16"])
def test_crop1024_against_oracle_after_1000_steps(storage):
    """The same crop over 1000 steps.  The flow is unstable (hot disks
    settling into a cold fluid), so differences grow: FP32's 1.5e-6 after 100
    steps is 1.8e-4 after 1000.  FP16 (11-bit mantissa) stays below 1e-2.
    BF16 (8 bits) drifts to rel-L2 0.25: the slow thermal diffusion adds
    increments below the resolution of the raw g near T = 1, so BF16 storage
    is for short horizons only."""
    wl = W.crop_1024()
    code = lbm.LBM_STORE_FP32 if storage == "fp32" else STORAGE[storage]
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=code)
    sim.step(1000)
    exp, eparts = _oracle_1000()
    errs = field_errors(sim.fields(), exp)
    gp = sim.particles()
    dpos = float(max(np.abs(gp["x"] - eparts["x"]).max(), np.abs(gp["y"] - eparts["y"]).max()))
    print("storage %s, 1024^2 x 300 disks, 1000 steps: %s; max centre error %.3e lu"
          % (storage, {k: "rel-L2 %.3e max-abs %.3e" % v for k, v in errs.items()}, dpos))
    bound, bpos = BOUND_1000[storage]
    for k, (rl2, _) in errs.items():
        assert rl2 <= bound, (storage, k, rl2)
    assert dpos <= bpos
    sim.close()


@pytest.mark.slow
@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_full_size_4000_cavity_two_steps_in_reduced_storage(storage):
    """The benchmark's 4000^2 / 4800-disk workload in 16-bit storage, in the
    launch configuration the benchmark's reduced-storage leg times (the
    staged stream-collide): owner map bit-exact at initialisation, every
    field within 5 unit roundoffs (rel-L2) of the FP64 oracle after two
    steps, centres within the FP32 bound."""
    wl = W.sedimentation_4000()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=STORAGE[storage])
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    assert np.array_equal(sim.owner(), ref.owner())
    sim.step(2)
    assert ref.step(2) == 0
    errs = field_errors(sim.fields(), ref.fields())
    print("storage %s, 4000^2 x 4800 disks, 2 steps: %s"
          % (storage, {k: "rel-L2 %.3e max-abs %.3e" % v for k, v in errs.items()}))
    for k, (rl2, _) in errs.items():
        assert rl2 <= TOL_FACTOR * UNIT_ROUNDOFF[storage], (storage, k, rl2)
    pg, po = sim.particles(), ref.particles()
    assert max(np.abs(pg["x"] - po["x"]).max(), np.abs(pg["y"] - po["y"]).max()) < 1e-4
    sim.close()
