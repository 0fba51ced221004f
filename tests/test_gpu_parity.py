"""GPU parity: the sm_103a library (through its C ABI) against the FP64 oracle.

Tolerances.  FP32 storage of f - w and g, FP32 collision: a single step from
a common state agrees to rel-L2 <= 1e-6 per field; the coupled 256^2 run
agrees to rel-L2 <= 1e-5 per field (rho - 1, ux, uy, T over the fluid nodes
both runs share) after 100 steps, and the particle centres to 1e-4 lattice
units.  Owner maps and the nodes of the fixed index array built from the
same positions are bit-exact; the FP32 wall fractions q of disks
(double-float |d|^2 - r^2, d.e and discriminant, FP32 square root, sum and
division) agree with the oracle's FP64 q within the per-link bound of
q_bound, derived from those operations' rounding errors.
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


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def compare_fields(sim, ref, tol, min_norm=1e-12):
    got, exp = sim.fields(), ref.fields()
    fluid = ~np.isnan(exp[0]) & ~np.isnan(got[0])
    assert fluid.mean() > 0.5
    errs = {}
    for name, a, b in zip(("rho-1", "ux", "uy", "T"), got, exp):
        a = a[fluid].astype(np.float64)
        b = b[fluid]
        if name == "rho-1":
            b = b - 1.0
        if np.linalg.norm(b) < min_norm * np.sqrt(b.size):
            errs[name] = np.abs(a - b).max()
            assert errs[name] < 1e-7, (name, errs[name])
            continue
        errs[name] = rel_l2(a, b)
        assert errs[name] <= tol, (name, errs[name])
    return errs


EX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
U32 = 2.0 ** -24  # largest relative error of one FP32 rounding


def q_bound(node, oq, nx, parts):
    """Per-slot bound on |q_gpu - q_oracle| for disks, derived from the
    kernels' arithmetic (c = |d|^2 - r^2, d.e and the discriminant in
    double-float; square root, sum and division in FP32; the oracle's FP64
    root rounded to FP32): 5.5 u q + (e_c + q e_de + q e_disc / (2 sqrt(disc)))
    / den with den = -d.e + sqrt(disc), e_c = 2e-9 s, e_de = 5e-11 s,
    e_disc = 1e-8 s, s = max(1, largest centre coordinate / 4096).  Zero for
    an ellipse, whose q both sides round from the same FP64 root."""
    out = np.zeros(len(node))
    base = 0
    for P in parts:
        N = orc.zone_size(P["r"])
        cap = 12 * N - 12
        sl = np.arange(cap)
        n = node[base:base + cap]
        ok = n >= 0
        k = np.where(sl < 4 * N, 1 + sl // N, 5 + (sl - 4 * N) // (2 * N - 3))
        if P["b"] > 0 and P["b"] != P["r"]:
            base += cap
            continue
        i, j = (n % nx).astype(float), (n // nx).astype(float)
        dx, dy = i - P["x"], j - P["y"]
        de = EX9[k] * dx + EY9[k] * dy
        c = dx * dx + dy * dy - P["r"] * P["r"]
        disc = np.maximum(de * de - (EX9[k] ** 2 + EY9[k] ** 2) * c, 0.0)
        sq = np.sqrt(disc)
        den = np.where(ok, sq - de, 1.0)
        q = oq[base:base + cap].astype(np.float64)
        sc = max(1.0, abs(P["x"]) / 4096, abs(P["y"]) / 4096)
        b = 5.5 * U32 * q + (2e-9 * sc + q * 5e-11 * sc + q * 1e-8 * sc / (2 * np.maximum(sq, 1e-300))) / den
        out[base:base + cap] = np.where(ok, b, 0.0)
        base += cap
    return out


def same_q(q, oq, node, nx, parts):
    return np.all(np.abs(q.astype(np.float64) - oq.astype(np.float64)) <= q_bound(node, oq, nx, parts))


def base_f():
    return orc.feq(1.0, 0.0, 0.0), orc.geq(1.0, 0.0, 0.0)


def test_loaded_device_code_is_sm_103():
    """The runtime loaded the library's sm_103a code on this GPU (no PTX JIT
    from another architecture): cudaFuncGetAttributes' binaryVersion."""
    assert lbm.lbm_binary_version() == 103


# --------------------------------------------------------------------------- lattice only
def test_rest_state_stays_exactly_at_rest():
    dom = W.cavity(133, 70)
    sim = lbm.Simulation(dom, None, W.base_params(0.05, 0.71, 1e-4))
    sim.step(100)
    drho, ux, uy, T = sim.fields()
    assert np.all(drho == 0.0) and np.all(ux == 0.0) and np.all(uy == 0.0) and np.all(T == 0.0)


@pytest.mark.parametrize("shape,periodic", [((300, 37), (0, 0)), ((257, 64), (1, 0)),
                                            ((129, 131), (1, 1)), ((5, 4), (0, 0)),
                                            ((520, 9), (0, 1))])
def test_single_step_from_a_random_state(shape, periodic):
    nx, ny = shape
    dom = W.cavity(nx, ny, T_wall=(0.3, 0.8, 1.0, 0.1), periodic_x=periodic[0],
                   periodic_y=periodic[1])
    prm = W.base_params(0.03, 0.71, 3e-3, body_fx=1e-5)
    f, g = W.random_state(nx, ny, 7, *base_f(), amp=2e-2)
    sim = lbm.Simulation(dom, None, prm)
    ref = orc.Oracle(dom, None, prm)
    sim.set_distributions(f, g)
    ref.set_state(f, g)
    compare_fields(sim, ref, 1e-6)
    for steps in (1, 3):
        sim.step(steps)
        ref.step(steps)
        compare_fields(sim, ref, 1e-6)


def test_poiseuille_profile_on_the_gpu():
    H, nu, Fx = 10, 0.1, 1e-6
    prm = W.base_params(nu, 1.0, 0.0, body_fx=Fx)
    sim = lbm.Simulation(W.cavity(64, H, periodic_x=1), None, prm)
    sim.step(20000)
    rho, ux, uy, T = sim.fields()
    y = np.arange(H)
    exact = Fx / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    assert np.abs(ux - exact[:, None]).max() / exact.max() < 1e-4
    assert np.abs(uy).max() < 1e-9


def test_linear_conduction_on_the_gpu():
    H = 8
    prm = W.base_params(0.1, 0.1 / 0.2, 0.0)
    sim = lbm.Simulation(W.cavity(40, H, T_wall=(0, 0, 1.0, 0.0), periodic_x=1), None, prm)
    sim.step(4000)
    T = sim.fields()[3]
    y = np.arange(H)
    assert np.abs(T - (1 - (y + 0.5) / H)[:, None]).max() < 2e-6


def test_mass_conservation_fp32_closed_box():
    prm = W.base_params(0.02, 0.71, 5e-4)
    sim = lbm.Simulation(W.cavity(96, 80, T_wall=(0, 0, 1.0, 0.0)), None, prm)
    n = 96 * 80
    m0 = n + np.nansum(sim.fields()[0].astype(np.float64))
    sim.step(2000)
    m1 = n + np.nansum(sim.fields()[0].astype(np.float64))
    assert abs(m1 - m0) / m0 < 1e-7


# --------------------------------------------------------------------------- geometry
def test_owner_map_and_fixed_slots_are_bit_exact():
    wl = W.parity_256()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    own0 = orc.raster(wl.nx, wl.ny, wl.particles)
    assert np.array_equal(sim.owner(), own0)
    sim.step(1)
    node, q = sim.slots()
    onode, oq, over = orc.build_slots(wl.nx, wl.ny, own0, wl.particles)
    assert over == 0
    assert np.array_equal(node, onode)
    assert same_q(q, oq, node, wl.nx, wl.particles)
    # later steps: slots of the last step equal the oracle's slots built from
    # the positions the GPU had at the start of that step
    for _ in range(3):
        sim.step(29)
        p = sim.particles()
        sim.step(1)
        own = orc.raster(wl.nx, wl.ny, p)
        onode, oq, _ = orc.build_slots(wl.nx, wl.ny, own, p)
        node, q = sim.slots()
        assert np.array_equal(node, onode)
        assert same_q(q, oq, node, wl.nx, p)
        assert np.array_equal(sim.owner(), orc.raster(wl.nx, wl.ny, sim.particles()))


@pytest.mark.parametrize("seed", range(4))
def test_slots_match_brute_force_links_for_random_radii(seed):
    rng = np.random.default_rng(seed)
    nx, ny = int(rng.integers(60, 140)), int(rng.integers(60, 140))
    n = int(rng.integers(2, 8))
    parts = W.rsa_disks(rng, n, rng.uniform(2.5, 12.0, n), 15, nx - 16, 15, ny - 16, 0.5)
    parts["rho"] = 1.5
    prm = W.base_params(0.05, 0.71, 0.0, fixed_particles=1)
    sim = lbm.Simulation(W.cavity(nx, ny), parts, prm)
    sim.step(1)
    own = orc.raster(nx, ny, parts)
    onode, oq, over = orc.build_slots(nx, ny, own, parts)
    node, q = sim.slots()
    assert over == 0 and np.array_equal(node, onode)
    assert same_q(q, oq, node, nx, parts)
    bn, bd, bp, bq = orc.links_bruteforce(nx, ny, own, parts)
    assert (node >= 0).sum() == len(bn)
    assert sim.counters()[7] == len(bn)


def test_largest_supported_disks_slots_and_forces():
    """Radii 28.0 and 28.4: link windows of 63 and 64 columns (zones of 59 and
    60 nodes plus the two-node margins), the limit of the 64-bit row masks, so
    both 32-column ballot words of every row are in use.  Owner map and slots
    bit-exact, q within its derived bound, every brute-force link found, first-step
    forces and fields as for the small disks."""
    nx, ny = 200, 160
    parts = np.zeros(2, W.PARTICLE_DTYPE)
    parts["x"], parts["y"] = [55.3, 140.6], [80.2, 78.9]
    parts["r"] = [28.0, 28.4]
    parts["rho"], parts["T"] = 1.5, 1.0
    assert [orc.zone_size(r) + 4 for r in parts["r"]] == [63, 64]
    prm = W.base_params(0.05, 0.71, 1e-4, fixed_particles=1)
    dom = W.cavity(nx, ny)
    sim = lbm.Simulation(dom, parts, prm)
    ref = orc.Oracle(dom, parts, prm)
    own = orc.raster(nx, ny, parts)
    assert np.array_equal(sim.owner(), own)
    f, g = W.random_state(nx, ny, 5, *base_f(), amp=1e-2)
    sim.set_distributions(f, g)
    ref.set_state(f, g)
    sim.step(1)
    ref.step(1)
    node, q = sim.slots()
    onode, oq, over = orc.build_slots(nx, ny, own, parts)
    assert over == 0 and np.array_equal(node, onode)
    assert same_q(q, oq, node, nx, parts)
    bn, bd, bp, bq = orc.links_bruteforce(nx, ny, own, parts)
    assert (node >= 0).sum() == len(bn) and sim.counters()[7] == len(bn)
    Fg, Fo = sim.forces(), ref.forces()
    assert np.abs(Fg[:, :2] - Fo[:, :2]).max() <= 1e-6 * np.abs(Fo[:, :2]).max()
    assert np.abs(Fg[:, 2] - Fo[:, 2]).max() <= 1e-5 * np.abs(Fo[:, 2]).max()
    compare_fields(sim, ref, 1e-6)
    sim.close()


def worst_link_disks(seed=5):
    """Disks (x, y, r) that put one link (i, j, k) at an extreme of the wall
    fraction's conditioning, centres near x = 3960 (where the FP32 spacing
    of the coordinates is 2^-12): the solid node B = A + e_k barely inside
    (depth 1e-9..1e-6) on a line within 1e-4 rad of tangent to the circle
    (q near 1, discriminant near 0), A barely outside (q near 0), or B
    barely inside (q near 1), for each direction; r = 28.4 on the axis
    directions' odd-numbered ones."""
    rng = np.random.default_rng(seed)
    out = []
    for kind in ("tangent", "q0", "q1"):
        for k in range(1, 9):
            r = 28.4 if k % 2 else float(rng.uniform(9.0, 28.4))
            e = np.array([EX9[k], EY9[k]], float)
            el = np.linalg.norm(e)
            perp = np.array([-e[1], e[0]]) / el
            for _ in range(1000):
                A = np.array([float(rng.integers(3930, 3990)), float(rng.integers(70, 180))])
                B = A + e
                if kind == "tangent":
                    delta, phi = float(rng.uniform(1e-9, 1e-6)), float(rng.uniform(-1e-4, 1e-4))
                    c = B + (r - delta) * (perp * np.cos(phi) - e / el * np.sin(phi))
                else:
                    ang = float(rng.uniform(0, 2 * np.pi))
                    n = np.array([np.cos(ang), np.sin(ang)])
                    c = (A + (r + float(rng.uniform(1e-8, 1e-5))) * n if kind == "q0"
                         else B + (r - float(rng.uniform(1e-8, 1e-5))) * n)
                if np.hypot(*(A - c)) > r >= np.hypot(*(B - c)):
                    out.append((float(c[0]), float(c[1]), r, int(A[0]), int(A[1]), k, kind))
                    break
    return out


def test_wall_fraction_within_its_derived_bound_at_worst_geometries():
    """The disk q of every link within the bound of q_bound, on disks built
    so that one link each sits at a tangent line (discriminant ~1e-5, where
    FP32 roundings of d.e^2 and c would give errors of ~1e-5), at q -> 0 and
    at q -> 1, with centres near x = 3960; slot nodes bit-exact."""
    nx, ny = 4064, 256
    cases = worst_link_disks()
    assert len(cases) == 24
    prm = W.base_params(0.05, 0.71, 0.0, fixed_particles=1)
    worst = 0.0
    for x, y, r, i, j, k, kind in cases:
        parts = np.zeros(1, W.PARTICLE_DTYPE)
        parts["x"], parts["y"], parts["r"], parts["rho"] = x, y, r, 1.5
        sim = lbm.Simulation(W.cavity(nx, ny), parts, prm)
        sim.step(1)
        node, q = sim.slots()
        own = orc.raster(nx, ny, parts)
        onode, oq, over = orc.build_slots(nx, ny, own, parts)
        assert over == 0 and np.array_equal(node, onode)
        assert j * nx + i in set(onode.tolist()), (kind, k)
        err = np.abs(q.astype(np.float64) - oq.astype(np.float64))
        b = q_bound(node, oq, nx, parts)
        assert np.all(err <= b), (kind, k, (err / np.where(b > 0, b, 1)).max())
        worst = max(worst, float((err / np.where(b > 0, b, 1)).max()))
        sim.close()
    print("largest error / bound: %.3f" % worst)


# --------------------------------------------------------------------------- coupled
def test_first_step_forces_match_the_oracle():
    wl = W.parity_256()
    prm = dict(wl.params, fixed_particles=1)
    sim = lbm.Simulation(wl.domain, wl.particles, prm)
    ref = orc.Oracle(wl.domain, wl.particles, prm)
    f, g = W.random_state(wl.nx, wl.ny, 3, *base_f(), amp=1e-2)
    sim.set_distributions(f, g)
    ref.set_state(f, g)
    sim.step(1)
    ref.step(1)
    Fg, Fo = sim.forces(), ref.forces()
    assert np.abs(Fg[:, :2] - Fo[:, :2]).max() <= 1e-6 * np.abs(Fo[:, :2]).max()
    assert np.abs(Fg[:, 2] - Fo[:, 2]).max() <= 1e-5 * np.abs(Fo[:, 2]).max()
    cg, co = sim.counters(), ref.counters()
    assert cg[7] == co[7] and cg[0] == co[0] and cg[1] == co[1] and cg[2] == co[2]
    compare_fields(sim, ref, 1e-6)


def test_cavity_256_eight_disks_100_steps():
    """256^2 cavity, 8 hot disks: fields rel-L2 <= 1e-5 and centres within
    1e-4 lattice units of the FP64 oracle after 100 steps."""
    wl = W.parity_256()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    for _ in range(4):
        sim.step(25)
        assert ref.step(25) == 0
        pg, po = sim.particles(), ref.particles()
        assert np.abs(pg["x"] - po["x"]).max() < 1e-4
        assert np.abs(pg["y"] - po["y"]).max() < 1e-4
    errs = compare_fields(sim, ref, 1e-5)
    print("rel-L2 after 100 steps:", errs)


@pytest.mark.slow
def test_cavity_256_eight_disks_1000_steps():
    """The same run over 1000 steps: particle centres stay within 1e-4
    lattice units of the FP64 oracle at every 100th step; the fields, which
    the settling flow amplifies, within rel-L2 1e-4."""
    wl = W.parity_256()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    worst = 0.0
    for _ in range(10):
        sim.step(100)
        assert ref.step(100) == 0
        pg, po = sim.particles(), ref.particles()
        worst = max(worst, np.abs(pg["x"] - po["x"]).max(), np.abs(pg["y"] - po["y"]).max())
        assert worst < 1e-4, worst
    errs = compare_fields(sim, ref, 1e-4)
    print("1000 steps: centres within %.2e lu, fields rel-L2 %s" % (worst, errs))


def test_moving_disk_refills_like_the_oracle():
    parts = np.zeros(2, W.PARTICLE_DTYPE)
    parts["x"], parts["y"] = [40.3, 90.6], [50.2, 47.7]
    parts["r"], parts["rho"], parts["T"] = 8.5, 1.5, 1.0
    parts["ux"], parts["uy"] = [0.04, -0.03], [-0.02, 0.035]
    dom = W.cavity(140, 100)
    prm = W.base_params(0.05, 0.71, 1e-4)
    sim = lbm.Simulation(dom, parts, prm)
    ref = orc.Oracle(dom, parts, prm)
    nb_g = nb_o = 0
    for _ in range(30):
        sim.step(1)
        ref.step(1)
        nb_g += sim.counters()[6]
        nb_o += ref.counters()[6]
    assert nb_o > 0 and nb_g == nb_o
    compare_fields(sim, ref, 1e-5)
    pg, po = sim.particles(), ref.particles()
    assert np.abs(pg["x"] - po["x"]).max() < 1e-6


def test_disks_leaving_the_side_columns_refill_like_the_oracle():
    """Disks that start over the first and last columns and the first row
    move off them: the uncovered side-column nodes are refilled by the
    general path from the newborn list, the fluid side-column nodes are
    pulled by the stream-collide kernel (wall rule across the side walls),
    and every field, the newborn count and the centres follow the oracle."""
    parts = np.zeros(4, W.PARTICLE_DTYPE)
    parts["x"], parts["y"] = [8.2, 170.8, 90.3, 60.4], [30.3, 62.7, 8.15, 55.0]
    parts["r"], parts["rho"], parts["T"] = 8.5, 1.5, 1.0
    parts["ux"], parts["uy"] = [0.12, -0.12, 0.0, 0.03], [0.0, 0.01, 0.12, -0.02]
    nx, ny = 180, 100
    own0 = orc.raster(nx, ny, parts)
    assert (own0[:, 0] == 0).any() and (own0[:, nx - 1] == 1).any() and (own0[0, :] == 2).any()
    dom = W.cavity(nx, ny, T_wall=(0.3, 0.8, 1.0, 0.1))
    prm = W.base_params(0.05, 0.71, 1e-4, eps_w=1e3)
    sim = lbm.Simulation(dom, parts, prm)
    ref = orc.Oracle(dom, parts, prm)
    nb_g = nb_o = 0
    for _ in range(25):
        sim.step(1)
        assert ref.step(1) == 0
        nb_g += sim.counters()[6]
        nb_o += ref.counters()[6]
    assert nb_o > 0 and nb_g == nb_o
    compare_fields(sim, ref, 1e-5)
    own = orc.raster(nx, ny, sim.particles())
    assert not (own[:, 0] == 0).any() and not (own[:, nx - 1] == 1).any()  # the side columns were uncovered
    pg, po = sim.particles(), ref.particles()
    assert np.abs(pg["x"] - po["x"]).max() < 1e-6 and np.abs(pg["y"] - po["y"]).max() < 1e-6


def state_flags(sim, nx, ny):
    """Node flags (0 fluid, 1 solid, 2 newborn) from the raw state image, laid
    out as include/lbm.h states: 14 FP32 planes of plane_stride elements, the
    int32 owner map [ny][nx], then the uint8 flags [ny][pitch]."""
    pitch = (nx + 31) // 32 * 32
    stride = (pitch * ny + 63) // 64 * 64
    buf = sim.get_state()
    off = 14 * stride * 4 + nx * ny * 4
    return buf[off:off + ny * pitch].reshape(ny, pitch)[:, :nx]


def test_node_flags_are_bit_exact():
    """After every step the flags are the node classes of Sec. 2.3 and 2.5
    from the owner maps before and after it: solid where a particle holds the
    node after the step, newborn where one held it before and none does
    after, fluid elsewhere; both owner maps from the oracle's raster of the
    GPU's positions.  Two translating disks and a translating, spinning
    ellipse uncover nodes every step, and two disks that start over the
    first column and the first row of the cavity uncover nodes of its frame
    (weak wall repulsion keeps them below a node per step)."""
    parts = np.zeros(5, W.PARTICLE_DTYPE)
    parts["x"], parts["y"] = [40.3, 90.6, 140.2, 8.2, 120.4], [50.2, 47.7, 52.9, 30.3, 8.15]
    parts["r"], parts["b"] = [8.5, 8.5, 11.0, 8.5, 8.5], [0.0, 0.0, 5.0, 0.0, 0.0]
    parts["theta"] = [0.0, 0.0, 0.7, 0.0, 0.0]
    parts["rho"], parts["T"] = 1.5, 1.0
    parts["ux"], parts["uy"] = [0.04, -0.03, 0.02, 0.12, 0.0], [-0.02, 0.035, -0.03, 0.0, 0.12]
    parts["omega"] = [0.0, 0.0, 0.02, 0.0, 0.0]
    nx, ny = 180, 100
    own0 = orc.raster(nx, ny, parts)
    assert (own0[:, 0] == 3).any() and (own0[0, :] == 4).any()  # frame nodes inside disks 3 and 4
    sim = lbm.Simulation(W.cavity(nx, ny), parts, W.base_params(0.05, 0.71, 1e-4, eps_w=1e3))
    assert np.array_equal(state_flags(sim, nx, ny), (orc.raster(nx, ny, parts) >= 0).astype(np.uint8))
    newborn = frame_newborn = 0
    for _ in range(25):
        p0 = sim.particles()
        sim.step(1)
        p1 = sim.particles()
        o0, o1 = orc.raster(nx, ny, p0), orc.raster(nx, ny, p1)
        exp = np.where(o1 >= 0, 1, np.where(o0 >= 0, 2, 0)).astype(np.uint8)
        assert np.array_equal(state_flags(sim, nx, ny), exp)
        assert sim.counters()[6] == (exp == 2).sum()
        newborn += int((exp == 2).sum())
        frame_newborn += int((exp[:, 0] == 2).sum() + (exp[0, :] == 2).sum())
    assert newborn > 0 and frame_newborn > 0
    sim.close()


# --------------------------------------------------------------------------- runtime
def test_runs_are_deterministic_and_graphs_match_direct_launches():
    """40 steps replayed as multi-step graphs, launched directly, and in
    chunks that mix multi-step and single-step graphs from both parities."""
    wl = W.parity_256()
    a = lbm.Simulation(wl.domain, wl.particles, wl.params)
    b = lbm.Simulation(wl.domain, wl.particles, wl.params, flags=lbm.LBM_FLAG_NO_GRAPH)
    c = lbm.Simulation(wl.domain, wl.particles, wl.params)
    a.step(40)
    b.step(40)
    for n in (1, 3, 4, 5, 8, 9, 10):
        c.step(n)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.get_state(), c.get_state())
    assert np.array_equal(a.particles(), c.particles())


def test_checkpoint_restore_is_bit_exact():
    wl = W.parity_256()
    a = lbm.Simulation(wl.domain, wl.particles, wl.params)
    a.step(30)
    snap = a.get_state()
    a.step(30)
    b = lbm.Simulation(wl.domain, wl.particles, wl.params)
    b.set_state(snap)
    b.step(30)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.particles(), b.particles())


def test_restore_with_newborn_nodes_keeps_the_flags_exact():
    """A state saved right after a step that uncovered nodes (its flags hold
    newborn nodes) and restored into a new handle: the next steps' flags are
    the node classes of the oracle's rasters, as in a run that never
    stopped, and the two runs stay bit-identical."""
    parts = np.zeros(2, W.PARTICLE_DTYPE)
    parts["x"], parts["y"] = [30.3, 70.6], [30.2, 28.7]
    parts["r"] = 7.5
    parts["rho"], parts["T"] = 1.5, 1.0
    parts["ux"], parts["uy"] = [0.05, -0.04], [0.03, 0.05]
    nx, ny = 100, 60
    dom, prm = W.cavity(nx, ny), W.base_params(0.05, 0.71, 1e-4)
    a = lbm.Simulation(dom, parts, prm)
    a.step(7)
    snap = a.get_state()
    assert (state_flags(a, nx, ny) == 2).any()
    b = lbm.Simulation(dom, parts, prm)
    b.set_state(snap)
    for _ in range(5):
        p0 = b.particles()
        a.step(1)
        b.step(1)
        o0, o1 = orc.raster(nx, ny, p0), orc.raster(nx, ny, b.particles())
        exp = np.where(o1 >= 0, 1, np.where(o0 >= 0, 2, 0)).astype(np.uint8)
        assert np.array_equal(state_flags(b, nx, ny), exp)
    assert np.array_equal(a.get_state(), b.get_state())


def test_async_particle_read_back_equals_the_synchronous_one():
    wl = W.parity_256()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    pinned = torch.empty(len(wl.particles) * lbm.PARTICLE_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    view = pinned.numpy().view(lbm.PARTICLE_DTYPE)
    snaps = []
    for _ in range(3):
        sim.step(7)
        lbm.lbm_get_particles_async(sim.h, view)
        sim.sync()
        snaps.append(view.copy())
        assert view.tobytes() == sim.particles().tobytes()
    assert snaps[0].tobytes() != snaps[2].tobytes()  # the disks moved
    sim.close()


def test_injected_nan_is_reported_and_held():
    """Host-side fault injection: a NaN handed to lbm_set_distributions inside
    a disk is ignored (solid nodes carry no distributions); at a fluid node
    the collision reports it as LBM_ENUMERIC, and the error stays set on the
    handle for the calls after it."""
    wl = W.parity_256()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    f, g = W.random_state(wl.nx, wl.ny, 3, *base_f(), amp=1e-2)
    own = sim.owner()
    js, is_ = np.nonzero(own >= 0)
    f_solid = f.copy()
    f_solid[3, js[0], is_[0]] = np.nan
    sim.set_distributions(f_solid, g)
    sim.step(5)
    assert np.isfinite(sim.particles()["x"]).all()
    jf, if_ = np.nonzero(own < 0)
    k = len(jf) // 2
    g_fluid = g.copy()
    g_fluid[2, jf[k], if_[k]] = np.nan
    with pytest.raises(lbm.LbmError) as e:
        sim.set_distributions(f, g_fluid)
    assert e.value.code == lbm.LBM_ENUMERIC
    with pytest.raises(lbm.LbmError) as e:
        sim.step(1)
        sim.particles()
    assert e.value.code == lbm.LBM_ENUMERIC
    sim.close()


def test_workspace_too_small_is_rejected():
    wl = W.parity_256()
    d = lbm.make_domain(**wl.domain)
    p = lbm.pack_particles(wl.particles)
    prm = lbm.make_params(**wl.params)
    need = lbm.lbm_query_footprint(d, p, prm)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_init(d, p, prm, ws.data_ptr(), need - 256, 0)
    assert e.value.code == lbm.LBM_ENOSPC


def test_kernel_timing_counts_launches():
    wl = W.parity_256()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    sim.kernel_timing(True)
    sim.step(5)
    t = sim.kernel_times()
    assert t["stream_collide"][1] == 5 and t["link_gather_bb_force"][1] == 5
    assert t["stream_collide"][0] > 0.0


# --------------------------------------------------------------------------- full size
@pytest.mark.slow
@pytest.mark.parametrize("make", [W.sedimentation_4000, W.paper_4800])
def test_full_size_4000_cavity_two_steps(make):
    """The 4000^2 / 4800-disk workloads (r = 10 at 9.4 % solid, and the
    paper's d = 40 at 37.7 %) in the benchmark's launch configuration: owner
    map bit-exact at init and every field within FP32 tolerance of the oracle
    after two steps."""
    wl = make()
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params)
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    assert np.array_equal(sim.owner(), ref.owner())
    sim.step(2)
    assert ref.step(2) == 0
    compare_fields(sim, ref, 1e-5)
    pg, po = sim.particles(), ref.particles()
    assert np.abs(pg["y"] - po["y"]).max() < 1e-8


def test_direct_addressing_matches_the_index_array():
    """The comparison of Sec. 3: links found by one thread per node, forces
    summed with atomics.  Same bounce-back values and link counts; forces
    equal to rounding, so the state after 100 steps matches the default to
    rel-L2 1e-6 and both meet the oracle bound."""
    wl = W.parity_256()
    a = lbm.Simulation(wl.domain, wl.particles, wl.params)
    b = lbm.Simulation(wl.domain, wl.particles, wl.params, flags=lbm.LBM_FLAG_DIRECT_LINKS)
    a.step(1)
    b.step(1)
    fa, fb = a.forces(), b.forces()
    assert np.allclose(fa, fb, rtol=1e-9, atol=1e-12)
    assert np.array_equal(a.counters(), b.counters())
    a.step(99)
    b.step(99)
    for x, y in zip(a.fields(), b.fields()):
        m = ~np.isnan(x)
        assert np.array_equal(m, ~np.isnan(y))
        assert rel_l2(x[m], y[m]) < 1e-6
    pa, pb = a.particles(), b.particles()
    assert np.abs(pa["x"] - pb["x"]).max() < 1e-9 and np.abs(pa["y"] - pb["y"]).max() < 1e-9
    ref = orc.Oracle(wl.domain, wl.particles, wl.params)
    ref.step(100)
    compare_fields(b, ref, 1e-5)
    a.close()
    b.close()
