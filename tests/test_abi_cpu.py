"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/lbm.h, and the pure-host calls (footprint and
argument validation) behave as documented.  No CUDA compute call is made."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2308_16597_gb300 import build as B
from paper_2308_16597_gb300 import lbm, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.library()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbm.exported_symbols())


def test_header_constants_match_the_binding():
    """Every LBM_* integer constant the header defines (error codes, storage
    formats, boundary and parameter flags) has the same value in the Python
    binding, and every one the binding defines is in the header."""
    import re
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    defs = {}
    for name, val in re.findall(r"#define (LBM_[A-Z0-9_]+) \(?(-?[0-9]+)u?\)?", text):
        defs[name] = int(val)
    assert len(defs) >= 20
    for name, val in defs.items():
        assert getattr(lbm, name) == val, name
    for name in dir(lbm):
        if re.fullmatch(r"LBM_(E[A-Z]+|OK|STORE_[A-Z0-9]+|FLAG_[A-Z_]+|BC_[A-Z_]+)", name):
            assert name in defs, name


def test_build_targets_sm_103a_only():
    """Every translation unit and the link step get exactly one -gencode,
    arch=compute_103a,code=sm_103a (the GPU-side check of the loaded code is
    test_gpu_parity::test_loaded_device_code_is_sm_103)."""
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("gencode" in f or "arch" in f for f in B.FLAGS)


def test_noalloc_rejects_sizes_beyond_its_static_array(lib):
    """Host-side checks of lbm_link_forces_noalloc come before any device
    call, so they run here without a GPU: 8000 disks of radius 20 need
    8000 * (12 * 43 - 12) slots, more than its 2,097,152, and nx * ny beyond
    2^31 - 1 would overflow its int32 node indices.  The pointers are never
    dereferenced (stand-in addresses)."""
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_link_forces_noalloc(16, 1 << 20, 1024, 16, 1000, 1000, 16, 8000, 20.0, 16, 0)
    assert e.value.code == lbm.LBM_ENOSPC
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_link_forces_noalloc(16, 50000 * 50000, 50000, 16, 50000, 50000, 16, 10, 10.0, 16, 0)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:  # pitch below nx
        lbm.lbm_link_forces_noalloc(16, 1 << 20, 999, 16, 1000, 1000, 16, 10, 10.0, 16, 0)
    assert e.value.code == lbm.LBM_EINVAL


def _setup(n_parts=3, nx=64, ny=48, r=5.0):
    rng = np.random.default_rng(1)
    parts = W.rsa_disks(rng, n_parts, r, r + 2, nx - 3 - r, r + 2, ny - 3 - r, 1.0)
    parts["rho"] = 1.5
    return lbm.make_domain(nx, ny), lbm.pack_particles(parts), lbm.make_params(0.05, 0.05)


def test_footprint_counts_every_buffer(lib):
    d, p, prm = _setup()
    b = lbm.lbm_query_footprint(d, p, prm)
    pitch = 64
    ps = pitch * 48
    minimum = 2 * 14 * ps * 4 + 2 * 64 * 48 * 4 + pitch * 48 + 3 * (12 * 13 - 12) * 8
    assert b >= minimum
    d2, p2, prm2 = _setup(n_parts=0)
    assert lbm.lbm_query_footprint(d2, p2, prm2) < b


@pytest.mark.parametrize("bad", ["nx", "nu", "alpha", "rate", "storage", "overlap", "wall", "radius",
                                 "reserved", "minor_below_1", "minor_above_r", "minor_negative",
                                 "minor_nan", "angle_out_of_range"])
def test_invalid_arguments_are_rejected(lib, bad):
    d, p, prm = _setup()
    if bad == "nx":
        d.nx = 3
    elif bad == "nu":
        prm.nu = 0.0
    elif bad == "alpha":
        prm.alpha = -1.0
    elif bad == "rate":
        prm.s_e = 2.5
    elif bad == "storage":
        prm.storage = 7
    elif bad == "overlap":
        p["x"][1], p["y"][1] = p["x"][0] + 3.0, p["y"][0]
    elif bad == "wall":
        p["x"][0] = 2.0
    elif bad == "radius":
        p["r"][0] = 0.5
    elif bad == "reserved":
        d.reserved = 1
    elif bad == "minor_below_1":
        p["b"][0] = 0.5
    elif bad == "minor_above_r":
        p["b"][0] = p["r"][0] + 0.5
    elif bad == "minor_negative":
        p["b"][0] = -1.0
    elif bad == "minor_nan":
        p["b"][0] = np.nan
    elif bad == "angle_out_of_range":
        p["b"][0], p["theta"][0] = 2.0, 2e6
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_query_footprint(d, p, prm)
    assert e.value.code == lbm.LBM_EINVAL


def test_disks_and_ellipses_are_accepted(lib):
    """b = 0 and b = r are disks; 1 <= b < r an ellipse (any angle up to
    1.6e6 rad); the footprint does not depend on b (the zone is the
    circumscribed disk's)."""
    d, p, prm = _setup()
    ref = lbm.lbm_query_footprint(d, p, prm)
    for b, th in ((0.0, 0.0), (5.0, 3.0), (1.0, -7.5), (4.99, 1.5e6)):
        p["b"][:] = b
        p["theta"][:] = th
        assert lbm.lbm_query_footprint(d, p, prm) == ref


def test_particle_struct_matches_the_dtype(lib):
    """lbm_particle is ten doubles: the Python record has the same layout."""
    assert lbm.PARTICLE_DTYPE.itemsize == 80
    assert lbm.PARTICLE_DTYPE.names[-1] == "b"
    assert W.PARTICLE_DTYPE == lbm.PARTICLE_DTYPE


def test_strerror_covers_every_code(lib):
    for code in range(0, -9, -1):  # LBM_OK .. LBM_EBOUNDS
        assert lbm.lbm_strerror(code) != "unknown error"


def test_kernel_names(lib):
    n = lib.lbm_kernel_count()
    names = [lib.lbm_kernel_name(k).decode() for k in range(n)]
    assert "stream_collide" in names and "link_gather_bb_force" in names


def test_product_path_has_no_oracle_import():
    """The package never reaches the oracle: no import of it anywhere under
    the package directory."""
    pkg = os.path.join(ROOT, "paper_2308_16597_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f
                assert "lbm_oracle" not in text, f


def test_bounds_checked_variant_builds_beside_the_default(lib, tmp_path):
    """build(extra=["-DLBM_CHECK"], out=dir) puts the checked library in dir,
    exporting the same entry points, and leaves the default library alone."""
    before = os.path.getmtime(lbm.LIB_PATH)
    path = B.build(force=True, extra=["-DLBM_CHECK"], out=str(tmp_path))
    assert os.path.dirname(path) == str(tmp_path) and os.path.exists(path)
    assert os.path.getmtime(lbm.LIB_PATH) == before
    checked = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(checked, name), name
