"""Host logic on the CPU: the synthetic workload generators of the batched
and served forms (valid, non-overlapping, seeded), the bench helpers, and
the argument checks of the batch and server entry points (which fail before
touching a device)."""
import ctypes as C
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2308_16597_gb300 import workloads as W  # noqa: E402


def _valid_layout(wl):
    p = wl.particles
    nx, ny = wl.nx, wl.ny
    assert np.all(p["x"] - p["r"] >= W.S_REP) and np.all(p["x"] + p["r"] <= nx - 1 - W.S_REP)
    assert np.all(p["y"] - p["r"] >= W.S_REP) and np.all(p["y"] + p["r"] <= ny - 1 - W.S_REP)
    d = np.hypot(p["x"][:, None] - p["x"][None], p["y"][:, None] - p["y"][None])
    rr = p["r"][:, None] + p["r"][None] + W.S_REP + 1.0
    np.fill_diagonal(d, np.inf)
    assert np.all(d >= rr - 1e-9)


def test_ensemble_matches_its_recipe():
    e = W.ensemble(64, seed=4)
    assert len(e) == 64
    for wl in e:
        assert wl.nx in (256, 512, 768, 1024) and wl.ny in (256, 512, 768, 1024)
        n = len(wl.particles)
        assert 1 <= n <= 400
        assert np.all((wl.particles["r"] >= 6.0) & (wl.particles["r"] <= 12.0))
        # g beta from the free-fall velocity on H = ny, and Ra from g
        u = wl.extra["u_ff"]
        assert 0.01 <= u <= 0.04
        p = wl.params
        assert p["g"] * p["beta"] == pytest.approx(u * u / wl.ny)
        assert wl.extra["Ra"] == pytest.approx(p["g"] * p["beta"] * wl.ny ** 3 / (p["nu"] * p["alpha"]))
        assert 1e4 <= wl.extra["Ra"] <= 3.1e6
        assert np.all(wl.particles["y"] >= 0.5 * wl.ny)
    for wl in e[:8]:
        _valid_layout(wl)
    # seeded: the same call gives the same ensemble
    f = W.ensemble(64, seed=4)
    assert all(a.particles.tobytes() == b.particles.tobytes() for a, b in zip(e, f))


def test_served_stream_matches_its_recipe():
    s = W.served_stream(40, seed=5)
    assert len(s) == 40
    t = [a for a, _, _ in s]
    assert all(b > a for a, b in zip(t, t[1:]))
    gaps = np.diff([0.0] + t)
    assert 0.02 < gaps.mean() < 0.08  # Poisson at 20/s
    for _, wl, steps in s:
        assert wl.nx == wl.ny and 512 <= wl.nx <= 2048 and wl.nx % 256 == 0
        assert 2000 <= steps <= 20000
        assert 1 <= len(wl.particles) <= 1500
        assert np.all(wl.particles["r"] == 10.0)
        assert math.sqrt(wl.params["g"] * wl.ny) == pytest.approx(0.04)
    _valid_layout(s[0][1])


def test_paper_shaped_benchmark_matches_its_recipe():
    """60 lines of 80 disks of diameter 40 on a 50 l.u. lattice in the upper
    part of the 4000^2 cavity: 37.7 % solid, clear of the walls and of each
    other by more than the repulsion range."""
    wl = W.paper_4800()
    p = wl.particles
    assert len(p) == 4800 and np.all(p["r"] == 20.0) and np.all(p["b"] == 0.0)
    assert len(np.unique(p["y"])) == 60 and len(np.unique(p["x"])) == 80
    assert len(p) * math.pi * 20.0 ** 2 / (4000.0 * 4000.0) == pytest.approx(0.377, abs=5e-4)
    assert np.all(p["x"] - 20.0 > W.S_REP) and np.all(p["x"] + 20.0 < 3999.0 - W.S_REP)
    assert np.all(p["y"] + 20.0 < 3999.0 - W.S_REP) and p["y"].min() > 1000.0
    # nearest neighbours on the lattice are 50 apart: a gap of 10 l.u.
    assert np.diff(np.unique(p["x"])).min() == 50.0 and np.diff(np.unique(p["y"])).min() == 50.0
    prm = wl.params
    assert prm["nu"] / prm["alpha"] == pytest.approx(5.0) and np.all(p["rho"] == 1.1)


def test_ellipse_cluster_matches_its_recipe():
    """One ellipse at (W/2, 3H/4) and rings of 6, 12, 18, 24, 31, 37 around
    it; semi-axes 25 and 12.5; circumscribed circles clear of each other."""
    wl = W.ellipse_cluster_129()
    p = wl.particles
    assert len(p) == 129 and np.all(p["r"] == 25.0) and np.all(p["b"] == 12.5)
    dist = np.hypot(p["x"] - 500.0, p["y"] - 1500.0)
    rings = np.round(dist / 56.0).astype(int)
    assert np.array_equal(np.bincount(rings), [1, 6, 12, 18, 24, 31, 37])
    d = np.hypot(p["x"][:, None] - p["x"][None], p["y"][:, None] - p["y"][None])
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 50.0 + W.S_REP
    assert np.all((p["theta"] >= 0.0) & (p["theta"] < math.pi))
    assert len(p) * math.pi * 25.0 * 12.5 / (1000.0 * 2000.0) == pytest.approx(0.063, abs=5e-4)


def test_weighted_percentile():
    import bench
    v = [3.0, 1.0, 2.0, 10.0]
    w = [1, 1, 1, 1]
    assert bench.weighted_percentile(v, w, 0.5) == 2.0
    assert bench.weighted_percentile(v, w, 0.99) == 10.0
    # a heavily weighted value dominates
    assert bench.weighted_percentile([1.0, 5.0], [99, 1], 0.5) == 1.0
    assert bench.weighted_percentile([1.0, 5.0], [1, 99], 0.5) == 5.0


def test_traffic_record_is_tied_to_the_kernel_source():
    import bench
    v = bench.profiled_traffic("stream_collide", "cavity4000_4800disks_r10")
    # either the record matches the current source or it is withheld
    assert v is None or 1.5e9 < v < 2.0e9
    assert bench.profiled_traffic("no_such_kernel", "cavity4000_4800disks_r10") is None
    # a record of one workload is not reported for another
    assert bench.profiled_traffic("stream_collide", "cavity1000x2000_129ellipses") is None


def test_batch_and_server_reject_bad_arguments():
    from paper_2308_16597_gb300 import lbm
    lib = lbm.library()
    h = C.c_void_p()
    size = C.c_size_t()
    assert lib.lbm_batch_footprint(None, 0, C.byref(size)) == lbm.LBM_EINVAL
    assert lib.lbm_batch_create(C.byref(h), None, 1, None, 0, None) == lbm.LBM_EINVAL
    assert lib.lbm_batch_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_batch_destroy(None) == lbm.LBM_EINVAL
    assert lib.lbm_server_create(C.byref(h), None, 1 << 20, 4, None) == lbm.LBM_EINVAL
    assert lib.lbm_server_create(C.byref(h), C.c_void_p(256), 1 << 20, 0, None) == lbm.LBM_EINVAL
    assert lib.lbm_server_create(C.byref(h), C.c_void_p(100), 1 << 20, 4, None) == lbm.LBM_EINVAL
    assert lib.lbm_server_submit(None, None, None, 0, None, 10, None) == lbm.LBM_EINVAL
    assert lib.lbm_server_tick(None, 10, None) == lbm.LBM_EINVAL
    assert lib.lbm_server_status(None, 1, None) == lbm.LBM_EINVAL
    assert lib.lbm_server_destroy(None) == lbm.LBM_EINVAL


def test_stream_collide_overrun_fits_the_tail_pad():
    """Launch geometry of the stream-collide fast path, restated: pitch = nx
    rounded up to 32, V nodes per thread (1 for FP32, 2 for 16-bit storage),
    128-thread blocks (fewer when a row has fewer threads), a warp wholly past
    the pitch returns before its first load.  A running warp reads its lanes'
    V-vectors and one element right of its last lane, so on the last row of
    the last plane it reads at most 32 V + 1 - (pitch - xw) elements past the
    buffer's planes; that must fit the 256-byte tail pad for every width."""
    pad_bytes = 256
    for V, es in ((1, 4), (2, 2)):
        worst = 0
        for nx in range(3, 2100):
            pitch = (nx + 31) // 32 * 32
            tx = pitch // V
            bx = min((tx + 31) // 32 * 32, 128)
            threads = (tx + bx - 1) // bx * bx
            for xw in range(0, threads * V, 32 * V):
                if xw >= pitch:
                    continue  # returns before its first load
                worst = max(worst, xw + 32 * V + 1 - pitch)
        assert worst * es <= pad_bytes, (V, worst)
        assert worst == (1 if V == 1 else 33)
    # without the early return the overhanging warps would read far past it
    # (16-bit storage, nx = 257: pitch 288, warps up to x = 448)
    pitch, V = 288, 2
    assert (448 + 32 * V + 1 - pitch) * 2 > pad_bytes


def test_staged_stream_collide_copies_are_aligned_and_in_bounds():
    """The staged stream-collide's bulk copies, restated: tile of W = 256
    nodes of a row, halo H = 16 bytes of elements on the side a plane pulls
    from (p with e_x = 1 reads from x_s - H, e_x = -1 up to x_e + H), source
    row clamped on non-periodic first and last rows, plus the flags.  Every
    copy must start on a 16-byte boundary in global and shared memory, move a
    multiple of 16 bytes, stay inside its buffer (planes and tail pad, or the
    flag map) and inside its shared-memory segment; and the announced byte
    count must equal the bytes the copies bring."""
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    pdx = ex + ex[:5]
    pdy = ey + ey[:5]
    pad_bytes = 256
    for es in (2, 4):
        W, H = (256 if es == 2 else 128), 16 // es
        seg_b = (W + 2 * H) * es
        shifted = sum(1 for d in pdx if d != 0)
        for nx in list(range(4, 700, 7)) + [4000, 4001, 2047]:
            for ny in (4, 5, 9, 37):
                pitch = (nx + 31) // 32 * 32
                ps = (pitch * ny + 63) // 64 * 64
                a_bytes = 14 * ps * es + pad_bytes
                ntx = (pitch + W - 1) // W
                for per_y in (0, 1):
                    for it in range(ntx * ny):
                        y, cx = divmod(it, ntx)
                        xs, xe = cx * W, min(cx * W + W, pitch)
                        got = xe - xs
                        assert y * pitch + xs >= 0 and (y * pitch + xs) % 16 == 0 and (xe - xs) % 16 == 0
                        assert y * pitch + xe <= pitch * ny
                        for p in range(14):
                            ys = y - pdy[p]
                            if ys < 0 or ys >= ny:
                                ys = (ys % ny) if per_y else min(max(ys, 0), ny - 1)
                            lo = xs - (H if pdx[p] == 1 else 0)
                            hi = xe + (H if pdx[p] == -1 else 0)
                            start = (p * ps + ys * pitch + lo) * es
                            size = (hi - lo) * es
                            assert start >= 0 and start + size <= a_bytes, (es, nx, ny, it, p)
                            assert start % 16 == 0 and size % 16 == 0
                            dst = (lo - xs + H) * es
                            assert dst % 16 == 0 and dst >= 0 and dst + size <= seg_b
                            got += size
                        assert got == (xe - xs) * (14 * es + 1) + shifted * 16


def test_batched_block_lookup_finds_every_tile():
    """The batched stream-collide's block -> (instance, tile) mapping,
    restated: per-instance first block and tiles per row gx with the
    multiplier m = floor(2^s / gx) + 1, s = 31 + ceil(log2 gx), and buckets
    of 2^shift blocks (at most 4 (n + 1) of them) holding the instance of
    their first block, then a forward step over the instances starting in
    the bucket.  Every block of random uneven batches lands on its own
    instance and tile."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(1, 70))
        gx = rng.integers(1, 400, n)
        gy = rng.integers(1, 300, n)
        blocks = gx * gy
        start = np.concatenate([[0], np.cumsum(blocks)])
        total = int(start[-1])
        ell = np.array([int(np.ceil(np.log2(g))) if g > 1 else 0 for g in gx])
        s = 31 + ell
        m = np.array([(1 << int(si)) // int(g) + 1 for si, g in zip(s, gx)], dtype=object)
        shift = 0
        while (total >> shift) + 1 > 4 * (n + 1):
            shift += 1
        bucket, i = [], 0
        for k in range((total >> shift) + 1):
            while i + 1 < n and start[i + 1] <= (k << shift):
                i += 1
            bucket.append(i)
        assert len(bucket) <= 4 * (n + 1)
        for g in rng.integers(0, total, 2000):
            i = bucket[int(g) >> shift]
            while i + 1 < n and start[i + 1] <= g:
                i += 1
            assert start[i] <= g < start[i + 1]
            local = int(g - start[i])
            by = (local * m[i]) >> int(s[i])
            bx = local - by * int(gx[i])
            assert (by, bx) == divmod(local, int(gx[i]))
