"""Serving (lbm_server_*): requests of different sizes, particle counts and
step budgets, arriving while others run, are admitted by device-memory
footprint, advanced together (continuous batching) and retired; each
result is exactly (bit for bit) what lbm_step gives the request alone, and
matches the FP64 oracle's run of the request (fields rel-L2 <= 1e-5, centres
within 1e-4 lattice units)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_16597_gb300 import lbm, workloads as W  # noqa: E402
from test_gpu_batch import check_against_oracle, oracle_run, small_ensemble  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def alone(wl, steps, storage=lbm.LBM_STORE_FP32):
    s = lbm.Simulation(wl.domain, wl.particles, wl.params, storage=storage)
    s.step(steps)
    out = (s.fields(), s.particles())
    s.close()
    return out


def same_result(got, ref):
    for a, b in zip(got[0], ref[0]):
        assert np.array_equal(a, b, equal_nan=True)
    assert got[1].tobytes() == ref[1].tobytes()


def footprint(wl, storage=lbm.LBM_STORE_FP32):
    d = lbm.make_domain(**wl.domain)
    p = lbm.make_params(**dict(wl.params, storage=storage))
    return lbm.lbm_query_footprint(d, lbm.pack_particles(wl.particles), p)


def run_until_done(srv, ids, max_steps, arrivals=()):
    """Tick until every id is done, submitting (tick, workload, steps) arrivals
    on their tick; returns {id: result}, the list of tick stats."""
    pending = list(arrivals)
    total = len(ids) + len(pending)
    out, stats, t = {}, [], 0
    while len(out) < total:
        while pending and pending[0][0] <= t:
            _, wl, steps, key = pending.pop(0)
            ids[key] = srv.submit(wl.domain, wl.particles, wl.params, steps)
        stats.append(srv.tick(max_steps))
        for key, rid in list(ids.items()):
            if key in out:
                continue
            state, err = srv.status(rid)
            assert state != lbm.SERVER_FAILED, err
            if state == lbm.SERVER_DONE:
                out[key] = srv.result(rid)
        t += 1
        assert t < 1000
    return out, stats


def test_results_are_the_same_alone_and_in_the_mix():
    wls = small_ensemble()
    budgets = {0: 30, 1: 45, 2: 20, 3: 37, 4: 26}
    refs = {k: alone(wls[k], budgets[k]) for k in budgets}
    srv = lbm.Server(2 << 30, max_active=8)
    ids = {0: srv.submit(wls[0].domain, wls[0].particles, wls[0].params, budgets[0]),
           1: srv.submit(wls[1].domain, wls[1].particles, wls[1].params, budgets[1])}
    arrivals = [(1, wls[2], budgets[2], 2), (2, wls[3], budgets[3], 3), (4, wls[4], budgets[4], 4)]
    out, stats = run_until_done(srv, ids, 8, arrivals)
    for k in budgets:
        same_result(out[k], refs[k])
        check_against_oracle(out[k][0], out[k][1], oracle_run(wls[k], budgets[k]), lbm.LBM_STORE_FP32)
    # requests overlapped on the device
    assert max(s["active"] + s["retired"] for s in stats) >= 3
    assert sum(s["admitted"] for s in stats) == 5
    srv.close()


def test_admission_waits_for_memory():
    """A pool that holds one request at a time serves them one after the
    other, with the same results."""
    wls = small_ensemble()
    pick = [1, 3]
    budgets = {1: 12, 3: 9}
    refs = {k: alone(wls[k], budgets[k]) for k in pick}
    biggest = max(footprint(wls[k]) for k in pick)
    srv = lbm.Server(biggest + (1 << 20) + (96 << 10), max_active=8)
    ids = {k: srv.submit(wls[k].domain, wls[k].particles, wls[k].params, budgets[k]) for k in pick}
    out, stats = run_until_done(srv, ids, 5)
    assert max(s["active"] + s["retired"] for s in stats) == 1
    for k in pick:
        same_result(out[k], refs[k])
    srv.close()


def test_oversized_request_is_refused():
    wl = small_ensemble()[3]
    srv = lbm.Server(footprint(wl) // 2, max_active=2)
    with pytest.raises(lbm.LbmError) as e:
        srv.submit(wl.domain, wl.particles, wl.params, 10)
    assert e.value.code == lbm.LBM_ENOSPC
    srv.close()


def test_failed_request_does_not_disturb_the_others():
    wls = small_ensemble()
    bad = wls[4].particles.copy()
    bad["ux"] = 10.0  # flung at a wall: the step raises LBM_EDOMAIN
    ref = alone(wls[0], 16)
    srv = lbm.Server(2 << 30, max_active=4)
    good = srv.submit(wls[0].domain, wls[0].particles, wls[0].params, 16)
    rid = srv.submit(wls[4].domain, bad, wls[4].params, 16)
    for _ in range(10):
        srv.tick(4)
    state, err = srv.status(rid)
    assert state == lbm.SERVER_FAILED and err in (lbm.LBM_EDOMAIN, lbm.LBM_ENUMERIC)
    with pytest.raises(lbm.LbmError):
        srv.result(rid)
    assert srv.status(good)[0] == lbm.SERVER_DONE
    same_result(srv.result(good), ref)
    srv.close()
