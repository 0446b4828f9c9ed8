"""Served mode: continuous batching of evolution requests (nr_server_*).

Requests that arrive while others are running are admitted at step
boundaries as the HBM budget and slots allow; all running requests advance
together in one batch.  Each result must be bitwise what the same request
gives run alone with nr_rk4_step, whatever shared the GPU with it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_00097_gb300 import binding as B  # noqa: E402
from paper_2505_00097_gb300 import build as BUILD  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


def _requests():
    reqs = []
    for k, (nr, masses, pos) in enumerate([
        (12, (1.0,), ((0, 0, 0),)),
        (20, (0.6, 0.4), ((0, 0, 0.4), (0, 0, -0.6))),
        (16, (0.8,), ((0, 0, 0),)),
        (24, (0.5, 0.5), ((0, 0, 0.5), (0, 0, -0.5))),
    ]):
        s = W.sinh_cylindrical((nr, 2, 2 * nr), rho_max=30.0, z_max=30.0)
        s.update(masses=masses, positions=pos)
        reqs.append(s)
    return reqs


def _alone(spec, t_final):
    g = B.Grid(spec)
    g.set_brill_lindquist(spec["masses"], spec["positions"])
    n = max(1, int(np.ceil(t_final / g.dt_cfl - 1e-9)))
    (g.ssprk3_step if spec.get("integrator") == "ssprk3" else g.rk4_step)(g.dt_cfl, n)
    st = np.empty(24 * g.T)
    g.get_state(st, True)
    T = g.T
    g.close()
    return st, n, T


@pytest.mark.parametrize("budget_gb,slots", [(80, 8), (80, 1)], ids=["mixed", "one-slot"])
def test_results_equal_alone_and_in_the_mix(budget_gb, slots):
    reqs = _requests()
    t_final = 0.8
    srv = B.Server(int(budget_gb * 2 ** 30), slots)
    srv.set_tile(32, 4)
    ids = [srv.submit(reqs[0], t_final, keep_state=True), srv.submit(reqs[1], t_final, keep_state=True)]
    srv.advance(3)                      # the first two start; the others arrive while they run
    ids += [srv.submit(reqs[2], t_final, keep_state=True), srv.submit(reqs[3], t_final, keep_state=True)]
    for _ in range(1000):
        nrun, nq = srv.advance(5)
        if nrun == 0 and nq == 0:
            break
    for rid, spec in zip(ids, reqs):
        info = srv.poll(rid)
        assert info["status"] == 2, info
        ref, n, T = _alone(spec, t_final)
        assert info["steps_done"] == n == info["steps_total"]
        got = srv.fetch_state(rid, 24 * T)
        assert np.array_equal(got, ref)
        assert np.isfinite(info["l2"]) and info["linf"] > 0.0
    srv.close()


def test_autotuned_server_and_oversized_request():
    reqs = _requests()
    srv = B.Server(int(0.05 * 2 ** 30), 4)   # 51 MiB: the small grids fit, a 1024x2x2048 grid never does
    big = W.sinh_cylindrical((1024, 2, 2048))
    big.update(masses=(1.0,), positions=((0, 0, 0),))
    rid_big = srv.submit(big, 0.5)
    rid = srv.submit(reqs[0], 0.5, keep_state=True)
    for _ in range(1000):
        nrun, nq = srv.advance(10)
        if nrun == 0 and nq == 0:
            break
    assert srv.poll(rid_big)["status"] == 3
    assert srv.poll(rid)["status"] == 2
    ref, n, T = _alone(reqs[0], 0.5)
    assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
    srv.close()


def _run_until_done(srv, rid, step=1):
    for _ in range(10000):
        srv.advance(step)
        if srv.poll(rid)["status"] in (2, 3):
            return
    raise AssertionError("request did not finish")


def test_srpt_preempts_a_long_request_and_keeps_results():
    long_spec, short_spec = _requests()[3], _requests()[0]   # 24x2x48 two punctures, 12x2x24 one
    t_final = 0.8
    srv = B.Server(int(80 * 2 ** 30), 8)
    srv.set_tile(32, 4)
    srv.set_policy("srpt", 1)          # one request at a time, least remaining work first
    a = srv.submit(long_spec, t_final, keep_state=True)
    srv.advance(2)
    assert srv.poll(a)["steps_done"] == 2
    b = srv.submit(short_spec, t_final, keep_state=True)
    _run_until_done(srv, b)
    assert srv.poll(b)["status"] == 2
    assert srv.poll(a)["steps_done"] == 2      # paused while the shorter request ran
    _run_until_done(srv, a, step=7)
    for rid, spec in ((a, long_spec), (b, short_spec)):
        ref, n, T = _alone(spec, t_final)
        assert srv.poll(rid)["steps_done"] == n
        assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
    srv.close()


def test_fifo_with_a_points_cap_runs_in_arrival_order():
    first, second = _requests()[0], _requests()[3]
    t_final = 0.8
    srv = B.Server(int(80 * 2 ** 30), 8)
    srv.set_tile(32, 4)
    nfirst = first["N"][0] * first["N"][1] * first["N"][2]
    srv.set_policy("fifo", nfirst)     # room for the first request only
    a = srv.submit(first, t_final, keep_state=True)
    b = srv.submit(second, t_final, keep_state=True)
    srv.advance(1)
    assert srv.poll(b)["status"] == 1 and srv.poll(b)["steps_done"] == 0   # resident, not advanced
    _run_until_done(srv, a)
    assert srv.poll(b)["steps_done"] == 0
    _run_until_done(srv, b, step=5)
    for rid, spec in ((a, first), (b, second)):
        ref, n, T = _alone(spec, t_final)
        assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
    srv.close()


def test_requests_of_every_kind_share_one_server():
    """Cylindrical grids with a two-point and with a wider azimuth and a spherical grid run in one
    server (one batch per kind of grid); each result is bitwise its result alone."""
    a = W.sinh_cylindrical((14, 2, 28), rho_max=30.0, z_max=30.0)
    a.update(masses=(1.0,), positions=((0, 0, 0),))
    b = W.sinh_cylindrical((10, 4, 20), rho_max=30.0, z_max=30.0)
    b.update(masses=(0.5, 0.5), positions=((0, 0.1, 0.5), (0, 0, -0.5)))
    c = W.sinh_spherical((16, 8, 2))
    c.update(masses=(1.0,), positions=((0, 0, 0),))
    t_final = 0.3
    srv = B.Server(int(80 * 2 ** 30), 8)
    srv.set_tile(32, 4)
    ids = [srv.submit(spec, t_final, keep_state=True) for spec in (a, b, c)]
    for _ in range(1000):
        nrun, nq = srv.advance(4)
        if nrun == 0 and nq == 0:
            break
    for rid, spec in zip(ids, (a, b, c)):
        assert srv.poll(rid)["status"] == 2
        ref, n, T = _alone(spec, t_final)
        assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
    srv.close()


def test_production_scheme_and_4th_order_requests_share_one_server():
    """8th-order SSPRK3 requests (the production scheme of Sec. 4.1), an 8th-order RK4 request
    and 4th-order RK4 requests in one server: one batch per kind, each result bitwise its result
    alone."""
    ko8 = [0.3] * 17 + [0.99] * 7
    specs = []
    for k, (nr, masses, pos) in enumerate([(14, (1.0,), ((0, 0, 0),)),
                                           (18, (0.6, 0.4), ((0, 0, 0.4), (0, 0, -0.6))),
                                           (12, (0.8,), ((0, 0, 0),)),
                                           (16, (0.5, 0.5), ((0, 0, 0.5), (0, 0, -0.5)))]):
        s = W.sinh_cylindrical((nr, 2, 2 * nr), rho_max=30.0, z_max=30.0)
        s.update(masses=masses, positions=pos)
        if k < 2:
            s.update(NG=5, ko_sigma=ko8, integrator="ssprk3", cfl=0.35)
        elif k == 2:
            s.update(NG=5, ko_sigma=ko8)
        specs.append(s)
    t_final = 0.5
    for policy in ("fifo", "srpt"):
        srv = B.Server(int(80 * 2 ** 30), 8)
        srv.set_tile(32, 4)
        srv.set_policy(policy)
        ids = [srv.submit(spec, t_final, keep_state=True) for spec in specs]
        for _ in range(1000):
            nrun, nq = srv.advance(3)
            if nrun == 0 and nq == 0:
                break
        for rid, spec in zip(ids, specs):
            p = srv.poll(rid)
            assert p["status"] == 2
            ref, n, T = _alone(spec, t_final)
            assert p["steps_total"] == n
            assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
        srv.close()


def _diverging():
    """a request whose CFL factor of 5 puts RK4 outside its stability region: non-finite within a few steps"""
    s = W.sinh_cylindrical((12, 2, 24), rho_max=30.0, z_max=30.0)
    s.update(masses=(1.0,), positions=((0, 0, 0),), cfl=5.0)
    return s


@pytest.mark.parametrize("every", [5, 0], ids=["guard-every-5", "guard-off"])
def test_a_diverging_request_fails_and_the_others_are_unaffected(every):
    """A request that goes non-finite is retired as failed with NR_ENONFINITE -- by the guard within
    its first checks (every 5 steps), or, with the guard off, at its retirement -- while every other
    request finishes with its result alone, bit for bit (state and digest)."""
    reqs = _requests()[:3]
    t_final = 2.0
    srv = B.Server(int(80 * 2 ** 30), 8)
    srv.set_tile(32, 4)
    srv.set_guard(every)
    ids = [srv.submit(reqs[0], t_final, keep_state=True, keep_digest=True),
           srv.submit(reqs[1], t_final, keep_state=True, keep_digest=True)]
    bad = srv.submit(_diverging(), 40.0, keep_state=True, keep_digest=True)
    srv.advance(3)
    ids.append(srv.submit(reqs[2], t_final, keep_state=True, keep_digest=True))
    for _ in range(1000):
        nrun, nq = srv.advance(5)
        if nrun == 0 and nq == 0:
            break
    p = srv.poll(bad)
    assert p["status"] == 3 and srv.request_error(bad) == 5        # NR_ENONFINITE
    if every:
        assert p["steps_done"] <= 3 + 2 * every < p["steps_total"]   # caught by the guard, not at the end
        assert np.isnan(p["l2"])
    else:
        assert p["steps_done"] == p["steps_total"]
    with pytest.raises(B.NrError):
        srv.fetch_state(bad, 1)
    for rid, spec in zip(ids, reqs):
        info = srv.poll(rid)
        assert info["status"] == 2 and srv.request_error(rid) == 0
        ref, n, T = _alone(spec, t_final)
        assert info["steps_done"] == n
        assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
        g = B.Grid(spec)
        g.set_state(ref, True)
        assert srv.fetch_digest(rid) == g.digest()
        g.close()
    srv.close()


def test_starvation_cap_lets_the_older_request_go_first():
    """SRPT with a starvation cap: once both requests have waited longer than the cap, the older one
    runs first although the newer one has less work left (plain SRPT would preempt it, as the test
    above shows); results stay bitwise those alone."""
    import time

    long_spec, short_spec = _requests()[3], _requests()[0]
    t_final = 0.8
    srv = B.Server(int(80 * 2 ** 30), 8)
    srv.set_tile(32, 4)
    srv.set_policy("srpt", 1)          # one request at a time
    srv.set_starvation_cap(1e-3)
    a = srv.submit(long_spec, t_final, keep_state=True)
    srv.advance(2)
    b = srv.submit(short_spec, t_final, keep_state=True)
    time.sleep(0.01)                   # both are now older than the cap
    srv.advance(3)
    assert srv.poll(a)["steps_done"] == 5 and srv.poll(b)["steps_done"] == 0
    _run_until_done(srv, a, step=7)
    assert srv.poll(b)["steps_done"] == 0
    _run_until_done(srv, b)
    for rid, spec in ((a, long_spec), (b, short_spec)):
        ref, n, T = _alone(spec, t_final)
        assert srv.poll(rid)["steps_done"] == n
        assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
    with pytest.raises(B.NrError):
        srv.set_starvation_cap(-1.0)
    srv.close()


@pytest.mark.parametrize("policy", ["fifo", "srpt"])
def test_background_setups_keep_results(policy):
    """With set-ups computed ahead by the worker thread (prefetch depth 2), requests that arrive while
    others run wait until their set-up is ready; every result is still bitwise its result alone, and
    the server's accounting sees every admission and retirement."""
    reqs = _requests()
    t_final = 0.8
    srv = B.Server(int(80 * 2 ** 30), 8)
    srv.set_tile(16, 8)
    srv.set_prefetch(2)
    srv.set_policy(policy, 2000)
    ids = [srv.submit(reqs[0], t_final, keep_state=True), srv.submit(reqs[1], t_final, keep_state=True)]
    srv.advance(3)
    ids += [srv.submit(reqs[2], t_final, keep_state=True), srv.submit(reqs[3], t_final, keep_state=True)]
    for _ in range(1000):
        nrun, nq = srv.advance(2)
        if nrun == 0 and nq == 0:
            break
    for rid, spec in zip(ids, reqs):
        assert srv.poll(rid)["status"] == 2
        ref, n, T = _alone(spec, t_final)
        assert np.array_equal(srv.fetch_state(rid, 24 * T), ref)
    st = srv.stats()
    assert st["admitted"] == 4 and st["retired"] == 4 and st["chunks"] > 0
    with pytest.raises(B.NrError):
        srv.set_prefetch(-1)
    srv.close()
