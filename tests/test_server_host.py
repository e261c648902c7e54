"""Host-only tests of the request server's scheduler (no GPU): admission,
continuous batching, per-call mode, injected launch failures, timeouts and
shutdown, driven through the C ABI with the simulated executor."""
import threading
import time

import pytest

from paper_2602_10262_gb300.server import Server, ServerError

FAKE = 0x100000            # device addresses are never touched by the simulator
OK, PENDING, ERR_INVALID, ERR_OOM, ERR_CUDA = 0, 1, -1, -5, -6


def _server(**kw):
    sim = kw.pop("simulate", (200.0, 0.0, 0))
    return Server(simulate=sim, **kw)


def _weight(s, N=4096, K=4096, sparse=False):
    return s.register_weight(N, K, FAKE, FAKE + 64, 1, W_meta=FAKE + 128 if sparse else None,
                             ldw=K // 2 if sparse else K)


def test_single_request_completes():
    with _server(num_tenants=2, latency_tenant=0) as s:
        w = _weight(s)
        t = s.submit(0, w, 16, FAKE, 4096, FAKE, 4096)
        r = s.wait(t, 5)
        assert r is not None and r.status == OK
        assert r.t_submit_us <= r.t_launch_us <= r.t_end_us
        assert r.t_end_us - r.t_launch_us >= 199.0          # simulated launch cost
        st = s.stats()
        assert st["submitted"] == st["completed"] == 1 and st["kernel_launches"] == 2
        assert st["pool_in_use"] == 0


def test_requests_arriving_during_a_batch_are_batched_together():
    # 20 ms per batch, one slot: the first request runs alone, the rest that
    # arrive meanwhile go out as one batch when the slot frees
    with _server(num_tenants=1, latency_tenant=-1, max_inflight=1,
                 simulate=(20000.0, 0.0, 0)) as s:
        w = _weight(s)
        first = s.submit(0, w, 8, FAKE, 4096, FAKE, 4096)
        time.sleep(0.005)
        rest = [s.submit(0, w, 8, FAKE, 4096, FAKE, 4096) for _ in range(10)]
        r0 = s.wait(first, 5)
        rs = [s.wait(t, 5) for t in rest]
        assert r0.batch_size == 1
        assert all(r.status == OK for r in rs)
        assert {r.batch_size for r in rs} == {10}
        assert len({r.t_end_us for r in rs}) == 1
        st = s.stats()
        assert st["batches"] == 2 and st["max_batch_seen"] == 10 and st["kernel_launches"] == 4


def test_max_batch_respected():
    with _server(num_tenants=1, latency_tenant=-1, max_inflight=1, max_batch=4,
                 simulate=(10000.0, 0.0, 0)) as s:
        w = _weight(s)
        ts = [s.submit(0, w, 8, FAKE, 4096, FAKE, 4096) for _ in range(13)]
        rs = [s.wait(t, 5) for t in ts]
        assert max(r.batch_size for r in rs) <= 4
        assert s.stats()["completed"] == 13


def test_latency_tenant_is_not_held_to_the_inflight_limit():
    # one in-flight slot, 20 ms per batch: the bulk tenant's requests wait for
    # the slot, the latency tenant's are all enqueued at once, one per batch
    with _server(num_tenants=2, latency_tenant=0, max_inflight=1, simulate=(20000.0, 0.0, 0)) as s:
        w = _weight(s)
        lat = [s.submit(0, w, 8, FAKE, 4096, FAKE, 4096) for _ in range(6)]
        bulk = [s.submit(1, w, 8, FAKE, 4096, FAKE, 4096) for _ in range(3)]
        rl = [s.wait(t, 5) for t in lat]
        rb = [s.wait(t, 5) for t in bulk]
        assert all(r.status == OK and r.batch_size == 1 for r in rl)
        assert max(r.t_launch_us for r in rl) - min(r.t_submit_us for r in rl) < 15000.0
        # the bulk tenant's requests went out as one batch, or the later ones
        # waited for its single slot
        assert len({r.t_launch_us for r in rb}) == 1 or \
            max(r.t_launch_us for r in rb) >= min(r.t_end_us for r in rb) - 1.0


def test_latency_pool_share_keeps_the_latency_tenant_admitted():
    # a 64 MiB pool with 16 MiB kept for the latency tenant: the bulk
    # tenant's 8 MiB requests fill at most 48 MiB, so a latency request that
    # arrives meanwhile is admitted at once instead of waiting for bulk work
    with _server(num_tenants=2, latency_tenant=0, max_inflight=8, pool_bytes=64 << 20,
                 latency_pool_bytes=16 << 20, simulate=(50000.0, 0.0, 0)) as s:
        w = _weight(s)
        bulk = [s.submit(1, w, 2048, FAKE, 4096, FAKE, 4096) for _ in range(10)]
        time.sleep(0.005)
        assert s.stats()["pool_in_use"] <= (48 << 20)
        t = s.submit(0, w, 16, FAKE, 4096, FAKE, 4096)
        r = s.wait(t, 5)
        assert r.status == OK and r.t_launch_us - r.t_submit_us < 20000.0
        assert all(s.wait(b, 5).status == OK for b in bulk)
        # a bulk request larger than the pool minus the latency share is refused
        with pytest.raises(ServerError) as e:
            s.submit(1, w, 13000, FAKE, 4096, FAKE, 4096)
        assert e.value.status == ERR_OOM


def test_latency_batches_capped():
    with _server(num_tenants=2, latency_tenant=0, latency_max_batch=4, simulate=(20000.0, 0.0, 0)) as s:
        w = _weight(s)
        first = s.submit(0, w, 8, FAKE, 4096, FAKE, 4096)
        time.sleep(0.005)
        ts = [s.submit(0, w, 8, FAKE, 4096, FAKE, 4096) for _ in range(11)]
        rs = [s.wait(t, 5) for t in [first] + ts]
        assert all(r.status == OK for r in rs)
        assert max(r.batch_size for r in rs) <= 4
        assert s.stats()["completed"] == 12


def test_per_call_mode_launches_every_request_alone():
    with _server(num_tenants=2, latency_tenant=0, batching=False) as s:
        w = _weight(s)
        ts = [s.submit(i % 2, w, 4, FAKE, 4096, FAKE, 4096) for i in range(9)]
        rs = [s.wait(t, 5) for t in ts]
        assert all(r.status == OK and r.batch_size == 1 for r in rs)
        st = s.stats()
        assert st["batches"] == 9 and st["kernel_launches"] == 18


def test_oversized_request_is_rejected():
    with _server(num_tenants=1, latency_tenant=-1, pool_bytes=1 << 20) as s:
        w = _weight(s, N=4096, K=4096)
        with pytest.raises(ServerError) as e:
            s.submit(0, w, 4096, FAKE, 4096, FAKE, 4096)      # 16 MiB of codes
        assert e.value.status == ERR_OOM
        assert s.stats()["rejected"] == 1


def test_admission_waits_for_pool_space():
    # each request needs ~128 KiB; the pool holds three at a time
    with _server(num_tenants=1, latency_tenant=-1, pool_bytes=3 * (128 * 1024 + 256),
                 max_inflight=8, simulate=(2000.0, 0.0, 0)) as s:
        w = _weight(s, N=4096, K=4096)
        ts = [s.submit(0, w, 32, FAKE, 4096, FAKE, 4096) for _ in range(12)]
        rs = [s.wait(t, 10) for t in ts]
        assert all(r.status == OK for r in rs)
        st = s.stats()
        assert st["pool_high_water"] <= st["pool_bytes"]
        assert st["pool_in_use"] == 0 and st["completed"] == 12


def test_injected_launch_failures_reach_the_requests():
    with _server(num_tenants=1, latency_tenant=-1, batching=False,
                 simulate=(100.0, 0.0, 3)) as s:
        w = _weight(s)
        ts = [s.submit(0, w, 4, FAKE, 4096, FAKE, 4096) for _ in range(9)]
        rs = [s.wait(t, 5) for t in ts]
        statuses = [r.status for r in rs]
        assert statuses.count(ERR_CUDA) == 3 and statuses.count(OK) == 6
        st = s.stats()
        assert st["failed"] == 3 and st["completed"] == 6 and st["pool_in_use"] == 0


def test_poll_pending_and_wait_timeout():
    with _server(num_tenants=1, latency_tenant=-1, simulate=(300000.0, 0.0, 0)) as s:
        w = _weight(s)
        t = s.submit(0, w, 4, FAKE, 4096, FAKE, 4096)
        assert s.poll(t) is None
        t0 = time.time()
        assert s.wait(t, 0.05) is None
        assert time.time() - t0 < 1.0
        with pytest.raises(ServerError) as e:
            s.poll(987654)
        assert e.value.status == ERR_INVALID


def test_bad_arguments():
    with _server(num_tenants=2, latency_tenant=1) as s:
        w = _weight(s)
        for args in [(2, w, 4), (0, 99, 4), (0, w, -1)]:
            with pytest.raises(ServerError):
                s.submit(args[0], args[1], args[2], FAKE, 4096, FAKE, 4096)
        with pytest.raises(ServerError):
            s.submit(0, w, 4, FAKE, 100, FAKE, 4096)          # ldx < K
        with pytest.raises(ServerError):
            s.register_weight(4096, 100, FAKE, FAKE, 1)        # K % 16 != 0
        with pytest.raises(ServerError):
            s.register_weight(4096, 4112, FAKE, FAKE, 1, W_meta=FAKE)   # sparse K % 128
        for bad in (2, -1):
            with pytest.raises(ServerError) as e:
                s.register_weight(4096, 4096, FAKE, FAKE, 1, w_format=bad)   # not E4M3 / E5M2
            assert e.value.status == ERR_INVALID
        w5 = s.register_weight(4096, 4096, FAKE, FAKE, 1, w_format=1)        # E5M2 accepted
        r = s.wait(s.submit(0, w5, 4, FAKE, 4096, FAKE, 4096), 5)
        assert r.status == OK
    with pytest.raises(ServerError):
        Server(num_tenants=0, simulate=(1, 0, 0))


def test_destroy_with_queued_requests_returns():
    s = _server(num_tenants=1, latency_tenant=-1, max_inflight=1, simulate=(50000.0, 0.0, 0))
    w = _weight(s)
    for _ in range(5):
        s.submit(0, w, 4, FAKE, 4096, FAKE, 4096)
    t0 = time.time()
    s.close()                       # waits for the running batch, fails the queued ones
    assert time.time() - t0 < 5.0


def test_concurrent_submitters():
    with _server(num_tenants=2, latency_tenant=0, simulate=(50.0, 0.0, 0)) as s:
        w = _weight(s)
        tickets, lock = [], threading.Lock()

        def client(tenant):
            for _ in range(50):
                t = s.submit(tenant, w, 8, FAKE, 4096, FAKE, 4096)
                with lock:
                    tickets.append(t)

        th = [threading.Thread(target=client, args=(i % 2,)) for i in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        rs = [s.wait(t, 10) for t in tickets]
        assert len(set(tickets)) == 200 and all(r.status == OK for r in rs)


def test_latency_tenant_not_blocked_by_bulk_queue():
    # the bulk tenant's stream is busy for a long time (30 ms per launch plus
    # 10 ms per GFLOP: >= 51 ms for a 2.1-GFLOP request, however the three
    # are batched); the latency tenant has its own stream and slots, so its
    # 0.03-GFLOP request finishes first
    with _server(num_tenants=2, latency_tenant=0, max_inflight=1,
                 simulate=(30000.0, 10000.0, 0)) as s:
        w = _weight(s)
        bulk = [s.submit(1, w, 64, FAKE, 4096, FAKE, 4096) for _ in range(3)]
        lat = s.submit(0, w, 1, FAKE, 4096, FAKE, 4096)
        rl = s.wait(lat, 5)
        rb = [s.wait(t, 5) for t in bulk]
        assert rl.t_end_us < max(r.t_end_us for r in rb)
        # 30 ms of its own; behind even one bulk batch it would take >= 60 ms
        # (the slack covers a loaded host delaying the scheduler thread)
        assert rl.t_end_us - rl.t_submit_us < 55000.0


def _res(a, b):
    from paper_2602_10262_gb300.server import Result
    return Result(OK, 1, 0.0, 0.0, b, a)


def test_overlap_efficiency_intervals():
    from paper_2602_10262_gb300.server import overlap_efficiency
    assert overlap_efficiency([]) == 0.0
    assert overlap_efficiency([_res(0, 10), _res(5, 15)]) == pytest.approx(5 / 15)
    assert overlap_efficiency([_res(0, 10), _res(10, 20)]) == 0.0          # touching only
    assert overlap_efficiency([_res(0, 10), _res(0, 10)]) == 0.0          # one batch, two requests
    assert overlap_efficiency([_res(0, 10), _res(2, 4)]) == pytest.approx(2 / 10)
    assert overlap_efficiency([_res(0, 4), _res(1, 3), _res(2, 6), _res(8, 9)]) == pytest.approx(3 / 7)


def test_batch_start_times_and_overlap_in_simulation():
    from paper_2602_10262_gb300.server import overlap_efficiency
    # 5 ms per launch; one tenant's batches queue on its stream, two tenants
    # run side by side
    with _server(num_tenants=2, latency_tenant=0, batching=0, simulate=(5000.0, 0.0, 0)) as s:
        w = _weight(s)
        t0 = [s.submit(0, w, 8, FAKE, 4096, FAKE, 4096) for _ in range(3)]
        rs0 = [s.wait(t, 5) for t in t0]
        for r in rs0:
            assert r.t_launch_us <= r.t_start_us < r.t_end_us
            assert r.t_end_us - r.t_start_us >= 4999.0
        spans = sorted((r.t_start_us, r.t_end_us) for r in rs0)
        assert all(spans[i][1] <= spans[i + 1][0] for i in range(2))    # serialised
        assert overlap_efficiency(rs0) == 0.0
        both = [s.submit(k % 2, w, 8, FAKE, 4096, FAKE, 4096) for k in range(4)]
        rs = [s.wait(t, 5) for t in both]
        assert overlap_efficiency(rs) > 0.5


def test_pool_stress_random_sizes():
    # a small pool and random request sizes: the first-fit pool fragments and
    # refills, FIFO admission waits for space, and every request completes
    # with the pool empty afterwards
    import random
    rng = random.Random(5)
    pool = 24 << 20
    with _server(num_tenants=2, latency_tenant=0, pool_bytes=pool, simulate=(20.0, 2.0, 0)) as s:
        w = _weight(s, N=4096, K=4096)
        tickets = [s.submit(rng.randrange(2), w, rng.randint(1, 1024), FAKE, 4096, FAKE, 4096)
                   for _ in range(300)]
        rs = [s.wait(t, 20) for t in tickets]
        assert all(r is not None and r.status == OK for r in rs)
        st = s.stats()
        assert st["completed"] == 300 and st["failed"] == 0
        assert st["pool_in_use"] == 0
        assert 0 < st["pool_high_water"] <= pool
