"""Admission and plan-cache logic of the solve server, in its scheduler test mode (no GPU).

With `simulate_us` > 0 the server plans nothing and issues no GPU work: an admitted
request holds its worker and its device-footprint reservation for
max_iter * simulate_us microseconds. Everything else -- footprints, the HBM budget,
first-come first-served admission with bounded backfill, the plan cache and its LRU
eviction, tickets, waiting and shutdown -- is the code the GPU server runs.
"""
import time

import numpy as np
import pytest

import __graft_entry__
from paper_2401_12890_gb300 import ssm

TICK_US = 2000   # simulated time per "iteration"


@pytest.fixture(scope="module", autouse=True)
def lib():
    __graft_entry__.build()
    return ssm.load_library()


def dictionary(P, Q, seed):
    return np.random.default_rng(seed).random((P, Q))


def problem(P, Q, dims, seed=0):
    N = int(np.prod(dims))
    return dictionary(P, Q, seed), np.zeros((P, N), np.float32)


BIG = (8, 16, (256, 256))      # (P, Q, dims)
SMALL = (4, 4, (8, 8))


def footprints():
    """Footprints (peak bytes) of the BIG and SMALL shapes, read back from the server."""
    out = []
    with ssm.Server(max_active=1, hbm_budget=1 << 40, simulate_us=1) as srv:
        for P, Q, dims in (BIG, SMALL):
            K, M = problem(P, Q, dims)
            t = srv.submit(K, M, dims, 0.01, 1.0, max_iter=1)
            _, info = srv.wait(t)
            out.append(info["footprint"])
    return out


def run_all(srv, reqs):
    tickets = [srv.submit(K, M, dims, 0.01, 1.0, max_iter=it) for K, M, dims, it in reqs]
    return [srv.wait(t)[1] for t in tickets]


def test_footprint_grows_with_the_problem():
    big, small = footprints()
    assert big > 10 * small > 0
    # state alone: z and d ping-pong, 4 x Q x N floats
    assert big >= 4 * 16 * 256 * 256 * 4


def test_fifo_when_everything_fits():
    with ssm.Server(max_active=1, hbm_budget=1 << 40, simulate_us=TICK_US,
                    cache_plans=False) as srv:
        reqs = [problem(*SMALL, seed=i) + (SMALL[2], 1) for i in range(6)]
        infos = run_all(srv, [(K, M, d, it) for K, M, d, it in reqs])
    assert [i["order"] for i in infos] == list(range(6))
    assert all(i["status"] == ssm.SSM_OK and i["iterations"] == 0 for i in infos)


def test_backfill_passes_a_head_that_does_not_fit():
    big, small = footprints()
    budget = int(1.5 * big)      # two BIG requests never fit together
    with ssm.Server(max_active=2, hbm_budget=budget, simulate_us=TICK_US,
                    cache_plans=False) as srv:
        a = srv.submit(*problem(*BIG[:2], BIG[2], 1), BIG[2], 0.01, 1.0, max_iter=40)
        time.sleep(0.02)         # A is admitted first
        b = srv.submit(*problem(*BIG[:2], BIG[2], 2), BIG[2], 0.01, 1.0, max_iter=5)
        c = srv.submit(*problem(*SMALL[:2], SMALL[2], 3), SMALL[2], 0.01, 1.0, max_iter=5)
        ia, ib, ic = (srv.wait(t)[1] for t in (a, b, c))
        st = srv.stats()
    assert (ia["order"], ic["order"], ib["order"]) == (0, 1, 2)
    assert st["peak_bytes_held"] <= budget
    assert st["completed"] == 3 and st["failed"] == 0


def test_bypass_limit_stops_backfill():
    big, small = footprints()
    budget = int(1.5 * big)
    with ssm.Server(max_active=2, hbm_budget=budget, simulate_us=TICK_US, cache_plans=False,
                    max_bypass=1) as srv:
        a = srv.submit(*problem(*BIG[:2], BIG[2], 1), BIG[2], 0.01, 1.0, max_iter=60)
        time.sleep(0.02)
        b = srv.submit(*problem(*BIG[:2], BIG[2], 2), BIG[2], 0.01, 1.0, max_iter=5)
        c = srv.submit(*problem(*SMALL[:2], SMALL[2], 3), SMALL[2], 0.01, 1.0, max_iter=2)
        d = srv.submit(*problem(*SMALL[:2], SMALL[2], 4), SMALL[2], 0.01, 1.0, max_iter=2)
        orders = [srv.wait(t)[1]["order"] for t in (a, b, c, d)]
    # C passes B once; then B holds the line and D follows B
    assert orders == [0, 2, 1, 3]


def test_budget_is_never_exceeded_under_load():
    big, small = footprints()
    budget = int(2.2 * big)
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(24):
        shape = BIG if rng.random() < 0.4 else SMALL
        reqs.append(problem(*shape[:2], shape[2], i) + (shape[2], int(rng.integers(1, 6))))
    with ssm.Server(max_active=4, hbm_budget=budget, simulate_us=TICK_US,
                    cache_plans=False) as srv:
        infos = run_all(srv, reqs)
        st = srv.stats()
    assert st["completed"] == 24 and st["peak_bytes_held"] <= budget
    assert sorted(i["order"] for i in infos) == list(range(24))
    assert len({i["slot"] for i in infos}) > 1           # solves ran side by side
    # at any admission instant, the running reservations fit in the budget
    spans = [(i["latency_ms"] - i["solve_ms"], i["latency_ms"], i["footprint"]) for i in infos]
    assert all(f <= budget for _, _, f in spans)


def test_oversize_request_is_rejected():
    big, small = footprints()
    with ssm.Server(max_active=1, hbm_budget=big // 2, simulate_us=1) as srv:
        with pytest.raises(ssm.SsmError) as e:
            srv.submit(*problem(*BIG[:2], BIG[2]), BIG[2], 0.01, 1.0)
        assert e.value.status == ssm.SSM_ENOMEM
        assert srv.stats()["rejected"] == 1


def test_plan_cache_reuse_and_lru_eviction():
    big, small = footprints()
    with ssm.Server(max_active=1, hbm_budget=int(1.5 * big), simulate_us=1) as srv:
        K1, M1 = problem(*BIG[:2], BIG[2], 11)
        K2, M2 = problem(*BIG[:2], BIG[2], 12)
        i1 = srv.wait(srv.submit(K1, M1, BIG[2], 0.01, 1.0, max_iter=1))[1]
        # same K and plan parameters, another stopping rule: reused
        i2 = srv.wait(srv.submit(K1.copy(), M1, BIG[2], 0.01, 1.0, max_iter=3,
                                 tol_primal=1e-3))[1]
        # another lambda: a new plan, which evicts the idle one (both do not fit)
        i3 = srv.wait(srv.submit(K1, M1, BIG[2], 0.02, 1.0, max_iter=1))[1]
        # another K: a new plan again
        i4 = srv.wait(srv.submit(K2, M2, BIG[2], 0.02, 1.0, max_iter=1))[1]
        st = srv.stats()
    assert (i1["plan_reused"], i2["plan_reused"], i3["plan_reused"], i4["plan_reused"]) == \
        (0, 1, 0, 0)
    assert st["plans_created"] == 3 and st["plans_reused"] == 1 and st["plans_evicted"] == 2


def test_wait_timeout_poll_and_unknown_ticket():
    with ssm.Server(max_active=1, hbm_budget=1 << 40, simulate_us=TICK_US) as srv:
        t = srv.submit(*problem(*SMALL[:2], SMALL[2]), SMALL[2], 0.01, 1.0, max_iter=50)
        assert srv.wait(t, timeout_ms=1.0) is None
        assert srv.poll(t) is None
        F, info = srv.wait(t)
        assert info["status"] == ssm.SSM_OK and info["latency_ms"] >= info["solve_ms"] > 0
        with pytest.raises(ssm.SsmError) as e:
            srv.wait(t)
        assert e.value.status == ssm.SSM_EINVAL


def test_destroy_waits_for_submitted_requests():
    srv = ssm.Server(max_active=2, hbm_budget=1 << 40, simulate_us=TICK_US)
    for i in range(5):
        srv.submit(*problem(*SMALL[:2], SMALL[2], i), SMALL[2], 0.01, 1.0, max_iter=3)
    t0 = time.perf_counter()
    srv.close()
    assert time.perf_counter() - t0 >= 0.9 * 3 * 3 * TICK_US * 1e-6   # 3 rounds of 2 workers


def test_invalid_server_config():
    with pytest.raises(ssm.SsmError):
        ssm.Server(max_active=0, simulate_us=1, hbm_budget=1)
    with pytest.raises(ssm.SsmError):
        ssm.Server(max_active=1, simulate_us=1, hbm_budget=0)


@pytest.mark.parametrize("reserved", [1, 0])
def test_reserved_worker_admits_small_requests_past_large_ones(reserved):
    """With a worker reserved for class-0 requests, a small request arriving while large
    ones hold (or wait for) the other workers is admitted at once; without it, it waits
    for a large one to finish."""
    big, small = footprints()
    with ssm.Server(max_active=2, hbm_budget=1 << 40, simulate_us=TICK_US, cache_plans=False,
                    small_bytes=2 * small, reserved_small=reserved) as srv:
        a = srv.submit(*problem(*BIG[:2], BIG[2], 1), BIG[2], 0.01, 1.0, max_iter=40)
        time.sleep(0.02)
        b = srv.submit(*problem(*BIG[:2], BIG[2], 2), BIG[2], 0.01, 1.0, max_iter=40)
        time.sleep(0.02)
        c = srv.submit(*problem(*SMALL[:2], SMALL[2], 3), SMALL[2], 0.01, 1.0, max_iter=2)
        ia, ib, ic = (srv.wait(t)[1] for t in (a, b, c))
    if reserved:
        # B waits for A's worker; C takes the reserved one right away
        assert (ia["order"], ic["order"], ib["order"]) == (0, 1, 2)
        assert ic["queue_ms"] < 10 * TICK_US * 1e-3
        assert ic["slot"] == 0 and ia["slot"] != 0 and ib["slot"] != 0
    else:
        assert (ia["order"], ib["order"], ic["order"]) == (0, 1, 2)
        # A (40 ticks) started 20 ticks before C arrived
        assert ic["queue_ms"] > 10 * TICK_US * 1e-3


def test_reserved_workers_never_take_every_worker():
    """reserved_small is capped at max_active - 1: large requests still run."""
    big, small = footprints()
    with ssm.Server(max_active=2, hbm_budget=1 << 40, simulate_us=TICK_US, cache_plans=False,
                    small_bytes=2 * small, reserved_small=5) as srv:
        info = srv.wait(srv.submit(*problem(*BIG[:2], BIG[2], 1), BIG[2], 0.01, 1.0,
                                   max_iter=2))[1]
    assert info["status"] == ssm.SSM_OK and info["slot"] == 1


def test_small_requests_are_admitted_as_groups():
    """group_small = 4: requests waiting behind a busy worker are admitted four at a time
    and solved as one group; large ones are never grouped."""
    big_b, small_b = footprints()
    with ssm.Server(max_active=1, hbm_budget=1 << 40, simulate_us=TICK_US, cache_plans=False,
                    small_bytes=2 * small_b, group_small=4) as srv:
        first = srv.submit(*problem(*SMALL[:2], SMALL[2], 0), SMALL[2], 0.01, 1.0, max_iter=30)
        time.sleep(0.01)
        rest = [srv.submit(*problem(*SMALL[:2], SMALL[2], i), SMALL[2], 0.01, 1.0, max_iter=3)
                for i in range(1, 6)]
        big = srv.submit(*problem(*BIG[:2], BIG[2], 9), BIG[2], 0.01, 1.0, max_iter=2)
        infos = [srv.wait(t)[1] for t in [first] + rest + [big]]
    sizes = [i["group_size"] for i in infos]
    assert sizes[0] == 1                 # alone when admitted: a group of one
    assert sizes[1:5] == [4, 4, 4, 4]    # the next four together
    assert sizes[5] == 1 and sizes[6] == 0
    orders = [i["order"] for i in infos]
    assert orders[1:5] == [1, 2, 3, 4]
    # the group ran as one solve: its members finished together
    assert max(i["latency_ms"] for i in infos[1:5]) - min(i["latency_ms"] for i in infos[1:5]) \
        < 10 * TICK_US * 1e-3


def test_groups_are_off_by_default():
    with ssm.Server(max_active=1, hbm_budget=1 << 40, simulate_us=TICK_US) as srv:
        infos = run_all(srv, [(*problem(*SMALL[:2], SMALL[2], i), SMALL[2], 2) for i in range(3)])
    assert [i["group_size"] for i in infos] == [0, 0, 0]
