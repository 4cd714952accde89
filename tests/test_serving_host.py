"""Host logic of the serving runtime, run in its dry-run mode (no device
work: each request holds its memory budget for a time proportional to n^3).
Covers admission by HBM budget, the slot limit, continuous batching, the
factor cache (hits, LRU eviction) and failure isolation."""
import numpy as np
import pytest

import paper_2010_05975_gb300 as g
from paper_2010_05975_gb300 import _native as nat


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_05975_gb300 import build
    build.build()


def req_bytes(n, nrhs):
    """The server's own estimate (persistent + transient), to size budgets."""
    per = n * n * 12 + n * 4 + 4096
    vs = n * nrhs
    trans = 2 * vs * 8 + vs * (8 + 4 + 8 * (2 * 30 + 2)) + (304 * nrhs * 4 + 32 * 16 * nrhs + 16 * nrhs) * 8 + 4096 + n * 2048
    return per + trans


def small_problem(n, nrhs=1):
    return np.eye(n), np.ones((n, nrhs))


def test_budget_never_exceeded_and_all_complete():
    budget = 3 * req_bytes(400, 4)
    with g.Server(budget, max_slots=4, dry_run=True) as srv:
        sizes = [400, 100, 300, 50, 400, 250, 64, 128, 399, 200] * 3
        tickets = [srv.enqueue(*small_problem(n, 4)) for n in sizes]
        res = srv.wait(tickets)
        st = srv.stats()
    assert all(r["status"] == "done" for r in res.values())
    assert st["completed"] == len(sizes) and st["failed"] == 0
    assert st["peak_bytes"] <= budget
    assert 1 < st["peak_running"] <= 4


def test_request_that_can_never_fit_is_rejected():
    with g.Server(req_bytes(100, 1), max_slots=2, dry_run=True) as srv:
        with pytest.raises(nat.LuError) as e:
            srv.enqueue(*small_problem(2000, 1))
        assert e.value.code == nat.LU_EBUSY
        t = srv.enqueue(*small_problem(50, 1))
        assert srv.wait([t])[t]["status"] == "done"


def test_continuous_batching_admits_new_work_while_busy():
    """A request enqueued while a long one runs starts before it finishes."""
    with g.Server(1 << 34, max_slots=2, dry_run=True) as srv:
        big = srv.enqueue(*small_problem(1500, 1))         # ~0.5 s simulated
        import time
        time.sleep(0.05)
        small = srv.enqueue(*small_problem(20, 1))
        r = srv.wait([small])[small]
        assert srv.poll(big)["status"] in ("running",)
        assert r["queue_s"] < 0.2
        srv.wait([big])


def test_factor_cache_hits_and_lru_eviction():
    budget = 2 * req_bytes(300, 1) + req_bytes(300, 1) // 2
    with g.Server(budget, max_slots=1, dry_run=True) as srv:
        A, B = small_problem(300, 1)
        t1 = srv.enqueue(A, B, matrix_id=7)
        srv.wait([t1])
        t2 = srv.enqueue(A, B, matrix_id=7)
        r2 = srv.wait([t2])[t2]
        assert r2["cache_hit"] == 1
        for mid in (8, 9, 10):                             # fill the cache past its budget
            t = srv.enqueue(A, B, matrix_id=mid)
            srv.wait([t])
        st = srv.stats()
        assert st["evictions"] >= 1 and st["peak_bytes"] <= budget
        t3 = srv.enqueue(A, B, matrix_id=7)                # evicted long ago: a miss
        assert srv.wait([t3])[t3]["cache_hit"] == 0


def test_failure_does_not_block_others():
    with g.Server(1 << 32, max_slots=2, dry_run=True) as srv:
        bad = srv.enqueue(*small_problem(200, 1), flags=nat.SERVE_FLAG_FAIL)
        good = [srv.enqueue(*small_problem(n, 2)) for n in (10, 200, 30)]
        res = srv.wait([bad] + good)
        assert res[bad]["status"] == "failed"
        assert all(res[t]["status"] == "done" for t in good)
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 3


def test_poll_retires_tickets():
    with g.Server(1 << 30, max_slots=1, dry_run=True) as srv:
        t = srv.enqueue(*small_problem(10, 1))
        srv.wait([t])
        with pytest.raises(nat.LuError) as e:
            srv.poll(t)
        assert e.value.code == nat.LU_ENOTFOUND
