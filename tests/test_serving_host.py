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


def req_bytes(n, nrhs, batched=None):
    """The server's own estimate (persistent + transient), to size budgets.
    batched: the shared-launch path (default for n <= 1024) or a slot."""
    if batched is None:
        batched = n <= 1024
    vs = n * nrhs
    per = n * n * 12 + n * 4 + 4096
    if batched:
        return per + vs * (3 * 8 + 4) + 16 * nrhs + 4096
    per += -(-n // 128) * 128 * 2048 + n * 4 + 4096
    trans = 2 * vs * 8 + vs * (8 + 4 + 8 * (2 * 30 + 2) + 16) + n * 16 * 4 + (304 * nrhs * 4 + 32 * 16 * nrhs + 16 * nrhs) * 8 \
        + 4096 + n * (4 * 1040 + 2048)
    return per + trans


def small_problem(n, nrhs=1):
    return np.eye(n), np.ones((n, nrhs))


def test_budget_never_exceeded_and_all_complete():
    """Every request on a slot of its own (batching off): the slot limit and
    the budget hold."""
    budget = 3 * req_bytes(400, 4, batched=False)
    with g.Server(budget, max_slots=4, dry_run=True, batch_n_max=-1) as srv:
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


def test_small_requests_share_batches_within_budget():
    """Small requests that queue while the batch worker is busy go out
    together in the next shared launch; the budget still holds."""
    budget = 12 * req_bytes(400, 4)
    with g.Server(budget, max_slots=2, dry_run=True) as srv:
        sizes = [400, 100, 300, 50, 400, 250, 64, 128, 399, 200] * 4
        tickets = [srv.enqueue(*small_problem(n, 4)) for n in sizes]
        res = srv.wait(tickets)
        st = srv.stats()
    assert all(r["status"] == "done" and r["batched"] == 1 for r in res.values())
    assert st["completed"] == len(sizes) and st["batched"] == len(sizes)
    assert st["batches"] < len(sizes)                    # some requests shared a launch
    assert st["peak_bytes"] <= budget


def test_batch_limit_and_large_requests_take_slots():
    with g.Server(1 << 36, max_slots=2, dry_run=True, batch_max=3) as srv:
        tickets = [srv.enqueue(*small_problem(200, 1)) for _ in range(10)]
        big = srv.enqueue(*small_problem(1100, 1))
        res = srv.wait(tickets + [big])
        st = srv.stats()
    assert res[big]["batched"] == 0 and res[big]["status"] == "done"
    assert all(res[t]["batched"] == 1 for t in tickets)
    assert st["batches"] >= 4                            # at most 3 per batch
    assert st["batched"] == 10


def test_batching_off():
    with g.Server(1 << 34, max_slots=2, dry_run=True, batch_n_max=-1) as srv:
        tickets = [srv.enqueue(*small_problem(64, 1)) for _ in range(5)]
        res = srv.wait(tickets)
        st = srv.stats()
    assert all(r["batched"] == 0 for r in res.values())
    assert st["batches"] == 0


def test_bad_batch_config_rejected():
    with pytest.raises(nat.LuError):
        g.Server(1 << 30, dry_run=True, batch_n_max=2048)
    with pytest.raises(nat.LuError):
        g.Server(1 << 30, dry_run=True, batch_max=-1)


def test_queue_bound_holds_per_path():
    """max_queue bounds each path's queue: a backlog of large requests turns
    further large ones away but still admits small ones."""
    import time
    with g.Server(1 << 38, max_slots=1, max_queue=2, dry_run=True) as srv:
        first = srv.enqueue(*small_problem(1500, 1))      # occupies the only slot (~0.5 s)
        time.sleep(0.05)
        queued = [srv.enqueue(*small_problem(1200, 1)) for _ in range(2)]
        with pytest.raises(nat.LuError) as e:
            srv.enqueue(*small_problem(1200, 1))
        assert e.value.code == nat.LU_EBUSY
        smalls = [srv.enqueue(*small_problem(64, 1)) for _ in range(2)]
        res = srv.wait(smalls + [first] + queued)
    assert all(r["status"] == "done" for r in res.values())


def test_budget_accounting_matches_cache_entries():
    """With every request done, the bytes the server still charges are
    exactly its cached entries' (the factors kept per matrix id)."""
    with g.Server(1 << 36, max_slots=2, dry_run=True) as srv:
        ids = [11, 12, 13]
        ts = [srv.enqueue(*small_problem(300, 2), matrix_id=i) for i in ids]          # batched path
        ts += [srv.enqueue(*small_problem(1100, 1), matrix_id=20 + i) for i in range(2)]   # slot path
        ts += [srv.enqueue(*small_problem(200, 1)) for _ in range(3)]                 # no cache
        srv.wait(ts)
        st = srv.stats()
    assert st["cache_entries"] == 5
    assert st["used_bytes"] == 3 * (300 * 300 * 12 + 300 * 4 + 4096) + \
        2 * (1100 * 1100 * 12 + 1100 * 4 + 4096 + 9 * 128 * 2048 + 1100 * 4 + 4096)
