"""Serving on the GPU: every request reaches 1e-12 backward error, its result
is the same alone and in the mix (bit for bit: each request runs the same
deterministic kernels on its own stream), the factor cache is reused, a
failing request does not disturb the others, and the budget holds."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import cuda_or_fail, lib

pytestmark = pytest.mark.gpu

WAIT_S = 240.0     # a request that takes longer than this is stuck, not slow


def problems():
    rng_sizes = [32, 100, 257, 512, 1000, 64, 2048, 300, 777, 128]
    out = []
    for i, n in enumerate(rng_sizes):
        kappa = 10.0 ** (1 + (i % 6))
        A, V1, V2, s = wl.householder_diag(n, kappa, seed=100 + i)
        nrhs = [1, 64, 7, 16, 3, 33, 16, 1, 8, 64][i]
        Xt = wl.matrix_normal(n, nrhs, seed=200 + i)
        out.append((A, A @ Xt, Xt, kappa))
    return out


def test_mix_equals_alone_and_reaches_tolerance(oracle_mod):
    cuda_or_fail()
    g = lib()
    probs = problems()
    budget = 24 << 30
    with g.Server(budget, max_slots=4) as srv:
        tickets = [srv.enqueue(A, B) for A, B, _, _ in probs]
        mixed = srv.wait(tickets, timeout_s=WAIT_S)
        st = srv.stats()
    assert st["peak_bytes"] <= budget and st["peak_running"] > 1
    # the small requests went through shared launches, several to a batch
    assert st["batched"] >= 2 and st["batches"] < st["batched"]
    alone = []
    with g.Server(budget, max_slots=1) as srv:
        for A, B, _, _ in probs:
            t = srv.enqueue(A, B)
            alone.append(srv.wait([t], timeout_s=WAIT_S)[t])
    for (A, B, Xt, kappa), t, ra in zip(probs, tickets, alone):
        rm = mixed[t]
        assert rm["status"] == "done" and ra["status"] == "done", (rm, ra)
        assert oracle_mod.backward_error(A, B, rm["X"]).max() <= 1e-12
        np.testing.assert_array_equal(rm["X"], ra["X"])
        fwd = np.abs(rm["X"] - Xt).max() / np.abs(Xt).max()
        assert fwd <= 10 * kappa * 1e-12


def test_factor_cache_reuse(oracle_mod):
    cuda_or_fail()
    g = lib()
    A, V1, V2, s = wl.householder_diag(700, 1e3, seed=5)
    B1 = wl.matrix_normal(700, 4, seed=6)
    B2 = wl.matrix_normal(700, 4, seed=7)
    with g.Server(8 << 30, max_slots=2) as srv:
        t1 = srv.enqueue(A, B1, matrix_id=42)
        r1 = srv.wait([t1], timeout_s=WAIT_S)[t1]
        t2 = srv.enqueue(A, B2, matrix_id=42)
        r2 = srv.wait([t2], timeout_s=WAIT_S)[t2]
    assert r1["cache_hit"] == 0 and r2["cache_hit"] == 1
    assert oracle_mod.backward_error(A, B2, r2["X"]).max() <= 1e-12


def test_singular_request_fails_alone():
    cuda_or_fail()
    g = lib()
    n = 300
    bad = np.zeros((n, n))
    good = [wl.householder_diag(n, 1e2, seed=i)[0] for i in range(3)]
    with g.Server(8 << 30, max_slots=2) as srv:
        tb = srv.enqueue(bad, np.ones((n, 1)))
        tg = [srv.enqueue(A, np.ones((n, 2))) for A in good]
        res = srv.wait([tb] + tg, timeout_s=WAIT_S)
    assert res[tb]["status"] == "failed"
    assert all(res[t]["status"] == "done" and res[t]["eta"] <= 1e-12 for t in tg)


def test_device_inputs():
    torch = cuda_or_fail()
    g = lib()
    A = wl.householder_diag(256, 1e2, seed=9)[0]
    B = wl.matrix_normal(256, 3, seed=10)
    with g.Server(4 << 30, max_slots=1) as srv:
        t = srv.enqueue(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
        r = srv.wait([t], timeout_s=WAIT_S)[t]
    assert r["status"] == "done" and r["eta"] <= 1e-12


def test_borrowed_inputs_match_copied():
    """SERVE_FLAG_BORROW reads the caller's buffers in place; same X as a copy."""
    torch = cuda_or_fail()
    g = lib()
    A = wl.householder_diag(500, 1e3, seed=21)[0]
    B = wl.matrix_normal(500, 5, seed=22)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with g.Server(4 << 30, max_slots=2) as srv:
        t1 = srv.enqueue(A, B)
        t2 = srv.enqueue(dA, dB, borrow=True)
        t3 = srv.enqueue(A, B, borrow=True)
        res = srv.wait([t1, t2, t3], timeout_s=WAIT_S)
    np.testing.assert_array_equal(res[t1]["X"], res[t2]["X"])
    np.testing.assert_array_equal(res[t1]["X"], res[t3]["X"])


def test_batched_requests_match_solo_slots(oracle_mod):
    """A small request solved in a shared batch equals the same request
    solved in a batch of its own, bit for bit, and both reach 1e-12; with
    batching off the slot path also reaches it."""
    cuda_or_fail()
    g = lib()
    probs = [p for p in problems() if p[0].shape[0] <= 1024]
    with g.Server(8 << 30, max_slots=1, batch_max=64) as srv:
        tickets = [srv.enqueue(A, B) for A, B, _, _ in probs]
        together = srv.wait(tickets, timeout_s=WAIT_S)
    with g.Server(8 << 30, max_slots=1) as srv:
        solo = []
        for A, B, _, _ in probs:
            t = srv.enqueue(A, B)
            solo.append(srv.wait([t], timeout_s=WAIT_S)[t])
    with g.Server(8 << 30, max_slots=2, batch_n_max=-1) as srv:
        slot = srv.wait([srv.enqueue(A, B) for A, B, _, _ in probs], timeout_s=WAIT_S)
    for (A, B, Xt, kappa), t, rs in zip(probs, tickets, solo):
        rt = together[t]
        assert rt["status"] == "done" and rs["status"] == "done"
        np.testing.assert_array_equal(rt["X"], rs["X"])
        assert oracle_mod.backward_error(A, B, rt["X"]).max() <= 1e-12
    assert all(r["status"] == "done" and r["batched"] == 0 and r["eta"] <= 1e-12 for r in slot.values())


def test_batched_cache_hit(oracle_mod):
    cuda_or_fail()
    g = lib()
    A, V1, V2, s = wl.householder_diag(400, 1e4, seed=15)
    B1 = wl.matrix_normal(400, 3, seed=16)
    B2 = wl.matrix_normal(400, 5, seed=17)
    with g.Server(4 << 30, max_slots=1) as srv:
        t1 = srv.enqueue(A, B1, matrix_id=77)
        r1 = srv.wait([t1], timeout_s=WAIT_S)[t1]
        t2 = srv.enqueue(A, B2, matrix_id=77)
        r2 = srv.wait([t2], timeout_s=WAIT_S)[t2]
        st = srv.stats()
    assert r1["batched"] == 1 and r2["batched"] == 1
    assert r1["cache_hit"] == 0 and r2["cache_hit"] == 1 and st["cache_entries"] == 1
    assert oracle_mod.backward_error(A, B2, r2["X"]).max() <= 1e-12
