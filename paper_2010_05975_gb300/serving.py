"""Python face of the serving C ABI (serve_create / enqueue / poll / destroy)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat

STATUS = {nat.SERVE_PENDING: "pending", nat.SERVE_RUNNING: "running", nat.SERVE_DONE: "done",
          nat.SERVE_FAILED: "failed"}


class Server:
    """Continuous-batching linear-solve server on the current CUDA device."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4, precision: int = 0, tol: float = 0.0,
                 max_queue: int = 0, dry_run: bool = False, batch_n_max: int = 0, batch_max: int = 0):
        """batch_n_max: requests with n up to this share batched launches
        (0: 1024, -1: every request takes a slot of its own); batch_max:
        most requests per shared batch (0: 256)."""
        self._lib = nat.library()
        cfg = nat.serve_cfg(int(hbm_budget_bytes), int(max_slots), int(precision), float(tol), int(max_queue),
                            1 if dry_run else 0, int(batch_n_max), int(batch_max))
        h = ctypes.c_void_p()
        nat.check("serve_create", self._lib.serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._shapes = {}
        self._borrowed = {}

    def enqueue(self, A, B, matrix_id: int = 0, tol: float = 0.0, precision: int = 0, flags: int = 0,
                borrow: bool = False) -> int:
        """Queue A X = B.  A, B: float64 numpy arrays (host) or CUDA tensors.
        borrow=True: the server reads A and B in place (no copy at enqueue);
        this object keeps them referenced until the ticket is retired.
        Returns the ticket.  Raises LuError (LU_EBUSY when it cannot fit)."""
        if borrow:
            flags |= nat.SERVE_FLAG_BORROW
        keep = []
        if hasattr(A, "is_cuda") and A.is_cuda:
            dev_in = 1
            B2 = B if B.dim() == 2 else B.view(-1, 1)
            pa, pb = A.data_ptr(), B2.data_ptr()
            n, nr, lda, ldb = A.shape[0], B2.shape[1], A.stride(0), B2.stride(0)
        else:
            dev_in = 0
            A = np.ascontiguousarray(A, dtype=np.float64)
            B2 = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1))
            keep = [A, B2]
            pa, pb = A.ctypes.data, B2.ctypes.data
            n, nr, lda, ldb = A.shape[0], B2.shape[1], A.shape[1], B2.shape[1]
        req = nat.serve_req(n, nr, pa, lda, pb, ldb, dev_in, int(matrix_id), float(tol), int(precision), int(flags))
        t = ctypes.c_uint64(0)
        rc = self._lib.serve_enqueue(self._h, ctypes.byref(req), ctypes.byref(t))
        nat.check("serve_enqueue", rc)
        self._shapes[t.value] = (n, nr)
        if borrow:
            self._borrowed[t.value] = (A, B2, keep)
        return t.value

    def poll(self, ticket: int):
        """Non-blocking.  Returns a dict; 'X' holds the solution once done."""
        st = nat.serve_status()
        n, nr = self._shapes.get(ticket, (0, 0))
        X = np.empty((n, nr), dtype=np.float64)
        rc = self._lib.serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(st),
                                  X.ctypes.data if n else None)
        nat.check("serve_poll", rc)
        out = {"status": STATUS[st.status], "error": st.error, "eta": st.eta, "latency_s": st.latency_s,
               "queue_s": st.queue_s, "iters": st.iters, "gmres_iters": st.gmres_iters, "path": st.path,
               "precision": st.precision, "cache_hit": st.cache_hit, "batched": st.batched}
        if st.status in (nat.SERVE_DONE, nat.SERVE_FAILED):
            self._shapes.pop(ticket, None)
            self._borrowed.pop(ticket, None)
            if st.status == nat.SERVE_DONE:
                out["X"] = X
        return out

    def stats(self) -> dict:
        s = nat.serve_stats()
        nat.check("serve_get_stats", self._lib.serve_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in nat.serve_stats._fields_}

    def close(self):
        if self._h:
            nat.check("serve_destroy", self._lib.serve_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def wait(self, tickets, timeout_s: float = 600.0, sleep_s: float = 0.001):
        """Poll until every ticket is retired; returns {ticket: result}."""
        import time
        out, left = {}, set(tickets)
        t0 = time.time()
        while left:
            for t in list(left):
                r = self.poll(t)
                if r["status"] in ("done", "failed"):
                    out[t] = r
                    left.discard(t)
            if left:
                if time.time() - t0 > timeout_s:
                    # say whether they sit in the queue or in a running solve
                    states = {t: self.poll(t)["status"] for t in sorted(left)}
                    raise TimeoutError(f"{len(left)} requests still pending after {timeout_s:.0f} s: "
                                       f"{states}; server {self.stats()}")
                time.sleep(sleep_s)
        return out
