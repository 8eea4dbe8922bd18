"""Serving loop over the native continuous-batching server of libfe2.

Requests (rve id, Fbar) arrive as macro Newton iterations emit them; the
server (fe2_server_*) batches queued requests per mesh size onto execution
lanes (own stream + workspace each) so that batches overlap on the device, and
reports per-request latency (completion - submission).  ``simulate`` replays
a Poisson arrival process in real time and returns p50/p99 latency and the
achieved throughput.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from .fe2 import Fe2Error, FE2_OK, _DP, _IP, fe2_last_error


class Server:
    def __init__(self, ctx, max_batch=1024, lanes=2, graphs=True, bucket=True, mixed=False):
        self.ctx = ctx
        self.lib = ctx.lib
        self.h = C.c_void_p()
        st = self.lib.fe2_server_create(ctx.h, int(max_batch), int(lanes), C.byref(self.h))
        if st != FE2_OK:
            raise Fe2Error(st, f"fe2_server_create: {fe2_last_error(ctx.h)}")
        self.lib.fe2_server_use_graphs(self.h, 1 if graphs else 0)
        self.lib.fe2_server_bucket(self.h, 1 if bucket else 0)
        self.lib.fe2_server_mixed_sizes(self.h, 1 if mixed else 0)
        self.dd = ctx.dim * ctx.dim

    def memory_stats(self):
        """(defined RVEs admitted, evicted, requests passed over for memory, device bytes held)."""
        a, e, dfr, b = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0), C.c_size_t(0)
        self.lib.fe2_server_memory_stats(self.h, C.byref(a), C.byref(e), C.byref(dfr), C.byref(b))
        return a.value, e.value, dfr.value, b.value

    def graph_stats(self):
        """(graphs captured, graph replays) of the lanes so far."""
        c, r = C.c_longlong(0), C.c_longlong(0)
        self.lib.fe2_server_graph_stats(self.h, C.byref(c), C.byref(r))
        return c.value, r.value

    def close(self):
        if self.h:
            self.lib.fe2_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, ids, Fbar):
        ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
        F = np.ascontiguousarray(np.asarray(Fbar, dtype=np.float64).reshape(len(ids), self.dd))
        tk = np.zeros(len(ids), dtype=np.int64)
        st = self.lib.fe2_server_submit(self.h, len(ids), ids.ctypes.data_as(_IP), F.ctypes.data_as(_DP),
                                        tk.ctypes.data_as(C.POINTER(C.c_longlong)))
        if st != FE2_OK:
            raise Fe2Error(st, f"fe2_server_submit: {fe2_last_error(self.ctx.h)}")
        return tk

    def pump(self):
        busy = C.c_int(0)
        st = self.lib.fe2_server_pump(self.h, C.byref(busy))
        if st != FE2_OK:
            raise Fe2Error(st, f"fe2_server_pump: {fe2_last_error(self.ctx.h)}")
        return busy.value

    def pending(self):
        return int(self.lib.fe2_server_pending(self.h))

    def take(self, max_n=65536):
        tk = np.zeros(max_n, dtype=np.int64)
        sig = np.zeros((max_n, self.dd))
        Cb = np.zeros((max_n, self.dd, self.dd))
        st = np.zeros(max_n, dtype=np.int32)
        lat = np.zeros(max_n)
        n = self.lib.fe2_server_take(self.h, max_n, tk.ctypes.data_as(C.POINTER(C.c_longlong)),
                                     sig.ctypes.data_as(_DP), Cb.ctypes.data_as(_DP), st.ctypes.data_as(_IP),
                                     lat.ctypes.data_as(_DP))
        return tk[:n], sig[:n], Cb[:n], st[:n], lat[:n]

    def drain(self, timeout_s=120.0):
        out = []
        t0 = time.perf_counter()
        while self.pending() > 0:
            self.pump()
            out.append(self.take())
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
        out.append(self.take())
        return [np.concatenate([o[i] for o in out]) for i in range(5)]


def simulate(server, ids, Fbar, arrivals):
    """Submit request k at wall time arrivals[k] (seconds from start), pump
    continuously, return (results dict, p50 ms, p99 ms, requests/s)."""
    n = len(ids)
    order = np.argsort(arrivals, kind="stable")
    t0 = time.perf_counter()
    k = 0
    res = []
    while k < n or server.pending() > 0:
        now = time.perf_counter() - t0
        j = k
        while j < n and arrivals[order[j]] <= now:
            j += 1
        if j > k:
            sel = order[k:j]
            server.submit(ids[sel], Fbar[sel])
            k = j
        server.pump()
        r = server.take()
        if len(r[0]):
            res.append(r)
    elapsed = time.perf_counter() - t0
    tk, sig, Cb, st, lat = [np.concatenate([r[i] for r in res]) for i in range(5)]
    return dict(tickets=tk, sigma=sig, Cbar=Cb, status=st, latency_ms=lat), \
        float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), n / elapsed
