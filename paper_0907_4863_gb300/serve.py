"""Continuous-batching solve server over the C ABI (requests of uneven grids and geometries).

A request is admitted as soon as (a) a slot is free, (b) its geometry has an idle solver handle
(the hierarchy, or one of up to `sets_per_geometry` work sets of it: handles that share the
hierarchy's levels and own one solve's work vectors each, made on demand), and (c) the
device-memory budget allows the hierarchy (built on a cache miss, least-recently-used idle
geometries are evicted), a new work set and the request's buffers.  Admitted requests run as
one device-loop graph launch each on their slot's stream, so the work of different requests,
of one geometry or of several, overlaps on the GPU while new requests keep being admitted.
The AMG hierarchy of a geometry is reused across its requests (Sec. 5.2, "reusing the
preconditioner").  Per request the server records the queueing time (arrival to admission),
the service time (admission to the moment its completion is observed) and their sum, the
latency.
"""
import collections
import statistics
import time

import torch

from . import inputs as I
from . import saamg as S


class Entry:
    """A cached geometry: its operator, hierarchy and work sets (handles[0] is the hierarchy)."""

    def __init__(self, op, h, nbytes):
        self.op = op
        self.handles = [h]
        self.busy = [False]
        self.bytes = nbytes
        self.prev = None      # latest finished solution of this geometry (warm start)

    def idle(self):
        for k, b in enumerate(self.busy):
            if not b:
                return k
        return None

    def any_busy(self):
        return any(self.busy)

    def free(self):
        for h in reversed(self.handles):
            h.free()
        self.op.free()


def _quantile(sorted_vals, p):
    return sorted_vals[min(len(sorted_vals) - 1, int(p * len(sorted_vals)))]


def _summary_ms(vals):
    if not vals:
        return dict(p50_ms=None, p99_ms=None, mean_ms=None)
    v = sorted(vals)
    return dict(p50_ms=1e3 * _quantile(v, 0.50), p99_ms=1e3 * _quantile(v, 0.99),
                mean_ms=1e3 * statistics.fmean(v))


class Server:
    def __init__(self, geometries, budget_bytes=120 << 30, slots=16, params=None, rtol=1e-8,
                 warm_start=False, keep_results=False, size_hints=None, sets_per_geometry=4):
        self.geoms = geometries
        self.budget = budget_bytes
        self.params = params or S.params_default(max_coarse=4096, precision=S.PREC_FP32, beta_rule=1)
        self.rtol = rtol
        self.warm = warm_start
        self.keep = keep_results
        self.max_sets = max(1, int(sets_per_geometry))
        self.cache = collections.OrderedDict()
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.used_bytes = 0
        self.peak_bytes = 0
        self.hits = 0
        self.misses = 0
        self.evictions = 0
        self.rejected = 0
        self.work_sets = 0
        self.max_inflight_same_geometry = 0
        self.results = {}
        # device bytes of each geometry's hierarchy and of one work set: measured after the
        # first build, else a bound
        self.sizes = dict(size_hints or {})
        self.set_sizes = {}

    def _request_bytes(self, g):
        return 2 * self.geoms[g].grid.nbox * 8

    def _evict_until(self, need):
        for key in list(self.cache.keys()):
            if self.used_bytes + need <= self.budget:
                break
            e = self.cache[key]
            if e.any_busy():
                continue
            e.free()
            self.used_bytes -= e.bytes
            del self.cache[key]
            self.evictions += 1
        return self.used_bytes + need <= self.budget

    def _charge(self, nbytes):
        self.used_bytes += nbytes
        self.peak_bytes = max(self.peak_bytes, self.used_bytes)

    def _entry(self, g, stream, extra=0):
        if g in self.cache:
            self.cache.move_to_end(g)
            self.hits += 1
            return self.cache[g]
        w = self.geoms[g]
        est = self.sizes.get(g, int(w.grid.nbox * 8 * 40))  # bound until measured
        if not self._evict_until(est + extra):
            return None
        self.misses += 1
        with torch.cuda.stream(stream):
            op = S.build_operator(S.make_domain(w.domain), S.make_grid(w.grid), w.mode,
                                  stream=stream.cuda_stream)
            h = S.setup(op, self.params, stream=stream.cuda_stream)
        info = h.info()
        nbytes = int(info["device_bytes"]) + w.grid.nbox * 8 * 4
        self.sizes[g] = nbytes
        e = Entry(op, h, nbytes)
        self.cache[g] = e
        self._charge(nbytes)
        return e

    def _handle(self, g, e, stream, extra):
        """An idle handle of geometry g (index into e.handles): an idle one, else a new work
        set while the geometry has fewer than sets_per_geometry and the budget allows it."""
        k = e.idle()
        if k is not None or len(e.handles) >= self.max_sets:
            return k
        est = self.set_sizes.get(g, int(self.geoms[g].grid.nbox * 8 * 12))
        if self.used_bytes + est + extra > self.budget and not self._evict_until(est + extra):
            return None
        w = S.hierarchy_work_set(e.handles[0], stream=stream.cuda_stream)
        nbytes = int(w.info()["device_bytes"])
        self.set_sizes[g] = nbytes
        e.handles.append(w)
        e.busy.append(False)
        e.bytes += nbytes
        self._charge(nbytes)
        self.work_sets += 1
        return len(e.handles) - 1

    def run(self, requests):
        """Serves the requests (sorted by arrival) and returns per-request records and stats."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        inflight = {}
        records = []
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # completions
            for slot, (req, e, k, phi, rho, t_admit) in list(inflight.items()):
                if S.solve_test(e.handles[k]):
                    info = S.solve_wait(e.handles[k])
                    t_done = time.perf_counter() - t0
                    records.append(dict(rid=req.rid, geometry=req.geometry, arrival=req.arrival,
                                        admit=t_admit, done=t_done, latency=t_done - req.arrival,
                                        queue=t_admit - req.arrival, service=t_done - t_admit,
                                        iters=info["iters"], converged=info["converged"],
                                        relres_true=info["relres_true"]))
                    if self.warm:
                        e.prev = phi
                    if self.keep:
                        self.results[req.rid] = phi
                    e.busy[k] = False
                    self.used_bytes -= self._request_bytes(req.geometry)
                    self.free_slots.append(slot)
                    del inflight[slot]
            # admissions (first come, first served among the requests that can start)
            kept = collections.deque()
            while waiting and self.free_slots:
                req = waiting.popleft()
                e = self.cache.get(req.geometry)
                if e is not None and e.idle() is None and len(e.handles) >= self.max_sets:
                    kept.append(req)
                    continue
                need = self._request_bytes(req.geometry)
                fits = self.used_bytes + need <= self.budget or self._evict_until(need)
                k = None
                slot = None
                if fits:
                    slot = self.free_slots.pop()
                    stream = self.streams[slot]
                    e = self._entry(req.geometry, stream, extra=need)
                    if e is not None:
                        k = self._handle(req.geometry, e, stream, need)
                    if k is None:
                        self.free_slots.append(slot)
                if k is None:
                    if not inflight:
                        # nothing left to wait for: the request cannot fit the budget at all
                        t_done = time.perf_counter() - t0
                        records.append(dict(rid=req.rid, geometry=req.geometry, arrival=req.arrival,
                                            admit=None, done=t_done, latency=t_done - req.arrival,
                                            queue=None, service=None, iters=0, converged=0,
                                            relres_true=None, rejected=True))
                        self.rejected += 1
                        continue
                    kept.append(req)
                    break
                w = self.geoms[req.geometry]
                c = (w.centre[0], w.centre[1], w.centre[2] + 0.005 * req.step)
                with torch.cuda.stream(stream):
                    rho = I.gaussian_bunch_torch(w.grid, c, w.sigma, req.seed)
                    phi = e.prev.clone() if (self.warm and e.prev is not None) else torch.zeros_like(rho)
                S.solve_async(e.handles[k], rho, phi, self.rtol, stream=stream.cuda_stream)
                t_admit = time.perf_counter() - t0
                e.busy[k] = True
                self.max_inflight_same_geometry = max(self.max_inflight_same_geometry, sum(e.busy))
                self._charge(need)
                inflight[slot] = (req, e, k, phi, rho, t_admit)
            waiting.extendleft(reversed(kept))
            if not inflight and not waiting and pending:
                time.sleep(max(0.0, min(0.001, pending[0].arrival - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        served = [r for r in records if not r.get("rejected")]
        lat = _summary_ms([r["latency"] for r in served])
        queue = _summary_ms([r["queue"] for r in served])
        service = _summary_ms([r["service"] for r in served])
        offered = (len(requests) / max(r.arrival for r in requests)) if requests else None
        return records, dict(requests=len(served), rejected=self.rejected, wall_s=wall,
                             solves_per_s=len(served) / wall, offered_per_s=offered,
                             p50_ms=lat["p50_ms"], p99_ms=lat["p99_ms"], mean_ms=lat["mean_ms"],
                             queue_p50_ms=queue["p50_ms"], queue_p99_ms=queue["p99_ms"],
                             queue_mean_ms=queue["mean_ms"],
                             service_p50_ms=service["p50_ms"], service_p99_ms=service["p99_ms"],
                             service_mean_ms=service["mean_ms"],
                             cache_hits=self.hits, cache_misses=self.misses,
                             evictions=self.evictions, work_sets=self.work_sets,
                             max_inflight_same_geometry=self.max_inflight_same_geometry,
                             peak_bytes=self.peak_bytes,
                             all_converged=all(r["converged"] for r in served))

    def close(self):
        for e in self.cache.values():
            e.free()
        self.cache.clear()
