"""Continuous-batching solve server over the C ABI (requests of uneven grids and geometries).

A request is admitted as soon as (a) a slot is free, (b) its geometry's hierarchy is not busy
(a hierarchy holds one solve's work vectors; the requests of one geometry are successive time
steps of one simulation anyway), and (c) the device-memory budget allows the hierarchy (built
on a cache miss, least-recently-used idle hierarchies are evicted) and the request's buffers.
Admitted requests run as one device-loop graph launch each on their slot's stream, so the work
of different requests overlaps on the GPU while new requests keep being admitted.  The AMG
hierarchy of a geometry is reused across its time steps (Sec. 5.2, "reusing the preconditioner").
Latency is measured from a request's arrival to the moment its completion is observed.
"""
import collections
import statistics
import time

import torch

from . import inputs as I
from . import saamg as S


class Entry:
    def __init__(self, op, h, nbytes):
        self.op = op
        self.h = h
        self.bytes = nbytes
        self.busy = False
        self.prev = None      # previous time step's solution (warm start)


class Server:
    def __init__(self, geometries, budget_bytes=120 << 30, slots=16, params=None, rtol=1e-8,
                 warm_start=False, keep_results=False, size_hints=None):
        self.geoms = geometries
        self.budget = budget_bytes
        self.params = params or S.params_default(max_coarse=4096, precision=S.PREC_FP32, beta_rule=1)
        self.rtol = rtol
        self.warm = warm_start
        self.keep = keep_results
        self.cache = collections.OrderedDict()
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.used_bytes = 0
        self.peak_bytes = 0
        self.hits = 0
        self.misses = 0
        self.evictions = 0
        self.rejected = 0
        self.results = {}
        # device bytes of each geometry's hierarchy: measured after a build, else a bound
        self.sizes = dict(size_hints or {})

    def _request_bytes(self, g):
        return 2 * self.geoms[g].grid.nbox * 8

    def _evict_until(self, need):
        for key in list(self.cache.keys()):
            if self.used_bytes + need <= self.budget:
                break
            e = self.cache[key]
            if e.busy:
                continue
            e.h.free()
            e.op.free()
            self.used_bytes -= e.bytes
            del self.cache[key]
            self.evictions += 1
        return self.used_bytes + need <= self.budget

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
        self.used_bytes += nbytes
        self.peak_bytes = max(self.peak_bytes, self.used_bytes)
        return e

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
            for slot, (req, e, phi, rho) in list(inflight.items()):
                if S.solve_test(e.h):
                    info = S.solve_wait(e.h)
                    t_done = time.perf_counter() - t0
                    records.append(dict(rid=req.rid, geometry=req.geometry, arrival=req.arrival,
                                        done=t_done, latency=t_done - req.arrival, iters=info["iters"],
                                        converged=info["converged"], relres_true=info["relres_true"]))
                    if self.warm:
                        e.prev = phi
                    if self.keep:
                        self.results[req.rid] = phi
                    e.busy = False
                    self.used_bytes -= self._request_bytes(req.geometry)
                    self.free_slots.append(slot)
                    del inflight[slot]
            # admissions (first come, first served among the geometries that are free)
            kept = collections.deque()
            while waiting and self.free_slots:
                req = waiting.popleft()
                e = self.cache.get(req.geometry)
                if e is not None and e.busy:
                    kept.append(req)
                    continue
                need = self._request_bytes(req.geometry)
                fits = self.used_bytes + need <= self.budget or self._evict_until(need)
                e = None
                slot = None
                if fits:
                    slot = self.free_slots.pop()
                    stream = self.streams[slot]
                    e = self._entry(req.geometry, stream, extra=need)
                    if e is None:
                        self.free_slots.append(slot)
                if e is None:
                    if not inflight:
                        # nothing left to wait for: the request cannot fit the budget at all
                        t_done = time.perf_counter() - t0
                        records.append(dict(rid=req.rid, geometry=req.geometry, arrival=req.arrival,
                                            done=t_done, latency=t_done - req.arrival, iters=0,
                                            converged=0, relres_true=None, rejected=True))
                        self.rejected += 1
                        continue
                    kept.append(req)
                    break
                w = self.geoms[req.geometry]
                c = (w.centre[0], w.centre[1], w.centre[2] + 0.005 * req.step)
                with torch.cuda.stream(stream):
                    rho = I.gaussian_bunch_torch(w.grid, c, w.sigma, req.seed)
                    phi = e.prev.clone() if (self.warm and e.prev is not None) else torch.zeros_like(rho)
                S.solve_async(e.h, rho, phi, self.rtol, stream=stream.cuda_stream)
                e.busy = True
                self.used_bytes += need
                self.peak_bytes = max(self.peak_bytes, self.used_bytes)
                inflight[slot] = (req, e, phi, rho)
            waiting.extendleft(reversed(kept))
            if not inflight and not waiting and pending:
                time.sleep(max(0.0, min(0.001, pending[0].arrival - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        served = [r for r in records if not r.get("rejected")]
        lat = sorted(r["latency"] for r in served)
        q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None  # noqa: E731
        return records, dict(requests=len(served), rejected=self.rejected, wall_s=wall,
                             solves_per_s=len(served) / wall,
                             p50_ms=1e3 * q(0.50) if lat else None,
                             p99_ms=1e3 * q(0.99) if lat else None,
                             mean_ms=1e3 * statistics.fmean(lat) if lat else None,
                             cache_hits=self.hits, cache_misses=self.misses,
                             evictions=self.evictions, peak_bytes=self.peak_bytes,
                             all_converged=all(r["converged"] for r in served))

    def close(self):
        for e in self.cache.values():
            e.h.free()
            e.op.free()
        self.cache.clear()
