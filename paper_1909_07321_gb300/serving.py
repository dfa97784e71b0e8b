"""Continuous-batching server for R -> K -> Omega requests.

A request is one partial wave (a pole set) and a batch of energies, solved in
direct or MQDT mode; its result is the Omega rows of those energies. The
server keeps a pool of slots; each slot is one rm_ctx on its own CUDA stream,
so the work of all admitted requests overlaps on the device. Requests are
admitted in arrival order as soon as a slot is free and the device-memory
budget covers their estimated footprint (pole set, operands, workspace,
Omega); a request that arrives while others run joins as soon as that holds.
Pole sets stay resident in the slot that loaded them (a per-slot cache keyed by
pole-set id, least-recently-used eviction) so repeated sets skip the upload.

Latency of a request = completion time on the host (Omega copied back)
minus its arrival time.
"""
import collections
import time

import numpy as np


class Request:
    def __init__(self, rid, set_id, pw, E, mode, t_arrival=0.0):
        self.id = rid
        self.set_id = set_id
        self.pw = pw
        self.E = np.ascontiguousarray(E, dtype=np.float64)
        self.mode = mode
        self.t_arrival = t_arrival
        self.t_admit = None
        self.t_done = None
        self.omega = None
        self.status = None

    def footprint(self, precision):
        n, N = self.pw["W"].shape
        nl = self.pw["n_levels"]
        b = n * N * 8 + N * 8 + 16 * n                      # pole set
        if precision != 0:
            b += n * (n + 1) // 2 * ((N + 63) // 64 * 64) * 4   # split pair operands
        b += self.E.size * (nl * (nl + 1) // 2 * 8 + 16)        # Omega, statuses
        return b


class Server:
    """Slots of (context, stream); `run` serves a list of requests whose
    arrival times are replayed in real time."""

    def __init__(self, n_slots=4, precision=0, mem_budget=8 << 30, slot_workspace=1 << 30,
                 cache_sets=4, device=0):
        import torch

        from . import rmgb

        self.torch = torch
        self.rmgb = rmgb
        self.precision = precision
        self.device = device
        self.mem_budget = mem_budget
        self.cache_sets = cache_sets
        self.slots = []
        for _ in range(n_slots):
            st = torch.cuda.Stream(device=device)
            ctx = rmgb.Context(precision=precision, stream=st.cuda_stream,
                               mem_budget=slot_workspace, device=device)
            self.slots.append(dict(ctx=ctx, stream=st, req=None, done_ev=None,
                                   cache=collections.OrderedDict(), workspace=slot_workspace))
        self.mem_used = n_slots * slot_workspace

    def close(self):
        for s in self.slots:
            s["ctx"].close()
        self.slots = []

    # -- pole-set cache -------------------------------------------------------
    def _ensure_loaded(self, slot, req):
        cache = slot["cache"]
        if req.set_id in cache:
            cache.move_to_end(req.set_id)
            return cache[req.set_id]["pw_index"]
        while len(cache) >= self.cache_sets:
            _, old = cache.popitem(last=False)
            self.mem_used -= old["bytes"]
        used = {v["pw_index"] for v in cache.values()}
        idx = next(i for i in range(self.cache_sets + 1) if i not in used)
        slot["ctx"].load_pw(idx, req.pw)
        n, N = req.pw["W"].shape
        b = n * N * 8 + N * 8 + 16 * n
        cache[req.set_id] = dict(pw_index=idx, bytes=b)
        self.mem_used += b
        return idx

    def _fits(self, req):
        return self.mem_used + req.footprint(self.precision) <= self.mem_budget

    def _launch(self, slot, req, now):
        """Loads the pole set if needed (the cache accounts for its bytes) and
        enqueues the solve; the request's other bytes are held until it ends."""
        torch = self.torch
        pw_index = self._ensure_loaded(slot, req)
        with torch.cuda.stream(slot["stream"]):
            st = torch.zeros(req.E.size, dtype=torch.int32, device="cuda:%d" % self.device)
            slot["ctx"].solve_energies(pw_index, req.E, req.mode, None, None, st)
            ev = torch.cuda.Event()
            ev.record(slot["stream"])
        slot.update(req=req, done_ev=ev, status=st)
        req.t_admit = now
        self.mem_used += req.footprint(self.precision) - self._cached_bytes(slot, req)

    def _cached_bytes(self, slot, req):
        c = slot["cache"].get(req.set_id)
        return c["bytes"] if c else 0

    def _finish(self, slot, now_fn):
        req = slot["req"]
        req.omega = slot["ctx"].collision_strengths(reset=True)
        req.status = slot["status"].cpu().numpy()
        req.t_done = now_fn()
        self.mem_used -= req.footprint(self.precision) - self._cached_bytes(slot, req)
        slot.update(req=None, done_ev=None, status=None)

    def run(self, requests, idle_sleep=2e-4):
        """Serve `requests`, replaying their arrival times (seconds from the
        start of the call) in real time. Returns them with results and timings
        filled in."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        queue = collections.deque()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0   # noqa: E731
        done = 0
        total = len(pending)
        while done < total:
            t = now()
            while pending and pending[0].t_arrival <= t:
                queue.append(pending.popleft())
            progressed = False
            for slot in self.slots:
                if slot["req"] is not None and slot["done_ev"].query():
                    self._finish(slot, now)
                    done += 1
                    progressed = True
            for slot in self.slots:
                if slot["req"] is None and queue and self._fits(queue[0]):
                    self._launch(slot, queue.popleft(), now())
                    progressed = True
                elif slot["req"] is None and queue and not any(s["req"] for s in self.slots):
                    # nothing running and the head still does not fit: run it alone
                    self._launch(slot, queue.popleft(), now())
                    progressed = True
            if not progressed:
                time.sleep(idle_sleep)
        return requests


def latency_stats(requests):
    """p50 / p99 / mean latency (s) and throughput (energy-solves/s) of served requests."""
    lat = np.array([r.t_done - r.t_arrival for r in requests])
    span = max(r.t_done for r in requests) - min(r.t_arrival for r in requests)
    n_e = sum(r.E.size for r in requests)
    return dict(p50_s=float(np.quantile(lat, 0.5)), p99_s=float(np.quantile(lat, 0.99)),
                mean_s=float(lat.mean()), requests=len(requests), energy_solves=int(n_e),
                wall_s=float(span), energy_solves_per_s=float(n_e / span))
