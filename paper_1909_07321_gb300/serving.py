"""Continuous-batching server for R -> K -> Omega requests.

A request is one partial wave (a pole set) and a batch of energies, solved in
direct or MQDT mode; its result is the Omega rows of those energies. The
server owns ONE library context with one lane per slot (rm_opts.lanes): each
lane has its own CUDA stream, workspace and Omega accumulator, and all lanes
share the context's partial waves, so a pole set is loaded once and every slot
uses it. Requests are admitted in arrival order as soon as a lane is free and
the device-memory budget covers what the request adds (its pole set if not
resident, exactly as rm_pw_bytes reports it once loaded); a request that
arrives while others run joins as soon as that holds, and its work overlaps
theirs on the device.

Before serving, every lane's workspace is sized once for the largest request
of the stream (rm_lane_reserve), so no solve in the mix allocates device
memory (a cudaMalloc would synchronise the whole device). Resident pole sets
are kept in least-recently-used order and evicted (rm_unload_pw) only when
no running request uses them.

Pole-set loads (rm_load_poles + rm_set_channels, which build the channel
tables) run synchronously in the admission loop; with the shared cache each
set is loaded once per residency, not once per slot.

Latency of a request = completion time on the host (Omega copied back)
minus its arrival time. A completed request's Omega goes to the server's
sink (a callable taking the request and its Omega rows) if one is given,
else to request.omega: a long stream's results (up to 8192 energies x 70k
level pairs each) need not all stay in host memory.
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

    def n_tri(self):
        nl = self.pw["n_levels"]
        return nl * (nl + 1) // 2


def estimate_set_bytes(pw, precision):
    """Device bytes of a pole set before it is loaded: poles and amplitudes,
    channel data, the channel tables (near-threshold nodes, open- and
    closed-side Chebyshev coefficients: about 85 KB per channel) and, with a
    tensor-core formation, the split operands (per-energy form: W in FP32 and
    split hi/lo). rm_pw_bytes replaces it once the set is loaded."""
    n, N = pw["W"].shape
    b = n * N * 8 + N * 16 + 64 * n
    if precision != 0:
        b += 85_000 * n
        kpad = (N + 63) // 64 * 64
        b += n * kpad * (4 + 4 + 4)
    return b


class Server:
    """One context with n_slots lanes; `run` serves a list of requests whose
    arrival times are replayed in real time."""

    def __init__(self, n_slots=4, precision=0, solve_precision=0, mem_budget=96 << 30,
                 lane_workspace=16 << 30, cache_sets=64, device=0, sink=None):
        from . import rmgb

        self.rmgb = rmgb
        self.sink = sink
        self.precision = precision
        self.device = device
        self.mem_budget = mem_budget
        self.cache_sets = cache_sets
        self.ctx = rmgb.Context(precision=precision, solve_precision=solve_precision, lanes=n_slots,
                                mem_budget=lane_workspace, device=device, stream=0)
        self.slots = [dict(lane=i, req=None) for i in range(n_slots)]
        self.lane_bytes = [0] * n_slots
        self.cache = collections.OrderedDict()     # set_id -> dict(pw_index, bytes, users)
        self.free_index = list(range(4095, -1, -1))
        self.loads = 0

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None

    # -- memory accounting -------------------------------------------------------
    def mem_used(self):
        return sum(self.lane_bytes) + sum(c["bytes"] for c in self.cache.values())

    def _need(self, req):
        """Bytes the request adds: its pole set if not resident, and its
        Omega rows on the host side are not device memory."""
        if req.set_id in self.cache:
            return 0
        return estimate_set_bytes(req.pw, self.precision)

    def _evictable(self):
        return [sid for sid, c in self.cache.items() if c["users"] == 0]

    def _make_room(self, need, new_set=True):
        """Evicts unused pole sets (least recently used first) until `need`
        more bytes fit the budget (and, for a set to be loaded, the cache has
        a free entry) or nothing more can be evicted."""
        while self.mem_used() + need > self.mem_budget or (new_set and len(self.cache) >= self.cache_sets):
            ev = self._evictable()
            if not ev:
                return False
            sid = ev[0]
            c = self.cache.pop(sid)
            self.ctx.unload_pw(c["pw_index"])
            self.free_index.append(c["pw_index"])
        return True

    # -- pole-set cache ----------------------------------------------------------
    def _ensure_loaded(self, req):
        c = self.cache.get(req.set_id)
        if c is not None:
            self.cache.move_to_end(req.set_id)
            return c
        idx = self.free_index.pop()
        self.ctx.load_pw(idx, req.pw)
        self.loads += 1
        c = dict(pw_index=idx, bytes=self.ctx.pw_bytes(idx), users=0)
        self.cache[req.set_id] = c
        return c

    def prepare(self, requests):
        """Sizes every lane's workspace for the largest request of the stream
        (most channels, then most energies) before serving."""
        big = max(requests, key=lambda r: (r.pw["W"].shape[0], r.E.size))
        n_e = max(r.E.size for r in requests)
        self._make_room(self._need(big))
        c = self._ensure_loaded(big)
        for s in self.slots:
            self.lane_bytes[s["lane"]] = self.ctx.lane_reserve(s["lane"], c["pw_index"], n_e)

    def _fits(self, req):
        resident = req.set_id in self.cache
        need = self._need(req)
        if self.mem_used() + need <= self.mem_budget and (resident or len(self.cache) < self.cache_sets):
            return True
        return self._make_room(need, new_set=not resident)

    def _launch(self, slot, req, now):
        c = self._ensure_loaded(req)
        c["users"] += 1
        self.ctx.lane_solve_energies(slot["lane"], c["pw_index"], req.E, req.mode)
        slot.update(req=req, cache=c)
        req.t_admit = now

    def _finish(self, slot, now_fn):
        req = slot["req"]
        om = np.empty((req.E.size, req.n_tri()), dtype=np.float64)
        self.ctx.lane_collision_strengths(slot["lane"], om, reset=True)
        req.t_done = now_fn()
        if self.sink is not None:
            self.sink(req, om)
        else:
            req.omega = om
        slot["cache"]["users"] -= 1
        slot.update(req=None, cache=None)

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
                if slot["req"] is not None and self.ctx.lane_query(slot["lane"]):
                    self._finish(slot, now)
                    done += 1
                    progressed = True
            for slot in self.slots:
                if slot["req"] is None and queue:
                    busy = any(s["req"] is not None for s in self.slots)
                    if self._fits(queue[0]) or not busy:
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
