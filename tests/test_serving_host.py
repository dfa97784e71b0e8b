"""Host logic of the continuous-batching server (serving.py) on the CPU, with
the device replaced by fakes: first-come admission, the memory budget (a
request waits until it fits, or runs alone), overlap of requests across
slots, the per-slot pole-set cache with least-recently-used eviction and its
byte accounting, and that every request gets its own result."""
import collections
import contextlib

import numpy as np

from paper_1909_07321_gb300 import serving, synth


class _Tensor:
    def __init__(self, a):
        self.a = a

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class _Event:
    """Completes after a fixed number of polls (the fake device's work)."""

    def __init__(self, polls):
        self.left = polls

    def record(self, stream):
        pass

    def query(self):
        self.left -= 1
        return self.left <= 0


class _Cuda:
    def __init__(self, owner):
        self.owner = owner

    def stream(self, s):
        return contextlib.nullcontext()

    def Event(self):
        return _Event(self.owner.next_polls)


class _Torch:
    int32 = np.int32

    def __init__(self):
        self.next_polls = 3
        self.cuda = _Cuda(self)

    def zeros(self, n, dtype=None, device=None):
        return _Tensor(np.zeros(n, dtype=np.int32))


def _result(pw, E):
    nl = pw["n_levels"]
    return np.outer(E, np.arange(nl * (nl + 1) // 2) + 1.0) * pw["g"] + pw["E_k"][0]


class _Ctx:
    def __init__(self, log):
        self.log = log
        self.waves = {}
        self.last = None

    def load_pw(self, idx, pw):
        self.waves[idx] = pw
        self.log.append(("load", id(pw), idx))

    def solve_energies(self, idx, E, mode, K, no, st):
        self.last = _result(self.waves[idx], E)

    def collision_strengths(self, reset=False):
        return self.last


class _Server(serving.Server):
    """The server with fake slots; records the budget state at every launch."""

    def __init__(self, n_slots, mem_budget, workspace, cache_sets):
        self.torch = _Torch()
        self.precision = 2
        self.device = 0
        self.mem_budget = mem_budget
        self.cache_sets = cache_sets
        self.log = []
        self.slots = [dict(ctx=_Ctx(self.log), stream=None, req=None, done_ev=None,
                           cache=collections.OrderedDict(), workspace=workspace)
                      for _ in range(n_slots)]
        self.mem_used = n_slots * workspace
        self.launches = []

    def _launch(self, slot, req, now):
        running = sum(1 for s in self.slots if s["req"] is not None)
        self.torch.next_polls = 2 + (req.id % 5)
        fits = self._fits(req)
        super()._launch(slot, req, now)
        self.launches.append((req.id, running, fits, self.mem_used))


def _requests(n, n_sets=3, seed=0):
    rng = np.random.default_rng(seed)
    sets = []
    for k in range(n_sets):
        pw = synth.random_pw(100 + k, 4 + 2 * k, 30 + 10 * k)
        pw["g"] = 1.0 + k
        sets.append(pw)
    reqs = []
    for i in range(n):
        sid = int(rng.integers(0, n_sets))
        E = np.sort(rng.uniform(0.0, 2.0, int(rng.integers(5, 40))))
        reqs.append(serving.Request(i, sid, sets[sid], E, int(rng.integers(0, 2)), t_arrival=0.0))
    return reqs


def test_every_request_gets_its_own_result_in_arrival_order():
    reqs = _requests(30)
    big = max(r.footprint(2) for r in reqs)
    srv = _Server(n_slots=3, mem_budget=3 * (1 << 20) + 2 * big + 3 * 50_000, workspace=1 << 20, cache_sets=2)
    srv.run(reqs, idle_sleep=0.0)
    for r in reqs:
        assert r.t_done is not None and r.omega is not None
        np.testing.assert_array_equal(r.omega, _result(r.pw, r.E))
    # first come, first admitted
    order = [rid for rid, *_ in srv.launches]
    assert order == sorted(order)
    # requests overlapped on the slots
    assert max(running for _, running, _, _ in srv.launches) >= 1
    # a launch either fitted the budget or ran alone
    for _, running, fits, _ in srv.launches:
        assert fits or running == 0


def test_budget_forces_one_at_a_time_and_bytes_are_returned():
    reqs = _requests(12, seed=1)
    small = min(r.footprint(2) for r in reqs)
    srv = _Server(n_slots=4, mem_budget=4 * (1 << 20) + small // 2, workspace=1 << 20, cache_sets=1)
    srv.run(reqs, idle_sleep=0.0)
    assert all(running == 0 for _, running, _, _ in srv.launches)
    # only the cached pole sets stay accounted once everything is done
    cached = sum(v["bytes"] for s in srv.slots for v in s["cache"].values())
    assert srv.mem_used == 4 * (1 << 20) + cached
    for r in reqs:
        np.testing.assert_array_equal(r.omega, _result(r.pw, r.E))


def test_pole_set_cache_evicts_least_recently_used():
    # one slot, room for two sets: A B A C A B -> C evicts B (least recent),
    # A stays, B is loaded again and evicts C
    pws = {}
    for r in _requests(40, n_sets=3, seed=3):
        pws.setdefault(r.set_id, r.pw)
    order = [0, 1, 0, 2, 0, 1]
    reqs = [serving.Request(i, sid, pws[sid], np.linspace(0.1, 1.0, 5), 0) for i, sid in enumerate(order)]
    srv = _Server(n_slots=1, mem_budget=1 << 40, workspace=1 << 20, cache_sets=2)
    srv.run(reqs, idle_sleep=0.0)
    loads = [pw_id for kind, pw_id, _ in srv.log if kind == "load"]
    assert loads == [id(pws[0]), id(pws[1]), id(pws[2]), id(pws[1])]
    assert list(srv.slots[0]["cache"].keys()) == [0, 1]
    for r in reqs:
        np.testing.assert_array_equal(r.omega, _result(r.pw, r.E))
