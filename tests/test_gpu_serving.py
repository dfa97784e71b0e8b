"""Continuous-batching server: requests of different channel counts, energy
batches and modes overlap on the device; every result equals the same request
solved alone, and admission under a tight memory budget still serves them all."""
import numpy as np
import pytest

from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb, serving
    build.build()
    return torch, rmgb, serving


def _requests(serving, n_req=14, rate=400.0):
    specs = synth.serving_requests(n_req, rate, n_range=(50, 140), ne_range=(256, 1200), n_sets=6)
    pws = {}
    out = []
    for s in specs:
        if s["set_id"] not in pws:
            pws[s["set_id"]] = synth.serving_pole_set(s["set_id"], s["n"])
        out.append(serving.Request(s["id"], s["set_id"], pws[s["set_id"]], s["E"], s["mode"],
                                   s["t_arrival"]))
    return out


def _alone(rmgb, req):
    with rmgb.Context() as ctx:
        ctx.load_pw(0, req.pw)
        ctx.solve_energies(0, req.E, req.mode)
        return ctx.collision_strengths()


@pytest.mark.parametrize("budget", [8 << 30, 1])
def test_results_same_alone_and_in_the_mix(rt, budget):
    torch, rmgb, serving = rt
    reqs = _requests(serving)
    srv = serving.Server(n_slots=4, mem_budget=budget, slot_workspace=256 << 20, cache_sets=2)
    try:
        srv.run(reqs)
    finally:
        srv.close()
    for r in reqs:
        ref = _alone(rmgb, r)
        assert r.omega.shape == ref.shape
        rel = np.linalg.norm(r.omega - ref) / max(np.linalg.norm(ref), 1e-300)
        assert rel <= 1e-12, (r.id, rel)
        assert r.t_done >= r.t_admit >= r.t_arrival - 1e-3
    st = serving.latency_stats(reqs)
    assert st["p50_s"] <= st["p99_s"] and st["energy_solves"] == sum(r.E.size for r in reqs)
    if budget == 1:      # nothing fits beside another request: strictly one at a time
        spans = sorted((r.t_admit, r.t_done) for r in reqs)
        assert all(b[0] >= a[1] - 1e-3 for a, b in zip(spans, spans[1:]))
