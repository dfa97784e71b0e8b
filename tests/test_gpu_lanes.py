"""Lanes of one context (rm_opts.lanes): solves enqueued on different lanes
overlap on the device and share the context's partial waves, yet each lane's
Omega equals what a context of its own computes; a lane sized by
rm_lane_reserve allocates no device memory during its solve; lane arguments
are checked."""
import numpy as np
import pytest

from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


def _waves():
    a = synth.workload_64ch(3000)
    b = synth.random_pw(777, 130, 3900, z=2.0, a=15.0, e_max=2.0, sigma=0.05, pole_lo=-2.0, pole_hi=60.0,
                        l_max=8)
    return [(a[0][0], a[1][::3].copy()), (b, synth.midpoint_grid(0.01, 2.5, 700))]


def _alone(rmgb, pw, E, mode, **kw):
    with rmgb.Context(**kw) as ctx:
        ctx.load_pw(0, pw)
        ctx.solve_energies(0, E, mode)
        return ctx.collision_strengths()


@pytest.mark.parametrize("prec,sp", [(0, 0), (2, 1)])
def test_lanes_overlap_and_equal_separate_contexts(rt, prec, sp):
    torch, rmgb = rt
    waves = _waves()
    jobs = [(0, 0, 0), (1, 1, 0), (2, 0, 1), (3, 1, 1)]    # (lane, wave, mode)
    with rmgb.Context(precision=prec, solve_precision=sp, lanes=4, stream=0) as ctx:
        for w, (pw, _) in enumerate(waves):
            ctx.load_pw(w, pw)
        for lane, w, mode in jobs:
            ctx.lane_solve_energies(lane, w, waves[w][1], mode)
        outs = {}
        for lane, w, mode in jobs:
            pw, E = waves[w]
            nl = pw["n_levels"]
            om = np.empty((E.size, nl * (nl + 1) // 2))
            ctx.lane_collision_strengths(lane, om, reset=True)
            assert ctx.lane_query(lane)
            outs[lane] = om
    for lane, w, mode in jobs:
        pw, E = waves[w]
        ref = _alone(rmgb, pw, E, mode, precision=prec, solve_precision=sp)
        np.testing.assert_array_equal(outs[lane], ref)


def test_reserved_lane_allocates_nothing(rt):
    torch, rmgb = rt
    pw, E = _waves()[1]
    with rmgb.Context(precision=2, solve_precision=1, lanes=2, stream=0, mem_budget=256 << 20) as ctx:
        ctx.load_pw(0, pw)
        # a first solve on lane 0 loads the kernels (lazy module loading
        # allocates device memory once per process)
        ctx.solve_energies(0, E[:64], 0)
        ctx.sync()
        b = ctx.lane_reserve(1, 0, E.size)
        assert b > 0
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ctx.lane_solve_energies(1, 0, Ed, 0)
        ctx.lane_sync(1)
        free1 = torch.cuda.mem_get_info()[0]
        assert free0 == free1, free0 - free1
        assert ctx.lane_reserve(1, 0, E.size) == b     # already sized: unchanged
        assert ctx.pw_bytes(0) > pw["W"].size * 8


def test_bad_lane_is_rejected(rt):
    torch, rmgb = rt
    pw, E = _waves()[1]
    with rmgb.Context(lanes=2, stream=0) as ctx:
        ctx.load_pw(0, pw)
        with pytest.raises(rmgb.RmError):
            ctx.lane_solve_energies(2, 0, E[:8], 0)
        with pytest.raises(rmgb.RmError):
            ctx.lane_query(-1)
        assert ctx.lane_stream(5) is None
        ctx.unload_pw(0)
        with pytest.raises(rmgb.RmError):
            ctx.lane_solve_energies(0, 0, E[:8], 0)
