"""A matching system that FP32 cannot hold is reported singular, not solved.

The per-energy status of Eq. match (Section "Overview") is RM_ESINGULAR when
the elimination meets a zero or non-finite pivot. Amplitudes scaled by 1e22
make R ~ 1e40 at every energy of the 4-channel workload: finite in FP64, past
the largest FP32 number. The FP64 solve of that system succeeds (K and Omega
finite); both FP32 solvers (the shared-memory one, whose factoring warp takes
the decision once per block of pivots, and the global-memory one) must mark
every such energy RM_ESINGULAR and add nothing to its Omega row."""
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


def _run(rt, pw, E, solver, sp):
    torch, rmgb = rt
    with rmgb.Context(precision=rmgb.RM_FP64, solver=solver, solve_precision=sp) as ctx:
        ctx.load_pw(0, pw)
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, E, rmgb.RM_DIRECT, None, None, st)
        om = ctx.collision_strengths()
    return st.cpu().numpy(), om


@pytest.mark.parametrize("solver", ["small", "large"])
def test_fp32_overflowing_system_is_singular(rt, solver):
    _, rmgb = rt
    sv = rmgb.RM_SOLVER_SMALL if solver == "small" else rmgb.RM_SOLVER_LARGE
    pws, E = synth.workload_small(64)
    pw = dict(pws[0])
    pw["W"] = pw["W"] * 1e22
    st64, om64 = _run(rt, pw, E, sv, rmgb.RM_FP64)
    ok = st64 == rmgb.RM_OK
    assert ok.sum() >= 60
    assert np.all(np.isfinite(om64)) and np.abs(om64[ok]).max() > 0.0
    st32, om32 = _run(rt, pw, E, sv, rmgb.RM_FP32)
    assert np.all(st32[ok] == rmgb.RM_ESINGULAR), np.unique(st32[ok])
    assert np.all(om32 == 0.0)


@pytest.mark.parametrize("solver", ["small", "large"])
def test_fp32_solve_after_singular_energies(rt, solver):
    """The same context then solves the unscaled workload: every energy that
    can be solved is (a singular energy of one launch leaves nothing behind
    for the next)."""
    torch, rmgb = rt
    sv = rmgb.RM_SOLVER_SMALL if solver == "small" else rmgb.RM_SOLVER_LARGE
    pws, E = synth.workload_small(64)
    big = dict(pws[0])
    big["W"] = big["W"] * 1e22
    with rmgb.Context(precision=rmgb.RM_FP64, solver=sv, solve_precision=rmgb.RM_FP32) as ctx:
        ctx.load_pw(0, big)
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, E, rmgb.RM_DIRECT, None, None, st)
        ctx.sync()
        s1 = st.cpu().numpy()
        assert np.all((s1 == rmgb.RM_ESINGULAR) | (s1 == rmgb.RM_ENEAR_POLE) | (s1 == rmgb.RM_ETHRESHOLD))
        ctx.collision_strengths(reset=True)
        ctx.load_pw(0, pws[0])
        ctx.solve_energies(0, E, rmgb.RM_DIRECT, None, None, st)
        om = ctx.collision_strengths()
        s2 = st.cpu().numpy()
    ok = s2 == rmgb.RM_OK
    assert ok.sum() >= 60
    assert np.all(np.isfinite(om)) and np.abs(om[ok]).max() > 0.0
