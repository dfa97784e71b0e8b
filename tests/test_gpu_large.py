"""Global-memory solver (any channel count) against the oracle and against the
shared-memory solver, in direct and MQDT modes, FP64 and mixed formation."""
import numpy as np
import pytest

import oracle
from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_K = 1e-9


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


def _close_rel(got, ref, tol):
    nrm = np.linalg.norm(ref)
    if nrm == 0:
        return np.abs(got).max(initial=0.0) == 0
    mx = np.abs(ref).max()
    return (np.linalg.norm(got - ref) <= tol * nrm and
            np.all(np.abs(got - ref) <= tol * np.maximum(np.abs(ref), mx)))


def _gpu(rt, pw, E, mode=0, solver=0, precision=0, mem_budget=0):
    torch, rmgb = rt
    n = pw["W"].shape[0]
    with rmgb.Context(precision=precision, solver=solver, mem_budget=mem_budget) as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, Ed, mode, K, no, st)
        om = ctx.collision_strengths()
    return dict(K=K.cpu().numpy().reshape(E.size, n, n), n_open=no.cpu().numpy(),
                status=st.cpu().numpy(), omega=om)


def _compare(res, ref, tol=TOL_K):
    assert np.array_equal(res["status"], ref["status"])
    assert np.array_equal(res["n_open"], ref["n_open"])
    bad = []
    for m in range(ref["status"].size):
        if ref["status"][m]:
            continue
        k = ref["n_open"][m]
        if not _close_rel(res["K"][m, :k, :k], ref["K"][m], tol):
            bad.append(("K", m))
        if not _close_rel(res["omega"][m], ref["omega"][m], tol):
            bad.append(("Omega", m))
    assert not bad, bad[:10]


def _pw150():
    pw = synth.random_pw(150, 150, 4500, z=2.0, a=18.0, e_max=2.0, sigma=0.04, pole_lo=-2.0,
                         pole_hi=60.0, l_max=8)
    # 3 channels per level for the Omega sums (levels share thresholds)
    lev = np.arange(150) // 3
    pw["level"] = lev.astype(np.int32)
    pw["n_levels"] = 50
    pw["e_thr"] = np.sort(pw["e_thr"])[::3][lev]
    pw["e_thr"][:3] = 0.0
    return pw


@pytest.mark.parametrize("mode", [0, 1])
def test_large_solver_forced_on_small_workload(rt, mode):
    pws, E = synth.workload_small(400)
    pw = pws[0]
    res = _gpu(rt, pw, E, mode=mode, solver=2, mem_budget=300 * 1024)
    ref = oracle.solve_energies(pw, E, mode=mode)
    _compare(res, ref)
    small = _gpu(rt, pw, E, mode=mode, solver=1)
    for m in range(E.size):
        if small["status"][m] == 0:
            k = small["n_open"][m]
            assert _close_rel(res["K"][m, :k, :k], small["K"][m, :k, :k], 1e-11)


def test_large_solver_forced_on_64ch_sample(rt):
    pws, E = synth.workload_64ch()
    pw = pws[0]
    rng = np.random.default_rng(12)
    Es = np.sort(E[rng.choice(E.size, 96, replace=False)])
    for mode in (0, 1):
        res = _gpu(rt, pw, Es, mode=mode, solver=2)
        ref = oracle.solve_energies(pw, Es, mode=mode)
        _compare(res, ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_150_channels_auto_large(rt, mode):
    pw = _pw150()
    E = np.sort(np.concatenate([synth.midpoint_grid(0.05, 2.3, 29),
                                pw["e_thr"][3::15][:6] - 0.004]))
    res = _gpu(rt, pw, E, mode=mode, mem_budget=12 * 2**20)   # several ragged blocks
    ref = oracle.solve_energies(pw, E, mode=mode)
    _compare(res, ref)


def test_150_channels_mixed_formation(rt):
    """bf16x3 tensor-core formation feeding the global-memory solver: same
    statuses, Omega within the mixed-precision band of the FP64 result."""
    pw = _pw150()
    E = synth.midpoint_grid(0.05, 2.3, 40)
    a = _gpu(rt, pw, E, precision=0)
    b = _gpu(rt, pw, E, precision=2)
    assert np.array_equal(a["status"], b["status"])
    rel = (np.linalg.norm(a["omega"] - b["omega"], axis=1) /
           np.maximum(np.linalg.norm(a["omega"], axis=1), 1e-300))
    assert np.median(rel) < 1e-3 and rel.max() < 0.5
