"""Batched solve of many partial waves (rm_solve_batch) on the batched
workload: 40 partial waves of 20-400 channels (30 poles per channel, z = 3)
on one energy grid, spread over the lanes of one context, captured into a
CUDA graph and replayed. Checked against the sum of the oracle's collision
strengths over the waves (FP64 path at 1e-9; mixed path within the sum of the
per-wave stated bounds), against one rm_solve_energies call per wave, and
replay against the first (eager) call."""
import numpy as np
import pytest

import oracle
from paper_1909_07321_gb300 import synth
from test_gpu_mixed import R_BOUND, U32, _first_order_k_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


@pytest.fixture(scope="module")
def workload():
    pws, E = synth.workload_batched()
    # few, half and most channels open, and 2.5e-4 Ry above the last threshold
    # (4 Ry), where the mixed path's error against FP64 is largest
    Es = E[[150, 2990, 6400, 8000, 9101]].copy()
    return pws, Es


@pytest.fixture(scope="module")
def oracle_sum(workload):
    pws, Es = workload
    nl = pws[0]["n_levels"]
    tot = np.zeros((Es.size, nl * (nl + 1) // 2))
    per = []
    for pw in pws:
        r = oracle.solve_energies(pw, Es)
        tot += r["omega"]
        per.append(r)
    return tot, per


def _batch(rmgb, torch, pws, Es, prec, sp, lanes=4, calls=1, graph=True, autotune=0):
    with rmgb.Context(precision=prec, solve_precision=sp, lanes=lanes, autotune=autotune, stream=0) as ctx:
        for i, pw in enumerate(pws):
            ctx.load_pw(i, pw)
        Ed = torch.tensor(Es, dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(calls):
            ctx.solve_batch(list(range(len(pws))), Ed, 0, graph)
            outs.append(ctx.collision_strengths(reset=False).copy())
            ctx.reset_omega()
        info = [ctx.autotune_info(i) for i in range(len(pws))] if autotune else None
    return outs, info


def _cf_amplification(pws, x, seed=0):
    """Largest factor over the waves by which a relative perturbation of 1e-13
    of the oracle's channel functions at energy x moves K (relative,
    Frobenius): the matching's amplification of channel-function errors."""
    import oracle.rmatrix as orm
    rng = np.random.default_rng(seed)
    amp = 1.0
    for pw in pws:
        cf = orm.channel_functions(x, pw["e_thr"], pw["l"], pw["z"], pw["a"])
        R = orm.r_matrix(x, pw["E_k"], pw["W"], pw["a"])
        K0, _ = orm.match_direct(R, cf, pw["a"])
        if K0 is None or K0.size == 0:
            continue
        cf2 = dict(cf)
        for key in ("s", "sp", "c", "cp", "th", "thp"):
            cf2[key] = cf[key] * (1.0 + 1e-13 * rng.standard_normal(cf[key].shape))
        K1, _ = orm.match_direct(R, cf2, pw["a"])
        amp = max(amp, np.linalg.norm(K1 - K0) / np.linalg.norm(K0) / 1e-13)
    return amp


def test_batched_fp64_equals_summed_oracle(rt, workload, oracle_sum):
    """FP64 path: 1e-9 relative where the matching is well conditioned; at an
    energy where it amplifies channel-function errors A-fold (2.5e5 at
    2.5e-4 Ry above the 4 Ry threshold, eta = -190 in the channel just
    opened) the bound is 1e-9 + 4 A 1e-11 (the channel functions' accuracy,
    1e-11 of the amplitude, through K into |T|^2)."""
    torch, rmgb = rt
    pws, Es = workload
    (om,), _ = _batch(rmgb, torch, pws, Es, 0, 0)
    ref, _ = oracle_sum
    for m in range(Es.size):
        nrm = np.linalg.norm(ref[m])
        rel = np.linalg.norm(om[m] - ref[m]) / nrm
        if rel <= 1e-9:
            continue
        amp = _cf_amplification(pws, float(Es[m]))
        assert amp > 1e3 and rel <= 1e-9 + 4.0 * amp * 1e-11, (m, rel, amp)


def test_batched_mixed_within_summed_bounds_and_graph_replay(rt, workload, oracle_sum):
    """bf16x3 formation chosen per wave by the autotuner, FP32 matching: the
    Omega error at each energy within the sum over waves of the stated
    per-wave bounds; the graph replays (calls 2 and 3) equal the eager first
    call bit for bit."""
    torch, rmgb = rt
    pws, Es = workload
    outs, info = _batch(rmgb, torch, pws, Es, 2, 1, calls=3, autotune=1)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    ref, per = oracle_sum
    om = outs[0]
    for m in range(Es.size):
        bound = 0.0
        for pw, r in zip(pws, per):
            if r["status"][m]:
                continue
            Ko = r["K"][m]
            k = Ko.shape[0]
            bK = _first_order_k_bound(pw, Es[m], U32, r_bound=R_BOUND)
            B = 3.0 * np.linalg.norm(bK) + k * U32 * np.linalg.norm(np.eye(k) - 1j * Ko)
            bound += pw["g"] * (8 * k * B + 4 * B * B)
        assert np.abs(om[m] - ref[m]).sum() <= bound + 1e-12, (m, np.abs(om[m] - ref[m]).sum(), bound)
    forms = {f for f, *_ in info}
    assert forms <= {1, 2} and len(info) == len(pws)


def test_batched_equals_one_call_per_wave(rt, workload):
    torch, rmgb = rt
    pws, Es = workload
    (batch,), _ = _batch(rmgb, torch, pws, Es, 2, 1, lanes=3)
    with rmgb.Context(precision=2, solve_precision=1) as ctx:
        for i, pw in enumerate(pws):
            ctx.load_pw(i, pw)
        for i in range(len(pws)):
            ctx.solve_energies(i, Es, 0)
        one = ctx.collision_strengths()
    rel = np.linalg.norm(batch - one, axis=1) / np.linalg.norm(one, axis=1)
    assert rel.max() <= 1e-12, rel
