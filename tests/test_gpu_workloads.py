"""Parity on the shapes of the batched and 1000-channel workloads, at energy
counts the oracle finishes quickly: several partial waves of uneven channel
counts accumulated into one Omega (4 channels per target level), and one
1000-channel partial wave with 30000 poles."""
import numpy as np
import pytest

import oracle
from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_batched_partial_waves_accumulate(rt):
    """Four partial waves of the batched workload (the smallest, the largest
    and two between) with the shared 100-level grid; Omega summed over them."""
    torch, rmgb = rt
    pws, E = synth.workload_batched(n_pw=40, n_energies=10000)
    sizes = np.array([p["W"].shape[0] for p in pws])
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), 5, 17]
    rng = np.random.default_rng(21)
    idx = np.sort(rng.choice(E.size, 12, replace=False))
    Es = E[idx]
    ref = np.zeros((Es.size, pws[0]["n_levels"] * (pws[0]["n_levels"] + 1) // 2))
    statuses = []
    for p in pick:
        r = oracle.solve_energies(pws[p], Es)
        ref += r["omega"]
        statuses.append(r["status"])
    with rmgb.Context() as ctx:
        for p in pick:
            ctx.load_pw(p, pws[p])
        for p in pick:
            st = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
            ctx.solve_energies(p, torch.tensor(Es, device="cuda"), 0, None, None, st)
            assert np.array_equal(st.cpu().numpy(), statuses[pick.index(p)])
        om = ctx.collision_strengths()
    for m in range(Es.size):
        assert _rel(om[m], ref[m]) <= TOL, m


@pytest.mark.slow
def test_1000_channel_partial_wave(rt):
    """The 1000-channel, 30000-pole partial wave at three energies (one
    below the highest thresholds, two across the band), FP64 path."""
    torch, rmgb = rt
    pws, E = synth.workload_1000ch(n_energies=5000)
    pw = pws[0]
    Es = np.array([E[700], E[2600], E[4300]])
    ref = oracle.solve_energies(pw, Es)
    n = pw["W"].shape[0]
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        K = torch.zeros((Es.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(Es.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, torch.tensor(Es, device="cuda"), 0, K, no, st)
        om = ctx.collision_strengths()
    K = K.cpu().numpy().reshape(Es.size, n, n)
    assert np.array_equal(st.cpu().numpy(), ref["status"])
    assert np.array_equal(no.cpu().numpy(), ref["n_open"])
    for m in range(Es.size):
        k = ref["n_open"][m]
        assert _rel(K[m, :k, :k], ref["K"][m]) <= TOL, m
        assert _rel(om[m], ref["omega"][m]) <= TOL, m
