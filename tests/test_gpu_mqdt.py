"""MQDT mode (closed channels eliminated through the unphysical K-matrix) on
the GPU, against the oracle's MQDT route and against the GPU's own direct
mode (the elimination is an exact identity, so both give the same K)."""
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


def _gpu(rt, pw, E, mode):
    torch, rmgb = rt
    n = pw["W"].shape[0]
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, Ed, mode, K, no, st)
        om = ctx.collision_strengths()
    return (K.cpu().numpy().reshape(E.size, n, n), no.cpu().numpy(), st.cpu().numpy(), om)


def _n_eliminated(pw, E):
    tot = 0
    for x in E:
        cf = oracle.channel_functions(float(x), pw["e_thr"], pw["l"], pw["z"], pw["a"])
        tot += int(oracle.mqdt_set(cf, pw["l"], a=pw["a"]).sum())
    return tot


@pytest.mark.parametrize("which", ["small", "64ch"])
def test_mqdt_vs_oracle_and_direct(rt, which):
    if which == "small":
        pws, E = synth.workload_small(600)
        Es = E
    else:
        pws, E = synth.workload_64ch()
        rng = np.random.default_rng(8)
        Es = np.sort(E[rng.choice(E.size, 120, replace=False)])
    pw = pws[0]
    assert _n_eliminated(pw, Es) > 20
    Km, nom, stm, omm = _gpu(rt, pw, Es, 1)
    Kd, nod, std, omd = _gpu(rt, pw, Es, 0)
    ref = oracle.solve_energies(pw, Es, mode=oracle.MODE_MQDT)
    assert np.array_equal(stm, ref["status"]) and np.array_equal(nom, ref["n_open"])
    bad = []
    for m in range(Es.size):
        if stm[m]:
            continue
        k = nom[m]
        if not _close_rel(Km[m, :k, :k], ref["K"][m], TOL_K):
            bad.append(("K vs oracle", m))
        if not _close_rel(omm[m], ref["omega"][m], TOL_K):
            bad.append(("Omega vs oracle", m))
        if std[m] == 0 and not _close_rel(Km[m, :k, :k], Kd[m, :k, :k], TOL_K):
            bad.append(("K vs direct", m))
    assert not bad, bad[:8]


def test_mqdt_fnumin_excludes_channels(rt):
    """With fnumin above every nu the MQDT mode reduces to the direct mode."""
    torch, rmgb = rt
    pws, E = synth.workload_small(200)
    pw = pws[0]
    n = pw["W"].shape[0]
    outs = []
    for mode, fnumin in [(1, 1e9), (0, 0.0)]:
        with rmgb.Context(fnumin=fnumin) as ctx:
            ctx.load_pw(0, pw)
            K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
            ctx.solve_energies(0, torch.tensor(E, device="cuda"), mode, K)
            outs.append((K.cpu().numpy(), ctx.collision_strengths()))
    # same arithmetic; the two kernel instantiations may contract FMAs differently
    np.testing.assert_allclose(outs[0][0], outs[1][0], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(outs[0][1], outs[1][1], rtol=1e-11, atol=1e-13)
