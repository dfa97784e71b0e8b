"""MQDT coarse-mesh interpolation on the GPU (rm_solve_energies_qdt) against
the oracle's restatement (oracle/qdt.py): same segments, nodes, weights and
elimination, so Omega agrees to the FP64 tolerance (norm-wise per energy
and per element against the row's largest), statuses and open counts
exactly."""
import numpy as np
import pytest

import oracle
from oracle import qdt
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


def _pw4():
    pw = synth.random_pw(4711, 4, 60, z=2.0, a=10.0, e_max=1.8, sigma=0.1, l_max=3)
    pw["e_thr"] = np.array([0.0, 0.6, 1.2, 1.8])
    return pw


def _pw12():
    """12 channels on 6 levels (two channels per level, distinct l), z = 2,
    a = 12: several channels eliminated at once below the upper thresholds."""
    pw = synth.random_pw(4712, 12, 240, z=2.0, a=12.0, e_max=2.0, sigma=0.08, l_max=4)
    lev = np.arange(12) // 2
    pw["e_thr"] = np.repeat(np.linspace(0.0, 2.0, 6), 2)
    pw["l"] = np.array([0, 1, 1, 2, 0, 3, 2, 4, 1, 3, 0, 2], dtype=np.int32)
    pw["level"] = lev.astype(np.int32)
    pw["n_levels"] = 6
    return pw


def _close(got, ref, tol):
    nrm = np.linalg.norm(ref)
    if nrm == 0:
        return np.abs(got).max(initial=0.0) <= 1e-300
    mx = np.abs(ref).max()
    return np.linalg.norm(got - ref) <= tol * nrm and np.all(np.abs(got - ref) <= tol * np.maximum(np.abs(ref), mx))


def _gpu(rt, pw, E, ieq, qetest, iqdt):
    torch, rmgb = rt
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies_qdt(0, E, ieq, qetest, iqdt, no, st)
        om = ctx.collision_strengths()
        return st.cpu().numpy(), no.cpu().numpy(), om


CASES = [("4ch", -6, 0.0, 1), ("4ch", -6, 0.0, 2), ("4ch", 25, 0.0, 1), ("4ch", -4, 0.004, 1),
         ("12ch", -5, 0.0, 1), ("12ch", 40, 0.002, 1), ("12ch", -5, 0.0, 2)]


@pytest.mark.parametrize("name,ieq,qetest,iqdt", CASES)
def test_qdt_matches_oracle(rt, name, ieq, qetest, iqdt):
    pw = _pw4() if name == "4ch" else _pw12()
    E = synth.midpoint_grid(0.3, 2.4, 700)
    E = np.sort(np.concatenate([E, pw["e_thr"][1:2]]))       # one energy on a threshold
    st, no, om = _gpu(rt, pw, E, ieq, qetest, iqdt)
    ref = qdt.solve_energies(pw, E, ieq=ieq, qetest=qetest, iqdt=iqdt)
    assert np.array_equal(st, ref["status"]), np.nonzero(st != ref["status"])[0][:10]
    assert np.array_equal(no, ref["n_open"])
    assert (st == oracle.RM_ETHRESHOLD).sum() == 1
    n_elim = sum(int(np.sum(c == qdt.CL_ELIM)) for _, _, c in ref["plan"]["segments"])
    assert n_elim > 0
    bad = [m for m in range(E.size) if st[m] == 0 and not _close(om[m], ref["omega"][m], TOL)]
    assert not bad, bad[:10]


def test_qdt_every_node_equals_plain_mqdt(rt):
    """ieq = -1 on the GPU against the GPU's own per-energy MQDT solve, at the
    energies where both treat the same channels by quantum-defect theory."""
    torch, rmgb = rt
    pw = _pw12()
    E = synth.midpoint_grid(0.3, 2.4, 400)
    st, no, om = _gpu(rt, pw, E, -1, 0.0, 1)
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        s2 = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, E, 1, None, None, s2)
        om2 = ctx.collision_strengths()
        s2 = s2.cpu().numpy()
    ok = np.ones(E.size, dtype=bool)
    for m, x in enumerate(E):
        c = qdt.classes(float(x), pw)
        el = np.nonzero(c == qdt.CL_ELIM)[0]
        if el.size:
            nu = pw["z"] / np.sqrt(pw["e_thr"][el] - x)
            ok[m] = np.all(np.abs(oracle.rmatrix.sincos_pi(nu)[0]) >= 1.01e-3)
    ok &= (st == 0) & (s2 == 0)
    assert ok.sum() > 300
    bad = [m for m in np.nonzero(ok)[0] if not _close(om[m], om2[m], TOL)]
    assert not bad, bad[:10]


def test_qdt_rejects_bad_input(rt):
    torch, rmgb = rt
    pw = _pw4()
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        with pytest.raises(rmgb.RmError) as ei:
            ctx.solve_energies_qdt(0, np.array([0.5, 0.4, 0.7]), -2)
        assert ei.value.code == rmgb.RM_EINVAL
        with pytest.raises(rmgb.RmError):
            ctx.solve_energies_qdt(0, np.array([0.4, 0.5]), 0)
        with pytest.raises(rmgb.RmError):
            ctx.solve_energies_qdt(0, np.array([0.4, 0.5]), -2, 0.0, 3)


@pytest.mark.parametrize("iqdt", [1, 2])
def test_qdt_on_propagated_wave_matches_oracle(rt, iqdt):
    """The coarse-mesh interpolation on a wave that carries the outer-region
    propagation (rm_set_multipoles: R carried from a to r1 by Numerov, the
    matching and the kappa r cap of the eliminated set at r1) against
    oracle/qdt.py on the same wave (R propagated by DOP853): with a = 10,
    r1 = 13 and 4000 steps Numerov's O(h^4) error is ~1e-13 of R, so Omega
    agrees to the FP64 tolerance, statuses and open counts exactly."""
    torch, rmgb = rt
    pw = _pw4()
    rng = np.random.default_rng(4713)
    A = rng.normal(0.0, 0.3, (2, 4, 4))
    A = 0.5 * (A + A.transpose(0, 2, 1))
    r1, steps = 13.0, 4000
    E = synth.midpoint_grid(0.3, 2.4, 160)
    E = E[np.abs(E[:, None] - pw["e_thr"][None, :]).min(axis=1) > 5e-3]
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        ctx.set_multipoles(0, A, r1, steps)
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies_qdt(0, E, -6, 0.0, iqdt, no, st)
        om = ctx.collision_strengths()
        st, no = st.cpu().numpy(), no.cpu().numpy()
    pwp = dict(pw)
    pwp["prop"] = (A, r1)
    ref = qdt.solve_energies(pwp, E, ieq=-6, qetest=0.0, iqdt=iqdt)
    assert np.array_equal(st, ref["status"]), np.nonzero(st != ref["status"])[0][:10]
    assert np.array_equal(no, ref["n_open"])
    n_elim = sum(int(np.sum(c == qdt.CL_ELIM)) for _, _, c in ref["plan"]["segments"])
    assert n_elim > 0 and (st == 0).sum() > 100
    bad = [m for m in range(E.size) if st[m] == 0 and not _close(om[m], ref["omega"][m], TOL)]
    assert not bad, bad[:10]
