"""Pins of the oracle's MQDT coarse-mesh interpolation (oracle/qdt.py).

What fixes it independently of its own code:
  * every fine energy a node (ieq = -1) reduces it to the plain MQDT solve
    of rmatrix.py at each energy (an exact identity);
  * a K_u that is linear in energy is reproduced exactly by the linear
    interpolation, inside and beyond the outer nodes (extrapolation), so the
    plan, the weights and the elimination at the fine energy are checked on
    their own;
  * the interpolation error of a smooth K_u falls as the square of the node
    spacing;
  * the segment and qetest rules on hand-made grids.
"""
import numpy as np
import pytest

import oracle
from oracle import qdt
from paper_1909_07321_gb300 import synth


def _pw():
    """4 channels, z = 2, a = 10: closed channels within 0.25 Ry of their
    thresholds are eliminated (kappa a <= 5, nu >= 4 > l + 0.1)."""
    pw = synth.random_pw(4711, 4, 60, z=2.0, a=10.0, e_max=1.8, sigma=0.1, l_max=3)
    pw["e_thr"] = np.array([0.0, 0.6, 1.2, 1.8])
    return pw


def _sin_ok(pw, E):
    """Energies at which every eliminated channel has |sin pi nu| >= 1e-3
    (where rmatrix's own MQDT set agrees with the segment classes)."""
    ok = np.ones(E.size, dtype=bool)
    for m, x in enumerate(E):
        c = qdt.classes(float(x), pw)
        el = np.nonzero(c == qdt.CL_ELIM)[0]
        if el.size:
            nu = pw["z"] / np.sqrt(pw["e_thr"][el] - x)
            ok[m] = np.all(np.abs(oracle.rmatrix.sincos_pi(nu)[0]) >= 1e-3)
    return ok


@pytest.mark.parametrize("iqdt", [1, 2])
def test_every_energy_a_node_equals_plain_mqdt(iqdt):
    pw = _pw()
    E = synth.midpoint_grid(0.35, 1.75, 120)
    res = qdt.solve_energies(pw, E, ieq=-1, iqdt=iqdt)
    ref = oracle.solve_energies(pw, E, mode=oracle.MODE_MQDT)
    ok = _sin_ok(pw, E) & (ref["status"] == 0)
    assert ok.sum() > 100
    n_elim = sum(int(np.sum(qdt.classes(float(x), pw) == qdt.CL_ELIM)) for x in E[ok])
    assert n_elim > 50
    for m in np.nonzero(ok)[0]:
        assert res["status"][m] == 0
        if iqdt == 2:
            np.testing.assert_allclose(res["K"][m], ref["K"][m], rtol=1e-12, atol=1e-12)
        scale = max(1.0, np.abs(ref["omega"][m]).max())
        np.testing.assert_allclose(res["omega"][m], ref["omega"][m], rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("iqdt", [1, 2])
def test_linear_node_matrix_is_reproduced(monkeypatch, iqdt):
    pw = _pw()
    rng = np.random.default_rng(3)
    A = rng.normal(size=(4, 4)); A = A + A.T
    B = rng.normal(size=(4, 4)); B = B + B.T
    if iqdt == 1:
        A = A + 1j * rng.normal(size=(4, 4))
        B = B + 1j * rng.normal(size=(4, 4))

    def mu(pw_, x, cls_seg, iqdt_):
        P = np.nonzero(cls_seg != qdt.CL_DECAY)[0]
        return (A + x * B)[np.ix_(P, P)]

    monkeypatch.setattr(qdt, "node_matrix", mu)
    E = synth.midpoint_grid(0.35, 1.75, 200)
    drop_first = {}

    def valid(pw_, x, cls_seg, **kw):
        # drop the first node of every segment: the energies before the next
        # node are then extrapolated
        key = tuple(cls_seg)
        if key not in drop_first:
            drop_first[key] = x
            return False
        return x != drop_first[key]

    monkeypatch.setattr(qdt, "node_valid", valid)
    for ieq in (-7, 5, 23):
        drop_first.clear()
        res = qdt.solve_energies(pw, E, ieq=ieq, iqdt=iqdt)
        pl = res["plan"]
        for m, x in enumerate(E):
            if pl["seg"][m] < 0 or res["status"][m]:
                continue
            s = pl["seg"][m]
            cls_seg = pl["segments"][s][2]
            P = np.nonzero(cls_seg != qdt.CL_DECAY)[0]
            xs = res["nodes_used"][s]
            # linear in energy is reproduced exactly; one remaining node holds
            x_int = pl["e_int"][m] if xs.size > 1 else xs[0]
            Mx = (A + x_int * B)[np.ix_(P, P)]
            if iqdt == 2:
                Kx = qdt.eliminate(Mx, cls_seg, float(x), pw)
                np.testing.assert_allclose(res["K"][m], Kx, rtol=1e-10, atol=1e-10)
            else:
                Sx = qdt.eliminate_s(Mx, cls_seg, float(x), pw)
                row = np.zeros_like(res["omega"][m])
                oracle.rmatrix.omega_add(row, Sx - np.eye(Sx.shape[0]), np.nonzero(cls_seg == 0)[0],
                                         pw["level"], pw["n_levels"], pw["g"])
                np.testing.assert_allclose(res["omega"][m], row, rtol=1e-10, atol=1e-10)
        n_extra = sum(int(np.sum(E[pl["seg"] == s] < xs[0])) for s, xs in enumerate(res["nodes_used"])
                      if xs.size > 1)
        assert n_extra > 0       # some energies were extrapolated


def test_interpolation_error_second_order():
    """S_u interpolation inside one segment (all four channels open above
    1.8 Ry; K passes through poles there, S does not) and away from the
    R-matrix poles (with these weak amplitudes each pole carries a narrow
    feature that no coarse mesh resolves): the error against the exact solve
    falls ~4x per halving of the node spacing."""
    pw = _pw()
    E = synth.midpoint_grid(2.25, 2.60, 193)
    assert np.min(np.abs(pw["E_k"][:, None] - E[None, :])) > 0.09
    exact = oracle.solve_energies(pw, E, mode=oracle.MODE_MQDT)
    errs = []
    for ieq in (-48, -24, -12):
        res = qdt.solve_energies(pw, E, ieq=ieq, iqdt=1)
        assert len(res["plan"]["segments"]) == 1
        errs.append(max(np.abs(res["omega"][m] - exact["omega"][m]).max() for m in range(E.size)))
    assert errs[0] > 1e-9
    assert 2.5 < errs[0] / errs[1] < 6.5 and 2.5 < errs[1] / errs[2] < 6.5, errs


def test_segments_and_thresholds():
    pw = _pw()
    E = np.array([0.2, 0.3, 0.6, 0.7, 1.19, 1.21, 1.3])   # 0.6 is a threshold
    pl = qdt.plan(pw, E, ieq=-1)
    assert pl["seg"][2] == -1
    # the open set changes at 0.6 and 1.2, the eliminated set where a channel
    # falls 0.25 Ry below its threshold
    for m in range(E.size - 1):
        if pl["seg"][m] >= 0 and pl["seg"][m] == pl["seg"][m + 1]:
            assert np.array_equal(qdt.classes(E[m], pw), qdt.classes(E[m + 1], pw))
    assert len(set(pl["seg"][pl["seg"] >= 0].tolist())) >= 4
    res = qdt.solve_energies(pw, E, ieq=-2)
    assert res["status"][2] == oracle.RM_ETHRESHOLD and not res["omega"][2].any()


def test_qetest_reuses_the_last_interpolation_energy():
    pw = _pw()
    E = 1.9 + 0.001 * np.arange(12)
    pl = qdt.plan(pw, E, ieq=-3, qetest=0.0025)
    # re-interpolated when the energy has moved by more than 0.0025 Ry
    expect = [E[0], E[0], E[0], E[3], E[3], E[3], E[6], E[6], E[6], E[9], E[9], E[9]]
    np.testing.assert_array_equal(pl["e_int"], expect)
    pl0 = qdt.plan(pw, E, ieq=-3, qetest=0.0)
    np.testing.assert_array_equal(pl0["e_int"], E)
    with pytest.raises(ValueError):
        qdt.plan(pw, E, ieq=0)


def test_every_energy_a_node_with_propagation():
    """With the outer-region propagation (pw["prop"] = (A, r1)) every fine
    energy a node still reduces the interpolation to the plain propagated
    MQDT solve of oracle/propagate.py (the matching radius r1 in both)."""
    from oracle import propagate
    pw = _pw()
    rng = np.random.default_rng(8)
    A = rng.normal(0.0, 0.3, (2, 4, 4))
    A = 0.5 * (A + A.transpose(0, 2, 1))
    r1 = 13.0
    pwp = dict(pw, prop=(A, r1))
    E = synth.midpoint_grid(0.35, 1.75, 80)
    res = qdt.solve_energies(pwp, E, ieq=-1, iqdt=2)
    ref = propagate.solve_energies(pw, E, A, r1, mode=oracle.MODE_MQDT)
    ok = _sin_ok(pwp, E) & (ref["status"] == 0)
    assert ok.sum() > 60
    n_elim = sum(int(np.sum(qdt.classes(float(x), pwp) == qdt.CL_ELIM)) for x in E[ok])
    assert n_elim > 15
    for m in np.nonzero(ok)[0]:
        assert res["status"][m] == 0
        np.testing.assert_allclose(res["K"][m], ref["K"][m], rtol=1e-12, atol=1e-12)
        scale = max(1.0, np.abs(ref["omega"][m]).max())
        np.testing.assert_allclose(res["omega"][m], ref["omega"][m], rtol=0, atol=1e-11 * scale)
    # and the propagation changes the answer
    plain = qdt.solve_energies(pw, E, ieq=-1, iqdt=2)
    assert max(np.abs(res["omega"][m] - plain["omega"][m]).max() for m in np.nonzero(ok)[0]) > 1e-4
